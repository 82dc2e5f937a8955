"""The C ABI without a GPU: the library loads, exports every entry point of
include/dr.h, and its host-side logic (validation, index arithmetic, zip
re-segmentation, take / drop) matches the oracle.  No call here touches the
device: containers are built over fake (never dereferenced) pointers."""
import ctypes
import os
import re

import pytest

import oracle
from paper_2406_00158_gb300 import _lib as L
from paper_2406_00158_gb300 import build as B
from paper_2406_00158_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def header_functions():
    text = open(os.path.join(ROOT, "include", "dr.h")).read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(dr_\w+)\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported_and_bound(lib):
    names = header_functions()
    assert len(names) >= 35
    for n in names:
        assert hasattr(lib, n), n
        assert n in L.PROTOTYPES, n
    assert set(L.PROTOTYPES) == set(names)
    assert lib.dr_version() == 1


def fake_ptrs(lens, base=1 << 32, esz=4):
    out, p = [], base
    for n in lens:
        out.append(p)
        p += ((n * esz + 255) // 256 + 1) * 256
    return out


def make_vec(lens, dtype=L.DR_F32, ptrs=None):
    ptrs = ptrs or fake_ptrs(lens)
    h = ctypes.c_void_p()
    rc = L.lib().dr_vec_create(dtype, len(lens), (ctypes.c_int64 * len(lens))(*lens),
                               (ctypes.c_void_p * len(lens))(*ptrs), ctypes.byref(h))
    return rc, h


def test_vec_create_validation(lib):
    rc, h = make_vec([4, 0, 5])
    assert rc == L.DR_OK
    n, ns, dt = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
    assert lib.dr_vec_info(h, ctypes.byref(dt), ctypes.byref(ns), ctypes.byref(n)) == 0
    assert (dt.value, ns.value, n.value) == (L.DR_F32, 3, 9)
    lib.dr_vec_destroy(h)
    assert make_vec([3, -1])[0] == L.DR_E_INVAL
    assert make_vec([3, 2], ptrs=[1 << 20, 0])[0] == L.DR_E_INVAL      # NULL non-empty segment
    assert make_vec([3, 0], ptrs=[1 << 20, 0])[0] == L.DR_OK           # NULL empty segment is fine
    assert make_vec([3], ptrs=[(1 << 20) + 2])[0] == L.DR_E_ALIGN     # not element aligned
    assert make_vec([3], dtype=9)[0] == L.DR_E_DTYPE
    h = ctypes.c_void_p()
    assert lib.dr_vec_create(0, 0, None, None, ctypes.byref(h)) == L.DR_E_INVAL
    assert "nseg" in L.last_error()


def test_block_lengths_ceil_partition(lib):
    for n, p in [(10, 3), (9, 3), (1, 4), (0, 2), (1 << 20, 8), (7, 7)]:
        out = (ctypes.c_int64 * p)()
        assert lib.dr_block_lengths(n, p, out) == 0
        b = -(-n // p)
        assert list(out) == inputs.block_segments(n, p)
        assert sum(out) == n and all(v <= b for v in out)


def test_locate_matches_bruteforce(lib):
    lens = [3, 0, 5, 1, 0, 4]
    _, h = make_vec(lens)
    owner = [(k, j) for k, L_ in enumerate(lens) for j in range(L_)]
    seg, off = ctypes.c_int(), ctypes.c_int64()
    for i, (k, j) in enumerate(owner):
        assert lib.dr_vec_locate(h, i, ctypes.byref(seg), ctypes.byref(off)) == 0
        assert (seg.value, off.value) == (k, j)
    assert lib.dr_vec_locate(h, len(owner), ctypes.byref(seg), ctypes.byref(off)) == L.DR_E_BOUNDS
    assert lib.dr_vec_locate(h, -1, ctypes.byref(seg), ctypes.byref(off)) == L.DR_E_BOUNDS
    lib.dr_vec_destroy(h)


def view_of(h):
    v = ctypes.c_void_p()
    assert L.lib().dr_view_of(h, ctypes.byref(v)) == 0
    return v


def pieces(view):
    n = ctypes.c_int()
    size = ctypes.c_int64()
    L.lib().dr_view_info(view, ctypes.byref(size), None, None, ctypes.byref(n))
    arr = (L.dr_piece * max(1, n.value))()
    assert L.lib().dr_view_segments(view, n.value, arr) == 0
    return size.value, [(p.seg[0], p.off[0], p.seg[1], p.off[1], p.len) for p in arr[:n.value]]


@pytest.mark.parametrize("trial", range(25))
def test_zip_resegmentation_matches_oracle(lib, trial):
    na, nb = 1 + trial % 6, 1 + (3 * trial) % 7
    la = inputs.random_cut_segments(300 + trial, 120, na)
    lb = inputs.random_cut_segments(400 + trial, 120 - (trial % 3) * 7, nb)
    if trial % 4 == 0:
        la = [0] + la + [0]
    _, ha = make_vec(la)
    _, hb = make_vec(lb, ptrs=fake_ptrs(lb, base=1 << 40))
    z = ctypes.c_void_p()
    assert lib.dr_view_zip(view_of(ha), view_of(hb), ctypes.byref(z)) == 0
    size, got = pieces(z)
    assert got == oracle.zip_segments_bruteforce(la, lb)
    assert size == min(sum(la), sum(lb))


def test_take_drop_trim_segments(lib):
    lens = [5, 3, 0, 6]
    _, h = make_vec(lens)
    v = view_of(h)
    for f in range(0, 15):
        for l in range(0, 15):
            t, d = ctypes.c_void_p(), ctypes.c_void_p()
            assert lib.dr_view_drop(v, f, ctypes.byref(d)) == 0
            assert lib.dr_view_take(d, l, ctypes.byref(t)) == 0
            size, got = pieces(t)
            lo = min(f, 14)
            hi = min(14, lo + l)
            assert size == hi - lo
            # the oracle's trimmed segment list (take(l) after drop(f) = trim to [lo, hi))
            exp = [[k, o, -1, 0, n] for k, o, n in oracle.trim_segments(lens, lo, hi)]
            assert [list(p) for p in got] == exp
            lib.dr_view_destroy(t)
            lib.dr_view_destroy(d)


def test_view_composition_rules(lib):
    _, ha = make_vec([8])
    _, hb = make_vec([8], dtype=L.DR_F64, ptrs=[1 << 44])
    va, vb = view_of(ha), view_of(hb)
    z = ctypes.c_void_p()
    assert lib.dr_view_zip(va, vb, ctypes.byref(z)) == L.DR_E_DTYPE
    _, hc = make_vec([4, 4], ptrs=[1 << 41, 1 << 42])
    assert lib.dr_view_zip(va, view_of(hc), ctypes.byref(z)) == 0
    t = ctypes.c_void_p()
    assert lib.dr_view_transform(z, L.DR_U_SCALE, 2.0, ctypes.byref(t)) == L.DR_E_INVAL  # raw zip
    zt = ctypes.c_void_p()
    assert lib.dr_view_zip_transform(z, L.DR_MUL, ctypes.byref(zt)) == 0
    arity = ctypes.c_int()
    lib.dr_view_info(zt, None, ctypes.byref(arity), None, None)
    assert arity.value == 1
    # chains are bounded
    cur = zt
    for k in range(4):
        nxt = ctypes.c_void_p()
        assert lib.dr_view_transform(cur, L.DR_U_ADD, 1.0, ctypes.byref(nxt)) == 0
        cur = nxt
    nxt = ctypes.c_void_p()
    assert lib.dr_view_transform(cur, L.DR_U_ADD, 1.0, ctypes.byref(nxt)) == L.DR_E_UNSUPPORTED
    # zip of a zip is outside this build
    assert lib.dr_view_zip(zt, va, ctypes.byref(nxt)) == L.DR_E_UNSUPPORTED


def test_md2_validation(lib):
    h = ctypes.c_void_p()
    rows = (ctypes.c_int64 * 2)(3, 4)
    ptrs = (ctypes.c_void_p * 2)(1 << 32, 1 << 33)
    assert lib.dr_md2_create(L.DR_F32, 7, 16, 2, rows, ptrs, ctypes.byref(h)) == 0
    lib.dr_md2_destroy(h)
    assert lib.dr_md2_create(L.DR_F32, 8, 16, 2, rows, ptrs, ctypes.byref(h)) == L.DR_E_INVAL
    assert lib.dr_md2_create(L.DR_F64, 7, 16, 2, rows, ptrs, ctypes.byref(h)) == L.DR_E_DTYPE
    bad = (ctypes.c_void_p * 2)(1 << 32, (1 << 33) + 2)
    assert lib.dr_md2_create(L.DR_F32, 7, 16, 2, rows, bad, ctypes.byref(h)) == L.DR_E_ALIGN


def test_status_knobs(lib):
    assert lib.dr_set_spin_limit(0) == L.DR_E_INVAL
    assert lib.dr_set_spin_limit(1 << 21) == 0
    assert lib.dr_debug_skip_publish(-5) == 0


# ----------------------------------------------------------------------------------
# k-ary zip, for_each and transform: host-side rules (no launch)
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("trial", range(12))
def test_zipn_resegmentation_matches_oracle(lib, trial):
    k = 2 + trial % 5
    lens_list, views = [], []
    for o in range(k):
        n = 150 - (o * trial) % 9
        lens = inputs.random_cut_segments(700 + 10 * trial + o, n, 1 + (trial + 2 * o) % 6)
        if (trial + o) % 3 == 0:
            lens = [0] + lens
        _, h = make_vec(lens, ptrs=fake_ptrs(lens, base=(o + 1) << 36))
        lens_list.append(lens)
        views.append(view_of(h))
    z = ctypes.c_void_p()
    assert lib.dr_view_zipn(k, (ctypes.c_void_p * k)(*views), ctypes.byref(z)) == 0
    size, got = pieces(z)
    exp = oracle.zip_segments_bruteforce_k(lens_list)
    assert size == min(sum(l) for l in lens_list)
    # dr_piece reports the first two operands; the cuts of all k show in the lengths
    assert got == [(s[0], f[0], s[1], f[1], n) for s, f, n in exp]
    arity = ctypes.c_int()
    lib.dr_view_info(z, None, ctypes.byref(arity), None, None)
    assert arity.value == k


def test_zipn_composition_rules(lib):
    _, ha = make_vec([8])
    _, hb = make_vec([8], ptrs=[1 << 41])
    _, hd = make_vec([8], dtype=L.DR_F64, ptrs=[1 << 42])
    va, vb, vd = view_of(ha), view_of(hb), view_of(hd)
    z = ctypes.c_void_p()
    arr = lambda *v: (ctypes.c_void_p * len(v))(*v)
    assert lib.dr_view_zipn(1, arr(va), ctypes.byref(z)) == L.DR_E_UNSUPPORTED
    assert lib.dr_view_zipn(7, arr(*([va] * 7)), ctypes.byref(z)) == L.DR_E_UNSUPPORTED
    assert lib.dr_view_zipn(2, arr(va, vd), ctypes.byref(z)) == L.DR_E_DTYPE
    assert lib.dr_view_zipn(2, arr(va, None), ctypes.byref(z)) == L.DR_E_INVAL
    t = ctypes.c_void_p()
    assert lib.dr_view_transform(va, L.DR_U_SCALE, 2.0, ctypes.byref(t)) == 0
    assert lib.dr_view_zipn(2, arr(va, t), ctypes.byref(z)) == L.DR_E_UNSUPPORTED  # transformed leaf
    z2 = ctypes.c_void_p()
    assert lib.dr_view_zipn(2, arr(va, vb), ctypes.byref(z2)) == 0
    assert lib.dr_view_zipn(2, arr(z2, va), ctypes.byref(z)) == L.DR_E_UNSUPPORTED  # zip of a zip
    # a 2-ary zipn is a zip: zip_transform applies
    zt = ctypes.c_void_p()
    assert lib.dr_view_zip_transform(z2, L.DR_MUL, ctypes.byref(zt)) == 0
    # trimmed leaves are allowed
    d = ctypes.c_void_p()
    assert lib.dr_view_drop(vb, 3, ctypes.byref(d)) == 0
    assert lib.dr_view_zipn(2, arr(va, d), ctypes.byref(z)) == 0
    size = ctypes.c_int64()
    lib.dr_view_info(z, ctypes.byref(size), None, None, None)
    assert size.value == 5


def test_for_each_validation(lib):
    F = {"copy": 0, "scale": 1, "add": 2, "triad": 3, "bs": 4}
    vs = [view_of(make_vec([64], ptrs=[(i + 1) << 36])[1]) for i in range(5)]
    arr = lambda *v: (ctypes.c_void_p * len(v))(*v)
    z3 = ctypes.c_void_p()
    assert lib.dr_view_zipn(3, arr(*vs[:3]), ctypes.byref(z3)) == 0
    q = (ctypes.c_double * 2)(3.0, 0.2)
    assert lib.dr_for_each(None, F["add"], q, 0, None) == L.DR_E_INVAL
    assert lib.dr_for_each(z3, 9, q, 2, None) == L.DR_E_INVAL                  # unknown function
    assert lib.dr_for_each(z3, F["copy"], q, 0, None) == L.DR_E_INVAL          # copy takes a 2-zip
    assert lib.dr_for_each(z3, F["bs"], q, 2, None) == L.DR_E_INVAL            # black-scholes a 5-zip
    assert lib.dr_for_each(z3, F["triad"], q, 0, None) == L.DR_E_INVAL         # triad needs q
    assert lib.dr_for_each(vs[0], F["copy"], q, 0, None) == L.DR_E_INVAL       # not a zip
    # integer vectors
    iv = [view_of(make_vec([64], dtype=L.DR_I64, ptrs=[(i + 1) << 38])[1]) for i in range(2)]
    zi = ctypes.c_void_p()
    assert lib.dr_view_zipn(2, arr(*iv), ctypes.byref(zi)) == 0
    assert lib.dr_for_each(zi, F["copy"], q, 0, None) == L.DR_E_DTYPE
    # a written operand overlapping another operand without coinciding: rejected
    _, hx = make_vec([64], ptrs=[1 << 40])
    _, hy = make_vec([64], ptrs=[(1 << 40) + 4 * 8])   # 8 elements further into the same memory
    zo = ctypes.c_void_p()
    assert lib.dr_view_zipn(2, arr(view_of(hx), view_of(hy)), ctypes.byref(zo)) == 0
    assert lib.dr_for_each(zo, F["copy"], q, 0, None) == L.DR_E_INVAL
    # an empty zip launches nothing
    ve = [view_of(make_vec([0], ptrs=[(i + 1) << 39])[1]) for i in range(3)]
    ze = ctypes.c_void_p()
    assert lib.dr_view_zipn(3, arr(*ve), ctypes.byref(ze)) == 0
    assert lib.dr_for_each(ze, F["add"], q, 0, None) == L.DR_OK


def test_transform_validation(lib):
    _, ha = make_vec([32])
    _, hb = make_vec([16], ptrs=[1 << 41])
    _, hd = make_vec([32], dtype=L.DR_F64, ptrs=[1 << 42])
    va = view_of(ha)
    assert lib.dr_transform(va, hb, None) == L.DR_E_INVAL     # output too short
    assert lib.dr_transform(va, hd, None) == L.DR_E_DTYPE
    assert lib.dr_transform(va, None, None) == L.DR_E_INVAL
    z = ctypes.c_void_p()
    _, hc = make_vec([32], ptrs=[1 << 43])
    assert lib.dr_view_zip(va, view_of(hc), ctypes.byref(z)) == 0
    assert lib.dr_transform(z, hc, None) == L.DR_E_INVAL      # raw zip
    _, hs = make_vec([32], ptrs=[(1 << 32) + 4])               # one element past a's start
    assert lib.dr_transform(va, hs, None) == L.DR_E_INVAL     # partial overlap


def test_sort_validation(lib):
    _, ha = make_vec([32])
    _, hb = make_vec([16], ptrs=[1 << 41])
    _, hd = make_vec([32], dtype=L.DR_F64, ptrs=[1 << 42])
    va = view_of(ha)
    assert lib.dr_sort(va, hb, None) == L.DR_E_INVAL      # output too short
    assert lib.dr_sort(va, hd, None) == L.DR_E_DTYPE
    assert lib.dr_sort(va, None, None) == L.DR_E_INVAL
    z = ctypes.c_void_p()
    assert lib.dr_view_zip(va, view_of(hb), ctypes.byref(z)) == 0
    assert lib.dr_sort(z, ha, None) == L.DR_E_INVAL       # raw zip
    _, he = make_vec([0])
    assert lib.dr_sort(view_of(he), he, None) == L.DR_OK  # nothing to sort, no launch
    big = [1 << 29, 1 << 29]                                # 2^30 elements: beyond the counters
    _, hbig = make_vec(big, ptrs=fake_ptrs(big, base=1 << 44))
    assert lib.dr_sort(view_of(hbig), hbig, None) == L.DR_E_UNSUPPORTED


def test_more_than_128_pieces_only_where_no_device_table(lib):
    # 129 segments: scan, reduce, transform and for_each keep their piece table in
    # device memory (tested on the GPU); sort and the dot adjoint refuse it on the
    # host, before any device work
    lens = [4] * 129
    _, h = make_vec(lens)
    _, o = make_vec([sum(lens)], ptrs=[1 << 45])
    v = view_of(h)
    assert lib.dr_sort(v, o, None) == L.DR_E_UNSUPPORTED
    assert b"128" in L.lib().dr_last_error()


def test_missing_library_fails_loudly(tmp_path):
    # no CPU fallback: every entry point raises when the CUDA library is absent
    import subprocess
    import sys
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_2406_00158_gb300 import _lib as L\n"
        "L.LIB_PATH = %r\n"
        "from paper_2406_00158_gb300 import api\n"
        "try:\n"
        "    api.block_lengths(10, 3)\n"
        "except RuntimeError as e:\n"
        "    print('raised:', e)\n"
        "    sys.exit(0)\n"
        "sys.exit(1)\n" % (ROOT, str(tmp_path / "absent.so")))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "no CPU fallback" in r.stdout


def test_batch_plan_validation(lib):
    # every rejection happens on the host, before the plan uploads anything
    P = ctypes.c_void_p
    arr = lambda *v: (P * len(v))(*v)
    _, a = make_vec([100])
    _, b = make_vec([100], ptrs=[1 << 41])
    _, c = make_vec([100], ptrs=[1 << 42])
    _, d64 = make_vec([100], dtype=L.DR_F64, ptrs=[1 << 43])
    _, short = make_vec([99], ptrs=[1 << 44])
    dots = P(1 << 45)
    h = P()
    assert lib.dr_batch_plan(0, arr(a), arr(b), arr(c), dots, None, ctypes.byref(h)) == L.DR_E_INVAL
    assert lib.dr_batch_plan(1, arr(a), arr(b), arr(c), None, None, ctypes.byref(h)) == L.DR_E_INVAL
    assert lib.dr_batch_plan(1, arr(a), arr(b), arr(c), P((1 << 45) + 2), None, ctypes.byref(h)) == L.DR_E_ALIGN
    bad = L.dr_tune(100, 16, 3, 0)                          # 100 threads: not a supported shape
    assert lib.dr_batch_plan(1, arr(a), arr(b), arr(c), dots, ctypes.byref(bad), ctypes.byref(h)) == L.DR_E_INVAL
    assert lib.dr_batch_plan(1, arr(a), arr(d64), arr(c), dots, None, ctypes.byref(h)) == L.DR_E_DTYPE
    assert lib.dr_batch_plan(1, arr(a), arr(short), arr(c), dots, None, ctypes.byref(h)) == L.DR_E_INVAL
    assert lib.dr_batch_plan(2, arr(a, None), arr(b, b), arr(c, c), dots, None, ctypes.byref(h)) == L.DR_E_INVAL
    many = [2] * 129                                        # one vector spanning 129 pieces
    _, m = make_vec(many, ptrs=fake_ptrs(many, base=1 << 46))
    _, mp = make_vec(many, ptrs=fake_ptrs(many, base=1 << 47))
    _, my = make_vec([sum(many)], ptrs=[1 << 44])
    assert lib.dr_batch_plan(1, arr(m), arr(mp), arr(my), dots, None, ctypes.byref(h)) == L.DR_E_UNSUPPORTED
    assert not h.value


def test_stencil_validation(lib):
    # rejected on the host, before the halo exchange launches anything
    def md2(base, rows=(3, 4), cols=16):
        h = ctypes.c_void_p()
        r = (ctypes.c_int64 * len(rows))(*rows)
        p = (ctypes.c_void_p * len(rows))(*[base + (k << 28) for k in range(len(rows))])
        assert lib.dr_md2_create(L.DR_F32, sum(rows), cols, len(rows), r, p, ctypes.byref(h)) == 0
        return h
    a, b, t = md2(1 << 36), md2(1 << 37), md2(1 << 38)
    other = md2(1 << 39, rows=(4, 3))
    wide = md2(1 << 40, cols=32)
    S = lib.dr_stencil5
    assert S(None, b, t, 1, 0.0, 0.25, None) == L.DR_E_INVAL
    assert S(a, b, t, 0, 0.0, 0.25, None) == L.DR_E_INVAL          # steps >= 1
    assert S(a, b, None, 2, 0.0, 0.25, None) == L.DR_E_INVAL       # tmp needed for > 1 step
    assert S(a, other, t, 1, 0.0, 0.25, None) == L.DR_E_INVAL      # different blocking
    assert S(a, wide, t, 1, 0.0, 0.25, None) == L.DR_E_INVAL       # different shape
    assert S(a, a, t, 1, 0.0, 0.25, None) == L.DR_E_INVAL          # in == out
    alias = md2(1 << 36)                                            # same storage as a
    assert S(a, alias, t, 1, 0.0, 0.25, None) == L.DR_E_INVAL
    assert lib.dr_stencil5_T(a, b, None, 3, 0.0, 0.25, None) == L.DR_E_INVAL
    # one rank's share of a taller grid: one step per call, in and out agree on the flags
    P = lib.dr_stencil5_part
    assert P(a, b, 3, 0.0, 0.25, None) == L.DR_E_INVAL               # unknown row part
    assert lib.dr_md2_set_external_halos(None, 1, 0) == L.DR_E_INVAL
    assert lib.dr_md2_set_external_halos(a, 1, 1) == L.DR_OK
    assert S(a, b, t, 2, 0.0, 0.25, None) == L.DR_E_INVAL            # exchange needed between steps
    assert "one step per call" in L.last_error()
    assert P(a, b, L.DR_ROWS_INNER, 0.0, 0.25, None) == L.DR_E_INVAL  # out's flags differ
    assert "external halos" in L.last_error()
    for h in (a, b, t, other, wide, alias):
        lib.dr_md2_destroy(h)


def test_scan_with_carry_validation(lib):
    _, x = make_vec([100, 28])
    _, o = make_vec([128], ptrs=[1 << 41])
    v = view_of(x)
    F = lib.dr_scan_with_carry
    assert F(v, o, L.DR_PLUS, 0, None, None) == L.DR_E_INVAL          # a carry is required
    assert F(v, o, L.DR_PLUS, 0, ctypes.c_void_p((1 << 42) + 2), None) == L.DR_E_ALIGN
    assert F(v, o, L.DR_MUL, 0, ctypes.c_void_p(1 << 42), None) == L.DR_E_INVAL
    _, o64 = make_vec([128], dtype=L.DR_F64, ptrs=[1 << 43])
    assert F(v, o64, L.DR_PLUS, 1, ctypes.c_void_p(1 << 42), None) == L.DR_E_DTYPE
    _, e = make_vec([0])
    _, eo = make_vec([0], ptrs=[1 << 44])
    assert F(view_of(e), eo, L.DR_PLUS, 1, ctypes.c_void_p(1 << 42), None) == L.DR_OK   # empty: no launch


def test_scale_by_partner_validation(lib):
    _, x = make_vec([64])
    _, y = make_vec([64], ptrs=[1 << 41])
    _, gx = make_vec([64], ptrs=[1 << 42])
    _, g64 = make_vec([64], dtype=L.DR_F64, ptrs=[1 << 43])
    _, gs = make_vec([63], ptrs=[1 << 44])
    g = ctypes.c_void_p(1 << 45)
    F = lib.dr_scale_by_partner
    assert F(None, y, g, gx, None, None) == L.DR_E_INVAL
    assert F(x, y, None, gx, None, None) == L.DR_E_INVAL
    assert F(x, y, g, None, None, None) == L.DR_OK            # nothing requested: no launch
    assert F(x, y, g, g64, None, None) == L.DR_E_DTYPE
    assert F(x, y, g, gs, None, None) == L.DR_E_INVAL         # lengths differ
    many = [1] * 129
    _, mx = make_vec(many, ptrs=fake_ptrs(many, base=1 << 46))
    _, my = make_vec([129], ptrs=[1 << 47])
    _, mg = make_vec([129], ptrs=[1 << 40])
    assert F(mx, my, g, mg, None, None) == L.DR_E_UNSUPPORTED


def test_kernel_geometry_host_only(lib):
    """Tile sizes the error bounds are derived from: 32 KB scan tiles (8192 fp32,
    4096 int64), 12 KB tiles for the scan of a fused view, 16 KB reduce tiles
    with a fixed 4 CTAs per SM."""
    assert L.kernel_geometry(L.DR_K_SCAN, L.DR_F32) == (8192, 0)
    assert L.kernel_geometry(L.DR_K_SCAN, L.DR_I64) == (4096, 0)
    assert L.kernel_geometry(L.DR_K_SCAN, L.DR_I32) == (8192, 0)
    assert L.kernel_geometry(L.DR_K_SCAN_VIEW, L.DR_F32) == (3072, 0)
    assert L.kernel_geometry(L.DR_K_SCAN_VIEW, L.DR_I64) == (1536, 0)
    assert L.kernel_geometry(L.DR_K_REDUCE, L.DR_F32) == (4096, 4)
    assert L.kernel_geometry(L.DR_K_REDUCE, L.DR_F64) == (2048, 4)
    t, _ = L.kernel_geometry(L.DR_K_FOREACH, L.DR_F64)
    assert t > 0 and L.kernel_geometry(L.DR_K_SORT, L.DR_F32)[0] > 0
    tt = ctypes.c_int64()
    assert lib.dr_kernel_geometry(9, L.DR_F32, ctypes.byref(tt), None) == L.DR_E_INVAL
    assert lib.dr_kernel_geometry(L.DR_K_SCAN, 7, ctypes.byref(tt), None) == L.DR_E_DTYPE
    assert lib.dr_kernel_geometry(L.DR_K_SCAN, L.DR_F32, None, None) == L.DR_OK


def test_strict_align_zip(lib):
    """DR_ZIP_STRICT_ALIGN refuses non-aligned operands (Sec. 4.4 "Zip": the
    distributed-memory runtime prohibits them) and accepts aligned ones;
    without the flag the zip re-cuts them as usual."""
    def zip_ex(la, lb, flags, take=None):
        _, ha = make_vec(la)
        _, hb = make_vec(lb, ptrs=fake_ptrs(lb, base=1 << 40))
        va, vb = view_of(ha), view_of(hb)
        if take is not None:
            ta, tb = ctypes.c_void_p(), ctypes.c_void_p()
            assert lib.dr_view_take(va, take, ctypes.byref(ta)) == 0
            assert lib.dr_view_take(vb, take, ctypes.byref(tb)) == 0
            va, vb = ta, tb
        z = ctypes.c_void_p()
        rc = lib.dr_view_zip_ex(va, vb, flags, ctypes.byref(z))
        if rc == 0:
            lib.dr_view_destroy(z)
        return rc
    S = L.DR_ZIP_STRICT_ALIGN
    assert zip_ex([4, 4], [4, 4], S) == L.DR_OK
    assert zip_ex([4, 0, 4], [4, 4], S) == L.DR_OK            # empty segments are not counted
    assert zip_ex([4, 4], [3, 5], S) == L.DR_E_ALIGN
    assert "not aligned" in L.last_error()
    assert zip_ex([8], [4, 4], S) == L.DR_E_ALIGN
    assert zip_ex([4, 4], [3, 5], 0) == L.DR_OK               # re-cut without the flag
    assert zip_ex([4, 4], [4, 6], S, take=6) == L.DR_OK       # aligned over the taken windows
    assert zip_ex([4, 4], [4, 6], S) == L.DR_E_ALIGN          # but not over the whole vectors
    assert zip_ex([4, 4], [4, 4], 2) == L.DR_E_INVAL


def test_vec_rebind_validation(lib):
    lens = [8, 0, 5]
    _, h = make_vec(lens)
    P = lambda ptrs: (ctypes.c_void_p * 3)(*ptrs)
    assert lib.dr_vec_rebind(None, P([1 << 40, 0, 1 << 41])) == L.DR_E_INVAL
    assert lib.dr_vec_rebind(h, None) == L.DR_E_INVAL
    assert lib.dr_vec_rebind(h, P([0, 0, 1 << 41])) == L.DR_E_INVAL          # non-empty segment, NULL
    assert lib.dr_vec_rebind(h, P([(1 << 40) + 2, 0, 1 << 41])) == L.DR_E_ALIGN
    assert lib.dr_vec_rebind(h, P([1 << 40, 0, 1 << 41])) == L.DR_OK
    ptr = ctypes.c_void_p()
    assert lib.dr_vec_segment(h, 2, ctypes.byref(ptr), None, None) == 0 and ptr.value == 1 << 41
