"""One segmented range sharded over several GPUs, one process per GPU.

In the paper's model every segment lives in a memory locale and has a rank
(Sec. 3); the distributed-memory runtime runs each algorithm SPMD, every
process working on the segments it owns (Sec. 4.3).  Here a rank's segments
sit in its GPU's HBM and every algorithm is the library's local kernels plus
the one exchange step the algorithm has:

* dot / reduce (Algorithm 3): one local transform_reduce over the owned
  segments; an all-gather of the N per-rank partials; every rank folds them in
  rank order with the library's reduce (the paper combines with MPI_Reduce).
* inclusive / exclusive scan (Algorithm 4): the owned segments form runs of
  consecutive segments; each run's total comes from a local reduce; an
  all-gather of the run totals (the paper gathers the segments' last elements
  on rank 0); each run's carry is the fold of the totals of the runs before it
  (the library's reduce over a zero-copy view of the gathered buffer); the
  local scan starts from that carry (dr_scan_with_carry).  Reads 12 B and
  writes 4 B per fp32 element, against the 16 B + 4 B of a local scan plus an
  offset pass.
* stencil for_each over a block_row array (Sec. 4.2.2): before each step the
  boundary rows go point-to-point into the neighbouring ranks' ghost rows,
  while the row blocks that do not read those ghost rows are updated.
* batched vectors: whole vectors are assigned to ranks; nothing is exchanged.

Collectives are torch.distributed calls (NCCL between GPUs, gloo between CPU
ranks in the tests); the local steps go through a backend object (the CUDA
library here; a CPU stand-in in the tests), so this module holds only the
placement and exchange logic.  With one rank no collective is issued.
"""
from __future__ import annotations

from typing import Optional, Sequence

import torch

# ---------------------------------------------------------------------------
# placement (host logic)
# ---------------------------------------------------------------------------


def block_owners(nitems: int, world: int) -> list[int]:
    """Items (segments, row blocks) 0..nitems-1 over `world` ranks in contiguous
    groups whose sizes differ by at most one: item k goes to rank k*world//nitems
    (rank k for nitems == world, the paper's one segment per locale)."""
    return [k * world // nitems for k in range(nitems)]


def runs(owners: Sequence[int], rank: int) -> list[tuple[int, int]]:
    """Maximal runs [a, b) of consecutive items owned by `rank`."""
    out, k = [], 0
    n = len(owners)
    while k < n:
        if owners[k] != rank:
            k += 1
            continue
        a = k
        while k < n and owners[k] == rank:
            k += 1
        out.append((a, k))
    return out


def run_heads(owners: Sequence[int]) -> list[tuple[int, int, int]]:
    """Every rank's runs in global order: (first item, owner, index of the run
    among the owner's runs)."""
    heads, count = [], {}
    k, n = 0, len(owners)
    while k < n:
        r = owners[k]
        heads.append((k, r, count.get(r, 0)))
        count[r] = count.get(r, 0) + 1
        while k < n and owners[k] == r:
            k += 1
    return heads


def balanced_owners(lengths: Sequence[int], world: int) -> list[int]:
    """Independent vectors over ranks: contiguous groups with about equal element
    totals (vector v goes to the rank whose share of the running total holds the
    vector's first element)."""
    total = sum(int(n) for n in lengths)
    out, s = [], 0
    for n in lengths:
        out.append(min(world - 1, (s * world) // total) if total else 0)
        s += int(n)
    return out


# ---------------------------------------------------------------------------
# communication
# ---------------------------------------------------------------------------


class TorchComm:
    """Collectives of one process group (torch.distributed): NCCL between GPUs,
    gloo between CPU processes."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.nccl = dist.get_backend(group) == "nccl"

    def all_gather(self, t: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """The ranks' tensors (equal sizes) concatenated in rank order (into `out`
        if given)."""
        if out is None:
            out = torch.empty(self.world * t.numel(), dtype=t.dtype, device=t.device)
        if self.nccl:
            self.dist.all_gather_into_tensor(out, t, group=self.group)
        else:
            parts = list(out.split(t.numel()))
            self.dist.all_gather(parts, t, group=self.group)
        return out

    def start_exchange(self, sends, recvs):
        """Posts point-to-point sends [(peer, tensor, tag)] and receives; returns
        the handles.  Both sides post in the same (global boundary) order."""
        if not sends and not recvs:
            return []
        if self.nccl:
            P2POp = self.dist.P2POp
            ops = [P2POp(self.dist.isend, t, peer, self.group, tag) for peer, t, tag in sends]
            ops += [P2POp(self.dist.irecv, t, peer, self.group, tag) for peer, t, tag in recvs]
            return self.dist.batch_isend_irecv(ops)
        reqs = [self.dist.isend(t, peer, group=self.group, tag=tag) for peer, t, tag in sends]
        reqs += [self.dist.irecv(t, peer, group=self.group, tag=tag) for peer, t, tag in recvs]
        return reqs

    @staticmethod
    def finish_exchange(reqs) -> None:
        """Waits for posted transfers (with NCCL: orders them before later work on
        the current stream, without a host synchronization)."""
        for r in reqs:
            r.wait()


class LocalComm:
    """The one-rank case: nothing to exchange."""
    rank, world = 0, 1

    def all_gather(self, t, out=None):
        if out is None:
            return t
        out.copy_(t)
        return out

    def start_exchange(self, sends, recvs):
        assert not sends and not recvs
        return []

    @staticmethod
    def finish_exchange(reqs) -> None:
        pass


# ---------------------------------------------------------------------------
# the local backend: the CUDA library
# ---------------------------------------------------------------------------


class CudaBackend:
    """Local steps as library calls on the current CUDA stream.  Views (and so
    their device workspaces) are created once per vector and reused by later
    calls."""

    def __init__(self):
        from . import api
        self.api = api
        self._folds = {}

    def vector(self, tensors):
        return self.api.SegmentedVector(list(tensors))

    def _view(self, v):
        w = getattr(v, "_shard_view", None)
        if w is None:
            w = v._shard_view = v.view()
        return w

    @staticmethod
    def default_device():
        return torch.device("cuda", torch.cuda.current_device())

    def scratch(self, k: int, dtype, device):
        return torch.empty(k, dtype=dtype, device=device)

    def reduce(self, v, op: str, out1: torch.Tensor) -> None:
        self.api.transform_reduce(self._view(v), out1, op=op, init=_identity(op, out1.dtype))

    def dot(self, x, y, out1: torch.Tensor) -> None:
        views = getattr(x, "_shard_dot", None)
        if views is None:
            views = x._shard_dot = {}
        key = id(y)
        if key not in views:
            views[key] = (y, self.api.dot_view(x, y))
        self.api.transform_reduce(views[key][1], out1)

    def fold(self, parts: Sequence[torch.Tensor], op: str, out1: torch.Tensor) -> None:
        """out1 = the fold of the one-element tensors `parts` in order (the
        identity if none): the library's reduce over a vector whose segments are
        those elements, wherever they live (no gather copy)."""
        segs = list(parts) if parts else [out1[:0]]
        key = tuple(t.data_ptr() for t in segs) + (len(segs), str(out1.dtype))
        v = self._folds.get(key)
        if v is None:
            if len(self._folds) > 256:
                self._folds.clear()
            v = self._folds[key] = self.api.SegmentedVector(segs)
        self.reduce(v, op, out1)

    def scan(self, x, out, op: str, carry1: Optional[torch.Tensor], exclusive: bool) -> None:
        if carry1 is None:
            self.api.inclusive_scan(self._view(x), out, op=op)
        else:
            self.api.scan_with_carry(self._view(x), out, carry1, op=op, exclusive=exclusive)

    def md(self, blocks, top: bool, bottom: bool):
        m = self.api.MdArray(list(blocks))
        m.set_external_halos(top, bottom)
        return m

    def stencil_part(self, a, b, part: str, wc: float, wn: float) -> None:
        self.api.stencil5_part(a, b, part, wc, wn)


def _identity(op: str, dtype):
    if op == "plus":
        return 0
    fl = dtype.is_floating_point
    if op == "min":
        return float("inf") if fl else torch.iinfo(dtype).max
    if op == "max":
        return float("-inf") if fl else torch.iinfo(dtype).min
    raise ValueError(op)


# ---------------------------------------------------------------------------
# sharded containers and algorithms
# ---------------------------------------------------------------------------


class ShardedVector:
    """This rank's share of a distributed vector: global segment sizes `lens`,
    segment k owned by rank owners[k]; `local` holds the owned segments' device
    tensors in segment order."""

    def __init__(self, comm, lens: Sequence[int], owners: Sequence[int], local: Sequence[torch.Tensor],
                 backend=None, dtype=None, device=None):
        self.comm = comm
        self.backend = backend or CudaBackend()
        self.lens = [int(n) for n in lens]
        self.owners = list(owners)
        assert len(self.owners) == len(self.lens)
        self.mine = [k for k, r in enumerate(self.owners) if r == comm.rank]
        local = list(local)
        assert len(local) == len(self.mine), "one local tensor per owned segment"
        for k, t in zip(self.mine, local):
            assert t.numel() == self.lens[k], (k, t.numel(), self.lens[k])
        self.seg = dict(zip(self.mine, local))
        self.runs = runs(self.owners, comm.rank)
        # a rank may own no segment: its element type and device are then given
        self.dtype = local[0].dtype if local else (dtype or torch.float32)
        self.device = local[0].device if local else (device or self.backend.default_device())
        self._all = None
        self._run_vecs = None
        self._scratch = {}

    def scratch(self, name: str, k: int, dtype=None) -> torch.Tensor:
        """A device buffer kept by this vector between calls (partials, gathered
        totals, carries)."""
        dtype = dtype or self.dtype
        t = self._scratch.get(name)
        if t is None or t.numel() != k or t.dtype != dtype:
            t = self._scratch[name] = self.backend.scratch(k, dtype, self.device)
        return t

    @classmethod
    def empty_like(cls, other: "ShardedVector", dtype=None) -> "ShardedVector":
        dtype = dtype or other.dtype
        local = [torch.empty(other.lens[k], dtype=dtype, device=other.device) for k in other.mine]
        return cls(other.comm, other.lens, other.owners, local, other.backend, dtype, other.device)

    def aligned_with(self, other: "ShardedVector") -> bool:
        """Same segment count, sizes and ranks (Sec. 4.4's alignment)."""
        return self.lens == other.lens and self.owners == other.owners

    def all_local(self):
        """The owned segments as one local vector (for order-free reductions)."""
        if self._all is None and self.mine:
            self._all = self.backend.vector([self.seg[k] for k in self.mine])
        return self._all

    def run_vectors(self):
        """One local vector per run of consecutive owned segments."""
        if self._run_vecs is None:
            self._run_vecs = [self.backend.vector([self.seg[k] for k in range(a, b)]) for a, b in self.runs]
        return self._run_vecs

    def local_offset(self, k: int) -> int:
        """Global index of the first element of segment k."""
        return sum(self.lens[:k])


def _check_same(x: ShardedVector, y: ShardedVector, who: str) -> None:
    if not x.aligned_with(y):
        raise ValueError(f"{who}: operands are not aligned (segment sizes or owners differ); the "
                         "distributed runtime prohibits zips of non-aligned ranges (Sec. 4.4)")


def dot(x: ShardedVector, y: ShardedVector, out1: torch.Tensor) -> torch.Tensor:
    """out1 = <x, y> on every rank (Algorithm 1 over Algorithm 3): local
    transform_reduce over the owned segments, all-gather of the partials, fold
    in rank order."""
    _check_same(x, y, "dot")
    comm, be = x.comm, x.backend
    if comm.world == 1:
        be.dot(x.all_local(), y.all_local(), out1)
        return out1
    part = x.scratch("part", 1, out1.dtype)
    if x.mine:
        be.dot(x.all_local(), y.all_local(), part)
    else:
        be.fold([], "plus", part)                 # a rank with no segments contributes 0
    gathered = comm.all_gather(part, x.scratch("gathered", comm.world, out1.dtype))
    be.fold([gathered[r:r + 1] for r in range(comm.world)], "plus", out1)
    return out1


def reduce(x: ShardedVector, out1: torch.Tensor, op: str = "plus") -> torch.Tensor:
    """out1 = the fold of the whole range with op, on every rank (Algorithm 3)."""
    comm, be = x.comm, x.backend
    if comm.world == 1:
        be.reduce(x.all_local(), op, out1)
        return out1
    part = x.scratch("part", 1, out1.dtype)
    if x.mine:
        be.reduce(x.all_local(), op, part)
    else:
        be.fold([], op, part)
    gathered = comm.all_gather(part, x.scratch("gathered", comm.world, out1.dtype))
    be.fold([gathered[r:r + 1] for r in range(comm.world)], op, out1)
    return out1


def scan(x: ShardedVector, out: ShardedVector, op: str = "plus", exclusive: bool = False,
         init=None) -> ShardedVector:
    """inclusive (or exclusive, with init) scan of the whole sharded range into
    `out` (aligned with x), following Algorithm 4: run totals, their exchange,
    carries, local scans that start from the carries."""
    _check_same(x, out, "scan")
    comm, be = x.comm, x.backend
    if comm.world == 1 and len(x.runs) == 1 and init is None and not exclusive:
        # one rank, one run: no carry (the plain local scan)
        be.scan(x.run_vectors()[0], out.run_vectors()[0], op, None, False)
        return out
    heads = run_heads(x.owners)
    rmax = max((i for _, r, i in heads), default=-1) + 1       # most runs of any rank
    dtype, dev = x.dtype, x.device
    totals = x.scratch("totals", max(rmax, 1))
    for i, v in enumerate(x.run_vectors()):
        be.reduce(v, op, totals[i:i + 1])
    gathered = comm.all_gather(totals, x.scratch("gathered_totals", comm.world * max(rmax, 1)))
    first = []
    if init is not None:
        first = [torch.tensor([init], dtype=dtype, device=dev)]    # a copy of the host value
    carries = x.scratch("carries", max(len(x.runs), 1))
    my = [a for a, r, _ in heads if r == comm.rank]
    for j, a in enumerate(my):
        # the carry of the run starting at segment a: init, then the totals of every
        # earlier run in global order
        parts = first + [gathered[r * rmax + i:r * rmax + i + 1] for h, r, i in heads if h < a]
        be.fold(parts, op, carries[j:j + 1])
        be.scan(x.run_vectors()[j], out.run_vectors()[j], op, carries[j:j + 1], exclusive)
    return out


# ---------------------------------------------------------------------------
# the stencil over a row-block array sharded by rows
# ---------------------------------------------------------------------------


class ShardedMdArray:
    """This rank's share of a row-block array: global block heights `seg_rows`,
    block k owned by rank owners[k]; `local` holds the owned blocks' device
    tensors ((rows_k + 2) x cols, ghost rows included) in block order."""

    def __init__(self, comm, seg_rows: Sequence[int], cols: int, owners: Sequence[int],
                 local: Sequence[torch.Tensor], backend=None):
        self.comm = comm
        self.backend = backend or CudaBackend()
        self.seg_rows = [int(r) for r in seg_rows]
        self.cols = int(cols)
        self.owners = list(owners)
        self.mine = [k for k, r in enumerate(self.owners) if r == comm.rank]
        local = list(local)
        assert len(local) == len(self.mine)
        self.blk = dict(zip(self.mine, local))
        self.runs = runs(self.owners, comm.rank)
        nb = len(self.seg_rows)
        # one local array per run; its outer ghost rows are external where the run
        # borders another rank's block
        self.mds = [self.backend.md([self.blk[k] for k in range(a, b)], a > 0, b < nb) for a, b in self.runs]

    @classmethod
    def empty_like(cls, other: "ShardedMdArray") -> "ShardedMdArray":
        local = [torch.zeros_like(other.blk[k]) for k in other.mine]
        return cls(other.comm, other.seg_rows, other.cols, other.owners, local, other.backend)

    def halo_plan(self):
        """Sends and receives of one exchange, in global boundary order: across
        every boundary between blocks b and b + 1 of different owners, block b's
        last own row goes to block b + 1's top ghost row and block b + 1's first
        own row to block b's bottom ghost row."""
        me = self.comm.rank
        sends, recvs = [], []
        for b in range(len(self.seg_rows) - 1):
            lo, hi = self.owners[b], self.owners[b + 1]
            if lo == hi:
                continue
            tag_dn, tag_up = 2 * b, 2 * b + 1
            if lo == me:
                t = self.blk[b]
                sends.append((hi, t[self.seg_rows[b]], tag_dn))           # last own row
                recvs.append((hi, t[self.seg_rows[b] + 1], tag_up))       # bottom ghost row
            if hi == me:
                t = self.blk[b + 1]
                sends.append((lo, t[1], tag_up))                          # first own row
                recvs.append((lo, t[0], tag_dn))                          # top ghost row
        return sends, recvs


def stencil5(a: ShardedMdArray, b: ShardedMdArray, steps: int, wc: float = 0.0,
             wn: float = 0.25) -> ShardedMdArray:
    """`steps` 5-point Jacobi steps of the whole sharded grid (zero outside it),
    ping-ponging between a and b; returns the array holding the result.  Each
    step: post the boundary-row exchange, update the inner row blocks, wait for
    the exchange, update the outer row blocks."""
    comm, be = a.comm, a.backend
    src, dst = a, b
    for _ in range(int(steps)):
        sends, recvs = src.halo_plan()
        reqs = comm.start_exchange(sends, recvs)
        for ms, md in zip(src.mds, dst.mds):
            be.stencil_part(ms, md, "inner", wc, wn)
        comm.finish_exchange(reqs)
        for ms, md in zip(src.mds, dst.mds):
            be.stencil_part(ms, md, "outer", wc, wn)
        src, dst = dst, src
    return src
