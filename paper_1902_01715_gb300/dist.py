"""Row-partitioned PCG with the V(1,1)-cycle over several processes (one GPU
each), for problems whose solve phase should be spread over GPUs.

Every rank builds the same hierarchy (the set-up is deterministic, so the
copies are bit-identical) and then owns a contiguous range of block rows of
every level: the fine ranges split the rows evenly, a coarser level's range
holds the coarse nodes whose fine nodes the rank owns (coarse nodes are
numbered in increasing fine index, so those are contiguous).  Vectors are
stored at full length on every rank, but a rank writes only its own rows.
Before each sparse product y = M x the rank receives the entries of x its
rows reference outside its own range (the halo) from their owners and sends
its own entries that other ranks reference: one exchange per product, point
to point.  Each inner product is the sum of the ranks' partial sums over their
own rows (one all-reduce of a scalar).  The last level is solved redundantly:
its right-hand side is gathered whole on every rank (one all-gather) and each
rank applies the coarse solve.

The local work goes through a backend: GpuBackend runs every product, vector
update and partial inner product as a kernel of the library (C ABI, FP64);
tests supply a host backend.  Communication uses torch.distributed (NCCL for
device tensors, gloo for host tensors).
"""
from __future__ import annotations

import numpy as np

# products of one level (the solve-phase matrices of Algorithm 2)
A_, G_, GT_, P_, R_ = "A", "G", "GT", "P", "R"
EP_SET, EP_SCALE, EP_RESID, EP_SADD, EP_ACC = 0, 1, 2, 3, 4


def row_ranges(n: int, world: int) -> list:
    """Contiguous, as even as possible, ranges [r0, r1) of n rows."""
    base, extra = divmod(n, world)
    out, r0 = [], 0
    for q in range(world):
        r1 = r0 + base + (1 if q < extra else 0)
        out.append((r0, r1))
        r0 = r1
    return out


def coarse_ranges(cf: np.ndarray, fine: list) -> list:
    """Coarse-node ranges induced by the fine ranges: rank q owns the coarse
    nodes of its fine nodes (coarse index = rank of the node among the C
    nodes in increasing fine index)."""
    csum = np.concatenate([[0], np.cumsum(np.asarray(cf) == 1)])
    return [(int(csum[r0]), int(csum[r1])) for r0, r1 in fine]


def owner_of(ranges: list) -> np.ndarray:
    """Rank that owns each row of a partition."""
    n = ranges[-1][1]
    own = np.empty(n, np.int64)
    for q, (r0, r1) in enumerate(ranges):
        own[r0:r1] = q
    return own


class Halo:
    """Exchange plan of one product y = M x: per peer, the block indices of x
    this rank receives (recv[q], owned by q, referenced by this rank's rows)
    and sends (send[q], owned here, referenced by q's rows).  Every rank
    holds the whole pattern, so both lists are formed locally."""

    def __init__(self, rowptr, col, row_parts: list, col_parts: list, me: int):
        rowptr = np.asarray(rowptr)
        col = np.asarray(col)
        own = owner_of(col_parts)
        world = len(row_parts)
        self.recv, self.send = {}, {}
        for q in range(world):
            if q == me:
                continue
            r0, r1 = row_parts[me]
            mine = np.unique(col[rowptr[r0]:rowptr[r1]])
            rv = mine[own[mine] == q] if len(mine) else mine
            q0, q1 = row_parts[q]
            theirs = np.unique(col[rowptr[q0]:rowptr[q1]])
            sd = theirs[own[theirs] == me] if len(theirs) else theirs
            if len(rv):
                self.recv[q] = rv.astype(np.int64)
            if len(sd):
                self.send[q] = sd.astype(np.int64)

    def volume(self) -> int:
        return sum(len(v) for v in self.recv.values())


class GpuBackend:
    """Local work of one rank on its GPU through the library (the handle of
    `solver`, FP64 V-cycle).  Exchange buffers live on the device for NCCL
    and are staged through host memory for gloo."""

    def __init__(self, solver, comm_device="cuda"):
        import ctypes as C

        import torch

        from . import _ptr, check, lib
        self.C, self.torch, self._ptr, self.check = C, torch, _ptr, check
        self.S, self.L = solver, lib()
        self.b = solver.b
        self.nlev = solver.nlev
        self._info = [solver.level_info(k) for k in range(self.nlev)]
        self.dev = torch.device("cuda")
        self.comm_device = torch.device(comm_device)
        self.stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    # hierarchy description
    def nr(self, k):
        return self._info[k]["nr"]

    def omega(self, k):
        return self._info[k]["omega"]

    def cf(self, k):
        return self.S.level_cf(k)

    def pattern(self, k, which):
        rp, col, _ = self.S.level_matrix(k, which)
        return rp, col

    # storage
    def vector(self, n):
        return self.torch.zeros(n, dtype=self.torch.float64, device=self.dev)

    def index(self, idx):
        return self.torch.as_tensor(np.asarray(idx, np.int64), device=self.dev)

    def comm_buffer(self, n):
        return self.torch.zeros(n, dtype=self.torch.float64, device=self.comm_device)

    # kernels
    def apply(self, k, which, ep, r0, r1, x, y, aux=None, w=0.0):
        code = {A_: 0, G_: 1, GT_: 2, P_: 3, R_: 4}[which]
        p = self._ptr
        self.check(self.L.amg_level_apply(self.S._h, k, code, ep, r0, r1, p(x), p(y), p(aux), w), "amg_level_apply")

    def coarse(self, y, z):
        self.check(self.L.amg_coarse_apply(self.S._h, self._ptr(y), self._ptr(z)), "amg_coarse_apply")

    def dot(self, n0, n1, x, y):
        out = self.torch.zeros(1, dtype=self.torch.float64, device=self.dev)
        self.check(self.L.amg_range_dot(n0, n1, self._ptr(x), self._ptr(y), self._ptr(out), self.stream),
                   "amg_range_dot")
        return out.to(self.comm_device)

    def axpby(self, n0, n1, a, x, b, y):
        self.check(self.L.amg_range_axpby(n0, n1, a, self._ptr(x), b, self._ptr(y), self.stream), "amg_range_axpby")

    def pack(self, idx, x):
        out = self.torch.empty(idx.numel(), dtype=self.torch.float64, device=self.dev)
        self.check(self.L.amg_gather(idx.numel(), self._ptr(idx), self._ptr(x), self._ptr(out), self.stream),
                   "amg_gather")
        return out.to(self.comm_device)

    def unpack(self, idx, buf, x):
        buf = buf.to(self.dev)
        self.check(self.L.amg_scatter(idx.numel(), self._ptr(idx), self._ptr(buf), self._ptr(x), self.stream),
                   "amg_scatter")

    def get_range(self, x, n0, n1):
        return x[n0:n1].to(self.comm_device)

    def set_range(self, x, n0, buf):
        x[n0:n0 + buf.numel()].copy_(buf.to(self.dev))

    def sync(self):
        self.torch.cuda.synchronize()


class DistSolver:
    """PCG with one V(1,1)-cycle per iteration (Algorithm 2, Sec. 4 stopping
    rule on the recurrence residual), row-partitioned over the ranks of a
    torch.distributed group."""

    def __init__(self, backend, group=None):
        import torch.distributed as td
        self.td, self.group, self.be = td, group, backend
        self.me = td.get_rank(group)
        self.world = td.get_world_size(group)
        be, b = backend, backend.b
        self.L = be.nlev - 1
        parts = [row_ranges(be.nr(0), self.world)]
        for k in range(self.L):
            parts.append(coarse_ranges(be.cf(k), parts[k]))
        self.parts = parts
        self.plans = {}
        keys = [(k, w) for k in range(self.L) for w in (A_, G_, GT_, P_, R_)]
        if self.L == 0:
            keys = [(0, A_)]
        for k, which in keys:
            rp, col = be.pattern(k, which)
            rows = parts[k + 1] if which == R_ else parts[k]
            cols = parts[k + 1] if which == P_ else parts[k]
            self.plans[(k, which)] = self._dof_plan(Halo(rp, col, rows, cols, self.me), b)
        self.halo_entries = sum(len(v[0]) for p in self.plans.values() for v in p[1].values())
        # level vectors (full length, own rows written)
        self.vec = []
        for k in range(be.nlev):
            n = b * be.nr(k)
            self.vec.append({name: be.vector(n) for name in ("y", "z", "s", "r", "t")})

    def _dof_plan(self, halo, b):
        def dofs(blocks):
            return (b * np.asarray(blocks)[:, None] + np.arange(b)[None, :]).reshape(-1)
        send = {q: (self.be.index(dofs(v)), None) for q, v in halo.send.items()}
        recv = {q: (self.be.index(dofs(v)), None) for q, v in halo.recv.items()}
        return send, recv

    def rows(self, k):
        return self.parts[k][self.me]

    # communication
    def exchange(self, x, key):
        send, recv = self.plans[key]
        if not send and not recv:
            return
        td = self.td
        ops, rbufs = [], []
        for q in sorted(send):
            ops.append(td.P2POp(td.isend, self.be.pack(send[q][0], x), q, self.group))
        for q in sorted(recv):
            buf = self.be.comm_buffer(recv[q][0].numel())
            ops.append(td.P2POp(td.irecv, buf, q, self.group))
            rbufs.append((q, buf))
        for req in td.batch_isend_irecv(ops):
            req.wait()
        for q, buf in rbufs:
            self.be.unpack(recv[q][0], buf, x)

    def allsum(self, t):
        self.td.all_reduce(t, group=self.group)
        return float(t.item())

    def dot(self, k, x, y):
        r0, r1 = self.rows(k)
        b = self.be.b
        return self.allsum(self.be.dot(b * r0, b * r1, x, y))

    def gather_full(self, k, x):
        """All-gather the owned slices of a level vector into x (every rank)."""
        b = self.be.b
        sizes = [b * (r1 - r0) for r0, r1 in self.parts[k]]
        mx = max(sizes)
        r0, r1 = self.rows(k)
        mine = self.be.comm_buffer(mx)
        mine[:b * (r1 - r0)].copy_(self.be.get_range(x, b * r0, b * r1))
        outs = [self.be.comm_buffer(mx) for _ in range(self.world)]
        self.td.all_gather(outs, mine, group=self.group)
        for q, (q0, q1) in enumerate(self.parts[k]):
            if q != self.me and q1 > q0:
                self.be.set_range(x, b * q0, outs[q][:b * (q1 - q0)])

    # V(1,1)-cycle of Algorithm 2 on this rank's rows
    def vcycle(self, k, y, z):
        be = self.be
        if k == self.L:
            self.gather_full(k, y)
            be.coarse(y, z)
            return
        V, C = self.vec[k], self.vec[k + 1]
        f0, f1 = self.rows(k)
        c0, c1 = self.rows(k + 1)
        w = be.omega(k)
        s, r, t = V["s"], V["r"], V["t"]
        self.exchange(y, (k, G_))
        be.apply(k, G_, EP_SET, f0, f1, y, t)                 # t = G y
        self.exchange(t, (k, GT_))
        be.apply(k, GT_, EP_SCALE, f0, f1, t, s, None, w)     # s = w G^T t
        self.exchange(s, (k, A_))
        be.apply(k, A_, EP_RESID, f0, f1, s, r, y)            # r = y - A s
        self.exchange(r, (k, R_))
        be.apply(k, R_, EP_SET, c0, c1, r, C["y"])            # y_c = P^T r
        self.vcycle(k + 1, C["y"], C["z"])
        self.exchange(C["z"], (k, P_))
        be.apply(k, P_, EP_ACC, f0, f1, C["z"], s)            # s += P z_c
        self.exchange(s, (k, A_))
        be.apply(k, A_, EP_RESID, f0, f1, s, r, y)            # r = y - A s
        self.exchange(r, (k, G_))
        be.apply(k, G_, EP_SET, f0, f1, r, t)                 # t = G r
        self.exchange(t, (k, GT_))
        be.apply(k, GT_, EP_SADD, f0, f1, t, z, s, w)         # z = s + w G^T t

    def solve(self, bvec, rtol=1e-8, maxit=1000):
        """x with K x = b (b: full-length level-0 vector, own rows read);
        returns (x with own rows, iterations, ||r|| / ||b||).  Every rank
        takes the same decisions (the scalars are all-reduced)."""
        be, b = self.be, self.be.b
        n0, n1 = (b * v for v in self.rows(0))
        n = b * be.nr(0)
        x, r, z, p, q = (be.vector(n) for _ in range(5))
        be.axpby(n0, n1, 1.0, bvec, 0.0, r)
        bn2 = self.dot(0, r, r)
        if bn2 == 0.0:
            return x, 0, 0.0
        self.vcycle(0, r, z)
        be.axpby(n0, n1, 1.0, z, 0.0, p)
        rz = self.dot(0, r, z)
        rr, it = bn2, 0
        while it < maxit:
            self.exchange(p, (0, A_))
            be.apply(0, A_, EP_SET, self.rows(0)[0], self.rows(0)[1], p, q)
            pq = self.dot(0, p, q)
            if not pq > 0.0:
                raise RuntimeError("PCG breakdown: p^T K p = %g" % pq)
            alpha = rz / pq
            be.axpby(n0, n1, alpha, p, 1.0, x)
            be.axpby(n0, n1, -alpha, q, 1.0, r)
            it += 1
            rr = self.dot(0, r, r)
            if rr <= rtol * rtol * bn2:
                break
            self.vcycle(0, r, z)
            rz2 = self.dot(0, r, z)
            beta = rz2 / rz
            rz = rz2
            be.axpby(n0, n1, 1.0, z, beta, p)
        return x, it, (rr / bn2) ** 0.5
