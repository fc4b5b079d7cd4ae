"""Host backend of the row-partitioned solve for CPU tests: the local products
of a rank use the oracle's hierarchy (scipy sparse rows of its level matrices,
the dense coarse solve by Cholesky), so the partitioning, the halo plans, the
exchanges and the distributed PCG run on CPU ranks (gloo) exactly as they do
around the GPU kernels.  Test infrastructure only."""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import torch


class HostBackend:
    def __init__(self, H):
        self.H = H
        self.b = H.params.b
        self.nlev = H.nlev
        self.info = [H.info(k) for k in range(self.nlev)]
        self.mats, self.pat = {}, {}
        b = self.b
        for k in range(self.nlev - 1):
            for which in ("A", "G", "GT", "P", "R"):
                M = H.matrix(k, which)
                nnzb = M.nnzb
                self.pat[(k, which)] = (M.rowptr, M.col[:nnzb])
                self.mats[(k, which)] = sp.bsr_matrix(
                    (M.val[:nnzb], M.col[:nnzb], M.rowptr), shape=(b * M.nr, b * M.nc)).tocsr()
        AL = H.matrix(self.nlev - 1, "A")
        self.pat[(self.nlev - 1, "A")] = (AL.rowptr, AL.col[:AL.nnzb])
        self.mats[(self.nlev - 1, "A")] = sp.bsr_matrix(
            (AL.val[:AL.nnzb], AL.col[:AL.nnzb], AL.rowptr), shape=(b * AL.nr, b * AL.nc)).tocsr()
        self.chol = sla.cho_factor(AL.todense())

    def nr(self, k):
        return self.info[k]["nr"]

    def omega(self, k):
        return self.info[k]["omega"]

    def cf(self, k):
        return self.H.cf(k)

    def pattern(self, k, which):
        return self.pat[(k, which)]

    def vector(self, n):
        return torch.zeros(n, dtype=torch.float64)

    def index(self, idx):
        return torch.as_tensor(np.asarray(idx, np.int64))

    def comm_buffer(self, n):
        return torch.zeros(n, dtype=torch.float64)

    def apply(self, k, which, ep, r0, r1, x, y, aux=None, w=0.0):
        b = self.b
        M = self.mats[(k, which)][b * r0:b * r1]
        mx = torch.as_tensor(M @ x.numpy())
        sl = slice(b * r0, b * r1)
        if ep == 0:
            y[sl] = mx
        elif ep == 1:
            y[sl] = w * mx
        elif ep == 2:
            y[sl] = aux[sl] - mx
        elif ep == 3:
            y[sl] = aux[sl] + w * mx
        else:
            y[sl] += mx

    def coarse(self, y, z):
        z[:] = torch.as_tensor(sla.cho_solve(self.chol, y.numpy()))

    def dot(self, n0, n1, x, y):
        return torch.tensor([float(x[n0:n1] @ y[n0:n1])], dtype=torch.float64)

    def axpby(self, n0, n1, a, x, b, y):
        y[n0:n1] = a * x[n0:n1] + b * y[n0:n1]

    def pack(self, idx, x):
        return x[idx].clone()

    def unpack(self, idx, buf, x):
        x[idx] = buf

    def get_range(self, x, n0, n1):
        return x[n0:n1].clone()

    def set_range(self, x, n0, buf):
        x[n0:n0 + buf.numel()] = buf

    def sync(self):
        pass
