"""Python access to the FP64 CPU oracle (test infrastructure only).

The oracle is plain C (``oracle/*.c``), compiled with ``-ffp-contract=off`` into
``oracle/_build/liboracle.so`` and loaded with ctypes.  Only the tests, the
smoke check and the CPU-baseline leg of ``bench.py`` may use it; the CUDA
library never does.

Block matrices travel as ``(rowptr, col, val)`` triples of numpy arrays with
``val`` shaped ``(nnzb, b, b)``; test spaces as ``(n, t)`` arrays (stored
column-major on the C side).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["o_util.c", "o_fe.c", "o_fsai.c", "o_srqcg.c", "o_coarsen.c",
            "o_dpls.c", "o_rap.c", "o_amg.c"]
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_NOT_SPD, ERR_BREAKDOWN, ERR_NOT_CONVERGED, ERR_MEM, ERR_COARSENING = (
    0, -1, -2, -3, -4, -5, -6)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no contraction, OpenMP row loops);
    returns the .so path."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES] + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(_LIB):
        if os.path.getmtime(_LIB) >= max(os.path.getmtime(s) for s in srcs):
            return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp] + [os.path.join(_HERE, s) for s in _SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class OBSR(C.Structure):
    _fields_ = [("nr", C.c_int), ("nc", C.c_int), ("b", C.c_int),
                ("rowptr", C.POINTER(C.c_int)), ("col", C.POINTER(C.c_int)),
                ("val", C.POINTER(C.c_double))]


class Params(C.Structure):
    _fields_ = [("b", C.c_int), ("k_g", C.c_int), ("rho_g", C.c_int), ("eps_g", C.c_double),
                ("k_i", C.c_int), ("rho_i", C.c_int), ("eps_i", C.c_double),
                ("omega_bar", C.c_double), ("rho_bar", C.c_double), ("max_refine", C.c_int),
                ("max_g_nodes", C.c_int), ("lanczos_m", C.c_int), ("omega_safety", C.c_double),
                ("n_tv", C.c_int), ("n_rq", C.c_int), ("k_ritz", C.c_int), ("theta", C.c_int),
                ("n_max", C.c_int), ("d_p", C.c_int), ("kappa_p", C.c_double),
                ("n_coarse", C.c_int), ("max_levels", C.c_int),
                ("max_coarse_ratio", C.c_double), ("seed", C.c_uint64)]


_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_up = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.POINTER(OBSR)
            sig = {
                "or_default_params": (None, [C.POINTER(Params), C.c_int]),
                "or_splitmix64": (C.c_uint64, [C.c_uint64, C.c_uint64]),
                "or_uniform_pm1": (C.c_double, [C.c_uint64, C.c_uint64]),
                "or_dot": (C.c_double, [C.c_int, _dp, _dp]),
                "or_spmv": (None, [P, _dp, _dp]),
                "or_transpose": (C.c_int, [P, P]),
                "or_bsr_free": (None, [P]),
                "or_chol": (C.c_int, [C.c_int, _dp, _dp]),
                "or_chol_solve": (None, [C.c_int, _dp, _dp, _dp]),
                "or_ke0": (C.c_int, [C.c_double] * 4 + [_dp]),
                "or_assemble": (C.c_int, [C.c_int] * 3 + [C.c_double] * 4 + [_dp, C.c_int, P, _ip]),
                "or_rbm": (C.c_int, [C.c_int] * 3 + [C.c_double] * 3 + [_ip, C.c_int, _dp]),
                "or_load_body": (C.c_int, [C.c_int] * 3 + [C.c_double] * 3 + [_dp, _ip, _dp]),
                "or_load_top_pressure": (C.c_int, [C.c_int] * 3 + [C.c_double] * 3 + [_dp, _ip, _dp]),
                "or_load_end_shear": (C.c_int, [C.c_int] * 3 + [C.c_double] * 4 + [_ip, _dp]),
                "or_afsai": (C.c_int, [P, P, C.c_int, C.c_int, C.c_double, C.c_int, P]),
                "or_lanczos_lmax": (C.c_double, [P, P, P, C.c_int, C.c_uint64, C.c_int]),
                "or_smoother_setup": (C.c_int, [P, C.POINTER(Params), C.c_int, P, P,
                                                C.POINTER(C.c_double), C.POINTER(C.c_double),
                                                C.POINTER(C.c_int)]),
                "or_srqcg": (C.c_int, [P, P, P, C.c_int, C.c_int, C.c_int, _dp, _dp]),
                "or_gen_eig": (C.c_int, [C.c_int, _dp, _dp, _dp, _dp]),
                "or_mgs": (None, [C.c_int, C.c_int, _dp]),
                "or_rq_line_min": (C.c_double, [C.c_double] * 6),
                "or_soc": (C.c_int, [P, C.c_int, _dp, _dp]),
                "or_filter": (C.c_int, [P, _dp, C.c_int, _up, _up]),
                "or_mis": (C.c_int, [P, _up, _ip]),
                "or_dpls": (C.c_int, [P, _up, _ip, C.c_int, _dp, C.c_int, C.c_int, C.c_double, P]),
                "or_rap": (C.c_int, [P, P, P]),
                "or_setup": (C.c_int, [C.POINTER(Params), P, C.c_int, _dp, C.POINTER(C.c_void_p)]),
                "or_free": (None, [C.c_void_p]),
                "or_vcycle": (C.c_int, [C.c_void_p, _dp, _dp]),
                "or_pcg": (C.c_int, [C.c_void_p, _dp, _dp, C.c_double, C.c_int,
                                     C.POINTER(C.c_int), C.POINTER(C.c_double)]),
                "or_h_nlev": (C.c_int, [C.c_void_p]),
                "or_h_level_info": (None, [C.c_void_p, C.c_int, _ip, C.POINTER(C.c_double),
                                           C.POINTER(C.c_double)]),
                "or_h_bsr_size": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int),
                                            C.POINTER(C.c_int), C.POINTER(C.c_int)]),
                "or_h_bsr_copy": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _ip, _ip, _dp]),
                "or_h_cf": (C.c_int, [C.c_void_p, C.c_int, _ip]),
                "or_h_V": (C.c_int, [C.c_void_p, C.c_int, _dp]),
                "or_h_coarse_factor": (C.c_int, [C.c_void_p, _dp]),
                "or_bsr_to_scalar": (C.c_int, [P, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


# ---------------------------------------------------------------- helpers

class Bsr:
    """A block matrix held in numpy arrays, viewable as an OBSR for C calls."""

    def __init__(self, rowptr, col, val, nc=None):
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        val = np.asarray(val, dtype=np.float64)
        self.b = int(val.shape[1]) if val.ndim == 3 else 1
        self.val = np.ascontiguousarray(val.reshape(-1, self.b, self.b))
        self.nr = len(self.rowptr) - 1
        self.nc = int(nc) if nc is not None else self.nr
        if len(self.col) == 0:
            self.col = np.zeros(1, np.int32)
            self.val = np.zeros((1, self.b, self.b))
            self._empty = True
        else:
            self._empty = False

    @property
    def nnzb(self):
        return int(self.rowptr[-1])

    def c(self) -> OBSR:
        s = OBSR()
        s.nr, s.nc, s.b = self.nr, self.nc, self.b
        s.rowptr = self.rowptr.ctypes.data_as(C.POINTER(C.c_int))
        s.col = self.col.ctypes.data_as(C.POINTER(C.c_int))
        s.val = self.val.ctypes.data_as(C.POINTER(C.c_double))
        return s

    def todense(self) -> np.ndarray:
        b = self.b
        D = np.zeros((self.nr * b, self.nc * b))
        for i in range(self.nr):
            for k in range(self.rowptr[i], self.rowptr[i + 1]):
                j = self.col[k]
                D[i * b:(i + 1) * b, j * b:(j + 1) * b] += self.val[k]
        return D

    def matvec(self, x: np.ndarray) -> np.ndarray:
        y = np.zeros(self.nr * self.b)
        lib().or_spmv(C.byref(self.c()), np.ascontiguousarray(x, dtype=np.float64), y)
        return y


def _take(s: OBSR) -> Bsr:
    """Copy a C-allocated OBSR into numpy and free the C storage."""
    nnzb = s.rowptr[s.nr]
    rowptr = np.ctypeslib.as_array(s.rowptr, shape=(s.nr + 1,)).copy()
    col = np.ctypeslib.as_array(s.col, shape=(max(nnzb, 1),)).copy()[:nnzb]
    val = np.ctypeslib.as_array(s.val, shape=(max(nnzb, 1) * s.b * s.b,)).copy()
    val = val[: nnzb * s.b * s.b].reshape(nnzb, s.b, s.b)
    out = Bsr(rowptr, col, val, nc=s.nc)
    lib().or_bsr_free(C.byref(s))
    return out


def default_params(b: int = 3, **over) -> Params:
    p = Params()
    lib().or_default_params(C.byref(p), b)
    for k, v in over.items():
        setattr(p, k, v)
    return p


# ---------------------------------------------------------------- FE

def ke0(nu, hx, hy, hz):
    K = np.zeros(576)
    rc = lib().or_ke0(nu, hx, hy, hz, K)
    assert rc == 0, rc
    return K.reshape(24, 24)


def assemble(nx, ny, nz, hx, hy, hz, nu, E, clamp_axis):
    E = np.ascontiguousarray(E, dtype=np.float64)
    assert E.size == nx * ny * nz
    node_map = np.zeros((nx + 1) * (ny + 1) * (nz + 1), np.int32)
    s = OBSR()
    rc = lib().or_assemble(nx, ny, nz, hx, hy, hz, nu, E, clamp_axis, C.byref(s), node_map)
    assert rc == 0, rc
    return _take(s), node_map


def rbm(nx, ny, nz, hx, hy, hz, node_map):
    nfree = int((node_map >= 0).sum())
    V = np.zeros(3 * nfree * 6)
    lib().or_rbm(nx, ny, nz, hx, hy, hz, node_map, nfree, V)
    return V.reshape(6, 3 * nfree).T.copy()


def load_body(nx, ny, nz, hx, hy, hz, g, node_map, f=None):
    nfree = int((node_map >= 0).sum())
    f = np.zeros(3 * nfree) if f is None else f
    lib().or_load_body(nx, ny, nz, hx, hy, hz, np.asarray(g, np.float64), node_map, f)
    return f


def load_top_pressure(nx, ny, nz, hx, hy, hz, p, node_map, f=None):
    nfree = int((node_map >= 0).sum())
    f = np.zeros(3 * nfree) if f is None else f
    lib().or_load_top_pressure(nx, ny, nz, hx, hy, hz,
                               np.ascontiguousarray(p, np.float64), node_map, f)
    return f


def load_end_shear(nx, ny, nz, hx, hy, hz, total, node_map, f=None):
    nfree = int((node_map >= 0).sum())
    f = np.zeros(3 * nfree) if f is None else f
    lib().or_load_end_shear(nx, ny, nz, hx, hy, hz, total, node_map, f)
    return f


# ---------------------------------------------------------------- pieces

def dot(x, y):
    return lib().or_dot(len(x), np.ascontiguousarray(x, np.float64), np.ascontiguousarray(y, np.float64))


def uniform_pm1(seed, counters):
    L = lib()
    return np.array([L.or_uniform_pm1(seed, int(c)) for c in counters])


def splitmix64(seed, counter):
    return lib().or_splitmix64(seed, counter)


def transpose(A: Bsr) -> Bsr:
    s = OBSR()
    lib().or_transpose(C.byref(A.c()), C.byref(s))
    return _take(s)


def to_scalar(A: Bsr) -> Bsr:
    s = OBSR()
    lib().or_bsr_to_scalar(C.byref(A.c()), C.byref(s))
    return _take(s)


def chol(M):
    M = np.ascontiguousarray(M, np.float64)
    m = M.shape[0]
    L = np.zeros_like(M)
    rc = lib().or_chol(m, M, L)
    return rc, L


def chol_solve(L, rhs):
    m = L.shape[0]
    x = np.zeros(m)
    lib().or_chol_solve(m, np.ascontiguousarray(L), np.ascontiguousarray(rhs, np.float64), x)
    return x


def afsai(A: Bsr, Gs: Bsr | None, k, rho, eps, max_nodes=24) -> Bsr:
    s = OBSR()
    gs = C.byref(Gs.c()) if Gs is not None else None
    rc = lib().or_afsai(C.byref(A.c()), gs, k, rho, eps, max_nodes, C.byref(s))
    assert rc == 0, rc
    return _take(s)


def lanczos_lmax(A: Bsr, G: Bsr, GT: Bsr, m=20, seed=20190205, level=0):
    return lib().or_lanczos_lmax(C.byref(A.c()), C.byref(G.c()), C.byref(GT.c()), m, seed, level)


def smoother_setup(A: Bsr, params: Params, level=0):
    G, GT = OBSR(), OBSR()
    om, lm, npass = C.c_double(), C.c_double(), C.c_int()
    rc = lib().or_smoother_setup(C.byref(A.c()), C.byref(params), level, C.byref(G), C.byref(GT),
                                 C.byref(om), C.byref(lm), C.byref(npass))
    assert rc == 0, rc
    return _take(G), _take(GT), om.value, lm.value, npass.value


def srqcg(A: Bsr, G: Bsr, GT: Bsr, V0, kmax=10, k_ritz=1):
    n, t = V0.shape
    V0c = np.ascontiguousarray(V0.T).reshape(-1)
    V = np.zeros(n * t)
    rc = lib().or_srqcg(C.byref(A.c()), C.byref(G.c()), C.byref(GT.c()), kmax, k_ritz, t, V0c, V)
    assert rc == 0, rc
    return V.reshape(t, n).T.copy()


def gen_eig(H, M):
    t = H.shape[0]
    U = np.zeros(t * t)
    lam = np.zeros(t)
    rc = lib().or_gen_eig(t, np.ascontiguousarray(H, np.float64).reshape(-1),
                          np.ascontiguousarray(M, np.float64).reshape(-1), U, lam)
    assert rc == 0, rc
    return lam, U.reshape(t, t)


def rq_line_min(a, b, c, d, e, f):
    return lib().or_rq_line_min(a, b, c, d, e, f)


def mgs(V):
    n, t = V.shape
    Vc = np.ascontiguousarray(V.T).reshape(-1).copy()
    lib().or_mgs(n, t, Vc)
    return Vc.reshape(t, n).T.copy()


def soc(A: Bsr, V):
    n, t = V.shape
    out = np.zeros(max(A.nnzb, 1))
    lib().or_soc(C.byref(A.c()), t, np.ascontiguousarray(V.T).reshape(-1), out)
    return out[:A.nnzb]


def filter_soc(A: Bsr, socv, theta):
    kept = np.zeros(max(A.nnzb, 1), np.uint8)
    strong = np.zeros(max(A.nnzb, 1), np.uint8)
    s = np.zeros(max(A.nnzb, 1))
    s[:A.nnzb] = socv
    lib().or_filter(C.byref(A.c()), s, theta, kept, strong)
    return kept[:A.nnzb], strong[:A.nnzb]


def mis(A: Bsr, strong):
    cf = np.zeros(A.nr, np.int32)
    st = np.zeros(max(A.nnzb, 1), np.uint8)
    st[:A.nnzb] = strong
    lib().or_mis(C.byref(A.c()), st, cf)
    return cf


def dpls(A: Bsr, strong, cf, V, n_max=5, d_p=2, kappa_p=50.0) -> Bsr:
    n, t = V.shape
    st = np.zeros(max(A.nnzb, 1), np.uint8)
    st[:A.nnzb] = strong
    s = OBSR()
    rc = lib().or_dpls(C.byref(A.c()), st, np.ascontiguousarray(cf, np.int32), t,
                       np.ascontiguousarray(V.T).reshape(-1), n_max, d_p, kappa_p, C.byref(s))
    assert rc == 0, rc
    return _take(s)


def rap(A: Bsr, P: Bsr) -> Bsr:
    s = OBSR()
    rc = lib().or_rap(C.byref(A.c()), C.byref(P.c()), C.byref(s))
    assert rc == 0, rc
    return _take(s)


# ---------------------------------------------------------------- hierarchy

class Hierarchy:
    """aSP-AMG hierarchy built by the oracle (Algorithm 1)."""

    def __init__(self, K: Bsr, V0: np.ndarray, params: Params | None = None):
        self.params = params if params is not None else default_params(K.b)
        n, t0 = V0.shape
        h = C.c_void_p()
        rc = lib().or_setup(C.byref(self.params), C.byref(K.c()), t0,
                            np.ascontiguousarray(V0.T).reshape(-1), C.byref(h))
        if rc != 0:
            raise RuntimeError("oracle setup failed: %d" % rc)
        self._h = h
        self.n = n

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.or_free(h)
            self._h = None

    @property
    def nlev(self):
        return lib().or_h_nlev(self._h)

    def info(self, k):
        info = np.zeros(6, np.int32)
        om, lm = C.c_double(), C.c_double()
        lib().or_h_level_info(self._h, k, info, C.byref(om), C.byref(lm))
        return dict(nr=int(info[0]), nnzb_A=int(info[1]), nnzb_G=int(info[2]),
                    nnzb_P=int(info[3]), nc=int(info[4]), npasses=int(info[5]),
                    omega=om.value, lmax=lm.value)

    def matrix(self, k, which):
        code = {"A": 0, "G": 1, "GT": 2, "P": 3, "R": 4}[which]
        nr, nc, nnzb = C.c_int(), C.c_int(), C.c_int()
        if lib().or_h_bsr_size(self._h, k, code, C.byref(nr), C.byref(nc), C.byref(nnzb)) != 0:
            return None
        b = self.params.b
        rowptr = np.zeros(nr.value + 1, np.int32)
        col = np.zeros(max(nnzb.value, 1), np.int32)
        val = np.zeros(max(nnzb.value, 1) * b * b)
        lib().or_h_bsr_copy(self._h, k, code, rowptr, col, val)
        return Bsr(rowptr, col[:nnzb.value], val[:nnzb.value * b * b].reshape(-1, b, b), nc=nc.value)

    def cf(self, k):
        cf = np.zeros(self.info(k)["nr"], np.int32)
        if lib().or_h_cf(self._h, k, cf) != 0:
            return None
        return cf

    def V(self, k):
        nr = self.info(k)["nr"]
        n = nr * self.params.b
        t = self.params.n_tv
        V = np.zeros(n * t)
        if lib().or_h_V(self._h, k, V) != 0:
            return None
        return V.reshape(t, n).T.copy()

    def vcycle(self, y):
        z = np.zeros(self.n)
        lib().or_vcycle(self._h, np.ascontiguousarray(y, np.float64), z)
        return z

    def pcg(self, b, rtol=1e-8, maxit=1000):
        x = np.zeros(self.n)
        it, rr = C.c_int(), C.c_double()
        rc = lib().or_pcg(self._h, np.ascontiguousarray(b, np.float64), x, rtol, maxit,
                          C.byref(it), C.byref(rr))
        return x, it.value, rr.value, rc

    def stats(self):
        """Grid and operator complexities (Sec. 4.1): sums over levels of rows
        and of stored entries, divided by the finest level's."""
        b = self.params.b
        rows = [self.info(k)["nr"] * b for k in range(self.nlev)]
        nnz = [self.info(k)["nnzb_A"] * b * b for k in range(self.nlev)]
        return dict(C_gd=sum(rows) / rows[0], C_op=sum(nnz) / nnz[0], levels=self.nlev,
                    rows=rows, nnz=nnz)
