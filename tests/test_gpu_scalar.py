"""The paper's scalar method (block size 1: every dof its own node, Sec. 3,
Algorithms 1-5 as printed) on the GPU against the oracle run with b = 1,
through the C ABI.

The GPU assembles the structured-hex K in 3x3 blocks and expands it to
scalar CSR on the device (amg_bsr_to_scalar); the oracle expands its own K.
Hierarchies must agree level by level (C/F splits and patterns bit for bit,
values within 1e-13, omega and passes exactly, test spaces within 1e-12), FP64
solutions within 1e-10 at rtol 1e-12."""
import numpy as np
import pytest

import workloads as W
from _problems import SMALL, compare_hierarchies, gpu_problem, oracle_problem, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1902_01715_gb300 as lib_
    lib_.build()
    lib_.lib()
    return lib_


def _scalar_both(A, orc, p, n_coarse=1536, **over):
    K, V0, f, nm = oracle_problem(orc, p)
    Ks = orc.to_scalar(K)
    H = orc.Hierarchy(Ks, V0, orc.default_params(1, n_coarse=n_coarse,
                                                  **{k: v for k, v in over.items() if k != "vcycle_prec"}))
    d = gpu_problem(A, p)
    srp, scol, sval = A.bsr_to_scalar(d["rowptr"], d["col"], d["vals"])
    S = A.Solver(srp, scol, sval, d["V0"], block=1, n_coarse=n_coarse, **over)
    return H, S, Ks, f, d, (srp, scol, sval)


def test_bsr_to_scalar_matches_oracle(A, orc):
    p = SMALL["beam"]()
    K, V0, f, nm = oracle_problem(orc, p)
    Ks = orc.to_scalar(K)
    d = gpu_problem(A, p)
    srp, scol, sval = A.bsr_to_scalar(d["rowptr"], d["col"], d["vals"])
    assert np.array_equal(srp.cpu().numpy(), Ks.rowptr)
    assert np.array_equal(scol.cpu().numpy(), Ks.col[:Ks.nnzb])
    assert np.array_equal(sval.cpu().numpy(), Ks.val[:Ks.nnzb].reshape(-1))


@pytest.mark.parametrize("name", list(SMALL))
def test_scalar_hierarchy_bit_exact(A, orc, name):
    H, S, Ks, f, d, _ = _scalar_both(A, orc, SMALL[name]())
    assert S.nlev >= 2
    compare_hierarchies(S, H)


@pytest.mark.parametrize("name", list(SMALL))
def test_scalar_solution_matches_oracle(A, orc, name):
    H, S, Ks, f, d, _ = _scalar_both(A, orc, SMALL[name]())
    xo, ito, rro, rco = H.pcg(f, 1e-8)
    xg, itg, rrg, rcg = S.solve(d["f"], 1e-8)
    assert rco == 0 and rcg == 0
    assert abs(itg[0] - ito) <= 1 and rrg[0] <= 1e-8
    xo12, _, _, _ = H.pcg(f, 1e-12)
    xg12, _, _, rc12 = S.solve(d["f"], 1e-12)
    x = xg12.cpu().numpy()
    assert rc12 == 0
    assert np.linalg.norm(x - xo12) <= 1e-10 * np.linalg.norm(xo12)
    assert np.linalg.norm(f - Ks.matvec(x)) <= 1e-10 * np.linalg.norm(f)


def test_scalar_vcycle_matches_oracle(A, orc):
    import torch
    H, S, Ks, f, d, _ = _scalar_both(A, orc, SMALL["beam"]())
    y = np.random.default_rng(44).normal(size=Ks.nr)
    zo = H.vcycle(y)
    zg = S.vcycle(torch.tensor(y, device="cuda")).cpu().numpy()
    Ac = H.matrix(H.nlev - 1, "A").todense()
    assert rel(zg, zo) <= 1e-10 + 2 * np.finfo(float).eps * np.linalg.cond(Ac)


def test_scalar_refinement_passes_bit_exact(A, orc):
    """An unreachable omega_bar forces the refinement passes of Algorithm 3
    (patterns up to 48 scalar entries per row with rho = 4)."""
    H, S, Ks, f, d, _ = _scalar_both(A, orc, SMALL["cube"](), omega_bar=10.0)
    assert H.info(0)["npasses"] > 0
    compare_hierarchies(S, H)


@pytest.mark.parametrize("prec", ["fp32", "bf16gp"])
def test_scalar_mixed_precision_reaches_tolerance(A, orc, prec):
    H, S64, Ks, f, d, sc = _scalar_both(A, orc, SMALL["beam"]())
    S = A.Solver(*sc, d["V0"], block=1, vcycle_prec=prec)
    x, it, rr, rc = S.solve(d["f"], 1e-8)
    assert rc == 0 and rr[0] <= 1e-8
    true_rel = np.linalg.norm(f - Ks.matvec(x.cpu().numpy())) / np.linalg.norm(f)
    assert abs(true_rel - rr[0]) <= 1e-10


def test_scalar_batched_matches_single(A, orc):
    """k = 5 right-hand sides through the batched path equal the single
    right-hand-side solves of the same columns."""
    import torch
    p = W.cube_batched(8, 5)
    K, V0, f0, nm = oracle_problem(orc, p, 0)
    d = gpu_problem(A, p, 0)
    srp, scol, sval = A.bsr_to_scalar(d["rowptr"], d["col"], d["vals"])
    from _problems import nodal_to_free
    F = np.column_stack([nodal_to_free(p, nm, c) for c in range(5)])
    Fg = torch.tensor(F, device="cuda")
    S = A.Solver(srp, scol, sval, d["V0"], block=1)
    X, its, rel_, rc = S.solve(Fg, 1e-12)
    assert rc == 0 and max(rel_) <= 1e-12
    for c in range(5):
        x1, it1, _, _ = S.solve(Fg[:, c].contiguous(), 1e-12)
        assert abs(it1[0] - its[c]) <= 1
        assert float(torch.linalg.norm(x1 - X[:, c]) / torch.linalg.norm(x1)) <= 1e-10
