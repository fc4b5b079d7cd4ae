"""Pattern work of the set-up on the GPU (graph.cu) against the oracle:
rows longer than the warp merges take (256 blocks), and DPLS candidate sets
at distances other than 2, each through a whole hierarchy that must equal
the oracle's bit for bit."""
import numpy as np
import pytest

import workloads as W
from _problems import SMALL, compare_hierarchies, gpu_problem, oracle_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1902_01715_gb300 as lib_
    lib_.build()
    lib_.lib()
    return lib_


def with_hub(K, hub, others, eps):
    """K plus a spring eps * I between node `hub` and each node of `others`
    (each spring adds [[eps I, -eps I], [-eps I, eps I]] on the two nodes:
    positive semidefinite, so the sum stays SPD).  Returns new CSR arrays
    (columns ascending)."""
    rows = [dict() for _ in range(K.nr)]
    for i in range(K.nr):
        for q in range(K.rowptr[i], K.rowptr[i + 1]):
            rows[i][int(K.col[q])] = K.val[q].copy()
    E = eps * np.eye(3)

    def add(i, j, B):
        if j in rows[i]:
            rows[i][j] = rows[i][j] + B
        else:
            rows[i][j] = B.copy()

    for j in others:
        add(hub, hub, E)
        add(j, j, E)
        add(hub, j, -E)
        add(j, hub, -E)
    rp, col, val = [0], [], []
    for i in range(K.nr):
        for j in sorted(rows[i]):
            col.append(j)
            val.append(rows[i][j])
        rp.append(len(col))
    return np.array(rp, np.int32), np.array(col, np.int32), np.array(val)


def test_long_rows_bit_exact(A, orc):
    """A node coupled to 300 others: its rows of A_0 (and of the products
    built from it) exceed 256 blocks, so the Galerkin patterns take the
    bitmap merge, the candidate sets the pattern-product path, and the
    transposes a long column; the hierarchy still equals the oracle's."""
    import torch
    p = SMALL["beam"]()
    K, V0, f, nm = oracle_problem(orc, p)
    n = K.nr
    others = list(range(1, n, max(1, (n - 1) // 300)))[:300]
    eps = 1e-2 * float(np.mean([K.val[q].trace() / 3 for q in range(K.nnzb)]))
    rp, col, val = with_hub(K, 0, others, eps)
    assert rp[1] - rp[0] > 256
    Kh = orc.Bsr(rp, col, val)
    H = orc.Hierarchy(Kh, V0, orc.default_params(3))
    dev = torch.device("cuda")
    S = A.Solver(torch.tensor(rp, device=dev), torch.tensor(col, device=dev),
                 torch.tensor(val.reshape(-1), device=dev), torch.tensor(V0, device=dev))
    compare_hierarchies(S, H)
    x, it, rr, rc = S.solve(torch.tensor(f, device=dev), 1e-8)
    assert rc == 0 and rr[0] <= 1e-8


@pytest.mark.parametrize("d_p", [1, 3])
@pytest.mark.parametrize("name", ["beam", "slab"])
def test_candidate_distance_bit_exact(A, orc, name, d_p):
    """DPLS candidate sets at distance 1 (the warp merge of one list) and 3
    (pattern products of the strong graph): hierarchy equal to the oracle's."""
    p = SMALL[name]()
    K, V0, f, nm = oracle_problem(orc, p)
    H = orc.Hierarchy(K, V0, orc.default_params(3, d_p=d_p))
    d = gpu_problem(A, p)
    S = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"], d_p=d_p)
    compare_hierarchies(S, H)


@pytest.mark.parametrize("ng", ["1", "2", "4", "8"])
def test_fsai_rows_per_warp_same_bits(A, orc, ng, monkeypatch):
    """The aFSAI kernel shares a warp among 1, 2, 4 or 8 node rows (chosen by
    level size; AMG_FSAI_NG pins it): the lanes only share out independent
    entries, so every choice gives the oracle's hierarchy bit for bit."""
    monkeypatch.setenv("AMG_FSAI_NG", ng)
    p = SMALL["beam"]()
    K, V0, f, nm = oracle_problem(orc, p)
    H = orc.Hierarchy(K, V0, orc.default_params(3))
    d = gpu_problem(A, p)
    S = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"])
    compare_hierarchies(S, H)



@pytest.mark.parametrize("ng", ["4", "8"])
def test_fsai_refinement_many_rounds_bit_exact(A, orc, ng, monkeypatch):
    """Algorithm 3's refinement passes (the layered slab refines twice) on a
    level with more rows than the aFSAI kernel has slots, so every slot takes
    several rows in turn and starts each from a row of the previous G: the
    hierarchy equals the oracle's bit for bit with 4 and 8 rows per warp."""
    monkeypatch.setenv("AMG_FSAI_NG", ng)
    p = W.slab(96, 96, 4)
    K, V0, f, nm = oracle_problem(orc, p)
    H = orc.Hierarchy(K, V0, orc.default_params(3))
    assert H.info(0)["npasses"] > 0
    d = gpu_problem(A, p)
    S = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"])
    compare_hierarchies(S, H)


def test_asymmetric_pattern_refused(A, orc):
    """K is symmetric: a pattern holding block (i, j) without (j, i) is
    refused with AMG_ERR_ARG before any set-up arithmetic."""
    import torch
    p = SMALL["beam"]()
    K, V0, f, nm = oracle_problem(orc, p)
    rp, col, val = np.asarray(K.rowptr), np.asarray(K.col[:K.nnzb]), np.asarray(K.val[:K.nnzb])
    i = 5
    k = next(q for q in range(rp[i], rp[i + 1]) if col[q] != i)  # an off-diagonal block of row i
    keep = np.ones(len(col), bool)
    keep[k] = False
    rp2 = rp.copy()
    rp2[i + 1:] -= 1
    dev = torch.device("cuda")
    with pytest.raises(A.AmgError) as e:
        A.Solver(torch.tensor(rp2, device=dev), torch.tensor(col[keep], device=dev),
                 torch.tensor(val[keep].reshape(-1), device=dev), torch.tensor(V0, device=dev))
    assert e.value.code == A.AMG_ERR_ARG
