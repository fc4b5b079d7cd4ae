"""Row-partitioned PCG (paper_1902_01715_gb300/dist.py) on CPU ranks over
gloo, with the host backend: the partitions and halo plans, and the
distributed solve against the oracle's single-process PCG on the same
hierarchy."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1902_01715_gb300 import dist as D


def test_row_ranges_cover_and_balance():
    for n, w in ((10, 3), (97, 4), (5, 5), (7, 1)):
        rr = D.row_ranges(n, w)
        assert rr[0][0] == 0 and rr[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(rr, rr[1:]))
        sizes = [r1 - r0 for r0, r1 in rr]
        assert max(sizes) - min(sizes) <= 1


def test_coarse_ranges_follow_fine_owners():
    cf = np.array([1, 0, 0, 1, 1, 0, 1, 0, 1, 1])
    fine = D.row_ranges(10, 3)
    cr = D.coarse_ranges(cf, fine)
    cidx = np.cumsum(cf) - 1
    own_f = D.owner_of(fine)
    own_c = D.owner_of(cr)
    for I in np.flatnonzero(cf == 1):
        assert own_c[cidx[I]] == own_f[I]


def test_halo_plans_are_exact_and_symmetric():
    rng = np.random.default_rng(3)
    nr, nc, world = 60, 40, 3
    rows = [np.unique(rng.choice(nc, size=rng.integers(1, 6), replace=False)) for _ in range(nr)]
    rowptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])])
    col = np.concatenate(rows)
    rp, cp = D.row_ranges(nr, world), D.row_ranges(nc, world)
    own = D.owner_of(cp)
    plans = [D.Halo(rowptr, col, rp, cp, me) for me in range(world)]
    for me in range(world):
        r0, r1 = rp[me]
        refs = np.unique(col[rowptr[r0]:rowptr[r1]])
        off = refs[own[refs] != me]
        got = np.sort(np.concatenate([v for v in plans[me].recv.values()])) if plans[me].recv else np.array([])
        assert np.array_equal(got, off)
        for q, v in plans[me].recv.items():
            assert np.all(own[v] == q)
            assert np.array_equal(plans[q].send[me], v)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out, block=3):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    import torch.distributed as td

    import oracle as orc
    import workloads as W
    from _dist_host import HostBackend
    from _problems import oracle_problem
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = W.beam(20, 5, 5)
        K, V0, f, nm = oracle_problem(orc, p)
        if block == 1:  # the paper's scalar form: one row per dof
            K = orc.to_scalar(K)
        H = orc.Hierarchy(K, V0, orc.default_params(block, n_coarse=200))
        S = D.DistSolver(HostBackend(H))
        import torch
        b = torch.as_tensor(f)
        x, it, rr = S.solve(b, rtol=1e-10)
        S.gather_full(0, x)
        if rank == 0:
            xo, ito, rro, rco = H.pcg(f, 1e-10)
            out.put((x.numpy().copy(), it, rr, xo, ito, H.nlev, S.halo_entries))
        td.barrier()
    finally:
        td.destroy_process_group()


@pytest.mark.parametrize("world,block", [(2, 3), (3, 3), (2, 1)])
def test_distributed_pcg_matches_single_process(world, block):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q, block)) for r in range(world)]
    for pr in procs:
        pr.start()
    x, it, rr, xo, ito, nlev, halo = q.get(timeout=300)
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    assert nlev >= 3 and halo > 0
    assert rr <= 1e-10
    assert abs(it - ito) <= 1
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)
