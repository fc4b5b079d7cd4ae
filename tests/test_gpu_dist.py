"""The GPU side of the row-partitioned solve: products restricted to block-row
ranges (amg_level_apply) against whole products, and the distributed PCG on
one rank through the library's kernels against amg_solve.  (Every run here
has one GPU; the multi-rank exchange is covered on CPU ranks in
test_dist.py.)"""
import os
import socket

import numpy as np
import pytest

import workloads as W
from _problems import gpu_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1902_01715_gb300 as lib_
    lib_.build()
    lib_.lib()
    return lib_


@pytest.mark.parametrize("block", [3, 1])
def test_row_range_products_equal_whole_products(A, block):
    import torch
    from paper_1902_01715_gb300 import dist as D
    d = gpu_problem(A, W.beam(32, 8, 8))
    if block == 1:
        rp, col, val = A.bsr_to_scalar(d["rowptr"], d["col"], d["vals"])
    else:
        rp, col, val = d["rowptr"], d["col"], d["vals"]
    S = A.Solver(rp, col, val, d["V0"], block=block)
    be = D.GpuBackend(S, comm_device="cpu")
    g = torch.Generator(device="cuda").manual_seed(5)
    for k in range(min(2, S.nlev - 1)):
        nr, b = be.nr(k), block
        nc = S.level_info(k)["nc"]
        for which in ("A", "G", "GT", "P", "R"):
            rows = nc if which == "R" else nr
            cols = nc if which == "P" else nr
            x = torch.randn(b * cols, dtype=torch.float64, device="cuda", generator=g)
            aux = torch.randn(b * rows, dtype=torch.float64, device="cuda", generator=g)
            for ep in range(5):
                y1 = aux.clone() if ep == 4 else torch.zeros(b * rows, dtype=torch.float64, device="cuda")
                y2 = y1.clone()
                be.apply(k, which, ep, 0, rows, x, y1, aux, 0.7)
                cut = [0, rows // 3 + 5, 2 * rows // 3 + 1, rows]  # not on slice boundaries
                for r0, r1 in zip(cut, cut[1:]):
                    be.apply(k, which, ep, r0, r1, x, y2, aux, 0.7)
                torch.cuda.synchronize()
                assert torch.equal(y1, y2), (k, which, ep)


def test_distributed_pcg_one_rank_matches_solve(A):
    import torch
    import torch.distributed as td
    from paper_1902_01715_gb300 import dist as D
    d = gpu_problem(A, W.beam(32, 8, 8))
    S = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"])
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=0, world_size=1)
    try:
        DS = D.DistSolver(D.GpuBackend(S, comm_device="cpu"))
        x, it, rr = DS.solve(d["f"], rtol=1e-10)
    finally:
        td.destroy_process_group()
    x1, it1, rr1, rc1 = S.solve(d["f"], 1e-10)
    assert rc1 == 0 and rr <= 1e-10
    assert abs(it - it1[0]) <= 1
    assert float(torch.linalg.norm(x - x1) / torch.linalg.norm(x1)) <= 1e-9
