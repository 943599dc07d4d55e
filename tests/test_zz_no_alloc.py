"""The no-allocation coarse solve against the regular one.

mg_coarse_solve_noalloc serves callers that cannot allocate device memory when
they solve (inside CUDA graph capture, under allocators that forbid growth, on
latency-critical paths): its workspace is a fixed array in the library's own
device memory.  Two calls in a row with different inputs must reproduce the
regular entry point's results (the array keeps the previous call's contents,
so the second call also checks that nothing stale leaks through), and a
coarse system too large for the array must be rejected with a clear error.
This file is collected last on purpose."""

import numpy as np
import pytest

import synth
from tests.gpu_util import torch_cuda, dev, host, rel

pytestmark = pytest.mark.gpu

DIMS = (8, 8, 8, 8)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_coarse_solve_matches_regular(prec):
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    u = synth.random_gauge_field(DIMS, 0.4, 91)
    s = G.Solver(dev(torch, u), 1.0, -0.2, n_levels=2, n_vec=(6,), setup_iters=1, precision=prec, seed=9)
    code = G.PRECISIONS[prec]
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    tol = 1e-12 if prec == "fp64" else 1e-6
    for seed in (92, 93):                     # two calls in a row
        bc = dev(torch, synth.random_spinor((2, 2, 2, 2), seed).reshape(16, 12), cdt)
        ref = torch.zeros_like(bc)
        out = torch.full_like(bc, 7.0)        # garbage in the output must not matter
        G.mg_coarse_solve(s.ctx, 1, bc, ref, code)
        G.mg_coarse_solve_noalloc(s.ctx, 1, bc, out, code)
        torch.cuda.synchronize()
        assert rel(host(out), host(ref)) < tol
    s.close()


def test_noalloc_rejects_oversized_system():
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    dims = (16, 16, 16, 32)
    u = synth.random_gauge_field(dims, 0.4, 94)
    s = G.Solver(dev(torch, u), 1.0, 0.0, n_levels=2, n_vec=(32,), setup_iters=0, coarse_iters=32)
    bc = torch.zeros((512, 64), dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(bc)
    with pytest.raises(G.MgError) as e:
        G.mg_coarse_solve_noalloc(s.ctx, 1, bc, out, G.MG_FP64)
    assert e.value.code == G.MG_ERR_ARG and "no-alloc scratch" in str(e.value)
    s.close()
