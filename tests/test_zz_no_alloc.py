"""The no-allocation coarse solve against the regular one and the oracle.

mg_coarse_solve_noalloc serves callers that cannot allocate device memory when
they solve (an allocator that forbids growth, a latency-critical path where an
allocation's synchronisation is not acceptable): its workspace is a fixed array
in the library's own device memory.  Two calls in a row with different inputs
must reproduce the regular entry point's results (the array keeps the previous
call's contents, so the second call also checks that nothing stale leaks
through); in FP64 both must equal the oracle's fixed-step GMRES (the Krylov
minimiser is unique); a coarse system too large for the array and a
three-level context must be rejected with a clear error.
This file is collected last on purpose."""

import numpy as np
import pytest

import synth
from oracle.dirac import WilsonClover
from oracle.aggregation import Aggregation
from oracle.coarse import CoarseOperator
from oracle.krylov import gmres_fixed
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


def test_noalloc_coarse_solve_matches_oracle_fp64():
    """FP64: the same Krylov minimiser as the oracle's GMRES on the oracle's
    D_c built from the same initial test vectors."""
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    u = synth.random_gauge_field(DIMS, 0.4, 95)
    iv = synth.test_vector_draw(DIMS, 6, 96)
    m0 = -0.2
    s = G.Solver(dev(torch, u), 1.0, m0, n_levels=2, n_vec=(6,), setup_iters=0, init_vectors=dev(torch, iv),
                 coarse_iters=12)
    c = CoarseOperator(WilsonClover(u, m0, 1.0), Aggregation(DIMS, (4, 4, 4, 4), (4, 3)).build(iv))
    for seed in (97, 98):
        bc = synth.random_spinor((2, 2, 2, 2), seed).reshape(16, 12)
        out = torch.zeros((16, 12), dtype=torch.complex128, device="cuda")
        G.mg_coarse_solve_noalloc(s.ctx, 1, dev(torch, bc), out, G.MG_FP64)
        torch.cuda.synchronize()
        ref = gmres_fixed(c.apply, bc.reshape(2, 2, 2, 2, 12), 12).reshape(16, 12)
        assert rel(host(out), ref) < 1e-11
    s.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_noalloc_against_fp16_basis_solve(prec):
    """Mixed form with 2N = 16: mg_coarse_solve keeps its Krylov basis in FP16
    (the FP16 operator copy exists), the no-alloc solve keeps it in FP32.  Both
    read the same FP16 operator, so they differ by the basis rounding only:
    FP16 keeps 11 significant bits (relative rounding 2^-11 = 4.9e-4), and a
    12-step GMRES result built on such a basis moves by a small multiple of
    that; 2e-2 is the bound the regular solve's own FP16-basis parity test
    uses against the oracle."""
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    u = synth.random_gauge_field(DIMS, 0.4, 99)
    s = G.Solver(dev(torch, u), 1.0, -0.2, n_levels=2, n_vec=(8,), setup_iters=1, precision=prec, seed=11,
                 coarse_iters=12)
    for seed in (100, 101):
        b = synth.random_spinor((2, 2, 2, 2), seed, nvec=2).reshape(2, 16, 12).transpose(1, 0, 2).reshape(16, 24)
        b = np.ascontiguousarray(b[:, :16])                 # 16 coarse sites x 2N = 16
        bc = dev(torch, b, torch.complex64)
        ref = torch.zeros_like(bc)
        out = torch.full_like(bc, 7.0)
        G.mg_coarse_solve(s.ctx, 1, bc, ref, G.MG_FP32)
        G.mg_coarse_solve_noalloc(s.ctx, 1, bc, out, G.MG_FP32)
        torch.cuda.synchronize()
        assert np.all(np.isfinite(host(out)))
        assert rel(host(out), host(ref)) < 2e-2
    s.close()


def test_noalloc_rejects_three_level_context():
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    dims = (16, 8, 8, 16)
    u = synth.random_gauge_field(dims, 0.4, 102)
    s = G.Solver(dev(torch, u), 1.0, -0.1, n_levels=3, n_vec=(6, 4), setup_iters=1, inner_iters=3,
                 coarse_iters=12, sap_block2=(2, 1, 1, 2), agg2=(2, 2, 2, 2))
    bc = torch.zeros((64, 12), dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(bc)
    with pytest.raises(G.MgError) as e:
        G.mg_coarse_solve_noalloc(s.ctx, 1, bc, out, G.MG_FP64)
    assert e.value.code == G.MG_ERR_STATE and "two-level" in str(e.value)
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
