"""GPU parity of the comparison solver (CG on the normal equations, the method
Sec. 4 compares with) and of D^dagger against the FP64 oracle, through the
C-ABI (dirac_apply with MG_DAGGER, mg_cgn_solve)."""

import numpy as np
import pytest

import synth
from oracle.dirac import WilsonClover
from oracle.krylov import cgn
from tests.gpu_util import torch_cuda, dev, host, rel, round_storage

pytestmark = pytest.mark.gpu

DIMS = (8, 8, 8, 8)
M0, CSW = 0.0, 1.0


@pytest.fixture(scope="module")
def field():
    u = synth.random_gauge_field(DIMS, 0.4, 31)
    return u, WilsonClover(u, M0, CSW)


@pytest.fixture(scope="module")
def ctxs(field):
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    u, _ = field
    plain = G.Solver(dev(torch, u), CSW, M0, n_levels=1, precision="fp64", nrhs_max=3)
    mixed = G.Solver(dev(torch, u), CSW, M0, n_levels=1, precision="bf16", nrhs_max=3)
    yield torch, G, plain, mixed
    plain.close()
    mixed.close()


def test_dagger_parity_and_adjointness(field, ctxs):
    """D^dagger on the GPU against the oracle's gamma5 D gamma5 (FP64 1e-13;
    FP32 against the oracle with the FP32-rounded fields' tolerance 2e-6), and
    <x, D y> = <D^dagger x, y> from the GPU's own outputs."""
    torch, G, plain, mixed = ctxs
    u, op = field
    x, y = synth.random_spinor(DIMS, 61, nvec=2)
    gx = plain.dirac(dev(torch, x), G.MG_FP64 | G.MG_DAGGER)
    gy = plain.dirac(dev(torch, y), G.MG_FP64)
    assert rel(host(gx), op.apply_dagger(x)) < 1e-13
    lhs = np.vdot(x, host(gy))
    rhs = np.vdot(host(gx), y)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    x32 = round_storage(x, "fp32")
    gx32 = mixed.dirac(dev(torch, x32, torch.complex64), G.MG_FP32 | G.MG_DAGGER)
    assert rel(host(gx32), op.apply_dagger(x32)) < 2e-6
    # the undaggered FP32 operator is unchanged by the new variants
    gy32 = mixed.dirac(dev(torch, x32, torch.complex64), G.MG_FP32)
    assert rel(host(gy32), op.apply(x32)) < 2e-6


def test_dagger_rejected_in_half_storage(ctxs):
    torch, G, plain, mixed = ctxs
    x = torch.zeros(DIMS[::-1] + (4, 3), dtype=torch.complex64, device="cuda")
    with pytest.raises(G.MgError) as e:
        mixed.dirac(x, G.MG_BF16 | G.MG_DAGGER)
    assert e.value.code == G.MG_ERR_ARG


@pytest.mark.parametrize("k", [1, 7, 30])
def test_cgn_iterates_match_the_oracle(field, ctxs, k):
    """After k iterations (the iteration cap) the FP64 iterate equals the
    oracle's k-th CGN iterate."""
    torch, G, plain, mixed = ctxs
    u, op = field
    b = synth.random_spinor(DIMS, 62)
    z, info, code = plain.cgn_solve(dev(torch, b), tol=1e-10, maxiter=k)
    assert code == G.MG_NOT_CONVERGED and info.iterations == k
    ref, it, _, _ = cgn(op.apply, op.apply_dagger, b, 1e-10, k)
    assert it == k
    assert rel(host(z), ref) < 1e-11


def test_cgn_fp64_solve_matches_the_oracle(field, ctxs):
    """A converged FP64 solve: the oracle's D confirms the tolerance, the
    iteration count equals the oracle's (the same stopping test), and the
    solutions agree."""
    torch, G, plain, mixed = ctxs
    u, op = field
    b = synth.random_spinor(DIMS, 63)
    z, info, code = plain.cgn_solve(dev(torch, b), tol=1e-10, maxiter=5000)
    assert code == 0
    z = host(z)
    assert np.linalg.norm(b - op.apply(z)) <= 1e-10 * np.linalg.norm(b)
    ref, it, relres, conv = cgn(op.apply, op.apply_dagger, b, 1e-10, 5000)
    assert conv and abs(info.iterations - it) <= 1, (info.iterations, it)
    assert rel(z, ref) < 1e-8
    assert info.relres <= 1e-10 and info.restarts == 1


def test_cgn_batch_equals_single_solves(field, ctxs):
    """Three right-hand sides at once (one zero, one twice another) give each
    system's single solve: the per-system scalars and partial sums do not
    depend on the batch."""
    torch, G, plain, mixed = ctxs
    u, op = field
    b = synth.random_spinor(DIMS, 64, nvec=3)
    b[1] = 0.0
    b[2] = 2.0 * b[0] + 1e-3 * b[2]
    zb, info, code = plain.cgn_solve(dev(torch, b), tol=1e-10, maxiter=5000)
    assert code == 0
    zb = host(zb)
    assert not np.any(zb[1])
    its = 0
    for k in (0, 2):
        z1, i1, c1 = plain.cgn_solve(dev(torch, b[k]), tol=1e-10, maxiter=5000)
        assert c1 == 0
        its += i1.iterations
        assert rel(zb[k], host(z1)) < 1e-13
        assert np.linalg.norm(b[k] - op.apply(zb[k])) <= 1e-10 * np.linalg.norm(b[k])
    assert info.iterations == its


def test_cgn_mixed_solve_reaches_the_fp64_tolerance(field, ctxs):
    """FP32 iteration with FP64 reliable updates: every system meets
    ||b - D z|| <= 1e-10 ||b|| under the oracle's D, with a few FP64 updates
    and an iteration count close to the FP64 form's."""
    torch, G, plain, mixed = ctxs
    u, op = field
    b = synth.random_spinor(DIMS, 65, nvec=3)
    z, info, code = mixed.cgn_solve(dev(torch, b), tol=1e-10, maxiter=5000, prec=G.MG_FP32)
    assert code == 0
    z = host(z)
    for k in range(3):
        assert np.linalg.norm(b[k] - op.apply(z[k])) <= 1e-10 * np.linalg.norm(b[k])
    z64, i64, c64 = plain.cgn_solve(dev(torch, b), tol=1e-10, maxiter=5000)
    assert c64 == 0
    assert info.restarts >= 3 and info.iterations <= 1.3 * i64.iterations, (info.iterations, i64.iterations)


def test_cgn_errors_and_cap(field, ctxs):
    torch, G, plain, mixed = ctxs
    u, op = field
    b = dev(torch, synth.random_spinor(DIMS, 66))
    z = torch.empty_like(b)
    for args, code in (((1, G.MG_FP64, 0.0, 10), G.MG_ERR_ARG), ((1, G.MG_FP64, 1e-10, 0), G.MG_ERR_ARG),
                       ((1, G.MG_BF16, 1e-10, 10), G.MG_ERR_ARG), ((1, G.MG_FP32, 1e-10, 10), G.MG_ERR_STATE)):
        with pytest.raises(G.MgError) as e:
            G.mg_cgn_solve(plain.ctx, b, z, *args)
        assert e.value.code == code
    bad = b.clone()
    bad.view(-1)[17] = float("nan")
    with pytest.raises(G.MgError) as e:
        G.mg_cgn_solve(plain.ctx, bad, z, 1, G.MG_FP64, 1e-10, 10)
    assert e.value.code == G.MG_ERR_NONFINITE
    code, info = G.mg_cgn_solve(mixed.ctx, b, z, 1, G.MG_FP32, 1e-10, 20)
    assert code == G.MG_NOT_CONVERGED and info.iterations == 20 and 1e-10 < info.relres < 1.0
