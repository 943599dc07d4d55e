"""GPU parity of the aggregation and coarse-grid components (Sec. 3), the
multilevel cycle and the outer solve (Sec. 4) against the FP64 oracle, through
the C-ABI entry points."""

import numpy as np
import pytest

import synth
from oracle.dirac import WilsonClover
from oracle.aggregation import Aggregation
from oracle.coarse import CoarseOperator
from oracle.krylov import gmres_fixed
from oracle.mg import Multigrid
from tests.gpu_util import torch_cuda, dev, host, rel, emax, round_storage

pytestmark = pytest.mark.gpu

DIMS = (8, 8, 8, 8)
M0, CSW = -0.2, 1.0


@pytest.fixture(scope="module")
def field():
    u = synth.random_gauge_field(DIMS, 0.4, 31)
    return u, WilsonClover(u, M0, CSW)


def _solver(torch, u, **kw):
    import paper_1202_2462_gb300 as G
    return G.Solver(dev(torch, u), CSW, M0, **kw)


def _vectors(torch, s, n):
    import paper_1202_2462_gb300 as G
    v = torch.zeros((n,) + s.lat + (4, 3), dtype=torch.complex128, device="cuda")
    G.mg_get_vectors(s.ctx, 0, v)
    return host(v)


def test_clover_export_parity(field):
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    u, op = field
    s = _solver(torch, u)
    a = torch.zeros(DIMS[::-1] + (2, 6, 6), dtype=torch.complex128, device="cuda")
    G.mg_clover_export(s.ctx, a)
    s.close()
    a = host(a)
    assert np.max(np.abs(a[..., 0, :, :] - op.a[..., :6, :6])) < 1e-14
    assert np.max(np.abs(a[..., 1, :, :] - op.a[..., 6:, 6:])) < 1e-14


def test_drawn_test_vectors_match_counter_generator():
    """With no set-up sweeps P is the local QR of the drawn vectors: the device
    draw (SplitMix64 counters) must equal the host draw bit for bit, so P agrees
    with the oracle's local orthonormalisation to rounding."""
    torch = torch_cuda()
    u = synth.random_gauge_field(DIMS, 0.4, 32)
    s = _solver(torch, u, n_levels=2, n_vec=(5,), setup_iters=0, seed=12345)
    v = _vectors(torch, s, 5)
    s.close()
    ref = Aggregation(DIMS, (4, 4, 4, 4), (4, 3)).build(synth.test_vector_draw(DIMS, 5, 12345)).columns()
    assert np.max(np.abs(v - ref)) < 1e-14


def test_bootstrap_setup_parity(field):
    """Bootstrap part 1 with identical initial vectors (FP64): P agrees."""
    torch = torch_cuda()
    u, op = field
    iv = synth.test_vector_draw(DIMS, 6, 33)
    s = _solver(torch, u, n_levels=2, n_vec=(6,), setup_iters=2, init_vectors=dev(torch, iv))
    v = _vectors(torch, s, 6)
    s.close()
    mg = Multigrid(op, dict(n_levels=2, n_vec=(6,), setup_iters=2, sap_block=((4, 4, 4, 4),),
                            agg=((4, 4, 4, 4),)), iv)
    assert np.max(np.abs(v - mg.levels[0].agg.columns())) < 1e-10


@pytest.fixture(scope="module")
def fp64_ctx(field):
    torch = torch_cuda()
    u, op = field
    iv = synth.test_vector_draw(DIMS, 6, 34)
    s = _solver(torch, u, n_levels=2, n_vec=(6,), setup_iters=0, init_vectors=dev(torch, iv))
    agg = Aggregation(DIMS, (4, 4, 4, 4), (4, 3)).build(iv)
    yield s, agg, CoarseOperator(op, agg)
    s.close()


def test_coarse_operator_parity(fp64_ctx):
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    s, agg, c = fp64_ctx
    m = torch.zeros((16, 9, 12, 12), dtype=torch.complex128, device="cuda")
    G.mg_get_coarse_op(s.ctx, 1, m)
    m = host(m)
    scale = np.max(np.abs(c.self_))
    assert np.max(np.abs(m[:, 0] - c.self_.reshape(16, 12, 12))) < 1e-14 * scale
    for mu in range(4):
        assert np.max(np.abs(m[:, 1 + 2 * mu] - c.fwd[mu].reshape(16, 12, 12))) < 1e-14 * scale
        assert np.max(np.abs(m[:, 2 + 2 * mu] - c.bwd[mu].reshape(16, 12, 12))) < 1e-14 * scale


def test_restrict_prolong_apply_parity(fp64_ctx):
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    s, agg, c = fp64_ctx
    r = synth.random_spinor(DIMS, 35)
    rc = torch.zeros((16, 12), dtype=torch.complex128, device="cuda")
    G.mg_restrict(s.ctx, 0, dev(torch, r), rc, G.MG_FP64)
    assert rel(host(rc), agg.restrict(r).reshape(16, 12)) < 1e-14
    ec = synth.random_spinor((2, 2, 2, 2), 36).reshape(16, 12)
    f = torch.zeros(DIMS[::-1] + (4, 3), dtype=torch.complex128, device="cuda")
    G.mg_prolong(s.ctx, 0, dev(torch, ec), f, G.MG_FP64)
    assert rel(host(f), agg.prolong(ec.reshape(2, 2, 2, 2, 12))) < 1e-14
    out = torch.zeros_like(rc)
    G.mg_coarse_apply(s.ctx, 1, dev(torch, ec), out, G.MG_FP64)
    assert rel(host(out), c.apply(ec.reshape(2, 2, 2, 2, 12)).reshape(16, 12)) < 1e-14


def test_coarse_gmres_parity(fp64_ctx):
    """Fixed-step GMRES (12 steps) from zero: the Krylov minimiser is unique."""
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    s, agg, c = fp64_ctx
    bc = synth.random_spinor((2, 2, 2, 2), 37).reshape(16, 12)
    out = torch.zeros((16, 12), dtype=torch.complex128, device="cuda")
    G.mg_coarse_solve(s.ctx, 1, dev(torch, bc), out, G.MG_FP64)
    ref = gmres_fixed(c.apply, bc.reshape(2, 2, 2, 2, 12), 12).reshape(16, 12)
    assert rel(host(out), ref) < 1e-11


@pytest.mark.parametrize("basis16", ["1", "0"])
def test_coarse_gmres_mixed_parity(basis16, monkeypatch):
    """Fixed-step GMRES in the mixed form (FP16 operator on the tensor cores),
    with the Krylov basis in FP16 (default) or FP32 (SAPMG_COARSE_BASIS_FP16=0),
    against the oracle's GMRES on the FP16-rounded operator (8^3 x 16 lattice,
    32 coarse sites, m0 = -3.9 so that 12 steps are far from an exact solve):
    the same Krylov minimiser up to the rounding of the basis and of the
    vectors fed to the tensor cores (FP16, 2^-11 relative), and a residual
    above the minimal one by no more than that rounding."""
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    monkeypatch.setenv("SAPMG_COARSE_BASIS_FP16", basis16)
    dims = (8, 8, 8, 16)
    u = synth.random_gauge_field(dims, 0.4, 59)
    iv = synth.test_vector_draw(dims, 8, 60)
    m0 = -3.9
    s = G.Solver(dev(torch, u), CSW, m0, n_levels=2, n_vec=(8,), setup_iters=0, precision="bf16",
                 init_vectors=dev(torch, iv), coarse_iters=12)
    c = CoarseOperator(WilsonClover(u, m0, CSW), Aggregation(dims, (4, 4, 4, 4), (4, 3)).build(iv))
    for name in ("self_", "fwd", "bwd"):
        setattr(c, name, round_storage(getattr(c, name), "fp16"))
    bc = synth.random_spinor((2, 2, 2, 4), 61).reshape(4, 2, 2, 2, 12)
    bc = np.concatenate([bc, bc[..., :4]], axis=-1).astype(np.complex64).astype(np.complex128)   # 16 dof
    out = torch.zeros((32, 16), dtype=torch.complex64, device="cuda")
    G.mg_coarse_solve(s.ctx, 1, dev(torch, bc.reshape(32, 16), torch.complex64), out, G.MG_FP32)
    torch.cuda.synchronize()
    s.close()
    ref = gmres_fixed(c.apply, bc, 12)
    got = host(out).astype(np.complex128).reshape(bc.shape)
    res_ref = np.linalg.norm(bc - c.apply(ref)) / np.linalg.norm(bc)
    res_got = np.linalg.norm(bc - c.apply(got)) / np.linalg.norm(bc)
    assert res_ref > 0.1                                    # not an exact solve: the minimiser matters
    tol = 2e-2 if basis16 == "1" else 2e-3
    assert rel(got, ref) < tol
    assert res_got <= res_ref * (1 + tol) + 2e-3


def test_cycle_parity(field, fp64_ctx):
    """One multilevel cycle z = M v with the same P (FP64)."""
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    u, op = field
    s, agg, c = fp64_ctx
    iv = synth.test_vector_draw(DIMS, 6, 34)
    mg = Multigrid(op, dict(n_levels=2, n_vec=(6,), setup_iters=0, sap_block=((4, 4, 4, 4),),
                            agg=((4, 4, 4, 4),)), iv)
    v = synth.random_spinor(DIMS, 38)
    z = torch.zeros(DIMS[::-1] + (4, 3), dtype=torch.complex128, device="cuda")
    G.mg_precondition(s.ctx, dev(torch, v), z, G.MG_FP64)
    assert rel(host(z), mg.cycle(0, v)) < 1e-11


def test_mixed_transfer_parity():
    """FP16-stored P with FP32 arithmetic against the oracle with the same rounded P."""
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    u = synth.random_gauge_field(DIMS, 0.4, 39)
    iv = synth.test_vector_draw(DIMS, 4, 40)
    s = _solver(torch, u, n_levels=2, n_vec=(4,), setup_iters=0, precision="fp16", init_vectors=dev(torch, iv))
    agg = Aggregation(DIMS, (4, 4, 4, 4), (4, 3)).build(iv)
    agg.q = round_storage(agg.q, "fp16")
    r = synth.random_spinor(DIMS, 41).astype(np.complex64)
    rc = torch.zeros((16, 8), dtype=torch.complex64, device="cuda")
    G.mg_restrict(s.ctx, 0, dev(torch, r), rc, G.MG_FP16)
    s.close()
    ref = agg.restrict(r.astype(np.complex128)).reshape(16, 8)
    assert rel(host(rc), ref) < 2e-6 and emax(host(rc), ref) < 6e-6


def _tf32(x):
    """Round float32 values to TF32 (10-bit mantissa, to nearest with ties away
    from zero), as the tensor-core kernels round their inputs."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    b = f.view(np.uint32)
    b = ((b.astype(np.uint64) + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return b.view(np.float32).astype(np.float64)


def _tf32c(z):
    return _tf32(np.real(z)) + 1j * _tf32(np.imag(z))


@pytest.mark.parametrize("nrhs,tf32", [(13, 1), (3, 1), (13, 0)])
def test_batched_transfer_parity(nrhs, tf32, monkeypatch):
    """Restriction and interpolation of several FP32 vectors at once (the form
    the cycle uses), FP16-stored P with N = 8, against the oracle's P^dagger
    and P with the same rounded P.  The tensor-core transfers take TF32
    inputs (FP16 values are exact in TF32), so the oracle transfers the
    TF32-rounded vectors; SAPMG_RESTRICT_TF32=0 selects the FP32 kernels."""
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    monkeypatch.setenv("SAPMG_RESTRICT_TF32", str(tf32))
    u = synth.random_gauge_field(DIMS, 0.4, 52)
    iv = synth.test_vector_draw(DIMS, 8, 53)
    s = _solver(torch, u, n_levels=2, n_vec=(8,), setup_iters=0, precision="fp16", init_vectors=dev(torch, iv),
                nrhs_max=16)
    agg = Aggregation(DIMS, (4, 4, 4, 4), (4, 3)).build(iv)
    agg.q = round_storage(agg.q, "fp16")
    r = synth.random_spinor(DIMS, 54, nvec=nrhs).astype(np.complex64)
    rc = torch.zeros((nrhs, 16, 16), dtype=torch.complex64, device="cuda")
    G.mg_restrict_batch(s.ctx, 0, dev(torch, r), rc, G.MG_FP16, nrhs)
    e = synth.random_spinor((2, 2, 2, 2), 55, nvec=nrhs).reshape(nrhs, 2, 2, 2, 2, 12)
    e = np.concatenate([e, e[..., :4] * 0.5], axis=-1).astype(np.complex64)         # 16 dof per site
    f = torch.zeros((nrhs,) + DIMS[::-1] + (4, 3), dtype=torch.complex64, device="cuda")
    G.mg_prolong_batch(s.ctx, 0, dev(torch, e), f, G.MG_FP16, nrhs)
    torch.cuda.synchronize()
    s.close()
    rin = _tf32c(r) if tf32 else r.astype(np.complex128)
    ref = agg.restrict(rin).reshape(nrhs, 16, 16)
    for k in range(nrhs):
        assert rel(host(rc)[k], ref[k]) < (1e-5 if tf32 else 2e-6), k
        assert emax(host(rc)[k], ref[k]) < (3e-5 if tf32 else 6e-6), k
    ein = _tf32c(e) if tf32 else e.astype(np.complex128)
    fref = agg.prolong(ein)
    for k in range(nrhs):
        assert rel(host(f)[k], fref[k]) < (1e-5 if tf32 else 2e-6), k
        assert emax(host(f)[k], fref[k]) < (3e-5 if tf32 else 6e-6), k


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
def test_solve_reaches_tolerance(field, prec):
    """Outer solve: the oracle's own D confirms ||b - D z|| <= 1e-10 ||b||."""
    torch = torch_cuda()
    u, op = field
    b = synth.random_spinor(DIMS, 42, nvec=2)
    s = _solver(torch, u, n_levels=2, n_vec=(8,), precision=prec, nrhs_max=2, seed=3)
    z, info, code = s.solve(dev(torch, b))
    s.close()
    assert code == 0
    z = host(z)
    for k in range(2):
        assert np.linalg.norm(b[k] - op.apply(z[k])) <= 1e-10 * np.linalg.norm(b[k])
    assert info.relres <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_two_pass_and_delayed_orthogonalisation_agree(field, prec, monkeypatch):
    """The outer Arnoldi with the delayed second Gram-Schmidt pass (default)
    and with two passes per step (SAPMG_DCGS2=0) both reach the tolerance under
    the oracle's D, on four right-hand sides of which one converges early
    (a multiple of another plus a small change), and give the same solution."""
    torch = torch_cuda()
    u, op = field
    b = synth.random_spinor(DIMS, 44, nvec=4)
    b[3] = 2.0 * b[0]
    zs = []
    for flag in ("1", "0"):
        monkeypatch.setenv("SAPMG_DCGS2", flag)
        s = _solver(torch, u, n_levels=2, n_vec=(8,), precision=prec, nrhs_max=4, seed=6, fgmres_m=8)
        z, info, code = s.solve(dev(torch, b))
        s.close()
        assert code == 0
        z = host(z)
        for k in range(4):
            assert np.linalg.norm(b[k] - op.apply(z[k])) <= 1e-10 * np.linalg.norm(b[k]), (flag, k)
        zs.append(z)
    assert rel(zs[0], zs[1]) < 1e-7


def test_fp64_and_mixed_solutions_agree(field):
    torch = torch_cuda()
    u, op = field
    b = synth.z2_spinor(DIMS, 43)
    s1 = _solver(torch, u, n_levels=2, n_vec=(8,), precision="fp64", seed=4)
    z1 = host(s1.solve(dev(torch, b))[0])
    s1.close()
    s2 = _solver(torch, u, n_levels=2, n_vec=(8,), precision="bf16", seed=4)
    z2 = host(s2.solve(dev(torch, b))[0])
    s2.close()
    assert rel(z2, z1) < 1e-7


def test_solve_zero_rhs(field):
    torch = torch_cuda()
    u, op = field
    s = _solver(torch, u, n_levels=2, n_vec=(4,))
    z, info, code = s.solve(torch.zeros(DIMS[::-1] + (4, 3), dtype=torch.complex128, device="cuda"))
    s.close()
    assert code == 0 and np.all(host(z) == 0) and info.relres == 0


def test_iteration_cap_reports_not_converged(field):
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    u, op = field
    b = synth.random_spinor(DIMS, 44)
    s = _solver(torch, u, n_levels=1, maxiter=3, fgmres_m=3)
    z, info, code = s.solve(dev(torch, b))
    s.close()
    assert code == G.MG_NOT_CONVERGED
    assert 1e-10 < info.relres < 1.0
    assert np.linalg.norm(b - op.apply(host(z))) < np.linalg.norm(b)


def test_nonfinite_gauge_field_rejected():
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    u = synth.random_gauge_field(DIMS, 0.4, 45)
    u[1, 2, 3, 4, 2, 1, 1] = np.nan
    with pytest.raises(G.MgError) as e:
        _solver(torch, u)
    assert e.value.code == G.MG_ERR_NONFINITE


def test_fp32_coarse_stencil_batched_parity():
    """The bulk-copy coarse stencil (FP32 operator) on 17 right-hand sides
    (batches of 12, 4 and 1) against the oracle's stencil with the same
    FP32-rounded entries."""
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    u = synth.random_gauge_field(DIMS, 0.4, 46)
    iv = synth.test_vector_draw(DIMS, 6, 47)
    s = _solver(torch, u, n_levels=2, n_vec=(6,), setup_iters=0, precision="fp32", init_vectors=dev(torch, iv))
    op = WilsonClover(u, M0, CSW)
    c = CoarseOperator(op, Aggregation(DIMS, (4, 4, 4, 4), (4, 3)).build(iv))
    for name in ("self_", "fwd", "bwd"):
        setattr(c, name, round_storage(getattr(c, name), "fp32"))
    x = synth.random_spinor((2, 2, 2, 2), 48, nvec=17).reshape(17, 2, 2, 2, 2, 12).astype(np.complex64)
    out = torch.zeros((17, 16, 12), dtype=torch.complex64, device="cuda")
    G.mg_coarse_apply_batch(s.ctx, 1, dev(torch, x), out, G.MG_FP32, 17)
    s.close()
    ref = c.apply(x.astype(np.complex128)).reshape(17, 16, 12)
    assert rel(host(out), ref) < 2e-6 and emax(host(out), ref) < 6e-6


@pytest.mark.parametrize("fp16", ["1", "0"])
def test_coarse_stencil_writes_only_its_rows(fp16, monkeypatch):
    """The tensor-core stencils run in batches of 16, 12, 8, 4 or 1 right-hand
    sides; a call with fewer (here 2, 6, 11, 14) must leave the memory after
    its output untouched (sentinel rows stay NaN) and give the same result as
    the call with exactly the batch width."""
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    monkeypatch.setenv("SAPMG_COARSE_FP16", fp16)
    u = synth.random_gauge_field(DIMS, 0.4, 62)
    iv = synth.test_vector_draw(DIMS, 8, 63)
    s = _solver(torch, u, n_levels=2, n_vec=(8,), setup_iters=0, precision="fp32", init_vectors=dev(torch, iv),
                nrhs_max=16)
    x = synth.random_spinor((2, 2, 2, 2), 64, nvec=16).reshape(16, 16, 12)
    x = dev(torch, np.concatenate([x, x[..., :4]], axis=-1), torch.complex64)          # 16 dof per site
    full = torch.zeros((16, 16, 16), dtype=torch.complex64, device="cuda")
    G.mg_coarse_apply_batch(s.ctx, 1, x, full, G.MG_FP32, 16)
    for nr in (2, 6, 11, 14):
        out = torch.full((nr + 4, 16, 16), float("nan"), dtype=torch.complex64, device="cuda")
        G.mg_coarse_apply_batch(s.ctx, 1, x[:nr].contiguous(), out, G.MG_FP32, nr)
        torch.cuda.synchronize()
        assert torch.isnan(out[nr:]).all(), nr
        assert torch.equal(out[:nr], full[:nr]), nr
    s.close()


def test_coarse_stencil_fp16_n2_40_parity():
    """The tensor-core stencil specialised for 2N = 40 (N = 20 test vectors, the
    benchmark's size), against the oracle's stencil on FP16-rounded entries and
    vectors, for 12 and 5 right-hand sides."""
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    u = synth.random_gauge_field(DIMS, 0.4, 56)
    iv = synth.test_vector_draw(DIMS, 20, 57)
    s = _solver(torch, u, n_levels=2, n_vec=(20,), setup_iters=0, precision="bf16", init_vectors=dev(torch, iv),
                nrhs_max=12)
    op = WilsonClover(u, M0, CSW)
    c = CoarseOperator(op, Aggregation(DIMS, (4, 4, 4, 4), (4, 3)).build(iv))
    for name in ("self_", "fwd", "bwd"):
        setattr(c, name, round_storage(getattr(c, name), "fp16"))
    x = synth.random_spinor((2, 2, 2, 2), 58, nvec=12).reshape(12, 2, 2, 2, 2, 12)
    x = np.concatenate([x, 0.5 * x, -x, x[..., :4]], axis=-1).astype(np.complex64)   # 40 dof per site
    xd = dev(torch, x)
    for nr in (12, 5):
        out = torch.zeros((nr, 16, 40), dtype=torch.complex64, device="cuda")
        G.mg_coarse_apply_batch(s.ctx, 1, xd[:nr].contiguous(), out, G.MG_FP32, nr)
        ref = c.apply(round_storage(x[:nr].astype(np.complex128), "fp16")).reshape(nr, 16, 40)
        assert rel(host(out), ref) < 5e-6 and emax(host(out), ref) < 1.5e-5, nr
    s.close()


@pytest.mark.parametrize("tf32,fp16", [(1, 1), (1, 0), (0, 0)])
def test_coarse_stencil_tensor_core_parity(tf32, fp16, monkeypatch):
    """n2 = 16 takes the tensor-core stencil: with the operator stored in FP16
    (default) the products are FP16 x FP16 with FP32 accumulation, so the
    oracle's stencil gets FP16-rounded entries and vectors; with
    SAPMG_COARSE_FP16=0 the FP32 operator and the vectors enter as TF32.  For
    13, 7, 3 and 1 right-hand sides (each batch width of the kernel).  With
    SAPMG_COARSE_TF32=0 the FP32 bulk-copy stencil runs and is compared with
    FP32-rounded entries."""
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    monkeypatch.setenv("SAPMG_COARSE_TF32", str(tf32))
    monkeypatch.setenv("SAPMG_COARSE_FP16", str(fp16))
    u = synth.random_gauge_field(DIMS, 0.4, 49)
    iv = synth.test_vector_draw(DIMS, 8, 50)
    s = _solver(torch, u, n_levels=2, n_vec=(8,), setup_iters=0, precision="fp32", init_vectors=dev(torch, iv))
    op = WilsonClover(u, M0, CSW)
    c = CoarseOperator(op, Aggregation(DIMS, (4, 4, 4, 4), (4, 3)).build(iv))
    if not tf32:
        rnd_m = rnd_x = lambda a: round_storage(a, "fp32")
    elif fp16:
        rnd_m = rnd_x = lambda a: round_storage(a, "fp16")        # FP16 operator and FP16 fragments
    else:
        rnd_m = rnd_x = _tf32c
    for name in ("self_", "fwd", "bwd"):
        setattr(c, name, rnd_m(getattr(c, name)))
    x = synth.random_spinor((2, 2, 2, 2), 51, nvec=13).reshape(13, 2, 2, 2, 2, 12)
    x = np.concatenate([x, x[:, ..., :4] * 0.5], axis=-1).astype(np.complex64)     # 16 dof per site
    xd = dev(torch, x)
    for nr in (13, 7, 3, 1):
        out = torch.zeros((nr, 16, 16), dtype=torch.complex64, device="cuda")
        G.mg_coarse_apply_batch(s.ctx, 1, xd[:nr].contiguous(), out, G.MG_FP32, nr)
        ref = c.apply(rnd_x(x[:nr].astype(np.complex128))).reshape(nr, 16, 16)
        assert rel(host(out), ref) < 5e-6 and emax(host(out), ref) < 1.5e-5, nr
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_solve_residual_history(field, prec):
    """mg_get_history: for every right-hand side the FP64-recomputed residuals
    end below the tolerance at the reported iteration count and match the
    solve's final relres (the systems run in lockstep, so the count is the
    batch's); each system's least-squares estimates start at iteration 1 and
    stop at or before it."""
    torch = torch_cuda()
    u, op = field
    s = _solver(torch, u, n_levels=2, n_vec=(8,), precision=prec, nrhs_max=2, seed=3)
    b = dev(torch, synth.random_spinor(DIMS, 43, nvec=2))
    z, info, code = s.solve(b)
    h = s.history()
    s.close()
    assert code == 0 and sorted(h) == [0, 1]
    total = 0
    worst = 0.0
    for q, d in h.items():
        k, r = d["fp64"][-1]
        assert r <= 1e-10
        worst = max(worst, r)
        total += k
        its = [it for it, _ in d["estimates"]]
        assert its and max(its) <= k and min(its) == 1
        assert 0 < d["rho"] < 1
    assert total == info.iterations and abs(worst - info.relres) <= 1e-12


def test_complex64_initial_vectors_match_complex128():
    """mg_params.init_vectors_prec = MG_FP32: initial test vectors given as
    complex64 are widened exactly, so the hierarchy equals the one built from
    the same values in complex128, bit for bit."""
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    dims = (8, 8, 8, 8)
    u = dev(torch, synth.random_gauge_field(dims, 0.4, 171))
    iv = torch.from_numpy(synth.test_vector_draw(dims, 6, 172).astype(np.complex64))
    ops = []
    for dt in (torch.complex64, torch.complex128):
        s = G.Solver(u, 1.0, -0.2, n_levels=2, n_vec=(6,), setup_iters=1, precision="fp64",
                     init_vectors=iv.to(dt).cuda())
        m = torch.empty((16, 9, 12, 12), dtype=torch.complex128, device="cuda")
        G.mg_get_coarse_op(s.ctx, 1, m)
        ops.append(m.cpu())
        s.close()
    assert torch.equal(ops[0], ops[1])


@pytest.mark.parametrize("levels", [2, 3])
def test_coarse_solve_graphs_match_plain_launches(levels, monkeypatch):
    """The mixed form replays its FP16-basis coarse GMRES as a captured CUDA
    graph (after one run with plain launches): two solves with graphs give
    the solution of the plain launches (SAPMG_GRAPHS=0) bit for bit, and the
    launch counter counts the graphs' kernels as launches."""
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    dims = (8, 8, 8, 16) if levels == 2 else (16, 8, 8, 16)
    kw = dict(n_levels=levels, n_vec=(12, 8) if levels == 3 else (12,), setup_iters=2, precision="bf16",
              nrhs_max=4, seed=6, coarse_iters=8, fgmres_m=10)
    if levels == 3:
        kw.update(sap_block2=(2, 1, 1, 2), agg2=(2, 2, 2, 2), inner_iters=3)
    u = dev(torch, synth.random_gauge_field(dims, 0.4, 181))
    b = dev(torch, synth.random_spinor(dims, 182, nvec=4))
    out = {}
    for flag in ("0", "1"):
        monkeypatch.setenv("SAPMG_GRAPHS", flag)
        s = G.Solver(u, 1.0, -0.1, **kw)
        zs, counts = [], []
        for _ in range(2):                       # the first solve runs plain, then the graphs
            torch.cuda.synchronize()
            l0 = G.mg_launch_count()
            z, info, code = s.solve(b)
            torch.cuda.synchronize()
            counts.append(G.mg_launch_count() - l0)
            assert code == 0
            zs.append(z)
        s.close()
        assert torch.equal(zs[0], zs[1])
        out[flag] = (zs[1], counts)
    assert torch.equal(out["0"][0], out["1"][0])
    assert out["0"][1] == out["1"][1]


@pytest.mark.parametrize("nrhs,m16", [(2, "1"), (3, "1"), (6, "0"), (6, "1"), (12, "0"), (12, "1")])
def test_level1_schwarz_all_rhs_per_cta_matches_one_rhs_per_cta(nrhs, m16, monkeypatch):
    """Three levels, mixed form: the level-1 Schwarz pass with every
    right-hand side in one CTA per box (each operator entry loaded once for
    all) gives the one-RHS-per-CTA solve bit for bit (same sums in the same
    order per right-hand side), for batch widths across its template bounds,
    with the FP16 (default) or the FP32 copy of the level-1 operator."""
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    monkeypatch.setenv("SAPMG_COARSE_SAP_FP16", m16)
    dims = (16, 8, 8, 16)
    kw = dict(n_levels=3, n_vec=(12, 8), setup_iters=2, precision="bf16", nrhs_max=nrhs, seed=7, coarse_iters=8,
              fgmres_m=10, sap_block2=(2, 1, 1, 2), agg2=(2, 2, 2, 2), inner_iters=3)
    u = dev(torch, synth.random_gauge_field(dims, 0.4, 191))
    b = dev(torch, synth.random_spinor(dims, 192, nvec=nrhs))
    out = {}
    for flag in ("0", "1"):
        monkeypatch.setenv("SAPMG_COARSE_SAP_MRHS", flag)
        s = G.Solver(u, 1.0, -0.1, **kw)
        z, info, code = s.solve(b)
        s.close()
        assert code == 0
        out[flag] = (z, info.iterations)
    assert torch.equal(out["0"][0], out["1"][0]) and out["0"][1] == out["1"][1]
