"""GPU parity of the Dirac operator (Sec. 1, Eq. 1.1) and of red-black Schwarz
sweeps (Sec. 2, Algorithm 1) against the FP64 oracle, through the C-ABI."""

import numpy as np
import pytest

import synth
from oracle.dirac import WilsonClover
from oracle.sap import BlockDecomposition, sap_sweep
from tests.gpu_util import torch_cuda, dev, host, rel, round_storage

pytestmark = pytest.mark.gpu

CASES = [((8, 8, 8, 8), 0.5, -0.2, False), ((8, 16, 8, 24), 0.7, 0.1, True)]


def _solver(torch, u, csw, m0, ap, **kw):
    from paper_1202_2462_gb300 import Solver
    return Solver(dev(torch, u), csw, m0, antiperiodic_t=int(ap), **kw)


@pytest.mark.parametrize("dims,eps,m0,ap", CASES)
def test_dirac_fp64_parity(dims, eps, m0, ap):
    torch = torch_cuda()
    u = synth.random_gauge_field(dims, eps, 11)
    op = WilsonClover(u, m0, 1.0, antiperiodic_t=ap)
    psi = synth.random_spinor(dims, 12, nvec=2)
    ref = op.apply(psi)
    s = _solver(torch, u, 1.0, m0, ap, nrhs_max=2)
    out = host(s.dirac(dev(torch, psi)))
    s.close()
    assert rel(out, ref) < 1e-14
    assert np.max(np.abs(out - ref)) < 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("dims,eps,m0,ap", CASES)
def test_dirac_fp64_on_fp32_units_parity(dims, eps, m0, ap):
    """MG_FP64_ON_FP32: the FP64 operator on FP64 data with double-float
    arithmetic (about 48 significand bits) against the oracle, element by
    element, and against the native FP64 kernel; an odd number of
    right-hand sides, and the flag refused with D^dagger or a non-FP64
    precision."""
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    u = synth.random_gauge_field(dims, eps, 15)
    op = WilsonClover(u, m0, 1.0, antiperiodic_t=ap)
    psi = synth.random_spinor(dims, 16, nvec=3)
    ref = op.apply(psi)
    s = _solver(torch, u, 1.0, m0, ap, nrhs_max=3, precision="bf16")
    x = dev(torch, psi)
    out = host(s.dirac(x, G.MG_FP64 | G.MG_FP64_ON_FP32))
    nat = host(s.dirac(x, G.MG_FP64))
    for bad in (G.MG_FP64 | G.MG_FP64_ON_FP32 | G.MG_DAGGER, G.MG_FP32 | G.MG_FP64_ON_FP32):
        with pytest.raises(G.MgError) as e:
            s.dirac(x, bad)
        assert e.value.code == G.MG_ERR_ARG
    s.close()
    assert np.max(np.abs(out - ref)) < 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(out - nat)) < 1e-12 * np.max(np.abs(nat))


@pytest.mark.parametrize("dims,eps,m0,ap", CASES)
def test_dirac_fp32_parity(dims, eps, m0, ap):
    """FP32 storage and arithmetic: <= 1e-5 relative against the exact FP64 operator."""
    torch = torch_cuda()
    from paper_1202_2462_gb300 import MG_FP32
    u = synth.random_gauge_field(dims, eps, 13)
    op = WilsonClover(u, m0, 1.0, antiperiodic_t=ap)
    psi = synth.random_spinor(dims, 14)
    ref = op.apply(psi)
    s = _solver(torch, u, 1.0, m0, ap, precision="fp32")
    out = host(s.dirac(dev(torch, psi, torch.complex64), MG_FP32)).astype(np.complex128)
    s.close()
    assert rel(out, ref) < 1e-6


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_dirac_half_storage_parity(prec):
    """FP16/BF16-stored links and clover with FP32 arithmetic: compared with the
    oracle applied to the identically rounded fields (1e-6), and with the exact
    operator at the storage format's accuracy."""
    torch = torch_cuda()
    from paper_1202_2462_gb300 import PRECISIONS
    dims = (8, 8, 8, 16)
    u = synth.random_gauge_field(dims, 0.6, 15)
    op = WilsonClover(u, -0.1, 1.0)
    opr = WilsonClover(round_storage(u, prec), -0.1, 1.0)
    opr.a = round_storage(op.a, prec)
    psi = synth.random_spinor(dims, 16).astype(np.complex64).astype(np.complex128)
    s = _solver(torch, u, 1.0, -0.1, False, precision=prec)
    out = host(s.dirac(dev(torch, psi, torch.complex64), PRECISIONS[prec])).astype(np.complex128)
    s.close()
    assert rel(out, opr.apply(psi)) < 2e-6
    assert rel(out, op.apply(psi)) < (2e-3 if prec == "fp16" else 1.5e-2)


def test_dirac_zero_field():
    torch = torch_cuda()
    dims = (8, 8, 8, 8)
    u = synth.random_gauge_field(dims, 0.5, 17)
    s = _solver(torch, u, 1.0, 0.0, False)
    out = host(s.dirac(torch.zeros((1, 8, 8, 8, 8, 4, 3), dtype=torch.complex128, device="cuda")))
    s.close()
    assert np.all(out == 0)


@pytest.mark.parametrize("dims,eps,m0,ap", CASES)
def test_sap_sweep_fp64_parity(dims, eps, m0, ap):
    torch = torch_cuda()
    u = synth.random_gauge_field(dims, eps, 21)
    op = WilsonClover(u, m0, 1.0, antiperiodic_t=ap)
    bl = BlockDecomposition(dims, (4, 4, 4, 4))
    b = synth.random_spinor(dims, 22)
    z0 = synth.random_spinor(dims, 23)
    ref = sap_sweep(op, bl, b, sap_sweep(op, bl, b, z0, 4), 4)
    s = _solver(torch, u, 1.0, m0, ap, n_mr=4)
    z = dev(torch, z0)
    s.smooth(dev(torch, b), z, 2)
    out = host(z)
    s.close()
    assert rel(out, ref) < 1e-13


@pytest.mark.parametrize("n_mr", [0, 1, 5])
def test_sap_sweep_fp32_parity(n_mr):
    torch = torch_cuda()
    dims = (8, 8, 16, 8)
    u = synth.random_gauge_field(dims, 0.5, 24)
    op = WilsonClover(u, 0.0, 1.0)
    bl = BlockDecomposition(dims, (4, 4, 4, 4))
    b = synth.random_spinor(dims, 25)
    z0 = np.zeros_like(b)
    ref = sap_sweep(op, bl, b, z0, n_mr)
    s = _solver(torch, u, 1.0, 0.0, False, n_mr=n_mr, precision="fp32")
    z = dev(torch, z0, torch.complex64)
    s.smooth(dev(torch, b, torch.complex64), z, 1)
    out = host(z).astype(np.complex128)
    s.close()
    if n_mr == 0:
        assert np.all(out == 0)
    else:
        assert rel(out, ref) < 2e-6


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_sap_sweep_half_storage_multi_rhs_parity(prec):
    """Two Schwarz sweeps on three right-hand sides at once with FP16/BF16
    fields, against the oracle's sweeps with the identically rounded fields,
    from a nonzero start."""
    torch = torch_cuda()
    dims = (8, 8, 16, 8)
    u = synth.random_gauge_field(dims, 0.5, 29)
    op = WilsonClover(round_storage(u, prec), 0.05, 1.0)
    op.a = round_storage(WilsonClover(u, 0.05, 1.0).a, prec)
    bl = BlockDecomposition(dims, (4, 4, 4, 4))
    b = synth.random_spinor(dims, 30, nvec=3).astype(np.complex64).astype(np.complex128)
    z0 = (0.1 * synth.random_spinor(dims, 31, nvec=3)).astype(np.complex64).astype(np.complex128)
    s = _solver(torch, u, 1.0, 0.05, False, n_mr=4, precision=prec, nrhs_max=3)
    z = dev(torch, z0, torch.complex64)
    s.smooth(dev(torch, b, torch.complex64), z, 2)
    out = host(z).astype(np.complex128)
    s.close()
    for k in range(3):
        ref = sap_sweep(op, bl, b[k], sap_sweep(op, bl, b[k], z0[k], 4), 4)
        assert rel(out[k], ref) < 5e-6, k


def test_sap_zero_rhs_block_stays_finite():
    """A block whose residual is exactly zero: MR takes alpha = 0 (no 0/0)."""
    torch = torch_cuda()
    dims = (8, 8, 8, 8)
    u = synth.random_gauge_field(dims, 0.5, 26)
    s = _solver(torch, u, 1.0, 0.0, False)
    b = torch.zeros((1, 8, 8, 8, 8, 4, 3), dtype=torch.complex128, device="cuda")
    z = torch.zeros_like(b)
    s.smooth(b, z, 3)
    out = host(z)
    s.close()
    assert np.all(out == 0)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_sap_multi_rhs_matches_single(prec):
    """Three right-hand sides in one launch equal three separate sweeps."""
    torch = torch_cuda()
    dims = (8, 8, 8, 16)
    u = synth.random_gauge_field(dims, 0.5, 27)
    s = _solver(torch, u, 1.0, 0.0, False, precision=prec, nrhs_max=3)
    b = dev(torch, synth.random_spinor(dims, 28, nvec=3), torch.complex64)
    z = torch.zeros_like(b)
    s.smooth(b, z, 2)
    for k in range(3):
        zk = torch.zeros_like(b[k:k + 1])
        s.smooth(b[k:k + 1].contiguous(), zk, 2)
        assert torch.equal(zk[0], z[k])
    s.close()


@pytest.mark.parametrize("shape", [0, 1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("prec,n_mr", [("fp32", 4), ("fp16", 1), ("bf16", 4), ("bf16", 2)])
def test_sap_pair_kernel_parity(prec, n_mr, shape, monkeypatch):
    """The paired Schwarz kernel (two right-hand sides per thread, packed
    two-wide FP32 arithmetic; every launch shape): two sweeps on four
    right-hand sides from a nonzero start, with FP32/FP16/BF16 fields, against
    the oracle's sweeps with the identically rounded fields.  n_MR = 1 takes
    the kernel's first-and-last MR step path, n_MR = 2 its first and last
    without a middle step.  Shape 6 (two threads per site) holds FP16/BF16
    fields only and refuses FP32 fields."""
    monkeypatch.setenv("SAPMG_SAP_SHAPE", str(shape))
    torch = torch_cuda()
    if shape == 6 and prec == "fp32":
        import paper_1202_2462_gb300 as G
        dims = (8, 8, 8, 16)
        s = _solver(torch, synth.random_gauge_field(dims, 0.5, 32), 1.0, 0.05, False, precision=prec, nrhs_max=2)
        b = dev(torch, synth.random_spinor(dims, 33, nvec=2), torch.complex64)
        with pytest.raises(G.MgError) as e:
            s.smooth(b, torch.zeros_like(b), 1)
        s.close()
        assert e.value.code == G.MG_ERR_ARG
        return
    dims = (8, 8, 16, 8)
    u = synth.random_gauge_field(dims, 0.5, 32)
    m0 = 0.05
    op = WilsonClover(round_storage(u, prec), m0, 1.0)
    op.a = round_storage(WilsonClover(u, m0, 1.0).a, prec)
    bl = BlockDecomposition(dims, (4, 4, 4, 4))
    b = synth.random_spinor(dims, 33, nvec=4).astype(np.complex64).astype(np.complex128)
    z0 = (0.1 * synth.random_spinor(dims, 34, nvec=4)).astype(np.complex64).astype(np.complex128)
    s = _solver(torch, u, 1.0, m0, False, n_mr=n_mr, precision=prec, nrhs_max=4)
    z = dev(torch, z0, torch.complex64)
    s.smooth(dev(torch, b, torch.complex64), z, 2)
    out = host(z).astype(np.complex128)
    s.close()
    for k in range(4):
        ref = sap_sweep(op, bl, b[k], sap_sweep(op, bl, b[k], z0[k], n_mr), n_mr)
        err = np.max(np.abs(out[k] - ref)) / np.max(np.abs(ref))
        assert err < 5e-6, (k, err)


def test_sap_pair_kernel_matches_single_kernel(monkeypatch):
    """Two right-hand sides through the paired kernel and through the
    one-RHS-per-CTA kernel (SAPMG_SAP_SHAPE=-1): the same sweep up to FP32
    rounding (the two order their sums differently)."""
    torch = torch_cuda()
    dims = (8, 8, 8, 16)
    u = synth.random_gauge_field(dims, 0.5, 35)
    b = dev(torch, synth.random_spinor(dims, 36, nvec=2), torch.complex64)
    outs = []
    for shape in ("0", "-1"):
        monkeypatch.setenv("SAPMG_SAP_SHAPE", shape)
        s = _solver(torch, u, 1.0, 0.0, False, precision="bf16", nrhs_max=2)
        z = torch.zeros_like(b)
        s.smooth(b, z, 2)
        outs.append(host(z))
        s.close()
    assert np.max(np.abs(outs[0] - outs[1])) / np.max(np.abs(outs[1])) < 2e-6


@pytest.mark.parametrize("prec,ap", [("fp32", False), ("fp16", False), ("bf16", True)])
def test_dirac_pair_kernel_parity(prec, ap):
    """Four right-hand sides (the paired Dirac kernel: two per thread, packed
    two-wide FP32 arithmetic) against the oracle with the identically rounded
    fields, element by element; with an antiperiodic time boundary too."""
    torch = torch_cuda()
    from paper_1202_2462_gb300 import PRECISIONS
    dims = (8, 8, 16, 8)
    m0 = 0.05
    u = synth.random_gauge_field(dims, 0.5, 37)
    op = WilsonClover(u, m0, 1.0, antiperiodic_t=ap)
    opr = WilsonClover(round_storage(u, prec), m0, 1.0, antiperiodic_t=ap)
    opr.a = round_storage(op.a, prec)
    psi = synth.random_spinor(dims, 38, nvec=4).astype(np.complex64).astype(np.complex128)
    s = _solver(torch, u, 1.0, m0, ap, precision=prec, nrhs_max=4)
    out = host(s.dirac(dev(torch, psi, torch.complex64), PRECISIONS[prec])).astype(np.complex128)
    s.close()
    for k in range(4):
        ref = opr.apply(psi[k])
        assert np.max(np.abs(out[k] - ref)) / np.max(np.abs(ref)) < 2e-6, k


def test_dirac_pair_kernel_matches_single_kernel(monkeypatch):
    """Two right-hand sides through the paired and the one-RHS-per-CTA Dirac
    kernels (SAPMG_DIRAC_PAIR=0): equal up to FP32 rounding."""
    torch = torch_cuda()
    from paper_1202_2462_gb300 import MG_FP32
    dims = (8, 8, 8, 16)
    u = synth.random_gauge_field(dims, 0.5, 39)
    psi = dev(torch, synth.random_spinor(dims, 40, nvec=2), torch.complex64)
    outs = []
    for flag in ("1", "0"):
        monkeypatch.setenv("SAPMG_DIRAC_PAIR", flag)
        s = _solver(torch, u, 1.0, 0.0, False, precision="fp32", nrhs_max=2)
        outs.append(host(s.dirac(psi, MG_FP32)))
        s.close()
    assert np.max(np.abs(outs[0] - outs[1])) / np.max(np.abs(outs[1])) < 2e-6


@pytest.mark.parametrize("shape", [0, 3, 5, 6])
def test_sap_pair_kernel_tiny_blocks_stay_finite(shape, monkeypatch):
    """Blocks whose residual is ~1e-21 make <p, p> a denormal FP32 number: the
    MR coefficient must still be finite (alpha by division; a reciprocal of
    the denormal overflows to inf and 0 * inf gives NaN).  Two right-hand
    sides with a block-wise scale from 1 down to 1e-21, one sweep from zero,
    against the oracle."""
    monkeypatch.setenv("SAPMG_SAP_SHAPE", str(shape))
    torch = torch_cuda()
    dims = (8, 8, 8, 16)
    u = synth.random_gauge_field(dims, 0.5, 41)
    m0 = 0.05
    op = WilsonClover(round_storage(u, "bf16"), m0, 1.0)
    op.a = round_storage(WilsonClover(u, m0, 1.0).a, "bf16")
    bl = BlockDecomposition(dims, (4, 4, 4, 4))
    scale = 10.0 ** (-(bl.block_id % 8) * 3)                    # 1, 1e-3, ..., 1e-21 per block
    b = synth.random_spinor(dims, 42, nvec=2) * scale[None, ..., None, None]
    b = b.astype(np.complex64).astype(np.complex128)
    s = _solver(torch, u, 1.0, m0, False, n_mr=4, precision="bf16", nrhs_max=2)
    z = torch.zeros((2,) + dims[::-1] + (4, 3), dtype=torch.complex64, device="cuda")
    s.smooth(dev(torch, b, torch.complex64), z, 1)
    out = host(z).astype(np.complex128)
    s.close()
    assert np.all(np.isfinite(out))
    for k in range(2):
        ref = sap_sweep(op, bl, b[k], np.zeros_like(b[k]), 4)
        assert np.max(np.abs(out[k] - ref)) / np.max(np.abs(ref)) < 5e-6, k
