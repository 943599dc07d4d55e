"""Failure detection of the bounded device waits, driven without a GPU fault.

The kernels that stage data with bulk copies wait on an mbarrier for at most a
bounded number of tries; one that gives up drains its copies in flight, skips
its work and raises the context's device flag, which the synchronising entry
points report as MG_ERR_TIMEOUT.  Here the bound is lowered to zero tries
(mg_set_wait_limit), so every such wait gives up at once; the call must report
MG_ERR_TIMEOUT and leave its output untouched, and after the bound is
restored the next call on the same context must succeed and match the
oracle."""

import numpy as np
import pytest

import synth
from oracle.aggregation import Aggregation
from oracle.coarse import CoarseOperator
from oracle.dirac import WilsonClover
from oracle.sap import BlockDecomposition, sap_sweep
from tests.gpu_util import torch_cuda, dev, host, rel, round_storage

pytestmark = pytest.mark.gpu

DIMS = (8, 8, 8, 8)


def test_coarse_stencil_wait_gives_up_then_recovers():
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    u = synth.random_gauge_field(DIMS, 0.4, 121)
    iv = synth.test_vector_draw(DIMS, 8, 122)
    m0 = -0.2
    s = G.Solver(dev(torch, u), 1.0, m0, n_levels=2, n_vec=(8,), setup_iters=0, precision="fp32",
                 init_vectors=dev(torch, iv))
    c = CoarseOperator(WilsonClover(u, m0, 1.0), Aggregation(DIMS, (4, 4, 4, 4), (4, 3)).build(iv))
    for name in ("self_", "fwd", "bwd"):
        setattr(c, name, round_storage(getattr(c, name), "fp16"))
    x = synth.random_spinor((2, 2, 2, 2), 123, nvec=3).reshape(3, 2, 2, 2, 2, 12)
    x = np.concatenate([x, x[..., :4] * 0.5], axis=-1).astype(np.complex64)          # 16 dof per site
    xd = dev(torch, x)
    out = torch.full((3, 16, 16), 7.0, dtype=torch.complex64, device="cuda")
    G.mg_set_wait_limit(s.ctx, 0)
    with pytest.raises(G.MgError) as e:
        G.mg_coarse_apply_batch(s.ctx, 1, xd, out, G.MG_FP32, 3)
    assert e.value.code == G.MG_ERR_TIMEOUT
    assert torch.all(out == 7.0)                       # the CTAs skipped their work
    G.mg_set_wait_limit(s.ctx, -1)
    G.mg_coarse_apply_batch(s.ctx, 1, xd, out, G.MG_FP32, 3)
    ref = c.apply(round_storage(x.astype(np.complex128), "fp16")).reshape(3, 16, 16)
    assert rel(host(out), ref) < 5e-6
    assert G.mg_sync(s.ctx) == G.MG_OK
    s.close()


def test_block_schwarz_wait_gives_up_then_recovers(monkeypatch):
    """The block-resident Schwarz pass (launch shape 3) on two right-hand sides."""
    monkeypatch.setenv("SAPMG_SAP_SHAPE", "3")
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    u = synth.random_gauge_field(DIMS, 0.5, 124)
    m0 = 0.05
    s = G.Solver(dev(torch, u), 1.0, m0, n_levels=1, n_mr=4, precision="bf16", nrhs_max=2)
    b = synth.random_spinor(DIMS, 125, nvec=2).astype(np.complex64).astype(np.complex128)
    z0 = (0.1 * synth.random_spinor(DIMS, 126, nvec=2)).astype(np.complex64).astype(np.complex128)
    bd = dev(torch, b, torch.complex64)
    z = dev(torch, z0, torch.complex64)
    G.mg_set_wait_limit(s.ctx, 0)
    s.smooth(bd, z, 1)
    with pytest.raises(G.MgError) as e:
        G.mg_sync(s.ctx)
    assert e.value.code == G.MG_ERR_TIMEOUT
    assert np.array_equal(host(z).astype(np.complex128), z0)        # no block was updated
    G.mg_set_wait_limit(s.ctx, -1)
    s.smooth(bd, z, 1)
    assert G.mg_sync(s.ctx) == G.MG_OK
    out = host(z).astype(np.complex128)
    s.close()
    op = WilsonClover(round_storage(u, "bf16"), m0, 1.0)
    op.a = round_storage(WilsonClover(u, m0, 1.0).a, "bf16")
    bl = BlockDecomposition(DIMS, (4, 4, 4, 4))
    for k in range(2):
        ref = sap_sweep(op, bl, b[k], z0[k], 4)
        assert np.max(np.abs(out[k] - ref)) / np.max(np.abs(ref)) < 5e-6, k
