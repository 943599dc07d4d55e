"""GPU parity of the three-level hierarchy (Sec. 3: the two-level construction
applied recursively to the coarse equation) against the FP64 oracle: level-1
bootstrap vectors, the level-2 Galerkin operator, level-1 transfers, the
level-1 solve (fixed-step flexible GMRES with the level-1 cycle), one full
cycle and complete solves."""

import numpy as np
import pytest

import synth
from oracle.dirac import WilsonClover
from oracle.mg import Multigrid
from tests.gpu_util import torch_cuda, dev, host, rel

pytestmark = pytest.mark.gpu

DIMS = (16, 8, 8, 16)          # level 1: 4 x 2 x 2 x 4, level 2: 2 x 1 x 1 x 2
M0, CSW = -0.1, 1.0
SAP2, AGG2 = (2, 1, 1, 2), (2, 2, 2, 2)
N0, N1 = 6, 4
PARAMS = dict(n_levels=3, n_vec=(N0, N1), setup_iters=2, inner_iters=3, coarse_iters=12)


@pytest.fixture(scope="module")
def three():
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    u = synth.random_gauge_field(DIMS, 0.4, 61)
    op = WilsonClover(u, M0, CSW)
    iv = synth.test_vector_draw(DIMS, N0, 62)
    mg = Multigrid(op, dict(PARAMS, sap_block=((4, 4, 4, 4), SAP2), agg=((4, 4, 4, 4), AGG2)), iv)
    s = G.Solver(dev(torch, u), CSW, M0, init_vectors=dev(torch, iv), sap_block2=SAP2, agg2=AGG2, **PARAMS)
    yield torch, G, s, op, mg
    s.close()


def test_level1_vectors(three):
    torch, G, s, op, mg = three
    w = torch.zeros((N1, 4, 2, 2, 4, 2 * N0), dtype=torch.complex128, device="cuda")
    G.mg_get_vectors(s.ctx, 1, w)
    assert np.max(np.abs(host(w) - mg.levels[1].agg.columns())) < 1e-9


def test_level2_operator(three):
    torch, G, s, op, mg = three
    c2 = mg.levels[2].op
    ns = int(np.prod(c2.lat))
    m = torch.zeros((ns, 9, 2 * N1, 2 * N1), dtype=torch.complex128, device="cuda")
    G.mg_get_coarse_op(s.ctx, 2, m)
    m = host(m)
    scale = np.max(np.abs(c2.self_))
    assert np.max(np.abs(m[:, 0] - c2.self_.reshape(ns, 2 * N1, 2 * N1))) < 1e-9 * scale
    for mu in range(4):
        assert np.max(np.abs(m[:, 1 + 2 * mu] - c2.fwd[mu].reshape(ns, 2 * N1, 2 * N1))) < 1e-9 * scale
        assert np.max(np.abs(m[:, 2 + 2 * mu] - c2.bwd[mu].reshape(ns, 2 * N1, 2 * N1))) < 1e-9 * scale


def test_level1_transfers(three):
    torch, G, s, op, mg = three
    agg = mg.levels[1].agg
    x1 = synth.random_spinor((4, 2, 2, 4), 63).reshape(4, 2, 2, 4, 12)
    out = torch.zeros((4, 2 * N1), dtype=torch.complex128, device="cuda")
    G.mg_restrict(s.ctx, 1, dev(torch, x1), out, G.MG_FP64)
    assert rel(host(out), agg.restrict(x1).reshape(4, 2 * N1)) < 1e-13
    e2 = synth.random_spinor((2, 1, 1, 2), 64).reshape(2, 1, 1, 2, 12)[..., :2 * N1]
    f = torch.zeros((4, 2, 2, 4, 12), dtype=torch.complex128, device="cuda")
    G.mg_prolong(s.ctx, 1, dev(torch, np.ascontiguousarray(e2)), f, G.MG_FP64)
    assert rel(host(f), agg.prolong(e2)) < 1e-13


def test_level1_solve(three):
    """Fixed-step flexible GMRES on level 1 with the level-1 cycle as preconditioner."""
    torch, G, s, op, mg = three
    vc = synth.random_spinor((4, 2, 2, 4), 65).reshape(4, 2, 2, 4, 12)
    out = torch.zeros((64, 12), dtype=torch.complex128, device="cuda")
    G.mg_coarse_solve(s.ctx, 1, dev(torch, vc.reshape(64, 12)), out, G.MG_FP64)
    assert rel(host(out), mg.coarse_solve(1, vc).reshape(64, 12)) < 1e-9


def test_three_level_cycle(three):
    torch, G, s, op, mg = three
    v = synth.random_spinor(DIMS, 66)
    z = torch.zeros(DIMS[::-1] + (4, 3), dtype=torch.complex128, device="cuda")
    G.mg_precondition(s.ctx, dev(torch, v), z, G.MG_FP64)
    assert rel(host(z), mg.cycle(0, v)) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_three_level_solve(prec):
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    u = synth.random_gauge_field(DIMS, 0.4, 67)
    op = WilsonClover(u, M0, CSW)
    b = synth.random_spinor(DIMS, 68, nvec=2)
    s = G.Solver(dev(torch, u), CSW, M0, sap_block2=SAP2, agg2=AGG2, precision=prec, nrhs_max=2, seed=5, **PARAMS)
    z, info, code = s.solve(dev(torch, b))
    s.close()
    assert code == 0
    z = host(z)
    for k in range(2):
        assert np.linalg.norm(b[k] - op.apply(z[k])) <= 1e-10 * np.linalg.norm(b[k])
