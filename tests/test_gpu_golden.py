"""The CUDA path against the stored expected values (tests/golden/, written
by the oracle only): the FP64 Dirac operator (Eq. 1.1), one FP64 Schwarz
sweep (Algorithm 1) and the FP64 coarse operator (Eq. 3.2) at the stored
sites, through the C ABI."""

import numpy as np
import pytest

import synth
from tests import golden_util as gu
from tests.gpu_util import torch_cuda, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    u = synth.random_gauge_field(gu.DIMS, gu.EPS, gu.GSEED)
    iv = synth.test_vector_draw(gu.DIMS, 4, gu.VSEED)
    s = G.Solver(dev(torch, u), gu.CSW, gu.M0, n_levels=2, n_vec=(4,), setup_iters=0, n_mr=4,
                 init_vectors=dev(torch, iv))
    yield torch, G, s
    s.close()


def test_dirac_against_stored_values(solver):
    torch, G, s = solver
    psi = dev(torch, synth.random_spinor(gu.DIMS, gu.PSEED))
    out = host(s.dirac(psi, G.MG_FP64))
    assert gu.compare_sites("dirac_8x8x8x8.txt", out) < 1e-13


def test_schwarz_sweep_against_stored_values(solver):
    torch, G, s = solver
    b = dev(torch, synth.random_spinor(gu.DIMS, gu.PSEED))
    z = torch.zeros_like(b)
    s.smooth(b, z, 1)
    assert gu.compare_sites("sap_sweep_8x8x8x8.txt", host(z)) < 1e-12


def test_coarse_operator_against_stored_values(solver):
    torch, G, s = solver
    m = torch.zeros((16, 9, 8, 8), dtype=torch.complex128, device="cuda")
    G.mg_get_coarse_op(s.ctx, 1, m)
    m = host(m)
    r = gu.rows("coarse_op_site0_8x8x8x8.txt")
    got = np.array([m[0, int(d), int(i), int(j)] for d, i, j, _, _ in r])
    ref = r[:, 3] + 1j * r[:, 4]
    assert np.max(np.abs(got - ref)) < 1e-13 * np.max(np.abs(ref))
