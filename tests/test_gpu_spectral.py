"""The paper's spectral experiments (Sec. 2, Fig. 2; Sec. 3, Fig. 4) through the
library's GPU entry points on an 8^4 lattice with the library's 4^4 Schwarz
blocks and aggregates, each compared with the oracle on the same lattice.

The field is a random gauge transformation of the unit field, so D has the
free spectrum in closed form (pinned in the oracle's tests) and its
eigenvectors are g(x) e^{i p.x} u c with u an eigenvector of sum_mu gamma_mu
sin p_mu and c a colour vector: exact eigenvectors with |lambda| from m0 to
m0 + 8, computed without an eigensolver.

* Fig. 2 (Sec. 2): one red-black Schwarz sweep of the smoother's iteration
  matrix (sap_smooth with b = 0, FP64) barely damps the eigenvectors with the
  smallest |lambda| and damps those with large |lambda| strongly; the GPU's
  swept vectors equal the oracle's.
* Fig. 4 (Sec. 3): after the bootstrap set-up the smallest eigenvalues of the
  Galerkin operator D_c (mg_get_coarse_op) come down to the smallest of D,
  while random test vectors leave them near the middle of the spectrum; the
  GPU's D_c has the oracle's spectrum (same initial vectors)."""

import numpy as np
import pytest

import synth
from oracle.dirac import GAMMA, WilsonClover
from oracle.mg import Multigrid
from oracle.sap import BlockDecomposition, sap_sweep
from tests.gpu_util import torch_cuda, dev, host

pytestmark = pytest.mark.gpu

DIMS = (8, 8, 8, 8)
M0 = 0.05


@pytest.fixture(scope="module")
def pure_gauge():
    g = synth.random_gauge_rotation(DIMS, 141)
    u = synth.gauge_transform(synth.unit_gauge_field(DIMS), g)
    return g, u, WilsonClover(u, M0, 1.0)


def _eigvec(g, n, k, col):
    """Eigenvector of D(U^g) for lattice momentum 2 pi n / L: (vector, eigenvalue)."""
    p = [2 * np.pi * n[i] / DIMS[i] for i in range(4)]
    w, v = np.linalg.eigh(sum(GAMMA[i] * np.sin(p[i]) for i in range(4)))
    t, z, y, x = np.meshgrid(*[np.arange(d) for d in DIMS[::-1]], indexing="ij")
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    c = np.zeros(3, complex)
    c[col] = 1.0
    free = ph[..., None, None] * v[:, k][:, None] * c[None, :]
    phi = np.einsum("tzyxab,tzyxsb->tzyxsa", g, free)
    lam = M0 + sum(1 - np.cos(q) for q in p) + 1j * w[k]
    return phi / np.linalg.norm(phi), lam


MODES = [((0, 0, 0, 0), 0, 0), ((0, 0, 0, 0), 3, 2), ((1, 0, 0, 0), 0, 1), ((0, 1, 1, 0), 2, 0),
         ((2, 2, 2, 2), 1, 2), ((4, 4, 0, 0), 0, 0), ((4, 4, 4, 0), 3, 1), ((4, 4, 4, 4), 2, 2)]


def test_fig2_schwarz_damping_by_eigenvalue_band(pure_gauge):
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    g, u, op = pure_gauge
    vecs, lams = zip(*[_eigvec(g, n, k, c) for n, k, c in MODES])
    for phi, lam in zip(vecs, lams):                    # they are eigenvectors of the oracle's D
        assert np.linalg.norm(op.apply(phi) - lam * phi) < 1e-12
    phis = np.stack(vecs)
    s = G.Solver(dev(torch, u), 1.0, M0, n_levels=1, n_mr=4, nrhs_max=len(MODES))
    z = dev(torch, phis)
    s.smooth(torch.zeros_like(z), z, 1)
    out = host(z)
    s.close()
    bl = BlockDecomposition(DIMS, (4, 4, 4, 4))
    damp = []
    for k, phi in enumerate(vecs):
        ref = sap_sweep(op, bl, np.zeros_like(phi), phi, 4)
        assert np.max(np.abs(out[k] - ref)) < 1e-12 * np.max(np.abs(ref)), k
        damp.append(np.linalg.norm(out[k]))
    damp, mag = np.array(damp), np.abs(np.array(lams))
    assert np.all(damp[mag < 0.1] > 0.9)                          # smallest |lambda|: hardly damped
    assert np.all((damp[(mag > 0.5) & (mag < 1.5)] > 0.4) & (damp[(mag > 0.5) & (mag < 1.5)] < 0.8))
    assert np.all(damp[mag > 4] < 0.25)                           # large |lambda|: damped strongly


@pytest.mark.parametrize("sweeps", [0, 8])
def test_fig4_coarse_spectrum_capture(pure_gauge, sweeps):
    torch = torch_cuda()
    import paper_1202_2462_gb300 as G
    g, u, op = pure_gauge
    iv = synth.test_vector_draw(DIMS, 8, 142)
    s = G.Solver(dev(torch, u), 1.0, M0, n_levels=2, n_vec=(8,), setup_iters=sweeps, init_vectors=dev(torch, iv))
    m = torch.empty((16, 9, 16, 16), dtype=torch.complex128, device="cuda")
    G.mg_get_coarse_op(s.ctx, 1, m)
    ms = host(m)
    s.close()
    # the dense coarse matrix of the stencil (coarse sites x, y, z, t = 2 x 2 x 2 x 2, x fastest)
    dc = np.zeros((16 * 16, 16 * 16), dtype=complex)
    for a in range(16):
        ct, cz, cy, cx = np.unravel_index(a, (2, 2, 2, 2))
        c = [cx, cy, cz, ct]
        dc[16 * a:16 * a + 16, 16 * a:16 * a + 16] += ms[a, 0]
        for mu in range(4):
            for d, step in ((1 + 2 * mu, 1), (2 + 2 * mu, -1)):
                cn = list(c)
                cn[mu] = (cn[mu] + step) % 2
                b = ((cn[3] * 2 + cn[2]) * 2 + cn[1]) * 2 + cn[0]
                dc[16 * a:16 * a + 16, 16 * b:16 * b + 16] += ms[a, d]
    ev = np.linalg.eigvals(dc)
    mg = Multigrid(op, dict(n_levels=2, n_vec=(8,), setup_iters=sweeps, sap_block=((4, 4, 4, 4),),
                            agg=((4, 4, 4, 4),)), iv)
    ref = np.linalg.eigvals(mg.levels[1].op.dense())
    dist = np.abs(ev[:, None] - ref[None, :])
    assert max(dist.min(axis=1).max(), dist.min(axis=0).max()) < 1e-7      # the same spectrum
    lowest = np.min(np.abs(ev)) / M0                              # the fine operator's lowest |lambda| is m0
    if sweeps:
        assert lowest < 1.5
    else:
        assert lowest > 50
