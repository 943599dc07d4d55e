"""Spectral experiments of the paper as tests, on the oracle (4^4 Wilson
lattice, 2^4 blocks and aggregates, the setting of Figs. 2 and 4).

* Sec. 2, Fig. 2: one red-black Schwarz sweep with exact block solves damps
  the error components along eigenvectors of large |lambda| well and leaves
  those of the smallest |lambda| essentially undamped.
* Sec. 3, Fig. 4: after the first set-up part (bootstrap sweeps on the test
  vectors) the smallest eigenvalues of D_c = P^dagger D P approximate the
  smallest eigenvalues of D; with unsmoothed random test vectors they do not.

Eigenpairs come from ARPACK (scipy) on the dense matrix of the oracle's D in
three bands (shift-invert at 0 for the smallest |lambda|, at 4 + m0 for the
middle of the spectrum and at 8 + m0 for its top), each checked against its
eigen-equation.
"""

import numpy as np
import pytest

import synth
from oracle.dirac import WilsonClover
from oracle.mg import Multigrid
from oracle.sap import BlockDecomposition, block_dense_matrices, sap_sweep

DIMS = (4, 4, 4, 4)
M0 = -0.3
K = 16


@pytest.fixture(scope="module")
def spectrum():
    sla = pytest.importorskip("scipy.sparse.linalg")
    u = synth.random_gauge_field(DIMS, 0.3, 71)
    op = WilsonClover(u, M0, 0.0)
    d = op.dense()
    bands = {}
    # shift-invert at 0, at the middle (4 + m0) and near the top (8 + m0) of the spectrum
    for name, sigma in (("small", 0.0), ("middle", 4.0 + M0), ("large", 8.0 + M0)):
        lam, vec = sla.eigs(d, k=K, sigma=sigma, tol=1e-12)
        order = np.argsort(np.abs(lam))
        lam, vec = lam[order], vec[:, order]
        assert np.max(np.linalg.norm(d @ vec - vec * lam, axis=0)) < 1e-9
        bands[name] = (lam, vec)
    return op, d, bands


def _fields(op, vec):
    return vec.T.reshape((vec.shape[1],) + op.lat + (4, 3))


def test_schwarz_sweep_damps_large_eigenvalues_but_not_small_ones(spectrum):
    """||S phi|| for unit eigenvectors phi, S the error propagator of one sweep
    (a sweep on D z = 0 from z = phi; exact block solves, 2^4 blocks)."""
    op, d, bands = spectrum
    blocks = BlockDecomposition(DIMS, (2, 2, 2, 2))
    exact = (block_dense_matrices(op, blocks, 0), block_dense_matrices(op, blocks, 1))
    rho = {}
    for name, (lam, vec) in bands.items():
        phi = _fields(op, vec)
        z = sap_sweep(op, blocks, np.zeros_like(phi), phi, 4, exact=exact)
        rho[name] = np.linalg.norm(z.reshape(len(lam), -1), axis=1)
    lam_large = bands["large"][0]
    assert np.min(np.abs(lam_large)) > 0.9 * np.max(np.abs(bands["middle"][0]))
    # the smallest |lambda| band is not reduced at all ...
    assert np.min(rho["small"][:8]) > 0.9, rho["small"]
    # ... while the middle and the top of the spectrum lose more than half
    assert np.max(rho["middle"]) < 0.5, rho["middle"]
    assert np.max(rho["large"]) < 0.5, rho["large"]
    # a second sweep reduces these large-|lambda| components further
    phi = _fields(op, bands["large"][1][:, :2])
    once = sap_sweep(op, blocks, np.zeros_like(phi), phi, 4, exact=exact)
    twice = sap_sweep(op, blocks, np.zeros_like(phi), once, 4, exact=exact)
    assert np.all(np.linalg.norm(twice.reshape(2, -1), axis=1) < np.linalg.norm(once.reshape(2, -1), axis=1))


@pytest.mark.parametrize("nu, bound", [(0, None), (3, 0.5)])
def test_coarse_operator_captures_the_smallest_eigenvalues_after_set_up(spectrum, nu, bound):
    """Relative distance from each of the 8 smallest eigenvalues of D to the
    nearest eigenvalue of D_c (2^4 aggregates x 2 chiralities x N = 8):
    below 0.5 after three bootstrap sweeps, above 5 with the raw random test
    vectors (nu = 0)."""
    op, d, bands = spectrum
    lam = bands["small"][0][:8]
    init = synth.test_vector_draw(DIMS, 8, 5)
    mg = Multigrid(op, dict(n_levels=2, sap_block=((2, 2, 2, 2),), agg=((2, 2, 2, 2),), n_vec=(8,),
                            setup_iters=nu), init_vectors=init)
    lc = np.linalg.eigvals(mg.levels[1].op.dense())
    dist = np.array([np.min(np.abs(lc - l)) / abs(l) for l in lam])
    if bound is None:
        assert np.min(dist) > 5.0, dist
    else:
        assert np.max(dist) < bound, dist
