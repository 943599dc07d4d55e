"""Pins of the oracle's aggregation, coarse operator, Krylov solvers and
multilevel solve (Sec. 3 and Sec. 4) against properties fixed by their
definitions: P^dagger P = 1, gamma_5 P = P gamma_5^c, uniqueness of the
local QR, the dense Galerkin product P^dagger D P, gamma_5^c-hermiticity,
nearest-neighbour sparsity, Galerkin orthogonality, the unitary special case,
and GMRES/FGMRES optimality."""

import numpy as np
import pytest

import synth
from oracle.dirac import WilsonClover
from oracle.aggregation import Aggregation, gamma5_coarse, orthonormalise
from oracle.coarse import CoarseOperator, galerkin_dense
from oracle.krylov import gmres_fixed, fgmres, fgmres_fixed
from oracle.mg import Multigrid


@pytest.fixture(scope="module")
def small():
    dims = (4, 4, 4, 4)
    op = WilsonClover(synth.random_gauge_field(dims, 0.5, 51), 0.1, 1.0)
    vecs = synth.test_vector_draw(dims, 3, 52)
    agg = Aggregation(dims, (2, 2, 2, 2), (4, 3)).build(vecs)
    return op, agg, vecs


def test_p_orthonormal(small):
    op, agg, vecs = small
    p = agg.dense()
    assert np.max(np.abs(np.conj(p.T) @ p - np.eye(p.shape[1]))) < 1e-13


def test_p_gamma5_compatible(small):
    """gamma_5 P = P gamma_5^c, exactly (a structural zero pattern)."""
    op, agg, vecs = small
    p = agg.dense()
    n_sites = p.shape[0] // 12
    g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), n_sites)
    g5c = np.tile(gamma5_coarse(agg.nvec), p.shape[1] // (2 * agg.nvec))
    assert np.max(np.abs(g5[:, None] * p - p * g5c[None, :])) == 0.0


def test_p_is_unique_qr(small):
    """Local MGS = thin QR with positive diagonal (numpy QR with signs fixed)."""
    op, agg, vecs = small
    x = agg.to_aggregates(vecs)                  # (N, S, 2, L)
    for s in (0, 5):
        for chi in (0, 1):
            a = x[:, s, chi, :].T                # L x N
            q, r = np.linalg.qr(a)
            ph = np.diag(r) / np.abs(np.diag(r))
            q = q * ph[None, :]
            assert np.max(np.abs(q - agg.q[:, s, chi, :].T)) < 1e-13


def test_p_span_contains_test_vectors(small):
    op, agg, vecs = small
    for v in vecs:
        assert np.max(np.abs(agg.prolong(agg.restrict(v)) - v)) < 1e-13


def test_coarse_stencil_equals_dense_galerkin(small):
    op, agg, vecs = small
    c = CoarseOperator(op, agg)
    assert np.max(np.abs(c.dense() - galerkin_dense(op, agg))) < 1e-13


def test_coarse_gamma5_hermitian(small):
    op, agg, vecs = small
    c = CoarseOperator(op, agg)
    d = c.dense()
    g = np.tile(gamma5_coarse(agg.nvec), d.shape[0] // (2 * agg.nvec))
    assert np.max(np.abs(g[:, None] * d * g[None, :] - np.conj(d.T))) < 1e-13


def test_coarse_nearest_neighbour_only():
    """On a 4x2x2x2 coarse grid, couplings between non-neighbouring aggregates are 0."""
    dims = (8, 4, 4, 4)
    op = WilsonClover(synth.random_gauge_field(dims, 0.4, 53), 0.0, 1.0)
    agg = Aggregation(dims, (2, 2, 2, 2), (4, 3)).build(synth.test_vector_draw(dims, 2, 54))
    g = galerkin_dense(op, agg)
    cl = agg.clat
    n2 = 2 * agg.nvec
    coords = np.array(np.unravel_index(np.arange(int(np.prod(cl))), cl)).T      # (t, z, y, x)
    dist = np.abs(coords[:, None, :] - coords[None, :, :])
    dist = np.minimum(dist, np.array(cl)[None, None, :] - dist).sum(-1)
    gb = g.reshape(len(coords), n2, len(coords), n2)
    far = dist > 1
    assert np.max(np.abs(gb.transpose(0, 2, 1, 3)[far])) == 0.0
    assert np.max(np.abs(gb.transpose(0, 2, 1, 3)[dist == 1])) > 1e-3


def test_galerkin_orthogonality(small):
    """After z = P D_c^{-1} P^dagger r: P^dagger (r - D z) = 0 (Eq. 3.2)."""
    op, agg, vecs = small
    c = CoarseOperator(op, agg)
    r = synth.random_spinor(op.dims, 55)
    rc = agg.restrict(r)
    ec = np.linalg.solve(c.dense(), rc.ravel()).reshape(rc.shape)
    z = agg.prolong(ec)
    assert np.max(np.abs(agg.restrict(r - op.apply(z)))) < 1e-12


def test_unitary_p_preserves_spectrum():
    """1-site aggregates with N = 6 make P square and unitary: spec(D_c) = spec(D)."""
    dims = (2, 2, 2, 2)
    op = WilsonClover(synth.random_gauge_field(dims, 0.6, 56), -0.1, 1.2)
    agg = Aggregation(dims, (1, 1, 1, 1), (4, 3)).build(synth.test_vector_draw(dims, 6, 57))
    c = CoarseOperator(op, agg)
    ea = np.sort_complex(np.round(np.linalg.eigvals(op.dense()), 9))
    eb = np.sort_complex(np.round(np.linalg.eigvals(c.dense()), 9))
    assert np.max(np.abs(ea - eb)) < 1e-8


def test_second_level_recursion_pins(small):
    """The coarse operator is again a stencil: a second aggregation of it
    passes the same Galerkin pin against the dense product."""
    op, agg, vecs = small
    c = CoarseOperator(op, agg)                       # coarse grid 2^4, 6 dof
    vc = np.stack([agg.restrict(v) for v in synth.test_vector_draw(op.dims, 2, 58)])
    agg2 = Aggregation(c.dims, (1, 1, 1, 2), (2 * agg.nvec,)).build(vc)
    c2 = CoarseOperator(c, agg2)
    assert np.max(np.abs(c2.dense() - galerkin_dense(c, agg2))) < 1e-13


def _rand_matrix(n, seed):
    a = synth.random_spinor((n, 1, 1, 1), seed, nvec=n).reshape(n, n * 12)[:, :n]
    return a / np.sqrt(n) + 3.0 * np.eye(n)


def test_gmres_full_space_is_exact():
    a = _rand_matrix(9, 60)
    b = _rand_matrix(9, 61)[:, 0]
    x = gmres_fixed(lambda v: a @ v, b, 9)
    assert np.max(np.abs(x - np.linalg.solve(a, b))) < 1e-12


def test_gmres_minimises_residual_over_krylov_space():
    a = _rand_matrix(12, 62)
    b = _rand_matrix(12, 63)[:, 0]
    k = 4
    x = gmres_fixed(lambda v: a @ v, b, k)
    kry = np.stack([np.linalg.matrix_power(a, i) @ b for i in range(k)], axis=1)
    q, _ = np.linalg.qr(kry)
    r = b - a @ x
    assert np.max(np.abs(np.conj((a @ q).T) @ r)) < 1e-12      # normal equations
    assert np.max(np.abs(x - q @ (np.conj(q.T) @ x))) < 1e-12  # x in K_k


def test_gmres_zero_rhs():
    assert np.all(gmres_fixed(lambda v: 2 * v, np.zeros(5, complex), 3) == 0)


def test_fgmres_fixed_identity_preconditioner_equals_gmres():
    a = _rand_matrix(10, 64)
    b = _rand_matrix(10, 65)[:, 0]
    x1 = gmres_fixed(lambda v: a @ v, b, 5)
    x2 = fgmres_fixed(lambda v: a @ v, lambda v: v, b, 5)
    assert np.max(np.abs(x1 - x2)) < 1e-12


def test_fgmres_restarted_converges():
    a = _rand_matrix(30, 66)
    b = _rand_matrix(30, 67)[:, 0]
    x, it, hist, ok = fgmres(lambda v: a @ v, lambda v: v, b, 5, 1e-11, 500)
    assert ok and np.linalg.norm(b - a @ x) <= 1e-11 * np.linalg.norm(b)
    assert hist[-1] <= 1e-11


def _min_residual_step(a, m_pre, r, k):
    """M y with y minimising ||r - A M y|| over K_k(A M, r): least squares on
    the explicit power basis (independent of any Arnoldi process)."""
    am = a @ m_pre
    basis = [r]
    for _ in range(k - 1):
        basis.append(am @ basis[-1])
    kr = np.stack(basis, axis=1)
    coef, *_ = np.linalg.lstsq(am @ kr, r, rcond=None)
    return m_pre @ (kr @ coef)


def test_fgmres_restart_cycles_are_krylov_minimisers():
    """Restarted flexible GMRES(m) with a fixed linear preconditioner M (Sec. 2,
    Sec. 4): every cycle adds the minimiser of the residual over
    M K_m(A M, r) for the true residual r at the restart, and the history
    holds the true residuals at the restarts."""
    a = _rand_matrix(30, 80)
    m_pre = np.eye(30) + 0.3 * _rand_matrix(30, 81)
    b = _rand_matrix(30, 82)[:, 0]
    m = 3
    x_ref = np.zeros(30, dtype=np.complex128)
    hist_ref = []
    for cycles in (1, 2, 3):
        x, it, hist, ok = fgmres(lambda v: a @ v, lambda v: m_pre @ v, b, m, 1e-14, m * cycles)
        r = b - a @ x_ref
        hist_ref.append(np.linalg.norm(r) / np.linalg.norm(b))
        x_ref = x_ref + _min_residual_step(a, m_pre, r, m)
        assert it == m * cycles and not ok
        assert np.max(np.abs(x - x_ref)) < 1e-10 * np.max(np.abs(x_ref))
        assert np.allclose(hist[:-1], hist_ref, rtol=1e-10, atol=0)
        assert abs(hist[-1] - np.linalg.norm(b - a @ x_ref) / np.linalg.norm(b)) < 1e-12
    # a restart that forgot the previous cycles' x, or restarted from b, would differ
    assert np.linalg.norm(b - a @ x_ref) < 0.9 * np.linalg.norm(b - a @ _min_residual_step(a, m_pre, b, m))


def test_global_orthonormalise():
    v = orthonormalise(list(synth.test_vector_draw((2, 2, 2, 2), 4, 68)))
    g = np.array([[np.vdot(a, b) for b in v] for a in v])
    assert np.max(np.abs(g - np.eye(4))) < 1e-14


def test_two_level_solve_small():
    """Full two-level solve on a 4^4 lattice (2^4 Schwarz blocks and aggregates)."""
    dims = (4, 4, 4, 4)
    op = WilsonClover(synth.random_gauge_field(dims, 0.4, 70), -0.1, 1.0)
    mg = Multigrid(op, dict(n_levels=2, sap_block=((2, 2, 2, 2),), agg=((2, 2, 2, 2),),
                            n_vec=(4,), setup_iters=2, fgmres_m=10),
                   synth.test_vector_draw(dims, 4, 71))
    b = synth.random_spinor(dims, 72)
    z, it, hist, ok = mg.solve(b)
    assert ok
    assert np.linalg.norm(b - op.apply(z)) <= 1e-10 * np.linalg.norm(b)
    d = op.dense()
    xs = np.linalg.solve(d, b.ravel())
    cond = np.linalg.cond(d)
    assert np.linalg.norm(z.ravel() - xs) <= 2e-10 * cond * np.linalg.norm(xs)


def test_three_level_solve_small():
    dims = (8, 4, 4, 8)
    op = WilsonClover(synth.random_gauge_field(dims, 0.4, 73), 0.0, 1.0)
    mg = Multigrid(op, dict(n_levels=3, sap_block=((2, 2, 2, 2), (1, 1, 1, 1)),
                            agg=((2, 2, 2, 2), (2, 1, 1, 2)), n_vec=(4, 4), setup_iters=2,
                            fgmres_m=10, inner_iters=3),
                   synth.test_vector_draw(dims, 4, 74))
    assert mg.levels[2].op.lat == (2, 2, 2, 2)
    b = synth.random_spinor(dims, 75)
    z, it, hist, ok = mg.solve(b)
    assert ok and np.linalg.norm(b - op.apply(z)) <= 1e-10 * np.linalg.norm(b)
