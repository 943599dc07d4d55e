"""Pins of the oracle's comparison solver (CG on the normal equations, Sec. 4)
and of D^dagger: the adjoint identity, the Krylov-space minimisation that
defines the CG iterates, a dense solve, and the degenerate cases."""

import numpy as np

import synth
from oracle.dirac import WilsonClover
from oracle.krylov import cgn

DIMS = (2, 2, 2, 4)          # (Lx, Ly, Lz, Lt): 384 unknowns


def _op(m0=0.1, antiperiodic_t=False, seed=1):
    u = synth.random_gauge_field(DIMS, 0.6, seed)
    return WilsonClover(u, m0, 1.0, antiperiodic_t=antiperiodic_t)


def test_dagger_is_the_adjoint():
    """<x, D y> = <D^dagger x, y> for random x, y (periodic and antiperiodic t),
    and the dense D^dagger is the conjugate transpose of the dense D."""
    for ap in (False, True):
        op = _op(-0.3, ap, 2)
        x, y = synth.random_spinor(DIMS, 3, nvec=2)
        lhs = np.vdot(x, op.apply(y))
        rhs = np.vdot(op.apply_dagger(x), y)
        assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    op = _op(0.2, False, 4)
    d = op.dense()
    n = d.shape[0]
    eye = np.eye(n, dtype=np.complex128).reshape((n,) + op.lat + (4, 3))
    ddag = op.apply_dagger(eye).reshape(n, n).T
    assert np.max(np.abs(ddag - d.conj().T)) < 1e-14


def _krylov_minimiser(d, b, k):
    """argmin ||b - D x|| over x in K_k(D^H D, D^H b), from an orthonormal
    basis of that space built by Arnoldi with two Gram-Schmidt passes (not by
    the CG recursion)."""
    a = d.conj().T @ d
    v = d.conj().T @ b
    basis = [v / np.linalg.norm(v)]
    for _ in range(k - 1):
        w = a @ basis[-1]
        for _pass in range(2):
            for q in basis:
                w = w - np.vdot(q, w) * q
        basis.append(w / np.linalg.norm(w))
    qm = np.stack(basis, axis=1)
    y = np.linalg.lstsq(d @ qm, b, rcond=None)[0]
    return qm @ y


def test_cgn_iterates_minimise_the_residual_over_the_krylov_space():
    """The k-th CGN iterate minimises ||b - D x|| over K_k(D^H D, D^H b): the
    defining property of CG applied to the normal equations."""
    op = _op(-0.2, False, 5)
    d = op.dense()
    b = synth.random_spinor(DIMS, 6)
    for k in (1, 2, 3, 5, 8):
        x, it, _, conv = cgn(op.apply, op.apply_dagger, b, 1e-14, k)
        assert it == k and not conv
        ref = _krylov_minimiser(d, b.ravel(), k).reshape(b.shape)
        assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref), k


def test_cgn_solves_to_the_tolerance():
    """Converged CGN against numpy's dense solve: the true residual meets the
    tolerance and the error is within kappa(D) times it."""
    op = _op(0.1, True, 7)
    d = op.dense()
    b = synth.random_spinor(DIMS, 8)
    x, it, relres, conv = cgn(op.apply, op.apply_dagger, b, 1e-10, 5000)
    assert conv and relres <= 1e-10 and 0 < it < 5000
    ref = np.linalg.solve(d, b.ravel()).reshape(b.shape)
    kappa = np.linalg.cond(d)
    assert np.linalg.norm(x - ref) <= 2 * kappa * 1e-10 * np.linalg.norm(ref)


def test_cgn_degenerate_cases():
    op = _op()
    x, it, relres, conv = cgn(op.apply, op.apply_dagger, np.zeros(op.lat + (4, 3), dtype=np.complex128), 1e-10, 10)
    assert conv and it == 0 and relres == 0.0 and not np.any(x)
    # a right-hand side D e_0 with D = the identity operator part: one step
    # solves b = c * (unit vector) exactly when D is a multiple of the identity
    ident = lambda f: 2.5 * f
    b = synth.random_spinor(DIMS, 9)
    x, it, relres, conv = cgn(ident, ident, b, 1e-12, 10)
    assert it == 1 and conv and np.max(np.abs(x - b / 2.5)) < 1e-15
