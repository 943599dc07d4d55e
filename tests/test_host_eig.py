"""The library's host eigen-solvers of set-up part 2 (Sec. 3), on the CPU:
harmonic Ritz pairs of a Hessenberg relation against the generalised
eigenproblem that defines them (scipy) and the Petrov-Galerkin condition,
and the Hermitian solver against numpy.linalg.eigh."""

import os

import numpy as np
import pytest


def _b():
    from paper_1202_2462_gb300 import binding
    if not os.path.exists(binding.LIB_PATH):
        pytest.skip("libsapmg.so not built")
    return binding


def _hessenberg(m, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    h = np.zeros((m + 1, m), dtype=np.complex128)
    for j in range(m):
        h[:j + 2, j] = rng.normal(size=j + 2) + 1j * rng.normal(size=j + 2)
    h[np.arange(m), np.arange(m)] += 3.0
    return h * scale


@pytest.mark.parametrize("m,seed", [(1, 0), (2, 1), (8, 2), (16, 3), (40, 4)])
def test_harmonic_ritz_matches_the_generalised_problem(m, seed):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    b = _b()
    h = _hessenberg(m, seed)
    theta, y = b.mg_harmonic_ritz(h)
    hm = h[:m, :m]
    a, bm = h.conj().T @ h, hm.conj().T
    ref, vl, vr = scipy_linalg.eig(a, bm, left=True, right=True)
    # condition number of each reference eigenvalue of the pencil
    cond = np.array([np.linalg.norm(vl[:, k]) * np.linalg.norm(vr[:, k]) / abs(vl[:, k].conj() @ bm @ vr[:, k])
                     for k in range(m)])
    assert np.all(np.diff(np.abs(theta)) >= -1e-12)
    scale = np.linalg.norm(a) + np.abs(theta).max() * np.linalg.norm(bm)
    left = list(range(m))
    for t in theta:
        # backward error: theta is an exact eigenvalue of a pencil within 1e-13 of (A, B)
        assert np.linalg.svd(a - t * bm, compute_uv=False)[-1] <= 1e-13 * scale
        # the same set as scipy's, within what each eigenvalue's conditioning allows
        k = min(left, key=lambda j: abs(t - ref[j]))
        assert abs(t - ref[k]) <= 1e-13 * cond[k] * scale + 1e-12, (t, ref[k], cond[k])
        left.remove(k)
    for k in range(m):
        yk = y[:, k]
        assert abs(np.linalg.norm(yk) - 1.0) < 1e-12
        # Hbar^H (Hbar y - theta [y; 0]) = 0: the Petrov-Galerkin condition in Arnoldi coordinates
        res = h @ yk - theta[k] * np.concatenate([yk, [0.0]])
        assert np.linalg.norm(h.conj().T @ res) < 1e-9 * np.linalg.norm(h) ** 2


def test_harmonic_ritz_of_an_invariant_space_are_eigenvalues():
    b = _b()
    h = _hessenberg(10, 5)
    h[10, 9] = 0.0
    theta, y = b.mg_harmonic_ritz(h)
    ref = np.linalg.eigvals(h[:10, :10])
    assert np.max(np.abs(np.sort_complex(theta) - np.sort_complex(ref))) < 1e-10
    for k in range(10):
        assert np.linalg.norm(h[:10, :10] @ y[:, k] - theta[k] * y[:, k]) < 1e-10


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (16, 2), (40, 3)])
def test_eigh_matches_numpy(n, seed):
    b = _b()
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    a = x @ x.conj().T
    w, v = b.mg_eigh(a)
    ref = np.linalg.eigvalsh(a)
    assert np.max(np.abs(w - ref)) < 1e-12 * max(1.0, np.abs(ref).max())
    assert np.max(np.abs(v.conj().T @ v - np.eye(n))) < 1e-12
    assert np.max(np.abs(a @ v - v * w)) < 1e-11 * max(1.0, np.abs(ref).max())


def test_eigh_with_degenerate_eigenvalues():
    b = _b()
    rng = np.random.default_rng(7)
    q, _ = np.linalg.qr(rng.normal(size=(12, 12)) + 1j * rng.normal(size=(12, 12)))
    d = np.array([1.0, 1.0, 1.0, 2.0, 2.0, 3.0, 4.0, 5.0, 5.0, 6.0, 7.0, 8.0])
    a = (q * d) @ q.conj().T
    w, v = b.mg_eigh(a)
    assert np.max(np.abs(w - d)) < 1e-12
    assert np.max(np.abs(a @ v - v * w)) < 1e-11


def test_bad_arguments_are_rejected():
    b = _b()
    with pytest.raises(b.MgError):
        b.mg_harmonic_ritz(np.zeros((1, 0), dtype=np.complex128))
