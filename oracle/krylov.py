"""Krylov solvers used by the method (Sec. 2 and Sec. 4).

* ``gmres_fixed``: GMRES from x0 = 0 with a fixed number k of iterations,
  used for the coarse-grid equation D_c z_c = b_c (Sec. 4: 12 iterations).
  Its result is by definition the minimiser of ||b - A x|| over the Krylov
  space K_k(A, b); it is computed here by Arnoldi with modified Gram-Schmidt
  and a dense least-squares solve (numpy.linalg.lstsq).  Arnoldi stops early
  if the new basis vector vanishes (the Krylov space is invariant).
* ``fgmres``: restarted flexible GMRES, right-preconditioned by a possibly
  varying preconditioner M (Sec. 2: the Schwarz method and the multilevel
  cycle are variable preconditioners, so the outer method must be flexible;
  Sec. 4: restart length 25, stop when the residual has dropped by 1e10).
  Reading taken: x0 = 0; the stopping test is ||b - A x|| <= tol ||b|| on the
  true residual, recomputed at every restart and whenever the least-squares
  residual estimate has reached the tolerance.
* ``cgn``: conjugate gradients on the normal equations A^H A x = A^H b, the
  method the multilevel solver is compared with in Sec. 4 (Tables 1-2: "CGN").
  Reading taken: x0 = 0; the residual r = b - A x is carried along by the
  recursion r -= alpha A p and the iteration stops when ||r|| <= tol ||b||
  (the same test as the flexible GMRES: the residual of A x = b, not of the
  normal equations) or at the iteration cap.
"""

import numpy as np


def _dot(a, b):
    return np.vdot(a, b)


def arnoldi_mgs(apply, b, k):
    """k Arnoldi steps from b: returns (basis list, H (j+1, j), beta, steps done)."""
    beta = np.sqrt(_dot(b, b).real)
    h = np.zeros((k + 1, k), dtype=np.complex128)
    if beta == 0.0:
        return [], h[:1, :0], beta, 0
    v = [b / beta]
    for j in range(k):
        w = apply(v[j])
        for i in range(j + 1):
            h[i, j] = _dot(v[i], w)
            w = w - h[i, j] * v[i]
        h[j + 1, j] = np.sqrt(_dot(w, w).real)
        if h[j + 1, j] == 0.0:
            return v, h[:j + 2, :j + 1], beta, j + 1
        v.append(w / h[j + 1, j])
    return v, h, beta, k


def gmres_fixed(apply, b, k):
    """x in K_k(A, b) minimising ||b - A x||, from x0 = 0."""
    v, h, beta, m = arnoldi_mgs(apply, b, k)
    if m == 0:
        return np.zeros_like(b)
    rhs = np.zeros(h.shape[0], dtype=np.complex128)
    rhs[0] = beta
    y = np.linalg.lstsq(h, rhs, rcond=None)[0]
    x = np.zeros_like(b)
    for i in range(m):
        x = x + y[i] * v[i]
    return x


def fgmres_fixed(apply, precond, b, k):
    """k steps of flexible GMRES from x0 = 0 without restart (no convergence test)."""
    beta = np.sqrt(_dot(b, b).real)
    if beta == 0.0:
        return np.zeros_like(b)
    v = [b / beta]
    z = []
    h = np.zeros((k + 1, k), dtype=np.complex128)
    m = k
    for j in range(k):
        z.append(precond(v[j]))
        w = apply(z[j])
        for i in range(j + 1):
            h[i, j] = _dot(v[i], w)
            w = w - h[i, j] * v[i]
        h[j + 1, j] = np.sqrt(_dot(w, w).real)
        if h[j + 1, j] == 0.0:
            m = j + 1
            break
        v.append(w / h[j + 1, j])
    rhs = np.zeros(m + 1, dtype=np.complex128)
    rhs[0] = beta
    y = np.linalg.lstsq(h[:m + 1, :m], rhs, rcond=None)[0]
    x = np.zeros_like(b)
    for i in range(m):
        x = x + y[i] * z[i]
    return x


def fgmres(apply, precond, b, m, tol, maxiter, x0=None):
    """Restarted right-preconditioned flexible GMRES(m).

    Each cycle: Arnoldi (modified Gram-Schmidt) on the flexible basis
    z_j = M v_j, w = A z_j; after every step the least-squares problem
    min ||beta e_1 - H y|| is solved densely (numpy.linalg.lstsq) and its
    residual serves as the estimate; the cycle ends when that estimate is
    <= tol ||b||, after m steps, at breakdown, or at the iteration cap; then
    x += Z y and the true residual is recomputed.

    Returns (x, total iterations, true relative residuals at every restart,
    converged flag)."""
    bnorm = np.sqrt(_dot(b, b).real)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    if bnorm == 0.0:
        return x, 0, [0.0], True
    it = 0
    history = []
    while True:
        r = b - apply(x)
        rnorm = np.sqrt(_dot(r, r).real)
        history.append(rnorm / bnorm)
        if rnorm <= tol * bnorm:
            return x, it, history, True
        if it >= maxiter:
            return x, it, history, False
        v = [r / rnorm]
        z = []
        h = np.zeros((m + 1, m), dtype=np.complex128)
        rhs = np.zeros(m + 1, dtype=np.complex128)
        rhs[0] = rnorm
        y = None
        for j in range(m):
            z.append(precond(v[j]))
            w = apply(z[j])
            for i in range(j + 1):
                h[i, j] = _dot(v[i], w)
                w = w - h[i, j] * v[i]
            h[j + 1, j] = np.sqrt(_dot(w, w).real)
            it += 1
            y = np.linalg.lstsq(h[:j + 2, :j + 1], rhs[:j + 2], rcond=None)[0]
            est = np.linalg.norm(rhs[:j + 2] - h[:j + 2, :j + 1] @ y)
            if est <= tol * bnorm or it >= maxiter or h[j + 1, j] == 0.0:
                break
            v.append(w / h[j + 1, j])
        for i in range(len(y)):
            x = x + y[i] * z[i]


def cgn(apply, apply_adj, b, tol, maxiter):
    """CG on A^H A x = A^H b from x0 = 0 (CGN).

    Hestenes-Stiefel CG for the Hermitian positive definite A^H A with the
    residual of A x = b kept alongside: r = b, s = A^H r, p = s; each step
    q = A p, alpha = ||s||^2 / ||q||^2, x += alpha p, r -= alpha q,
    s = A^H r, beta = ||s_new||^2 / ||s_old||^2, p = s + beta p.

    Returns (x, iterations, true relative residual ||b - A x|| / ||b||,
    converged flag)."""
    x = np.zeros_like(b, dtype=np.complex128)
    bnorm = np.sqrt(_dot(b, b).real)
    if bnorm == 0.0:
        return x, 0, 0.0, True
    r = np.array(b, dtype=np.complex128)
    s = apply_adj(r)
    p = s.copy()
    gam = _dot(s, s).real
    it = 0
    while np.sqrt(_dot(r, r).real) > tol * bnorm and it < maxiter:
        q = apply(p)
        alpha = gam / _dot(q, q).real
        x = x + alpha * p
        r = r - alpha * q
        s = apply_adj(r)
        gam_new = _dot(s, s).real
        p = s + (gam_new / gam) * p
        gam = gam_new
        it += 1
    true = b - apply(x)
    rel = np.sqrt(_dot(true, true).real) / bnorm
    return x, it, rel, rel <= tol
