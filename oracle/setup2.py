"""Bootstrap set-up, part 2 (Sec. 3): refinement of the test vectors by
harmonic Ritz pairs of the coarse operator.

TEST INFRASTRUCTURE ONLY: plain FP64 numpy restatement, used by the tests,
never by the library.

The paper's steps, for a two-level hierarchy built by part 1 (the paper runs
the procedure once, starting on the coarsest grid):

1. N approximations (lambda_i, phi_i) to the eigenpairs of D_c = P^dagger D P
   of smallest magnitude, as harmonic Ritz values and vectors.  Reading: from
   an Arnoldi space of D_c of dimension m = 2N (when m reaches the coarse
   dimension, or Arnoldi meets an invariant subspace, they are exact
   eigenpairs; a subdiagonal entry below 1e-12 of the largest Hessenberg entry
   is read as that breakdown).  The pairs are defined through an orthonormal
   basis of the Krylov space, so the Arnoldi process here orthogonalises twice
   (two modified Gram-Schmidt passes): with one pass the basis of this
   non-normal operator loses orthogonality (1.7e-10 after 12 steps on the 8^4
   test case) and the computed values move by 1e-6.  A harmonic Ritz pair (theta, phi = V_m y) of a space V_m
   satisfies the Petrov-Galerkin condition D_c phi - theta phi perpendicular
   to D_c V_m; with D_c V_m = V_{m+1} Hbar this is the generalised problem
   Hbar^H Hbar y = theta H_m^H y (H_m the square part of Hbar).
2. Each phi_i is interpolated (P phi_i) and smoothed towards lambda_i by iota
   Schwarz sweeps of the iteration matrix S(lambda_i) of D - lambda_i: sweeps
   on (D - lambda_i) x = 0 started at x = P phi_i, whose block solves are
   B_j(lambda_i) = I [I^T (D - lambda_i) I]^{-1} I^T (here n_MR MR steps on
   the shifted block systems, or exact solves).
3. V = {S(lambda_i)^iota P phi_i} together with the current test vectors
   {S^nu v_j} of part 1 (2N vectors).
4. Reduced to N vectors: reading, V is orthonormalised first (global modified
   Gram-Schmidt), so that the eigenvectors y_k of the Hermitian 2N x 2N
   matrix (DV)^dagger DV for its N smallest eigenvalues (the squared N
   smallest singular values of DV) give the new vectors V y_k.
5. P and D_c are rebuilt from the N new vectors.
(The three-level reading is stated with ``part2``.)
"""

import numpy as np
import scipy.linalg

from .aggregation import Aggregation, orthonormalise
from .coarse import CoarseOperator
from .sap import block_dense_matrices, sap_sweep


def arnoldi_reorth(apply, start, m):
    """m Arnoldi steps from start with two modified Gram-Schmidt passes per
    step: (basis list, Hbar (m+1, m), steps done; fewer if the new vector
    vanishes exactly)."""
    beta = np.sqrt(np.vdot(start, start).real)
    h = np.zeros((m + 1, m), dtype=np.complex128)
    v = [np.array(start, dtype=np.complex128) / beta]
    for j in range(m):
        w = apply(v[j])
        for _ in range(2):
            for i, q in enumerate(v):
                c = np.vdot(q, w)
                h[i, j] += c
                w = w - c * q
        h[j + 1, j] = np.sqrt(np.vdot(w, w).real)
        if h[j + 1, j] == 0.0:
            return v, h[:j + 2, :j + 1], j + 1
        v.append(w / h[j + 1, j])
    return v, h, m


def harmonic_ritz(apply, start, m):
    """Harmonic Ritz pairs of the operator from the Arnoldi space K_m(A, start).

    A subdiagonal entry h_{j+1,j} below 1e-12 max|h| ends the space there: it
    is then (numerically) invariant and its pairs are eigenpairs.

    Returns (theta, vectors): all pairs of the space, sorted by |theta|;
    vectors[k] is the unit-norm field V_m y_k (shape of ``start``)."""
    v, h, steps = arnoldi_reorth(apply, start, m)
    scale = np.max(np.abs(h)) if h.size else 0.0
    for j in range(steps):
        if abs(h[j + 1, j]) <= 1e-12 * scale:
            steps = j + 1
            h = h[:j + 2, :j + 1].copy()
            h[j + 1, j] = 0.0
            break
    hm = h[:steps, :steps]
    theta, y = scipy.linalg.eig(np.conj(h.T) @ h, np.conj(hm.T))
    order = np.argsort(np.abs(theta))
    theta, y = theta[order], y[:, order]
    vecs = []
    for k in range(steps):
        x = np.zeros_like(start, dtype=np.complex128)
        for j in range(steps):
            x = x + y[j, k] * v[j]
        vecs.append(x / np.sqrt(np.vdot(x, x).real))
    return theta, vecs


class Shifted:
    """The operator D - lambda (same lattice attributes as D)."""

    def __init__(self, op, lam):
        self.op, self.lam = op, complex(lam)
        self.lat, self.tail, self.dof_shape, self.dims = op.lat, op.tail, op.dof_shape, op.dims

    def apply(self, x):
        return self.op.apply(x) - self.lam * x


def shifted_smoothing(op, blocks, x, lam, iota, n_mr, exact=False):
    """S(lambda)^iota x: iota sweeps on (D - lambda) z = 0 from z = x, with
    n_MR MR steps per shifted block system (exact: dense solves of them)."""
    sop = Shifted(op, lam)
    dense = (block_dense_matrices(sop, blocks, 0), block_dense_matrices(sop, blocks, 1)) if exact else None
    z = np.array(x, dtype=np.complex128)
    for _ in range(iota):
        z = sap_sweep(sop, blocks, np.zeros_like(z), z, n_mr, exact=dense)
    return z


def reduce_vectors(apply, vectors, n):
    """Steps 4: orthonormalise the vectors, then the n combinations of smallest
    ||D x|| from the eigenvectors of (DV)^dagger DV.  Returns (new vectors,
    the n smallest eigenvalues of (DV)^dagger DV)."""
    q = orthonormalise([np.array(x) for x in vectors])
    w = np.stack([apply(x).ravel() for x in q], axis=1)
    g = np.conj(w.T) @ w
    mu, y = np.linalg.eigh(g)
    out = []
    for k in range(n):
        x = np.zeros_like(q[0])
        for j in range(len(q)):
            x = x + y[j, k] * q[j]
        out.append(x)
    return out, mu[:n]


def part2(mg, iota, start, n_mr=None, exact=False):
    """Run the second set-up part once on the oracle hierarchy ``mg``
    (oracle.mg.Multigrid with two or three levels, built by part 1) and
    rebuild it in place.  ``start``: the start vector of the Arnoldi process
    on the coarsest operator (shape of a coarsest-level field).  Returns the
    harmonic Ritz values used.

    Reading for three levels (the paper ran two): the procedure starts on the
    coarsest grid, as the paper says -- the harmonic Ritz vectors of the
    coarsest operator are interpolated through every level to the finest,
    smoothed and reduced there with the finest level's part-1 vectors; the
    finest P and the level-1 operator are rebuilt from the result, and the
    coarser level is then rebuilt as part 1 builds it (the new fine vectors
    restricted, its own smoother sweeps, P_1 and the coarsest operator)."""
    levels = mg.levels
    lev, coarsest = levels[0], levels[-1]
    n = len(lev.vectors)
    n_mr = mg.p["n_mr"] if n_mr is None else n_mr
    nc = int(np.prod(coarsest.op.lat)) * coarsest.op.dof_shape[0]
    theta, phis = harmonic_ritz(coarsest.op.apply, start, min(2 * n, nc))

    def to_fine(x):
        for l in range(len(levels) - 2, -1, -1):
            x = levels[l].agg.prolong(x)
        return x

    new = [shifted_smoothing(lev.op, lev.blocks, to_fine(phis[i]), theta[i], iota, n_mr, exact)
           for i in range(min(n, len(phis)))]
    vhat, _ = reduce_vectors(lev.op.apply, new + list(lev.vectors), n)
    nxt = mg.bootstrap_level(0, vhat, sweeps=0)          # P and the level-1 operator from the new vectors
    if nxt is not None:
        mg.bootstrap_level(1, nxt)                        # the coarser level rebuilt as part 1 builds it
    return theta[:n]
