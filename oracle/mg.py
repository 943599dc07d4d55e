"""The SAP-multilevel method: cycle, bootstrap set-up part 1 and outer solve (Sec. 3, Sec. 4).

Readings taken where the paper leaves the choice open (it says only that a
two-level method alternates smoother and subspace correction, recursing until
the coarsest operator is solved directly, Sec. 3):

* Cycle on level l for the residual equation A_l z = v:
  1. v_c = P^dagger v;
  2. e_c = approximate solve of A_{l+1} e_c = v_c: GMRES with a fixed number
     of iterations from zero on the coarsest level (Sec. 4: 12 iterations),
     otherwise a fixed number of flexible GMRES steps preconditioned by the
     cycle on level l+1;
  3. z = P e_c  (the subspace correction of Eq. 3.2 from z = 0);
  4. nu_post Schwarz sweeps (Algorithm 1) on A_l z = v starting from z.
  With one level the cycle is nu_post Schwarz sweeps from zero.
  The block systems of the sweeps are solved by n_MR minimal-residual steps
  (``block_solver="mr"``, the method's reading) or exactly by dense LU
  (``block_solver="exact"``: B_i = I D_i^{-1} I^T of Sec. 2), which makes the
  cycle a linear map whose error propagator the tests compare with the dense
  product of the Schwarz and coarse-correction propagators.
* Bootstrap set-up, part 1 (Sec. 3): N test vectors (random, drawn by the
  caller) -> per round: one Schwarz sweep of the smoother's iteration matrix
  on every vector (a sweep on A x = 0 started at x = v), then global modified
  Gram-Schmidt ("kept orthonormal"); after ``setup_iters`` rounds, P from the
  locally orthonormalised vectors, D_c = P^dagger A P; the smoothed vectors
  restricted with P^dagger start the next level.
* Outer solve: FGMRES(m) on D z = b with the cycle as right preconditioner,
  x0 = 0, ||b - D z|| <= tol ||b|| (Sec. 4).
"""

import numpy as np

from .sap import BlockDecomposition, block_dense_matrices, sap, sap_sweep
from .aggregation import Aggregation, orthonormalise
from .coarse import CoarseOperator
from .krylov import gmres_fixed, fgmres_fixed, fgmres


DEFAULTS = dict(
    n_levels=2,
    sap_block=((4, 4, 4, 4), (2, 2, 2, 2)),
    agg=((4, 4, 4, 4), (2, 2, 2, 2)),
    n_vec=(8, 8),
    setup_iters=3,
    n_mr=4,
    nu_post=2,
    coarse_iters=12,
    inner_iters=8,
    fgmres_m=20,
    tol=1e-10,
    maxiter=500,
    block_solver="mr",
)


class Level:
    def __init__(self, op, sap_block):
        self.op = op
        self.blocks = BlockDecomposition(op.dims, sap_block)
        self.agg = None
        self.vectors = None
        self.exact = None


class Multigrid:
    """Oracle multilevel hierarchy built by bootstrap set-up part 1.

    ``op``: the fine operator (oracle.dirac.WilsonClover);
    ``init_vectors``: list per non-coarsest level, or just the fine-level
    array (N, Lt, Lz, Ly, Lx, 4, 3) of initial test vectors (the coarser levels
    then start from the restricted smoothed vectors).
    """

    def __init__(self, op, params, init_vectors=None):
        p = dict(DEFAULTS)
        p.update(params)
        self.p = p
        if p["block_solver"] not in ("mr", "exact"):
            raise ValueError(f"unknown block solver {p['block_solver']!r}")
        self.levels = [Level(op, p["sap_block"][0])]
        init = init_vectors
        for l in range(p["n_levels"] - 1):
            init = self.bootstrap_level(l, init)

    def bootstrap_level(self, l, init, sweeps=None):
        """Bootstrap part 1 on level l from the initial vectors ``init``:
        ``sweeps`` (default setup_iters) rounds of one smoother sweep on
        A_l x = 0 per vector, each round followed by global modified
        Gram-Schmidt; then P_l from the locally orthonormalised vectors and
        A_{l+1} = P_l^dagger A_l P_l, which replaces level l+1 (and drops the
        levels below it).  Returns the next level's initial vectors, the
        smoothed vectors restricted with P_l^dagger (None on the last pair)."""
        p = self.p
        lev = self.levels[l]
        v = [np.array(x) for x in init[:p["n_vec"][l]]]
        for _ in range(p["setup_iters"] if sweeps is None else sweeps):
            v = [sap_sweep(lev.op, lev.blocks, np.zeros_like(x), x, p["n_mr"], self.exact_blocks(l)) for x in v]
            v = orthonormalise(v)
        lev.vectors = v
        lev.agg = Aggregation(lev.op.dims, p["agg"][l], lev.op.dof_shape).build(np.stack(v))
        cop = CoarseOperator(lev.op, lev.agg)
        del self.levels[l + 1:]
        if l + 1 < p["n_levels"] - 1:
            blk = p["sap_block"][l + 1] if l + 1 < len(p["sap_block"]) else p["sap_block"][-1]
            self.levels.append(Level(cop, blk))
            return [lev.agg.restrict(x) for x in v]
        nxt = Level.__new__(Level)
        nxt.op, nxt.blocks, nxt.agg, nxt.vectors, nxt.exact = cop, None, None, None, None
        self.levels.append(nxt)
        return None

    def exact_blocks(self, l):
        """Dense block matrices of both colours on level l when the block
        solver is exact (built once), else None (MR block solves)."""
        if self.p["block_solver"] != "exact":
            return None
        lev = self.levels[l]
        if getattr(lev, "exact", None) is None:
            lev.exact = tuple(block_dense_matrices(lev.op, lev.blocks, c) for c in (0, 1))
        return lev.exact

    def coarse_solve(self, l, vc):
        """Approximate solve on level l (l >= 1)."""
        p = self.p
        lev = self.levels[l]
        if l == len(self.levels) - 1:
            return gmres_fixed(lev.op.apply, vc, p["coarse_iters"])
        return fgmres_fixed(lev.op.apply, lambda w: self.cycle(l, w), vc, p["inner_iters"])

    def cycle(self, l, v):
        """Approximate A_l^{-1} v by the multilevel cycle."""
        p = self.p
        lev = self.levels[l]
        if len(self.levels) == 1:
            return sap(lev.op, lev.blocks, v, np.zeros_like(v), p["nu_post"], p["n_mr"], self.exact_blocks(l))
        vc = lev.agg.restrict(v)
        ec = self.coarse_solve(l + 1, vc)
        z = lev.agg.prolong(ec)
        return sap(lev.op, lev.blocks, v, z, p["nu_post"], p["n_mr"], self.exact_blocks(l))

    def solve(self, b):
        """Outer FGMRES(m) with the cycle as preconditioner."""
        p = self.p
        op = self.levels[0].op
        return fgmres(op.apply, lambda v: self.cycle(0, v), b, p["fgmres_m"], p["tol"], p["maxiter"])
