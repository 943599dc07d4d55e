"""Pins of the oracle's multilevel cycle and of its bootstrap set-up part 1
(Sec. 3, Eq. 3.2; Sec. 2, Algorithm 1) against dense error propagators built
here from the dense Dirac matrix alone.

With exact block solves (B_i = I D_i^{-1} I^T, Sec. 2) and an exact coarse
solve the cycle is a linear map M, and the method fixes its error propagator:
the coarse-grid correction of Eq. 3.2 is C = P (P^dagger D P)^{-1} P^dagger,
one red-black Schwarz sweep propagates errors by
S = (1 - K_1 D)(1 - K_0 D) with K_c = sum over the colour-c blocks of B_i
(colour 0 first), and the cycle "coarse correction from zero, then nu_post
sweeps" gives 1 - M D = S^nu_post (1 - C D) and M = C when nu_post = 0.
Every matrix on the right is formed here with numpy from op.dense() and the
block index sets computed from the coordinates, not by the oracle's Schwarz,
restriction or Krylov code, so a dropped term, a wrong start vector, a wrong
ordering or a wrong sign in Multigrid.cycle fails one of these tests; each
such mistake is planted below and shown to fail.

Bootstrap part 1 with exact block solves is also linear between its
orthonormalisations: x -> S x per sweep (the smoother's iteration matrix on
D x = 0), and modified Gram-Schmidt after every sweep.  Re-orthonormalising
after each sweep changes the vectors by an upper-triangular factor with a
positive diagonal, so after nu sweeps the vectors are the Q factor (positive
real diagonal) of the thin QR of S^nu X, X the initial vectors.
"""

import numpy as np
import pytest

import synth
from oracle.dirac import WilsonClover
from oracle.mg import Multigrid
from oracle.sap import sap

DIMS = (4, 4, 4, 4)                 # (Lx, Ly, Lz, Lt)
BLOCK = 2                           # 2^4 Schwarz blocks and aggregates
NVEC = 4


def _block_index_sets(dims, bs):
    """Dof indices of every block, per colour, from the site coordinates
    (canonical order: x fastest, then 12 spin-colour dof per site)."""
    lx, ly, lz, lt = dims
    sets = {0: {}, 1: {}}
    for t in range(lt):
        for z in range(lz):
            for y in range(ly):
                for x in range(lx):
                    site = ((t * lz + z) * ly + y) * lx + x
                    b = (x // bs, y // bs, z // bs, t // bs)
                    colour = sum(b) % 2
                    sets[colour].setdefault(b, []).extend(range(12 * site, 12 * site + 12))
    return sets


class _SchwarzPropagator:
    """S = (1 - K_1 D)(1 - K_0 D), K_c the direct sum of the inverses of the
    colour-c diagonal blocks of D, applied to vectors or to n x k matrices
    (the dense n x n product is never formed)."""

    def __init__(self, d, dims, bs):
        self.d = d
        self.kinv = []
        for colour in (0, 1):
            blocks = []
            for idx in _block_index_sets(dims, bs)[colour].values():
                ix = np.array(idx)
                blocks.append((ix, np.linalg.inv(d[np.ix_(ix, ix)])))
            self.kinv.append(blocks)

    def __call__(self, x, nu=1):
        for _ in range(nu):
            for colour in (0, 1):
                r = self.d @ x
                y = x.copy()
                for ix, inv in self.kinv[colour]:
                    y[ix] -= inv @ r[ix]
                x = y
        return x


@pytest.fixture(scope="module")
def setup():
    op = WilsonClover(synth.random_gauge_field(DIMS, 0.4, 81), 0.05, 1.0)
    init = synth.test_vector_draw(DIMS, NVEC, 82)
    d = op.dense()
    s = _SchwarzPropagator(d, DIMS, BLOCK)
    return op, init, d, s


def _mg(op, init, nu_post, setup_iters=2, cls=Multigrid):
    ncoarse = (DIMS[0] // BLOCK) ** 4 * 2 * NVEC      # coarse dimension: exact GMRES
    return cls(op, dict(n_levels=2, sap_block=((BLOCK,) * 4,), agg=((BLOCK,) * 4,), n_vec=(NVEC,),
                        setup_iters=setup_iters, nu_post=nu_post, coarse_iters=ncoarse,
                        block_solver="exact"), init)


def _coarse_correction(mg, d):
    """x -> C x = P (P^dagger D P)^{-1} P^dagger x, from the dense P and D."""
    p = mg.levels[0].agg.dense()
    ph = np.conj(p.T)
    dc = ph @ d @ p
    return lambda x: p @ np.linalg.solve(dc, ph @ x)


def _cycle_matrix_error(mg, d, s, nu_post, xs):
    """max over the probe vectors x of |(x - M D x) - S^nu (1 - C D) x| / |x|."""
    c = _coarse_correction(mg, d)
    err = 0.0
    for x in xs:
        xv = x.ravel()
        lhs = xv - mg.cycle(0, (d @ xv).reshape(x.shape)).ravel()
        rhs = s(xv - c(d @ xv), nu_post)
        err = max(err, np.max(np.abs(lhs - rhs)) / np.max(np.abs(xv)))
    return err


def _probes():
    return [synth.random_spinor(DIMS, 90 + k) for k in range(2)]


def test_cycle_without_smoothing_is_the_coarse_correction(setup):
    """nu_post = 0: M v = P (P^dagger D P)^{-1} P^dagger v (Eq. 3.2)."""
    op, init, d, s = setup
    mg = _mg(op, init, 0)
    c = _coarse_correction(mg, d)
    for v in _probes():
        got = mg.cycle(0, v).ravel()
        want = c(v.ravel())
        assert np.max(np.abs(got - want)) < 1e-10 * np.max(np.abs(want))


@pytest.mark.parametrize("nu_post", [1, 2])
def test_cycle_error_propagator(setup, nu_post):
    """1 - M D = S^nu_post (1 - C D), applied to probe vectors."""
    op, init, d, s = setup
    assert _cycle_matrix_error(_mg(op, init, nu_post), d, s, nu_post, _probes()) < 1e-10


def _norm_lower_bound(apply, n, seed, steps=12):
    """A lower bound on the spectral norm of a linear map: ||A w|| / ||w|| for
    the power-iteration vectors w (each ratio is at most ||A||_2)."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    best = 0.0
    for _ in range(steps):
        w = w / np.linalg.norm(w)
        aw = apply(w)
        best = max(best, np.linalg.norm(aw))
        w = aw
    return best


def test_propagator_factors_are_not_trivial(setup):
    """The pin can only fail a wrong cycle if S and 1 - C D are far from the
    identity and do not commute (lower bounds of the spectral norms)."""
    op, init, d, s = setup
    mg = _mg(op, init, 1)
    c = _coarse_correction(mg, d)
    n = d.shape[0]
    e = lambda x: x - c(d @ x)
    assert _norm_lower_bound(lambda x: s(x) - x, n, 1) > 0.5
    assert _norm_lower_bound(lambda x: e(x) - x, n, 2) > 0.5
    assert _norm_lower_bound(lambda x: s(e(x)) - e(s(x)), n, 3) > 0.1


# ---- planted mistakes: each must fail the propagator pin --------------------

class _SmoothFromZero(Multigrid):
    """Mistake: the Schwarz sweeps start from 0 instead of P e_c."""
    def cycle(self, l, v):
        lev = self.levels[l]
        self.coarse_solve(l + 1, lev.agg.restrict(v))
        return sap(lev.op, lev.blocks, v, np.zeros_like(v), self.p["nu_post"], self.p["n_mr"],
                   self.exact_blocks(l))


class _PostCorrection(Multigrid):
    """Mistake: smooth first, then add the coarse correction of the new residual."""
    def cycle(self, l, v):
        lev = self.levels[l]
        z = sap(lev.op, lev.blocks, v, np.zeros_like(v), self.p["nu_post"], self.p["n_mr"],
                self.exact_blocks(l))
        r = v - lev.op.apply(z)
        return z + lev.agg.prolong(self.coarse_solve(l + 1, lev.agg.restrict(r)))


class _SmoothZeroRhs(Multigrid):
    """Mistake: the sweeps solve D z = 0 from P e_c instead of D z = v."""
    def cycle(self, l, v):
        lev = self.levels[l]
        z = lev.agg.prolong(self.coarse_solve(l + 1, lev.agg.restrict(v)))
        return sap(lev.op, lev.blocks, np.zeros_like(v), z, self.p["nu_post"], self.p["n_mr"],
                   self.exact_blocks(l))


class _ConjugateRestriction(Multigrid):
    """Mistake: the restriction omits the complex conjugate of the test vectors."""
    def cycle(self, l, v):
        lev = self.levels[l]
        agg = lev.agg
        ra = agg.to_aggregates(v)
        vc = np.einsum("ksxl,sxl->sxk", agg.q, ra).reshape(agg.clat + (2 * agg.nvec,))
        z = agg.prolong(self.coarse_solve(l + 1, vc))
        return sap(lev.op, lev.blocks, v, z, self.p["nu_post"], self.p["n_mr"], self.exact_blocks(l))


@pytest.mark.parametrize("cls", [_SmoothFromZero, _PostCorrection, _SmoothZeroRhs, _ConjugateRestriction])
def test_planted_cycle_mistakes_fail_the_pin(setup, cls):
    op, init, d, s = setup
    assert _cycle_matrix_error(_mg(op, init, 1, cls=cls), d, s, 1, _probes()) > 1e-3


# ---- bootstrap set-up part 1 ------------------------------------------------

def _positive_qr(a):
    q, r = np.linalg.qr(a)
    ph = np.diag(r) / np.abs(np.diag(r))
    return q * ph[None, :]


@pytest.mark.parametrize("nu", [1, 2])
def test_bootstrap_vectors_are_qr_of_smoothed_initial_vectors(setup, nu):
    op, init, d, s = setup
    mg = _mg(op, init, 1, setup_iters=nu)
    x = np.stack([v.ravel() for v in init[:NVEC]], axis=1)
    q = _positive_qr(s(x, nu))
    got = np.stack([v.ravel() for v in mg.levels[0].vectors], axis=1)
    assert np.max(np.abs(got - q)) < 1e-9


class _InverseIterationBootstrap(Multigrid):
    """Mistake: each set-up sweep solves D x = v from 0 (the alternative
    reading) instead of applying the iteration matrix to v."""
    def __init__(self, op, params, init_vectors=None):
        import oracle.mg as mgmod
        orig = mgmod.sap_sweep
        mgmod.sap_sweep = lambda o, blk, b, z, n, exact=None: orig(o, blk, z, np.zeros_like(z), n, exact)
        try:
            super().__init__(op, params, init_vectors)
        finally:
            mgmod.sap_sweep = orig


def test_planted_bootstrap_mistake_fails_the_pin(setup):
    op, init, d, s = setup
    mg = _mg(op, init, 1, setup_iters=1, cls=_InverseIterationBootstrap)
    x = np.stack([v.ravel() for v in init[:NVEC]], axis=1)
    q = _positive_qr(s(x))
    got = np.stack([v.ravel() for v in mg.levels[0].vectors], axis=1)
    assert np.max(np.abs(got - q)) > 1e-3


def test_mr_cycle_equals_exact_cycle_when_mr_converges(setup):
    """The default (MR block solver) cycle tends to the exact one as n_MR
    grows: the two share every step but the block solve."""
    op, init, d, s = setup
    v = _probes()[0]
    mg = _mg(op, init, 1, setup_iters=1)
    ex = mg.cycle(0, v)
    errs = []
    for n_mr in (2, 40):
        mg.p = dict(mg.p, block_solver="mr", n_mr=n_mr)          # same hierarchy, MR block solves
        errs.append(np.max(np.abs(mg.cycle(0, v) - ex)) / np.max(np.abs(ex)))
    assert errs[1] < 1e-6 < errs[0]
