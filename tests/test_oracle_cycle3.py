"""Pins of the oracle's three-level method (Sec. 3: the two-level method
applied recursively to the coarse equation) against dense matrices built here
from the dense Dirac matrix and the dense interpolations alone.

Hierarchy: the 4^4 Wilson-clover lattice with 2^4 Schwarz blocks and
aggregates and N = 4 test vectors; level 1 is the 2^4 lattice of aggregates
(8 dof per site) with single-site Schwarz blocks and single-site aggregates
and N = 2; level 2 (64 dof) is solved by GMRES with as many steps as its
dimension, i.e. exactly.  Block solves are exact (dense LU).

With A_1 = P_0^dagger D P_0 and A_2 = P_1^dagger A_1 P_1 formed here, the
level-1 cycle is the linear map M_1 with 1 - M_1 A_1 = S_1^nu (1 - C_1 A_1)
(C_1 = P_1 A_2^{-1} P_1^dagger, S_1 the level-1 red-black Schwarz propagator;
the two-level identity that test_oracle_cycle.py pins on level 0).  The
level-1 solve inside the level-0 cycle is k steps of flexible GMRES from zero
preconditioned by M_1; with a fixed linear preconditioner that is GMRES on
A_1 M_1, so its result is M_1 y with y the minimiser of ||v_c - A_1 M_1 y||
over the Krylov space K_k(A_1 M_1, v_c), computed here by least squares on the
explicit power basis (not by the oracle's Arnoldi process).  The level-0 cycle
then gives x with x - D^{-1} v = S_0^nu (P_0 e_c - D^{-1} v).

Bootstrap on level 1 starts from the restriction of the final level-0 test
vectors; with exact block solves each round applies S_1 (sweep on A_1 x = 0)
and re-orthonormalises, so the level-1 vectors are the positive-diagonal QR
factor of S_1^nu P_0^dagger V_0.

Planted mistakes, each of which fails a pin: the level-1 solve without its
preconditioner, the level-1 cycle without its Schwarz sweep, and a level-1
bootstrap that starts from unrestricted random vectors."""

import numpy as np
import pytest

import synth
from oracle.dirac import WilsonClover
from oracle.mg import Multigrid
from oracle.krylov import fgmres_fixed

DIMS = (4, 4, 4, 4)
NVEC = (4, 2)
SETUP_ITERS = 2


def _positive_qr(a):
    q, r = np.linalg.qr(a)
    ph = np.diag(r) / np.abs(np.diag(r))
    return q * ph[None, :]


def _schwarz_level0(d):
    """S_0 = (1 - K_1 D)(1 - K_0 D) for 2^4 blocks of the 4^4 lattice, as a
    function on vectors (K_c: inverses of the colour-c diagonal blocks)."""
    lx, ly, lz, lt = DIMS
    sets = {0: {}, 1: {}}
    for t in range(lt):
        for z in range(lz):
            for y in range(ly):
                for x in range(lx):
                    site = ((t * lz + z) * ly + y) * lx + x
                    b = (x // 2, y // 2, z // 2, t // 2)
                    sets[sum(b) % 2].setdefault(b, []).extend(range(12 * site, 12 * site + 12))
    kinv = [[(np.array(ix), np.linalg.inv(d[np.ix_(ix, ix)])) for ix in sets[c].values()] for c in (0, 1)]

    def apply(x, nu=1):
        for _ in range(nu):
            for c in (0, 1):
                r = d @ x
                y = x.copy()
                for ix, inv in kinv[c]:
                    y[ix] -= inv @ r[ix]
                x = y
        return x
    return apply


def _schwarz_level1(a1):
    """S_1 = (1 - K_1 A_1)(1 - K_0 A_1) on the 2^4 level-1 lattice with
    single-site blocks: site s = ((t*2 + z)*2 + y)*2 + x has colour
    (x + y + z + t) mod 2, the parity of the bits of s."""
    n = a1.shape[0]
    dof = n // 16
    eye = np.eye(n, dtype=np.complex128)
    s = eye
    for c in (0, 1):
        k = np.zeros_like(a1)
        for site in range(16):
            if bin(site).count("1") % 2 == c:
                ix = np.arange(dof * site, dof * site + dof)
                k[np.ix_(ix, ix)] = np.linalg.inv(a1[np.ix_(ix, ix)])
        s = (eye - k @ a1) @ s
    return s


def _mg(op, init, inner_iters, cls=Multigrid):
    return cls(op, dict(n_levels=3, sap_block=((2, 2, 2, 2), (1, 1, 1, 1)), agg=((2, 2, 2, 2), (1, 1, 1, 1)),
                        n_vec=NVEC, setup_iters=SETUP_ITERS, nu_post=1, coarse_iters=16 * 2 * NVEC[1],
                        inner_iters=inner_iters, block_solver="exact"), init)


@pytest.fixture(scope="module")
def setup():
    op = WilsonClover(synth.random_gauge_field(DIMS, 0.4, 81), 0.05, 1.0)
    init = synth.test_vector_draw(DIMS, NVEC[0], 82)
    d = op.dense()
    return op, init, d, _schwarz_level0(d)


def _dense_hierarchy(mg, d):
    p0 = mg.levels[0].agg.dense()
    a1 = np.conj(p0.T) @ d @ p0
    p1 = mg.levels[1].agg.dense()
    a2 = np.conj(p1.T) @ a1 @ p1
    return p0, a1, p1, a2


def _expected_cycle(mg, d, s0, v, k):
    """The level-0 cycle of the three-level method, from dense matrices."""
    p0, a1, p1, a2 = _dense_hierarchy(mg, d)
    n1 = a1.shape[0]
    c1 = p1 @ np.linalg.solve(a2, np.conj(p1.T))
    s1 = _schwarz_level1(a1)
    m1 = (np.eye(n1) - s1 @ (np.eye(n1) - c1 @ a1)) @ np.linalg.inv(a1)       # nu_post = 1
    vc = np.conj(p0.T) @ v
    b = a1 @ m1
    basis = [vc]
    for _ in range(k - 1):
        basis.append(b @ basis[-1])
    kr = np.stack(basis, axis=1)
    coef, *_ = np.linalg.lstsq(b @ kr, vc, rcond=None)
    ec = m1 @ (kr @ coef)
    xs = np.linalg.solve(d, v)
    return xs + s0(p0 @ ec - xs)


def _cycle_error(mg, d, s0, k):
    err = 0.0
    for seed in (90, 91):
        v = synth.random_spinor(DIMS, seed)
        got = mg.cycle(0, v).ravel()
        want = _expected_cycle(mg, d, s0, v.ravel(), k)
        err = max(err, np.max(np.abs(got - want)) / np.max(np.abs(want)))
    return err


def test_level1_operator_is_the_galerkin_product(setup):
    op, init, d, s0 = setup
    mg = _mg(op, init, 1)
    p0, a1, p1, a2 = _dense_hierarchy(mg, d)
    assert np.max(np.abs(mg.levels[1].op.dense() - a1)) < 1e-12 * np.max(np.abs(a1))
    assert np.max(np.abs(mg.levels[2].op.dense() - a2)) < 1e-12 * np.max(np.abs(a2))


@pytest.mark.parametrize("k", [1, 2])
def test_three_level_cycle_matches_dense_composition(setup, k):
    op, init, d, s0 = setup
    assert _cycle_error(_mg(op, init, k), d, s0, k) < 1e-9


def test_level1_factors_are_not_trivial(setup):
    """The pin can only tell a wrong level-1 solve apart if M_1 is far from a
    multiple of the identity and its sweep and coarse correction matter."""
    op, init, d, s0 = setup
    mg = _mg(op, init, 1)
    p0, a1, p1, a2 = _dense_hierarchy(mg, d)
    n1 = a1.shape[0]
    s1 = _schwarz_level1(a1)
    e1 = np.eye(n1) - p1 @ np.linalg.solve(a2, np.conj(p1.T)) @ a1
    assert np.linalg.norm(s1 - np.eye(n1), 2) > 0.5
    assert np.linalg.norm(e1 - np.eye(n1), 2) > 0.5
    assert np.linalg.norm(s1 @ e1 - e1 @ s1, 2) > 0.1


def test_level1_vectors_are_qr_of_smoothed_restricted_vectors(setup):
    op, init, d, s0 = setup
    mg = _mg(op, init, 1)
    p0, a1, p1, a2 = _dense_hierarchy(mg, d)
    v0 = np.stack([v.ravel() for v in mg.levels[0].vectors[:NVEC[1]]], axis=1)
    x1 = np.conj(p0.T) @ v0
    q = _positive_qr(np.linalg.matrix_power(_schwarz_level1(a1), SETUP_ITERS) @ x1)
    got = np.stack([v.ravel() for v in mg.levels[1].vectors], axis=1)
    assert np.max(np.abs(got - q)) < 1e-9


# ---- planted mistakes ----------------------------------------------------------

class _UnpreconditionedLevel1(Multigrid):
    """Mistake: the level-1 solve is flexible GMRES without the level-1 cycle."""
    def coarse_solve(self, l, vc):
        if l == len(self.levels) - 1:
            return super().coarse_solve(l, vc)
        return fgmres_fixed(self.levels[l].op.apply, lambda w: w, vc, self.p["inner_iters"])


class _Level1WithoutSweep(Multigrid):
    """Mistake: the level-1 cycle stops after its coarse correction."""
    def cycle(self, l, v):
        if l != 1:
            return super().cycle(l, v)
        lev = self.levels[l]
        return lev.agg.prolong(self.coarse_solve(l + 1, lev.agg.restrict(v)))


class _Level1FromRandomVectors(Multigrid):
    """Mistake: the level-1 bootstrap starts from fresh random vectors rather
    than the restricted level-0 vectors."""
    def bootstrap_level(self, l, init, sweeps=None):
        if l == 1:
            rng = np.random.default_rng(5)
            init = [rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape) for x in init]
        return super().bootstrap_level(l, init, sweeps)


@pytest.mark.parametrize("cls", [_UnpreconditionedLevel1, _Level1WithoutSweep])
def test_planted_level1_cycle_mistakes_fail_the_pin(setup, cls):
    op, init, d, s0 = setup
    assert _cycle_error(_mg(op, init, 2, cls=cls), d, s0, 2) > 1e-3


def test_planted_level1_bootstrap_mistake_fails_the_pin(setup):
    op, init, d, s0 = setup
    mg = _mg(op, init, 1, cls=_Level1FromRandomVectors)
    p0, a1, p1, a2 = _dense_hierarchy(mg, d)
    v0 = np.stack([v.ravel() for v in mg.levels[0].vectors[:NVEC[1]]], axis=1)
    q = _positive_qr(np.linalg.matrix_power(_schwarz_level1(a1), SETUP_ITERS) @ (np.conj(p0.T) @ v0))
    got = np.stack([v.ravel() for v in mg.levels[1].vectors], axis=1)
    assert np.max(np.abs(got - q)) > 1e-3
