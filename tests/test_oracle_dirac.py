"""Pins of the oracle's Dirac operator (Sec. 1, Eq. 1.1) against mathematics
that does not depend on the oracle's own formula: the Clifford algebra, the
closed-form free-field spectrum, gamma_5-hermiticity, gauge covariance and the
closed-form clover term of a uniform abelian field."""

import numpy as np
import pytest

import synth
from oracle import dirac
from oracle.dirac import WilsonClover, GAMMA, GAMMA5


def _match_spectra(a, b, tol):
    a = np.sort_complex(np.round(a, 9))
    b = np.sort_complex(np.round(b, 9))
    return np.max(np.abs(a - b)) < tol


def test_gamma_basis():
    for mu in range(4):
        for nu in range(4):
            ac = GAMMA[mu] @ GAMMA[nu] + GAMMA[nu] @ GAMMA[mu]
            assert np.allclose(ac, 2.0 * np.eye(4) * (mu == nu), atol=0)
        assert np.allclose(GAMMA[mu], np.conj(GAMMA[mu].T))
    assert np.allclose(GAMMA5, np.diag([1, 1, -1, -1]))


@pytest.mark.parametrize("dims,antiperiodic", [((3, 3, 2, 4), False), ((2, 3, 3, 4), True)])
def test_free_field_spectrum(dims, antiperiodic):
    """At U = 1 the clover term vanishes and the spectrum is
    m0 + sum(1 - cos p) +- i sqrt(sum sin^2 p), each 6-fold."""
    m0 = 0.137
    op = WilsonClover(synth.unit_gauge_field(dims), m0, c_sw=1.7, antiperiodic_t=antiperiodic)
    ev = np.linalg.eigvals(op.dense())
    ref = dirac.free_spectrum(dims, m0, antiperiodic)
    assert _match_spectra(ev, ref, 1e-8)


def test_free_field_plane_wave_small_dims_periodic_vs_antiperiodic_differ():
    """Sanity of the boundary flag: the two spectra differ."""
    dims = (2, 2, 2, 3)
    a = dirac.free_spectrum(dims, 0.1, False)
    b = dirac.free_spectrum(dims, 0.1, True)
    assert not _match_spectra(a, b, 1e-6)


def _random_op(dims=(4, 4, 2, 2), seed=11, m0=-0.3, c_sw=1.3, antiperiodic=False):
    return WilsonClover(synth.random_gauge_field(dims, 0.7, seed), m0, c_sw, antiperiodic)


@pytest.mark.parametrize("antiperiodic", [False, True])
def test_gamma5_hermiticity(antiperiodic):
    """gamma_5 D gamma_5 = D^dagger, i.e. <gamma_5 D gamma_5 x, y> = <x, D y>."""
    op = _random_op(antiperiodic=antiperiodic)
    x = synth.random_spinor(op.dims, 1)
    y = synth.random_spinor(op.dims, 2)
    lhs = np.vdot(op.apply_gamma5(op.apply(op.apply_gamma5(x))), y)
    rhs = np.vdot(x, op.apply(y))
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def test_gauge_covariance():
    """D(U^g) (g psi) = g (D(U) psi) with U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dagger."""
    dims = (4, 2, 4, 2)
    u = synth.random_gauge_field(dims, 0.6, 21)
    g = synth.random_gauge_rotation(dims, 22)
    psi = synth.random_spinor(dims, 23)
    op = WilsonClover(u, 0.05, 1.1)
    opg = WilsonClover(synth.gauge_transform(u, g), 0.05, 1.1)
    gpsi = np.einsum("...ab,...sb->...sa", g, psi)
    lhs = opg.apply(gpsi)
    rhs = np.einsum("...ab,...sb->...sa", g, op.apply(psi))
    assert np.max(np.abs(lhs - rhs)) < 1e-12


def test_pure_gauge_has_free_spectrum():
    """U_mu(x) = g(x) g(x+mu)^dagger is a gauge transform of U = 1."""
    dims = (3, 2, 2, 3)
    g = synth.random_gauge_rotation(dims, 5)
    u = synth.gauge_transform(synth.unit_gauge_field(dims), g)
    op = WilsonClover(u, -0.2, 1.9)
    ev = np.linalg.eigvals(op.dense())
    assert _match_spectra(ev, dirac.free_spectrum(dims, -0.2), 1e-8)


def _flux_field(dims, mu, nu, n):
    """Uniform abelian field in the mu-nu plane: every mu-nu plaquette equals
    exp(i f E), E = diag(1, -1, 0), f = 2 pi n / (L_mu L_nu) (periodic wrap made
    consistent by a twist on the last mu-slice)."""
    u = synth.unit_gauge_field(dims).copy()
    lat = dims[::-1]
    coords = np.meshgrid(*[np.arange(k) for k in lat], indexing="ij")  # t, z, y, x
    xm, xn = coords[3 - mu], coords[3 - nu]
    lm, ln = dims[mu], dims[nu]
    f = 2 * np.pi * n / (lm * ln)
    e = np.array([1.0, -1.0, 0.0])
    ph_nu = f * xm
    ph_mu = np.where(xm == lm - 1, -f * lm * xn, 0.0)
    for d, ph in ((nu, ph_nu), (mu, ph_mu)):
        u[..., d, :, :] = 0.0
        for c in range(3):
            u[..., d, c, c] = np.exp(1j * ph * e[c])
    return u, f


@pytest.mark.parametrize("mu,nu,sigma_diag", [(0, 1, (-1, 1, -1, 1)), (2, 3, (1, -1, -1, 1))])
def test_clover_uniform_abelian_closed_form(mu, nu, sigma_diag):
    """For the uniform flux field, Q = 4 exp(i f E), Fhat = i sin(f) E and
    A(x) = (4 + m0) - (c_sw/2) sin(f) sigma_{mu nu} (x) E everywhere, with
    sigma_xy = diag(-1, 1, -1, 1) and sigma_zt = diag(1, -1, -1, 1) in the
    chiral basis (worked out by hand from gamma_mu gamma_nu)."""
    dims = (4, 4, 4, 4)
    m0, c_sw = 0.2, 1.37
    u, f = _flux_field(dims, mu, nu, 1)
    op = WilsonClover(u, m0, c_sw)
    e = np.diag([1.0, -1.0, 0.0])
    expect = (4 + m0) * np.eye(12) - 0.5 * c_sw * np.sin(f) * np.kron(np.diag(sigma_diag), e)
    assert np.max(np.abs(op.a - expect)) < 1e-13


def test_clover_zero_at_unit_field():
    op = WilsonClover(synth.unit_gauge_field((2, 2, 2, 2)), 0.3, 2.0)
    assert np.max(np.abs(op.a - 4.3 * np.eye(12))) == 0.0


def test_clover_hermitian_chiral_blocks():
    """A(x) is Hermitian and commutes with gamma_5: two 6x6 chiral blocks."""
    op = _random_op()
    a = op.a
    assert np.max(np.abs(a - np.conj(np.swapaxes(a, -1, -2)))) < 1e-14
    assert np.max(np.abs(a[..., :6, 6:])) < 1e-15
    assert np.max(np.abs(a[..., 6:, :6])) < 1e-15


def test_clover_covariant():
    dims = (2, 4, 2, 4)
    u = synth.random_gauge_field(dims, 0.8, 31)
    g = synth.random_gauge_rotation(dims, 32)
    a = WilsonClover(u, 0.0, 1.0).a.reshape(dims[::-1] + (4, 3, 4, 3))
    ag = WilsonClover(synth.gauge_transform(u, g), 0.0, 1.0).a.reshape(dims[::-1] + (4, 3, 4, 3))
    expect = np.einsum("...ab,...sbtc,...dc->...satd", g, a, np.conj(g))
    assert np.max(np.abs(ag - expect)) < 1e-13


# --- planted mistakes: each must break one of the pins above -----------------

def test_planted_missing_dagger_breaks_gamma5_hermiticity(monkeypatch):
    orig = WilsonClover.hop

    def bad_hop(self, psi, mu, step):
        if step > 0:
            return orig(self, psi, mu, step)
        nb = dirac.shift(psi, mu, -1, 2)
        ub = dirac.shift(self.u[..., mu, :, :], mu, -1, 2)
        c = np.einsum("...ab,...sb->...sa", ub, nb)          # U instead of U^dagger
        return -0.5 * np.einsum("st,...tb->...sb", dirac.ONE4 + GAMMA[mu], c)

    monkeypatch.setattr(WilsonClover, "hop", bad_hop)
    op = _random_op()
    x = synth.random_spinor(op.dims, 1)
    y = synth.random_spinor(op.dims, 2)
    lhs = np.vdot(op.apply_gamma5(op.apply(op.apply_gamma5(x))), y)
    rhs = np.vdot(x, op.apply(y))
    assert abs(lhs - rhs) > 1e-3 * abs(rhs)


def test_planted_wrong_leaf_orientation_breaks_clover_closed_form(monkeypatch):
    orig = dirac.plaquette_sum

    def bad(u, mu, nu):
        q = orig(u, mu, nu)
        um, un = u[..., mu, :, :], u[..., nu, :, :]
        s = lambda f, d, k: dirac.shift(f, d, k, 2)
        leaf1 = um @ s(un, mu, 1) @ dirac.dagger(s(um, nu, 1)) @ dirac.dagger(un)
        return q - leaf1 + dirac.dagger(leaf1)                 # first leaf reversed

    monkeypatch.setattr(dirac, "plaquette_sum", bad)
    u, f = _flux_field((4, 4, 4, 4), 0, 1, 1)
    op = WilsonClover(u, 0.2, 1.37)
    e = np.diag([1.0, -1.0, 0.0])
    expect = 4.2 * np.eye(12) - 0.5 * 1.37 * np.sin(f) * np.kron(np.diag((-1, 1, -1, 1)), e)
    assert np.max(np.abs(op.a - expect)) > 1e-3


def test_planted_wrong_hop_sign_breaks_free_spectrum(monkeypatch):
    orig = WilsonClover.hop
    monkeypatch.setattr(WilsonClover, "hop", lambda self, psi, mu, step: -orig(self, psi, mu, step)
                        if mu == 2 else orig(self, psi, mu, step))
    dims = (2, 2, 3, 3)
    op = WilsonClover(synth.unit_gauge_field(dims), 0.1, 1.0)
    ev = np.linalg.eigvals(op.dense())
    assert not _match_spectra(ev, dirac.free_spectrum(dims, 0.1), 1e-6)
