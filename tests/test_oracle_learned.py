"""Pins of the learned set-up's oracle (gauge-covariant convolutional network):
finite-difference gradients, gauge covariance, reduction of one layer to the
(independently pinned) Wilson hopping term, identity layers, adjointness of
the transports."""

import numpy as np

import synth
from oracle import learned as L
from oracle.dirac import GAMMA, ONE4, WilsonClover

DIMS = (2, 2, 2, 4)          # (Lx, Ly, Lz, Lt)


def _field(seed=1, eps=0.7):
    return synth.random_gauge_field(DIMS, eps, seed)


def _spinors(seed, n):
    return synth.random_spinor(DIMS, seed, nvec=n)


def test_transports_are_adjoint_pairs():
    u = _field()
    a, b = _spinors(2, 2)
    for h in range(L.N_HOPS):
        lhs = np.vdot(L.transport(u, a, h), b)
        rhs = np.vdot(a, L.transport(u, b, L.adjoint_hop(h)))
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_identity_layer():
    u = _field()
    x = _spinors(3, 3)
    w = np.zeros((3, 3, L.N_HOPS, 4, 4), dtype=np.complex128)
    for a in range(3):
        w[a, a, 0] = np.eye(4)
    assert np.max(np.abs(L.layer(u, w, x) - x)) < 1e-15


def test_layer_reproduces_wilson_hopping_term():
    """W[+mu] = -(1 - gamma_mu)/2, W[-mu] = -(1 + gamma_mu)/2: the layer is D - A."""
    u = _field(4)
    op = WilsonClover(u, 0.3, 1.0)
    psi = _spinors(5, 1)[0]
    w = np.zeros((1, 1, L.N_HOPS, 4, 4), dtype=np.complex128)
    for mu in range(4):
        w[0, 0, 1 + 2 * mu] = -0.5 * (ONE4 - GAMMA[mu])
        w[0, 0, 2 + 2 * mu] = -0.5 * (ONE4 + GAMMA[mu])
    out = L.layer(u, w, psi[None])[0]
    ref = op.apply(psi) - op.local(psi)
    assert np.max(np.abs(out - ref)) < 1e-13 * np.max(np.abs(ref))


def test_network_is_gauge_covariant():
    u = _field(6)
    g = synth.random_gauge_rotation(DIMS, 7)
    ug = synth.gauge_transform(u, g)
    eta = _spinors(8, 1)[0]
    ws = L.init_weights([(3, 1), (3, 3), (1, 3)], 9)
    out, _ = L.forward(u, ws, eta)
    rot = lambda f: np.einsum("...ab,...sb->...sa", g, f)
    outg, _ = L.forward(ug, ws, rot(eta))
    assert np.max(np.abs(outg - rot(out))) < 1e-12 * np.max(np.abs(out))


def test_gate_is_a_radial_squashing():
    x = _spinors(10, 2) * 3.0
    y = L.gate(x)
    nx = np.sqrt(np.sum(np.abs(x) ** 2, axis=(-2, -1)))
    ny = np.sqrt(np.sum(np.abs(y) ** 2, axis=(-2, -1)))
    assert np.allclose(ny, nx / np.sqrt(1 + nx ** 2), rtol=1e-14)
    # same direction at every site
    dots = np.sum(np.conj(x) * y, axis=(-2, -1))
    assert np.allclose(np.imag(dots), 0, atol=1e-12) and np.all(np.real(dots) > 0)


def _params_dot(g, d):
    return sum(np.real(np.vdot(a, b)) for a, b in zip(g, d))


def test_gradients_match_finite_differences():
    u = _field(11)
    eta = _spinors(12, 1)[0]
    target = _spinors(13, 1)[0]
    ws = L.init_weights([(3, 1), (3, 3), (1, 3)], 14)
    val, grads = L.backward(u, ws, eta, target)
    rng = np.random.default_rng(15)
    for trial in range(3):
        d = [rng.normal(size=w.shape) + 1j * rng.normal(size=w.shape) for w in ws]
        e = 1e-6
        lp = L.loss(L.forward(u, [w + e * dd for w, dd in zip(ws, d)], eta)[0], target)[0]
        lm = L.loss(L.forward(u, [w - e * dd for w, dd in zip(ws, d)], eta)[0], target)[0]
        fd = (lp - lm) / (2 * e)
        an = _params_dot(grads, d)
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (trial, fd, an)


def test_loss_gradient_in_the_output():
    """G_out of the loss against finite differences in one output entry (real and imaginary)."""
    out = _spinors(16, 1)[0]
    t = _spinors(17, 1)[0]
    val, g = L.loss(out, t)
    idx = (1, 0, 1, 0, 2, 1)
    for unit in (1.0, 1j):
        e = 1e-6
        o1 = out.copy(); o1[idx] += e * unit
        o2 = out.copy(); o2[idx] -= e * unit
        fd = (L.loss(o1, t)[0] - L.loss(o2, t)[0]) / (2 * e)
        an = np.real(np.conj(g[idx]) * unit)
        assert abs(fd - an) < 1e-8
