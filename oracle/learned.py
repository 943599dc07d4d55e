"""Gauge-covariant convolutional network that proposes near-kernel test
vectors for the set-up (the learned set-up of the multilevel solver; the
paper's own set-up is the bootstrap of Sec. 3, which this network is trained
to imitate and which stays the fallback).

TEST INFRASTRUCTURE ONLY: plain FP64 numpy restatement, used by the tests
and the smoke check, never by the library.

Definitions (fields of shape (C, Lt, Lz, Ly, Lx, 4, 3): C channels of spinor
fields; gauge field (Lt, Lz, Ly, Lx, 4, 3, 3); periodic boundaries):

* parallel transport along hop h (h = 0: none; h = 1 + 2 mu: +mu;
  h = 2 + 2 mu: -mu, the ordering of the coarse stencil's directions):
      (T_0 psi)(x) = psi(x),
      (T_{+mu} psi)(x) = U_mu(x) psi(x + mu),
      (T_{-mu} psi)(x) = U_mu(x - mu)^dagger psi(x - mu);
  T_{+mu} and T_{-mu} are each other's adjoints, and T_h (g psi) = g T_h psi
  under U_mu(x) -> g(x) U_mu(x) g(x + mu)^dagger;
* layer: out_a = sum_b sum_h W[a, b, h] T_h in_b, W[a, b, h] a complex 4 x 4
  matrix acting on the spin index (colour untouched), so every layer is
  gauge covariant;
* gate between layers, per channel and site (gauge invariant scaling):
      psi(x) -> psi(x) / sqrt(1 + |psi(x)|^2),  |.| the norm over spin and colour;
* network: eta (1 channel) -> layer -> gate -> layer -> gate -> ... -> layer
  (1 channel);
* loss: L = ||f(eta) - t||^2 / ||t||^2 with t the target vector (the
  bootstrap's smoothed vector for the same eta).

Gradients use the convention G_z = dL/dRe z + i dL/dIm z (steepest descent is
z -= lr G_z); for y = A x (A complex linear) G_x = A^dagger G_y, for
y = W z, G_W = G_y z^dagger.  The backward pass below is the reverse of each
forward step written out; its pin is a finite-difference test.
"""

import numpy as np

from .dirac import shift

N_HOPS = 9


def hop_of(h):
    """(mu, step) of hop h >= 1."""
    return (h - 1) // 2, (1 if (h - 1) % 2 == 0 else -1)


def adjoint_hop(h):
    """The hop whose transport is the adjoint of T_h."""
    if h == 0:
        return 0
    return h + 1 if (h - 1) % 2 == 0 else h - 1


def transport(u, psi, h):
    """T_h psi for psi of shape (..., Lt, Lz, Ly, Lx, 4, 3)."""
    if h == 0:
        return psi
    mu, step = hop_of(h)
    umu = u[..., mu, :, :]
    if step > 0:
        return np.einsum("...ab,...sb->...sa", umu, shift(psi, mu, 1, 2))
    ub = shift(umu, mu, -1, 2)
    return np.einsum("...ba,...sb->...sa", np.conj(ub), shift(psi, mu, -1, 2))


def layer(u, w, x):
    """out_a = sum_b sum_h W[a, b, h] T_h x_b; w: (Cout, Cin, 9, 4, 4), x: (Cin, ...)."""
    cout, cin = w.shape[:2]
    out = np.zeros((cout,) + x.shape[1:], dtype=np.complex128)
    for b in range(cin):
        for h in range(N_HOPS):
            t = transport(u, x[b], h)
            out += np.einsum("ast,...tc->a...sc", w[:, b, h], t)
    return out


def layer_backward(u, w, x, gy):
    """(G_x, G_W) of out = layer(u, w, x) given G_out."""
    cout, cin = w.shape[:2]
    gx = np.zeros_like(x, dtype=np.complex128)
    gw = np.zeros_like(w, dtype=np.complex128)
    for b in range(cin):
        for h in range(N_HOPS):
            t = transport(u, x[b], h)
            # G_W[a, b, h] = sum_{x, c} G_out_a(x)[s, c] conj(T_h x_b(x)[t, c])
            gw[:, b, h] = np.einsum("axsc,xtc->ast", gy.reshape(cout, -1, 4, 3), np.conj(t).reshape(-1, 4, 3))
            # G_{T_h x_b} = sum_a W[a, b, h]^dagger G_out_a; G_x_b += T_h^dagger of it
            gt = np.einsum("ats,a...tc->...sc", np.conj(w[:, b, h]), gy)
            gx[b] += transport(u, gt, adjoint_hop(h))
    return gx, gw


def gate(x):
    """psi / sqrt(1 + |psi|^2) per channel and site."""
    n = np.sum(np.abs(x) ** 2, axis=(-2, -1), keepdims=True)
    return x / np.sqrt(1.0 + n)


def gate_backward(x, gy):
    """G_x of y = gate(x): s G_y - (1 + n)^(-3/2) Re<G_y, x>_site x, s = (1 + n)^(-1/2)."""
    n = np.sum(np.abs(x) ** 2, axis=(-2, -1), keepdims=True)
    re = np.sum(np.real(np.conj(gy) * x), axis=(-2, -1), keepdims=True)
    return gy / np.sqrt(1.0 + n) - re * (1.0 + n) ** -1.5 * x


def forward(u, weights, eta):
    """Network output and the activations (inputs of every layer)."""
    x = eta[None] if eta.ndim == 6 else eta
    acts = []
    for i, w in enumerate(weights):
        acts.append(x)
        y = layer(u, w, x)
        x = gate(y) if i + 1 < len(weights) else y
    return x[0], acts


def loss(out, target):
    """||out - target||^2 / ||target||^2 and its gradient G_out."""
    tn = np.vdot(target, target).real
    d = out - target
    return np.vdot(d, d).real / tn, 2.0 * d / tn


def backward(u, weights, eta, target):
    """Loss and the gradients G_W of every layer."""
    out, acts = forward(u, weights, eta)
    val, g = loss(out, target)
    g = g[None]
    grads = [None] * len(weights)
    for i in range(len(weights) - 1, -1, -1):
        if i + 1 < len(weights):
            # the layer's output went through the gate
            y = layer(u, weights[i], acts[i])
            g = gate_backward(y, g)
        g, grads[i] = layer_backward(u, weights[i], acts[i], g)
    return val, grads


def init_weights(shapes, seed):
    """Seeded complex Gaussian weights, scaled by 1/sqrt(fan-in)."""
    rng = np.random.default_rng(seed)
    out = []
    for cout, cin in shapes:
        std = 1.0 / np.sqrt(cin * N_HOPS * 4)
        w = rng.normal(size=(cout, cin, N_HOPS, 4, 4)) + 1j * rng.normal(size=(cout, cin, N_HOPS, 4, 4))
        out.append(w * std / np.sqrt(2.0))
    return out
