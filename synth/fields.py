"""Seeded synthetic gauge and spinor fields.

Gauge links follow the recipe U_mu(x) = exp(i eps H_mu(x)) with H traceless
Hermitian, H = (M + M^dagger)/2 - tr(.)/3, where M has i.i.d. complex Gaussian
entries (N(0,1) + i N(0,1))/sqrt(2).  The exponential is the plain PyTorch CPU
matrix exponential in float64; for traceless Hermitian H the result is in
SU(3) to rounding.  The paper's gauge ensembles (Tables 1 and 2) are not
available; these fields stand in for them.
"""

import numpy as np
import torch

from .rng import (
    counter_u64, uniform_pm1, gaussian,
    STREAM_GAUGE, STREAM_SPINOR, STREAM_TESTVEC, STREAM_GAUGE_TRANSFORM, STREAM_Z2,
)


def spinor_shape(dims):
    lx, ly, lz, lt = dims
    return (lt, lz, ly, lx, 4, 3)


def gauge_shape(dims):
    lx, ly, lz, lt = dims
    return (lt, lz, ly, lx, 4, 3, 3)


def _volume(dims):
    return int(np.prod(dims))


def _su3_exp(g, eps):
    """SU(3) matrices exp(i eps H) from rows of 18 Gaussian deviates."""
    n = g.shape[0]
    m = (g[:, 0::2] + 1j * g[:, 1::2]).reshape(n, 3, 3) / np.sqrt(2.0)
    h = 0.5 * (m + np.conj(np.swapaxes(m, 1, 2)))
    tr = np.trace(h, axis1=1, axis2=2).real / 3.0
    h = h - tr[:, None, None] * np.eye(3)[None]
    t = torch.from_numpy(1j * eps * h)
    return torch.linalg.matrix_exp(t).numpy()


def random_su3(n, eps, seed, stream=STREAM_GAUGE, offset=0, chunk=1 << 19):
    """n matrices exp(i eps H); matrix l uses Gaussian indices 18*(offset+l)+0..17."""
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        l = np.arange(offset + s, offset + e, dtype=np.uint64)
        j = l[:, None] * np.uint64(18) + np.arange(18, dtype=np.uint64)[None, :]
        out[s:e] = _su3_exp(gaussian(seed, stream, j), eps)
    return out


def random_gauge_field(dims, eps, seed):
    """Gauge field U_mu(x) = exp(i eps H_mu(x)); link (site, mu) is matrix site*4+mu."""
    v = _volume(dims)
    u = random_su3(4 * v, eps, seed, STREAM_GAUGE)
    return u.reshape(gauge_shape(dims))


def unit_gauge_field(dims):
    """The free field U_mu(x) = 1."""
    u = np.zeros(gauge_shape(dims), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def gauge_transform(u, g):
    """U^g_mu(x) = g(x) U_mu(x) g(x + mu)^dagger for g of shape (Lt,Lz,Ly,Lx,3,3)."""
    out = np.empty_like(u)
    for mu in range(4):
        axis = 3 - mu
        g_fwd = np.roll(g, -1, axis=axis)
        out[..., mu, :, :] = g @ u[..., mu, :, :] @ np.conj(np.swapaxes(g_fwd, -1, -2))
    return out


def random_gauge_rotation(dims, seed, eps=1.0):
    """Random SU(3) field g(x), shape (Lt, Lz, Ly, Lx, 3, 3)."""
    lx, ly, lz, lt = dims
    v = _volume(dims)
    return random_su3(v, eps, seed, STREAM_GAUGE_TRANSFORM).reshape(lt, lz, ly, lx, 3, 3)


def random_spinor(dims, seed, nvec=None):
    """Complex Gaussian spinor(s): real and imaginary parts i.i.d. N(0, 1)."""
    v = _volume(dims)
    n = 1 if nvec is None else nvec
    j = np.arange(n * v * 24, dtype=np.uint64)
    g = gaussian(seed, STREAM_SPINOR, j).reshape(n, v * 12, 2)
    psi = (g[..., 0] + 1j * g[..., 1]).reshape((n,) + spinor_shape(dims))
    return psi[0] if nvec is None else psi


def uniform_spinor(dims, seed, nvec, stream):
    """Spinors with real and imaginary parts uniform_pm1 of counters
    i = ((k*V + site)*12 + spin*3 + colour)*2 + (0 for re, 1 for im)."""
    v = _volume(dims)
    i = np.arange(nvec * v * 24, dtype=np.uint64)
    x = uniform_pm1(counter_u64(seed, stream, i)).reshape(nvec, v * 12, 2)
    return (x[..., 0] + 1j * x[..., 1]).reshape((nvec,) + spinor_shape(dims))


def test_vector_draw(dims, nvec, seed):
    """The random initial test vectors of the bootstrap set-up (uniform in [-1,1)
    per real component, stream STREAM_TESTVEC).  The CUDA library draws the same
    values from the same counters when no initial vectors are supplied."""
    return uniform_spinor(dims, seed, nvec, STREAM_TESTVEC)


def z2_spinor(dims, seed):
    """Z2 noise: every real component +1 or -1 (top bit of counter i), imaginary 0."""
    v = _volume(dims)
    i = np.arange(v * 12, dtype=np.uint64)
    bit = (counter_u64(seed, STREAM_Z2, i) >> np.uint64(63)).astype(np.float64)
    return (1.0 - 2.0 * bit).astype(np.complex128).reshape(spinor_shape(dims))


def point_sources(dims, origin=(0, 0, 0, 0)):
    """The 12 spin-colour point sources at ``origin`` = (x, y, z, t)."""
    src = np.zeros((12,) + spinor_shape(dims), dtype=np.complex128)
    x, y, z, t = origin
    for s in range(4):
        for c in range(3):
            src[s * 3 + c, t, z, y, x, s, c] = 1.0
    return src
