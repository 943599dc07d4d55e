"""Clover-improved Wilson-Dirac operator (Sec. 1, Eq. 1.1).

The paper names the operator (Wilson discretisation D = D(U) + m with clover
improvement and coefficient c_sw) but prints no formula.  Reading taken here,
the standard Sheikholeslami-Wohlert form:

    (D psi)(x) = (4 + m0) psi(x)
                 - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                              + (1 + gamma_mu) U_mu(x - mu)^dagger psi(x - mu) ]
                 + c_sw (i/2) sum_{mu<nu} sigma_{mu nu} Fhat_{mu nu}(x) psi(x)

with sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu] and
Fhat_{mu nu}(x) = (Q_{mu nu}(x) - Q_{mu nu}(x)^dagger) / 8, Q the sum of the four
plaquettes of the mu-nu plane that start and end at x, all traversed in the
same (mu first, then nu) sense.  Gamma matrices are in the chiral basis,
gamma_k = [[0, -i s_k], [i s_k, 0]] (k = 1, 2, 3; s_k the Pauli matrices),
gamma_4 = [[0, 1], [1, 0]], gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 =
diag(1, 1, -1, -1).  Boundary conditions are periodic; optionally the
fermion field is antiperiodic in t (a factor -1 on every hop that crosses the
t boundary).

This oracle deliberately uses the full 4x4 gamma matrices and a full 12x12
clover matrix per site: no spin projection, no chiral-block packing.
"""

import numpy as np

_S1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_S2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_S3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)

#: gamma_mu for mu = 0..3 <-> x, y, z, t (the paper's gamma_1..gamma_4)
GAMMA = [np.block([[_Z2, -1j * s], [1j * s, _Z2]]) for s in (_S1, _S2, _S3)] + \
        [np.block([[_Z2, _I2], [_I2, _Z2]])]
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ONE4 = np.eye(4, dtype=np.complex128)


def sigma(mu, nu):
    """sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu]."""
    return 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])


def dagger(m):
    return np.conj(np.swapaxes(m, -1, -2))


def shift(f, mu, step, tail):
    """f(x + step * mu) for a field of shape (..., Lt, Lz, Ly, Lx, *tail)."""
    return np.roll(f, -step, axis=-tail - 1 - mu)


def plaquette_sum(u, mu, nu):
    """Q_{mu nu}(x): the four mu-nu plaquettes at x, all in the same sense.

    Leaves (corners visited in order):
      x -> x+mu -> x+mu+nu -> x+nu -> x
      x -> x+nu -> x+nu-mu -> x-mu -> x
      x -> x-mu -> x-mu-nu -> x-nu -> x
      x -> x-nu -> x-nu+mu -> x+mu -> x
    """
    um = u[..., mu, :, :]
    un = u[..., nu, :, :]
    s = lambda f, d, k: shift(f, d, k, 2)
    q = um @ s(un, mu, 1) @ dagger(s(um, nu, 1)) @ dagger(un)
    q = q + un @ dagger(s(s(um, nu, 1), mu, -1)) @ dagger(s(un, mu, -1)) @ s(um, mu, -1)
    q = q + dagger(s(um, mu, -1)) @ dagger(s(s(un, mu, -1), nu, -1)) @ s(s(um, mu, -1), nu, -1) \
        @ s(un, nu, -1)
    q = q + dagger(s(un, nu, -1)) @ s(um, nu, -1) @ s(s(un, nu, -1), mu, 1) @ dagger(um)
    return q


def field_strength(u, mu, nu):
    """Fhat_{mu nu}(x) = (Q - Q^dagger)/8 (anti-Hermitian 3x3 per site)."""
    q = plaquette_sum(u, mu, nu)
    return (q - dagger(q)) / 8.0


def clover_matrix(u, m0, c_sw):
    """A(x) = (4 + m0) 1 + c_sw (i/2) sum_{mu<nu} sigma_{mu nu} (x) Fhat_{mu nu}(x).

    Returns an array (Lt, Lz, Ly, Lx, 12, 12) indexed [spin*3 + colour].
    """
    lat = u.shape[:4]
    a = np.zeros(lat + (4, 3, 4, 3), dtype=np.complex128)
    for mu in range(4):
        for nu in range(mu + 1, 4):
            f = field_strength(u, mu, nu)
            a += 0.5j * c_sw * np.einsum("st,...ab->...satb", sigma(mu, nu), f)
    a = a.reshape(lat + (12, 12))
    a += (4.0 + m0) * np.eye(12)
    return a


class WilsonClover:
    """The operator D of Eq. 1.1 on a periodic 4D lattice.

    ``u``: gauge field (Lt, Lz, Ly, Lx, 4, 3, 3); ``m0``: bare mass;
    ``c_sw``: clover coefficient; ``antiperiodic_t``: fermion boundary sign in t.
    Fields it acts on have shape (..., Lt, Lz, Ly, Lx, 4, 3).
    """

    tail = 2

    def __init__(self, u, m0, c_sw, antiperiodic_t=False):
        self.u = np.asarray(u, dtype=np.complex128)
        self.lat = self.u.shape[:4]                # (Lt, Lz, Ly, Lx)
        self.dims = self.lat[::-1]                 # (Lx, Ly, Lz, Lt)
        self.m0 = float(m0)
        self.c_sw = float(c_sw)
        self.antiperiodic_t = bool(antiperiodic_t)
        self.a = clover_matrix(self.u, m0, c_sw)
        self.dof_shape = (4, 3)

    # -- the pieces of D ------------------------------------------------------
    def _bc(self, f, mu, step):
        """Apply the t-boundary sign to a field already shifted by step*mu."""
        if mu != 3 or not self.antiperiodic_t:
            return f
        f = f.copy()
        lt = self.lat[0]
        if step > 0:
            f[..., lt - 1, :, :, :, :, :] *= -1.0   # psi(x+t) with x_t = Lt-1 wrapped
        else:
            f[..., 0, :, :, :, :, :] *= -1.0        # psi(x-t) with x_t = 0 wrapped
        return f

    def local(self, psi):
        """The site-diagonal part A(x) psi(x)."""
        sh = psi.shape
        p = psi.reshape(sh[:-2] + (12, 1))
        return np.matmul(self.a, p).reshape(sh)

    def hop(self, psi, mu, step):
        """One hopping term of D.

        step = +1: -1/2 (1 - gamma_mu) U_mu(x) psi(x + mu)
        step = -1: -1/2 (1 + gamma_mu) U_mu(x - mu)^dagger psi(x - mu)
        """
        umu = self.u[..., mu, :, :]
        if step > 0:
            nb = self._bc(shift(psi, mu, 1, 2), mu, 1)
            c = np.matmul(nb, np.swapaxes(umu, -1, -2))            # c[s, a] = sum_b U[a, b] psi[s, b]
            spin = ONE4 - GAMMA[mu]
        else:
            nb = self._bc(shift(psi, mu, -1, 2), mu, -1)
            ub = shift(umu, mu, -1, 2)
            c = np.matmul(nb, np.conj(ub))                         # c[s, a] = sum_b conj(U[b, a]) psi[s, b]
            spin = ONE4 + GAMMA[mu]
        return -0.5 * np.matmul(spin, c)

    def apply(self, psi):
        """D psi."""
        out = self.local(psi)
        for mu in range(4):
            out = out + self.hop(psi, mu, 1) + self.hop(psi, mu, -1)
        return out

    def apply_gamma5(self, psi):
        return np.einsum("st,...tb->...sb", GAMMA5, psi)

    def apply_dagger(self, psi):
        """D^dagger psi, as gamma5 D gamma5 psi: D is gamma5-Hermitian (the
        hopping projectors satisfy gamma5 (1 - gamma_mu) gamma5 = 1 + gamma_mu,
        and the clover term is Hermitian and commutes with gamma5)."""
        return self.apply_gamma5(self.apply(self.apply_gamma5(psi)))

    def chirality_of_dof(self):
        """Chirality index (0: gamma_5 = +1, spins 0,1; 1: spins 2,3) per dof."""
        return np.repeat(np.array([0, 0, 1, 1]), 3).reshape(4, 3)

    def dense(self):
        """The full matrix of D (small lattices only), index site*12 + spin*3 + colour."""
        n = int(np.prod(self.lat)) * 12
        eye = np.eye(n, dtype=np.complex128).reshape((n,) + self.lat + (4, 3))
        cols = self.apply(eye).reshape(n, n)
        return cols.T


def free_spectrum(dims, m0, antiperiodic_t=False):
    """Closed-form eigenvalues of D at U = 1 (the clover term vanishes there):
    m0 + sum_mu (1 - cos p_mu) +- i sqrt(sum_mu sin^2 p_mu), each with
    multiplicity 6, p_mu = 2 pi n / L_mu (t: (2n+1) pi / L_t if antiperiodic)."""
    axes = []
    for mu, l in enumerate(dims):
        n = np.arange(l)
        if mu == 3 and antiperiodic_t:
            axes.append((2 * n + 1) * np.pi / l)
        else:
            axes.append(2 * np.pi * n / l)
    p = np.meshgrid(*axes, indexing="ij")
    re = m0 + sum(1 - np.cos(q) for q in p)
    im = np.sqrt(sum(np.sin(q) ** 2 for q in p))
    ev = np.concatenate([re.ravel() + 1j * im.ravel(), re.ravel() - 1j * im.ravel()])
    return np.repeat(ev, 6)


def patch(field, origin, size, lat_axes=4):
    """The periodic sub-box of a field (Lt, Lz, Ly, Lx, ...) starting at origin
    (x, y, z, t) with edge ``size`` (indices wrap around the lattice)."""
    out = field
    for mu in range(4):
        axis = 3 - mu
        n = field.shape[axis]
        idx = (origin[mu] + np.arange(size)) % n
        out = np.take(out, idx, axis=axis)
    return out


def apply_at_sites(u, psi, m0, c_sw, sites, antiperiodic_t=False, round_fields=None):
    """(D psi)(x) for a list of sites x = (x, y, z, t), each evaluated on its own
    5^4 periodic patch centred on x: the clover term at x reaches two sites
    out, the hops one, so the patch wrap never touches them.  Returns an array
    (len(sites), 4, 3).  ``round_fields`` (a function) is applied to the links
    of the hops and to the clover matrix, to mimic reduced storage.

    An antiperiodic time boundary is not supported here (the patch loses the
    global position of the boundary)."""
    if antiperiodic_t:
        raise NotImplementedError("site evaluation supports periodic boundaries only")
    out = []
    for x in sites:
        origin = tuple(c - 2 for c in x)
        up = patch(u, origin, 5)
        pp = patch(psi, origin, 5)
        op = WilsonClover(up, m0, c_sw)
        if round_fields is not None:
            op.a = round_fields(op.a)
            op.u = round_fields(op.u)
        out.append(op.apply(pp)[2, 2, 2, 2])
    return np.array(out)
