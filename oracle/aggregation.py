"""Aggregation-based interpolation P and restriction R = P^dagger (Sec. 3).

* Aggregates are a block decomposition of the lattice (independent of the
  Schwarz blocks), each split by chirality so that gamma_5 P = P gamma_5^c
  (Sec. 3): on the fine level chirality 0 = spins {0, 1} (gamma_5 = +1),
  chirality 1 = spins {2, 3}; on a coarse level with 2N dof per site the first
  N dof have gamma_5^c = +1 and the last N have -1.
* P e_j is test vector v_{((j-1) mod N)+1} restricted to aggregate
  A_{ceil(j/N)} (Sec. 3, the formula beside Fig. 3).  The paper prints the
  restriction operator there; what is meant is the restricted vector embedded
  back into the full space (I_A I_A^T v), which is how it is read here.
* To have P^dagger P = 1 the test vectors are orthonormalised on every
  aggregate (Sec. 3).  Reading taken: modified Gram-Schmidt over the vectors in
  their order k = 1..N, each normalised to a positive real norm, i.e. the
  unique thin QR factor with positive diagonal.
* Coarse dof ordering per coarse site: index chi*N + k (chirality chi, vector k).
"""

import numpy as np


class Aggregation:
    """Aggregates of size ``agg`` on lattice ``dims``; fields carry ``dof_shape`` per site.

    ``dof_shape`` is (4, 3) on the fine level (chirality = spin // 2) or
    (2N_prev,) on a coarse level (chirality = dof // N_prev).
    """

    def __init__(self, dims, agg, dof_shape):
        dims = tuple(int(d) for d in dims)
        agg = tuple(int(a) for a in agg)
        for d, a in zip(dims, agg):
            if a <= 0 or d % a != 0:
                raise ValueError(f"aggregate {agg} does not divide lattice {dims}")
        self.dims, self.agg = dims, agg
        self.cdims = tuple(d // a for d, a in zip(dims, agg))
        self.lat, self.clat = dims[::-1], self.cdims[::-1]
        self.dof_shape = tuple(dof_shape)
        self.tail = len(self.dof_shape)

    # -- views --------------------------------------------------------------
    def _chiral_split(self, x):
        """(..., *dof_shape) -> (..., 2, half)."""
        lead = x.shape[:-self.tail]
        if self.dof_shape == (4, 3):
            return x.reshape(lead + (2, 6))
        n2 = self.dof_shape[0]
        return x.reshape(lead + (2, n2 // 2))

    def to_aggregates(self, x):
        """Field (..., Lt, Lz, Ly, Lx, *dof) -> (..., coarse sites, 2, local dof)."""
        lead = x.shape[:x.ndim - 4 - self.tail]
        (ax, ay, az, at), (cx, cy, cz, ct) = self.agg, self.cdims
        y = self._chiral_split(x)
        half = y.shape[-1]
        y = y.reshape(lead + (ct, at, cz, az, cy, ay, cx, ax, 2, half))
        k = len(lead)
        perm = tuple(range(k)) + tuple(k + i for i in (0, 2, 4, 6, 8, 1, 3, 5, 7, 9))
        y = y.transpose(perm)                                # (..., ct,cz,cy,cx, 2, at,az,ay,ax, half)
        return y.reshape(lead + (ct * cz * cy * cx, 2, at * az * ay * ax * half))

    def from_aggregates(self, y):
        """Inverse of ``to_aggregates``."""
        lead = y.shape[:-3]
        (ax, ay, az, at), (cx, cy, cz, ct) = self.agg, self.cdims
        half = y.shape[-1] // (at * az * ay * ax)
        y = y.reshape(lead + (ct, cz, cy, cx, 2, at, az, ay, ax, half))
        k = len(lead)
        perm = tuple(range(k)) + tuple(k + i for i in (0, 5, 1, 6, 2, 7, 3, 8, 4, 9))
        y = y.transpose(perm)                                # (..., ct,at,cz,az,cy,ay,cx,ax, 2, half)
        return y.reshape(lead + self.lat + self.dof_shape)

    # -- construction -------------------------------------------------------
    def build(self, vectors):
        """Locally orthonormalise the N test vectors (N, Lt, Lz, Ly, Lx, *dof) -> P.

        Stores ``self.q`` of shape (N, coarse sites, 2, local dof).
        """
        q = self.to_aggregates(np.array(vectors, dtype=np.complex128))
        n = q.shape[0]
        for k in range(n):
            for j in range(k):
                c = np.sum(np.conj(q[j]) * q[k], axis=-1, keepdims=True)
                q[k] = q[k] - c * q[j]
            nrm = np.sqrt(np.sum((np.conj(q[k]) * q[k]).real, axis=-1, keepdims=True))
            q[k] = q[k] / nrm
        self.q = q
        self.nvec = n
        return self

    def columns(self):
        """The locally orthonormalised test vectors as fine fields (N, Lt, Lz, Ly, Lx, *dof)."""
        return self.from_aggregates(self.q)

    # -- P and P^dagger -----------------------------------------------------
    def restrict(self, r):
        """(P^dagger r)[a, chi*N + k] = sum over aggregate a, chirality chi of conj(v_k) r."""
        ra = self.to_aggregates(r)                                   # (..., S, 2, L)
        c = np.einsum("ksxl,...sxl->...sxk", np.conj(self.q), ra, optimize=True)    # (..., S, 2, N)
        lead = c.shape[:-3]
        return c.reshape(lead + self.clat + (2 * self.nvec,))

    def prolong(self, e):
        """(P e)(x) = sum_k v_k(x)|_chi e[a(x), chi*N + k]."""
        lead = e.shape[:-5]
        ec = e.reshape(lead + (-1, 2, self.nvec))                    # (..., S, 2, N)
        fa = np.einsum("ksxl,...sxk->...sxl", self.q, ec, optimize=True)
        return self.from_aggregates(fa)

    def dense(self):
        """P as a dense matrix (fine dof x coarse dof), for small tests."""
        nc = int(np.prod(self.clat)) * 2 * self.nvec
        eye = np.eye(nc, dtype=np.complex128).reshape((nc,) + self.clat + (2 * self.nvec,))
        cols = self.prolong(eye).reshape(nc, -1)
        return cols.T

    # -- geometry used by the coarse operator --------------------------------
    def face_mask(self, mu, step):
        """1 at sites whose neighbour x + step*mu lies in another aggregate."""
        lat = self.lat
        coords = np.meshgrid(*[np.arange(n) for n in lat], indexing="ij")  # t, z, y, x
        c = coords[3 - mu]
        a = self.agg[mu]
        if step > 0:
            m = (c % a) == a - 1
        else:
            m = (c % a) == 0
        return m.astype(np.float64)

    def chirality_projector(self, chi):
        """Per-dof 0/1 mask of chirality chi, shape dof_shape."""
        if self.dof_shape == (4, 3):
            m = np.zeros((4, 3))
            m[2 * chi:2 * chi + 2, :] = 1.0
            return m
        n2 = self.dof_shape[0]
        m = np.zeros(n2)
        m[chi * (n2 // 2):(chi + 1) * (n2 // 2)] = 1.0
        return m


def gamma5_coarse(nvec):
    """gamma_5^c on one coarse site: diag(+1 x N, -1 x N)."""
    return np.concatenate([np.ones(nvec), -np.ones(nvec)])


def orthonormalise(vectors):
    """Global modified Gram-Schmidt of a list of fields, in order (set-up part 1)."""
    out = []
    for v in vectors:
        w = np.array(v, dtype=np.complex128)
        for q in out:
            w = w - np.vdot(q, w) * q
        out.append(w / np.sqrt(np.vdot(w, w).real))
    return out
