"""Petrov-Galerkin coarse operator D_c = R D P with R = P^dagger (Sec. 3).

Because P is aggregate-block-diagonal and D couples nearest neighbours only,
D_c couples only neighbouring aggregates: it is again a nearest-neighbour
stencil on the regular 4D grid of aggregates (Sec. 3), with per coarse site a
self-coupling 2N x 2N matrix and one 2N x 2N matrix per direction +-mu:

    (D_c x)(a) = S(a) x(a) + sum_mu [ F_mu(a) x(a + mu) + B_mu(a) x(a - mu) ].

Entries are built from the pieces of D applied to the columns of P:
S(a) = P_a^dagger (A + hops that stay inside a) P_a,
F_mu(a) = P_a^dagger H_{+mu} P_{a+mu} (the +mu hop from a's +mu face),
B_mu(a) = P_a^dagger H_{-mu} P_{a-mu}.  The tests pin this stencil against the
dense product P^dagger D P.

The stencil offers the same ``local`` / ``hop`` / ``apply`` interface as the
fine operator, so the construction recurses to the next coarser level.
"""

import numpy as np

from .dirac import shift


class CoarseOperator:
    tail = 1

    def __init__(self, fine_op, agg):
        n = agg.nvec
        n2 = 2 * n
        self.nvec = n
        self.lat = agg.clat
        self.dims = agg.cdims
        self.dof_shape = (n2,)
        self.self_ = np.zeros(self.lat + (n2, n2), dtype=np.complex128)
        self.fwd = np.zeros((4,) + self.lat + (n2, n2), dtype=np.complex128)
        self.bwd = np.zeros((4,) + self.lat + (n2, n2), dtype=np.complex128)
        cols = agg.columns()
        fine_tail = len(agg.dof_shape)
        faces = {(mu, s): agg.face_mask(mu, s).reshape(agg.lat + (1,) * fine_tail)
                 for mu in range(4) for s in (1, -1)}
        # all 2N columns at once: column j = chi*N + k is v_k restricted to chirality chi
        proj = np.stack([agg.chirality_projector(chi) for chi in (0, 1)])          # (2, *dof)
        proj = proj.reshape((2, 1, 1, 1, 1, 1) + agg.dof_shape)
        u = (proj * cols[None]).reshape((n2,) + cols.shape[1:])                    # (2N, lat, dof)
        to_cols = lambda r: np.moveaxis(r, 0, -1)                                   # (2N, clat, 2N_i) -> (clat, i, j)
        self.self_ += to_cols(agg.restrict(fine_op.local(u)))
        for mu in range(4):
            for s in (1, -1):
                h = fine_op.hop(u, mu, s)
                f = faces[(mu, s)]
                self.self_ += to_cols(agg.restrict(h * (1.0 - f)))
                tgt = self.fwd if s > 0 else self.bwd
                tgt[mu] += to_cols(agg.restrict(h * f))

    def local(self, x):
        return np.einsum("...ij,...j->...i", self.self_, x)

    def hop(self, x, mu, step):
        if step > 0:
            return np.einsum("...ij,...j->...i", self.fwd[mu], shift(x, mu, 1, 1))
        return np.einsum("...ij,...j->...i", self.bwd[mu], shift(x, mu, -1, 1))

    def apply(self, x):
        out = self.local(x)
        for mu in range(4):
            out = out + self.hop(x, mu, 1) + self.hop(x, mu, -1)
        return out

    def apply_gamma5(self, x):
        g = np.concatenate([np.ones(self.nvec), -np.ones(self.nvec)])
        return x * g

    def dense(self):
        n = int(np.prod(self.lat)) * self.dof_shape[0]
        eye = np.eye(n, dtype=np.complex128).reshape((n,) + self.lat + self.dof_shape)
        return self.apply(eye).reshape(n, n).T


def galerkin_dense(fine_op, agg):
    """Brute force P^dagger D P as a dense matrix: D applied to every column of P."""
    p = agg.dense()
    nc = p.shape[1]
    cols = p.T.reshape((nc,) + agg.lat + agg.dof_shape)
    dp = fine_op.apply(cols).reshape(nc, -1).T
    return np.conj(p.T) @ dp
