"""Block decomposition, block solvers and red-black Schwarz (Sec. 2).

* A block decomposition {L_i} of the lattice with trivial embeddings I_{L_i};
  the block operator is D_i = I^T D I (every hop that leaves the block is
  dropped) and the block solver B_i = I D_i^{-1} I^T (Sec. 2).
* Blocks are two-coloured so that no two blocks of one colour touch; then a
  residual update on one block leaves the residual on the other blocks of its
  colour unchanged, and all blocks of a colour can be solved at once
  (Algorithm 1).  Colour of block (bx, by, bz, bt) = (bx + by + bz + bt) mod 2;
  colour 0 (the block at the origin) goes first.
* Reading taken: the block systems are solved approximately by n_MR steps of
  the minimal-residual method (MR), e = 0, rho = r and per step
  p = D_i rho, alpha = <p, rho>/<p, p>, e += alpha rho, rho -= alpha p, with
  <a, b> = sum conj(a) b and alpha = 0 when <p, p> = 0.  The paper's own runs
  used a few GMRES steps (Sec. 2 and Sec. 4); one MR step equals one GMRES
  step.  An exact (dense LU) block solve is provided for the tests.

The operator objects passed in need ``apply(x)`` on fields of shape
(..., Lt, Lz, Ly, Lx, *dof) and attributes ``lat`` and ``tail`` (number of
per-site dof axes).
"""

import numpy as np


class BlockDecomposition:
    """Blocks of size ``block`` = (bx, by, bz, bt) on a lattice ``dims`` = (Lx, Ly, Lz, Lt).

    Needs an even number (>= 2) of blocks in every direction, so that the
    two-colouring survives the periodic wrap.
    """

    def __init__(self, dims, block):
        dims = tuple(int(d) for d in dims)
        block = tuple(int(b) for b in block)
        for d, b in zip(dims, block):
            if b <= 0 or d % b != 0 or (d // b) % 2 != 0:
                raise ValueError(f"lattice {dims} cannot be cut into an even number of blocks {block}")
        self.dims, self.block = dims, block
        self.nb = tuple(d // b for d, b in zip(dims, block))          # blocks per direction (x..t)
        lat = dims[::-1]
        t, z, y, x = np.meshgrid(*[np.arange(n) for n in lat], indexing="ij")
        bx, by, bz, bt = x // block[0], y // block[1], z // block[2], t // block[3]
        self.colour = (bx + by + bz + bt) % 2                             # (Lt, Lz, Ly, Lx)
        self.block_id = ((bt * self.nb[2] + bz) * self.nb[1] + by) * self.nb[0] + bx
        self.nblocks = int(np.prod(self.nb))
        self.block_colour = np.zeros(self.nblocks, dtype=int)
        self.block_colour[self.block_id.ravel()] = self.colour.ravel()

    def mask(self, colour):
        return (self.colour == colour).astype(np.float64)

    def block_sums(self, f):
        """Sum a per-site field f (..., Lt, Lz, Ly, Lx) over each block -> (..., nblocks)."""
        lead = f.shape[:-4]
        (nbx, nby, nbz, nbt), (bx, by, bz, bt) = self.nb, self.block
        g = f.reshape(lead + (nbt, bt, nbz, bz, nby, by, nbx, bx))
        k = len(lead)
        g = g.sum(axis=(k + 1, k + 3, k + 5, k + 7))
        return g.reshape(lead + (self.nblocks,))

    def per_site(self, b):
        """Broadcast per-block values (..., nblocks) back onto sites (..., Lt, Lz, Ly, Lx)."""
        return b[..., self.block_id]


def _expand(site_field, tail):
    return site_field.reshape(site_field.shape + (1,) * tail)


def colour_operator(op, blocks, colour):
    """x -> sum_{i: colour(i) = c} I_i D_i I_i^T x.

    Same-coloured blocks never touch, so masking D on both sides with the
    union of colour-c blocks gives exactly the direct sum of the block
    operators D_i = I^T D I.
    """
    m = _expand(blocks.mask(colour), op.tail)
    return lambda x: m * op.apply(m * x)


def block_mr(op, blocks, colour, r, n_mr):
    """e ~ sum_{i: colour c} B_i r by n_mr MR steps on every colour-c block."""
    tail = op.tail
    dc = colour_operator(op, blocks, colour)
    m = _expand(blocks.mask(colour), tail)
    axes = tuple(range(-tail, 0))
    e = np.zeros_like(r)
    rho = m * r
    for _ in range(n_mr):
        p = dc(rho)
        pr = blocks.block_sums(np.sum(np.conj(p) * rho, axis=axes))
        pp = blocks.block_sums(np.sum((np.conj(p) * p).real, axis=axes))
        alpha = np.where(pp > 0, pr / np.where(pp > 0, pp, 1.0), 0.0)
        a = _expand(blocks.per_site(alpha), tail)
        e = e + a * rho
        rho = rho - a * p
    return e


def block_dense_matrices(op, blocks, colour):
    """Dense D_i = I^T D I of every block i of the colour: dict block -> (dof indices, matrix).

    Column j of every D_i is probed at once by a unit vector placed at the
    j-th local dof of every colour-c block (they do not interact).
    """
    lat = op.lat
    dof = int(np.prod(op.dof_shape))
    ids = blocks.block_id.ravel()
    members = [b for b in range(blocks.nblocks) if blocks.block_colour[b] == colour]
    sites = np.stack([np.nonzero(ids == b)[0] for b in members])          # (nblk, sites per block)
    cols = (sites[:, :, None] * dof + np.arange(dof)[None, None, :]).reshape(len(members), -1)
    n = cols.shape[1]
    dc = colour_operator(op, blocks, colour)
    e = np.zeros((n, int(np.prod(lat)) * dof), dtype=np.complex128)
    for k in range(len(members)):
        e[np.arange(n), cols[k]] = 1.0
    de = dc(e.reshape((n,) + lat + op.dof_shape)).reshape(n, -1)
    return {b: (cols[k], de[:, cols[k]].T) for k, b in enumerate(members)}


def block_exact(op, blocks, colour, r, dense=None):
    """e = sum_{i: colour c} B_i r with every D_i solved by dense LU (numpy.linalg.solve)."""
    if dense is None:
        dense = block_dense_matrices(op, blocks, colour)
    flat = r.reshape(r.shape[:r.ndim - 4 - op.tail] + (-1,))
    e = np.zeros_like(flat)
    for b, (cols, mat) in dense.items():
        e[..., cols] = np.linalg.solve(mat, flat[..., cols].T).T if flat.ndim > 1 else \
            np.linalg.solve(mat, flat[cols])
    return e.reshape(r.shape)


def sap_sweep(op, blocks, b, z, n_mr, exact=None):
    """One red-black Schwarz iteration (Algorithm 1) on D z = b.

    For colour c = 0, 1: r <- b - D z, then z <- z + B_i r on every block of
    colour c.  ``exact`` (a pair of dense-block dicts, one per colour) selects
    exact block solves instead of MR.
    """
    for c in (0, 1):
        r = b - op.apply(z)
        if exact is None:
            e = block_mr(op, blocks, c, r, n_mr)
        else:
            e = block_exact(op, blocks, c, r, exact[c])
        z = z + e
    return z


def sap(op, blocks, b, z0, n_sweeps, n_mr, exact=None):
    """n_sweeps red-black Schwarz iterations from z0 (``exact``: as in sap_sweep)."""
    z = z0
    for _ in range(n_sweeps):
        z = sap_sweep(op, blocks, b, z, n_mr, exact)
    return z


def mr_on_mask(op, mask, r, n_mr):
    """n_mr MR steps on the single block selected by the 0/1 site mask (the
    operator mask D mask), from e = 0; returns e."""
    m = _expand(mask, op.tail)
    axes = tuple(range(-op.tail - 4, 0))
    e = np.zeros_like(r)
    rho = m * r
    for _ in range(n_mr):
        p = m * op.apply(m * rho)
        pr = np.sum(np.conj(p) * rho, axis=axes)
        pp = np.sum((np.conj(p) * p).real, axis=axes)
        alpha = pr / pp if pp > 0 else 0.0
        e = e + alpha * rho
        rho = rho - alpha * p
    return e


def colour_pass_on_block(u, m0, c_sw, b, z, block_origin, n_mr, round_fields=None):
    """One Schwarz colour pass (Algorithm 1) restricted to the 4^4 block at
    block_origin = (x, y, z, t) of a periodic lattice: r = b - D z on the block,
    n_mr MR steps with the block operator, z + e on the block.  Evaluated on an
    8^4 patch with the block at offset 2, far enough from the patch wrap for
    the clover term and the hops.  Returns the block's new z, (4, 4, 4, 4, 4, 3)
    indexed (t, z, y, x)."""
    from .dirac import WilsonClover, patch
    origin = tuple(c - 2 for c in block_origin)
    up = patch(u, origin, 8)
    op = WilsonClover(up, m0, c_sw)
    if round_fields is not None:
        op.a = round_fields(op.a)
        op.u = round_fields(op.u)
    bp = patch(b, origin, 8)
    zp = patch(z, origin, 8)
    mask = np.zeros((8, 8, 8, 8))
    mask[2:6, 2:6, 2:6, 2:6] = 1.0
    r = (bp - op.apply(zp)) * mask[..., None, None]
    e = mr_on_mask(op, mask, r, n_mr)
    return (zp + e)[2:6, 2:6, 2:6, 2:6]
