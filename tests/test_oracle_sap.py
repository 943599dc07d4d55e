"""Pins of the oracle's Schwarz method (Sec. 2, Eq. 2.1, Algorithm 1): dense-LU
block solves, the dense error propagator on a 4^4 lattice with 2^4 blocks
(the setting of Fig. 2), the independence of same-coloured blocks, and MR
special cases."""

import numpy as np
import pytest

import synth
from oracle.dirac import WilsonClover
from oracle import sap as osap
from oracle.sap import BlockDecomposition, block_mr, block_exact, block_dense_matrices, sap_sweep

DIMS = (4, 4, 4, 4)


@pytest.fixture(scope="module")
def setting():
    op = WilsonClover(synth.random_gauge_field(DIMS, 0.5, 41), 0.2, 1.0)
    bl = BlockDecomposition(DIMS, (2, 2, 2, 2))
    dense_blocks = [block_dense_matrices(op, bl, c) for c in (0, 1)]
    d = op.dense()
    return op, bl, dense_blocks, d


def test_blocks_need_even_count():
    with pytest.raises(ValueError):
        BlockDecomposition((6, 4, 4, 4), (2, 2, 2, 2))     # 3 blocks in x
    with pytest.raises(ValueError):
        BlockDecomposition((4, 4, 4, 4), (4, 2, 2, 2))     # 1 block in x
    bl = BlockDecomposition((8, 4, 4, 8), (4, 2, 2, 4))
    assert bl.nblocks == 16 and np.sum(bl.block_colour) == 8


def test_colouring_no_touching_blocks():
    bl = BlockDecomposition((8, 4, 4, 8), (4, 2, 2, 4))
    for mu in range(4):
        nb = np.roll(bl.colour, -1, axis=3 - mu)
        nbid = np.roll(bl.block_id, -1, axis=3 - mu)
        crossing = nbid != bl.block_id
        assert np.all(nb[crossing] != bl.colour[crossing])


def test_block_matrix_is_restriction_of_dense(setting):
    op, bl, dense_blocks, d = setting
    for c in (0, 1):
        for b, (cols, mat) in dense_blocks[c].items():
            assert np.max(np.abs(mat - d[np.ix_(cols, cols)])) == 0.0


def test_mr_converges_to_dense_lu(setting):
    op, bl, dense_blocks, d = setting
    r = synth.random_spinor(DIMS, 3)
    e_lu = block_exact(op, bl, 1, r, dense_blocks[1])
    e_mr = block_mr(op, bl, 1, r, 300)
    assert np.max(np.abs(e_mr - e_lu)) < 1e-12 * np.max(np.abs(e_lu))
    # second check of the LU path itself
    b0 = next(iter(dense_blocks[1]))
    cols, mat = dense_blocks[1][b0]
    assert np.allclose(mat @ e_lu.ravel()[cols], r.ravel()[cols], atol=1e-12)
    # nothing leaks onto the other colour
    assert np.max(np.abs(e_mr * (bl.colour == 0)[..., None, None])) == 0.0


def test_sap_error_propagator_dense(setting):
    """One sweep with exact block solves: e_new = (1 - B_1 D)(1 - B_0 D) e_old, and
    this equals the multiplicative Schwarz product over all blocks of Eq. 2.1 taken
    colour by colour (same-coloured factors commute).  Both operators are applied
    to random probe vectors, built from the dense D and dense block inverses: a
    matrix difference that vanishes on random probes vanishes with probability 1."""
    op, bl, dense_blocks, d = setting
    n = d.shape[0]
    inv = [[(np.asarray(cols), np.linalg.inv(mat)) for cols, mat in dense_blocks[c].values()]
           for c in (0, 1)]

    def colour_factor(c, x):                 # (1 - B_c D) x, B_c the colour-c block sum
        r = d @ x
        y = x.copy()
        for cols, bi in inv[c]:
            y[cols] -= bi @ r[cols]
        return y

    def prop(x):
        return colour_factor(1, colour_factor(0, x))

    def mult(x):                             # colour 0 blocks first, then colour 1
        for c in (0, 1):
            for cols, bi in inv[c]:
                x = x.copy()
                x[cols] -= bi @ (d[cols] @ x)
        return x

    rng = np.random.default_rng(7)
    v = rng.standard_normal((n, 8)) + 1j * rng.standard_normal((n, 8))
    pv = prop(v)
    assert np.max(np.abs(pv - mult(v))) < 1e-11 * np.max(np.abs(pv))
    assert np.max(np.abs(pv - v)) > 0.1 * np.max(np.abs(v))    # the factor is not the identity
    b = synth.random_spinor(DIMS, 4)
    z0 = synth.random_spinor(DIMS, 5)
    xs = np.linalg.solve(d, b.ravel())
    z1 = sap_sweep(op, bl, b, z0, 0, exact=dense_blocks)
    assert np.max(np.abs((z1.ravel() - xs) - prop(z0.ravel() - xs))) < 1e-11


def test_same_colour_blocks_independent(setting):
    """B_1 D B_2 D = 0 for two blocks of one colour.  B_i is the inverse of the
    block's diagonal part embedded at its rows and columns, so the product's only
    nonzero rows are block 1's: inv(D_11) D_12 inv(D_22) D[block 2 rows, :]."""
    op, bl, dense_blocks, d = setting
    items = list(dense_blocks[0].items())
    (c1, m1), (c2, m2) = items[0][1], items[1][1]
    c1, c2 = np.asarray(c1), np.asarray(c2)
    prod = np.linalg.inv(m1) @ d[np.ix_(c1, c2)] @ np.linalg.inv(m2) @ d[c2]
    assert np.max(np.abs(prod)) < 1e-12
    # the blocks of the other colour do touch block 1
    touching = [np.max(np.abs(d[np.ix_(c1, np.asarray(c))])) for c, _ in dense_blocks[1].values()]
    assert max(touching) > 0.1


def test_mr_step_matches_definition_on_one_block(setting):
    """Two MR steps on one block, written out with the dense block matrix."""
    op, bl, dense_blocks, d = setting
    r = synth.random_spinor(DIMS, 6)
    e = block_mr(op, bl, 0, r, 2).ravel()
    blk, (cols, mat) = next(iter(dense_blocks[0].items()))
    rho = r.ravel()[cols]
    ee = np.zeros_like(rho)
    for _ in range(2):
        p = mat @ rho
        alpha = np.vdot(p, rho) / np.vdot(p, p)
        ee = ee + alpha * rho
        rho = rho - alpha * p
    assert np.max(np.abs(e[cols] - ee)) < 1e-13


def test_mr_zero_block_gives_zero_not_nan(setting):
    op, bl, dense_blocks, d = setting
    r = synth.random_spinor(DIMS, 7)
    blk = next(iter(dense_blocks[0]))
    r = r * (bl.block_id != blk)[..., None, None]        # one block with r = 0
    e = block_mr(op, bl, 0, r, 4)
    assert np.all(np.isfinite(e))
    assert np.max(np.abs(e * (bl.block_id == blk)[..., None, None])) == 0.0


def test_sap_fixed_point(setting):
    """The exact solution is a fixed point of a sweep."""
    op, bl, dense_blocks, d = setting
    b = synth.random_spinor(DIMS, 8)
    xs = np.linalg.solve(d, b.ravel()).reshape(b.shape)
    z = sap_sweep(op, bl, b, xs, 4)
    assert np.max(np.abs(z - xs)) < 1e-12


def test_planted_colour_order_breaks_propagator(setting, monkeypatch):
    """Recomputing the residual only once per sweep (additive across colours)
    is a different method; the propagator pin detects it."""
    op, bl, dense_blocks, d = setting

    def additive(op_, blocks, b, z, n_mr, exact=None):
        r = b - op_.apply(z)
        return z + sum(osap.block_exact(op_, blocks, c, r, exact[c]) for c in (0, 1))

    b = synth.random_spinor(DIMS, 4)
    z0 = synth.random_spinor(DIMS, 5)
    good = sap_sweep(op, bl, b, z0, 0, exact=dense_blocks)
    bad = additive(op, bl, b, z0, 0, exact=dense_blocks)
    assert np.max(np.abs(good - bad)) > 1e-3
