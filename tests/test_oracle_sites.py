"""Pins of the oracle's site-wise and block-wise evaluations (used for the
full-size GPU checks) against the oracle's whole-lattice operator and Schwarz
sweep on a small lattice."""

import numpy as np

import synth
from oracle.dirac import WilsonClover, apply_at_sites
from oracle.sap import BlockDecomposition, block_mr, colour_pass_on_block


def test_apply_at_sites_matches_full_operator():
    dims = (8, 8, 8, 8)
    u = synth.random_gauge_field(dims, 0.6, 81)
    psi = synth.random_spinor(dims, 82)
    full = WilsonClover(u, -0.3, 1.2).apply(psi)
    sites = [(0, 0, 0, 0), (7, 3, 0, 5), (4, 7, 7, 7), (1, 2, 3, 4)]
    got = apply_at_sites(u, psi, -0.3, 1.2, sites)
    for k, (x, y, z, t) in enumerate(sites):
        assert np.max(np.abs(got[k] - full[t, z, y, x])) < 1e-13


def test_colour_pass_on_block_matches_full_pass():
    dims = (8, 8, 8, 8)
    u = synth.random_gauge_field(dims, 0.5, 83)
    op = WilsonClover(u, 0.1, 1.0)
    bl = BlockDecomposition(dims, (4, 4, 4, 4))
    b = synth.random_spinor(dims, 84)
    z = synth.random_spinor(dims, 85)
    r = b - op.apply(z)
    e = block_mr(op, bl, 0, r, 3)
    znew = z + e
    for origin in [(0, 0, 0, 0), (4, 4, 0, 0), (4, 0, 4, 0), (0, 4, 0, 4)]:   # colour-0 blocks
        got = colour_pass_on_block(u, 0.1, 1.0, b, z, origin, 3)
        x, y, zz, t = origin
        ref = znew[t:t + 4, zz:zz + 4, y:y + 4, x:x + 4]
        assert np.max(np.abs(got - ref)) < 1e-12
