"""The oracle against the stored expected values (tests/golden/): the closed
free-field spectrum against the oracle's dense operator, and the oracle's
Dirac operator, Schwarz sweep and coarse operator against the values it
recorded when the fixtures were written (a change to the oracle's arithmetic
must come with regenerated fixtures and a reason)."""

import numpy as np

import synth
from oracle.dirac import WilsonClover
from oracle.sap import BlockDecomposition, sap_sweep
from oracle.aggregation import Aggregation
from oracle.coarse import CoarseOperator
from tests import golden_util as gu


def test_free_spectrum_file_matches_dense_operator():
    r = gu.rows("free_spectrum_2x2x2x2.txt")
    ref = np.sort(np.repeat(r[:, 0] + 1j * r[:, 1], r[:, 2].astype(int)).real)
    u = synth.unit_gauge_field((2, 2, 2, 2))
    ev = np.linalg.eigvals(WilsonClover(u, 0.1, 1.0).dense())
    assert np.max(np.abs(np.sort(ev.real) - ref)) < 1e-12
    assert np.max(np.abs(ev.imag)) < 1e-12


def _inputs():
    u = synth.random_gauge_field(gu.DIMS, gu.EPS, gu.GSEED)
    return u, WilsonClover(u, gu.M0, gu.CSW), synth.random_spinor(gu.DIMS, gu.PSEED)


def test_oracle_reproduces_stored_dirac_and_sweep():
    u, op, psi = _inputs()
    assert gu.compare_sites("dirac_8x8x8x8.txt", op.apply(psi)) < 1e-13
    z = sap_sweep(op, BlockDecomposition(gu.DIMS, (4, 4, 4, 4)), psi, np.zeros_like(psi), 4)
    assert gu.compare_sites("sap_sweep_8x8x8x8.txt", z) < 1e-13


def test_oracle_reproduces_stored_coarse_operator():
    u, op, psi = _inputs()
    c = CoarseOperator(op, Aggregation(gu.DIMS, (4, 4, 4, 4), (4, 3)).build(synth.test_vector_draw(gu.DIMS, 4,
                                                                                                   gu.VSEED)))
    r = gu.rows("coarse_op_site0_8x8x8x8.txt")
    blocks = [c.self_] + [x for mu in range(4) for x in (c.fwd[mu], c.bwd[mu])]
    got = np.array([blocks[int(d)][0, 0, 0, 0][int(i), int(j)] for d, i, j, _, _ in r])
    ref = r[:, 3] + 1j * r[:, 4]
    assert np.max(np.abs(got - ref)) < 1e-13 * np.max(np.abs(ref))
