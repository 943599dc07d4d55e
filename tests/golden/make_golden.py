"""Writes the stored expected values under tests/golden/ from the FP64 oracle
(and the seeded input generators) only.  Run from the repository root:

    python tests/golden/make_golden.py

Each file starts with comment lines naming the passage it restates, the
inputs and this command; data lines are whitespace-separated numbers.
"""

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle.dirac import WilsonClover, free_spectrum  # noqa: E402
from oracle.sap import BlockDecomposition, sap_sweep  # noqa: E402
from oracle.aggregation import Aggregation  # noqa: E402
from oracle.coarse import CoarseOperator  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
DIMS = (8, 8, 8, 8)
M0, CSW, EPS, GSEED, PSEED = -0.2, 1.0, 0.4, 301, 302
SITES = [(0, 0, 0, 0), (7, 7, 7, 7), (3, 4, 5, 6), (4, 0, 0, 7), (1, 2, 3, 4), (6, 5, 4, 3),
         (0, 7, 0, 7), (5, 1, 6, 2)]


def _write(name, header, rows):
    with open(os.path.join(HERE, name), "w") as f:
        for h in header:
            f.write("# " + h + "\n")
        f.write("# written by: python tests/golden/make_golden.py\n")
        for r in rows:
            f.write(" ".join(repr(float(v)) if isinstance(v, (float, np.floating)) else str(v) for v in r) + "\n")


def _site_rows(field):
    rows = []
    for (x, y, z, t) in SITES:
        for s in range(4):
            for c in range(3):
                v = field[t, z, y, x, s, c]
                rows.append((x, y, z, t, s, c, v.real, v.imag))
    return rows


def main():
    u = synth.random_gauge_field(DIMS, EPS, GSEED)
    op = WilsonClover(u, M0, CSW)
    psi = synth.random_spinor(DIMS, PSEED)
    inputs = f"8^4 lattice, gauge field synth.random_gauge_field(dims, {EPS}, {GSEED}), m0 = {M0}, c_sw = {CSW}, " \
             f"periodic; spinor synth.random_spinor(dims, {PSEED})"
    _write("dirac_8x8x8x8.txt",
           ["(D psi)(x) of the clover-improved Wilson operator, Sec. 1, Eq. 1.1 (Sheikholeslami-Wohlert form,",
            "chiral gamma basis), at sampled sites", inputs,
            "columns: x y z t spin colour Re Im"], _site_rows(op.apply(psi)))
    z = sap_sweep(op, BlockDecomposition(DIMS, (4, 4, 4, 4)), psi, np.zeros_like(psi), 4)
    _write("sap_sweep_8x8x8x8.txt",
           ["one red-black Schwarz sweep (Sec. 2, Algorithm 1) on D z = psi from z = 0, 4^4 blocks, colour 0 first,",
            "4 minimal-residual steps per block, at sampled sites", inputs,
            "columns: x y z t spin colour Re Im"], _site_rows(z))
    iv = synth.test_vector_draw(DIMS, 4, 303)
    c = CoarseOperator(op, Aggregation(DIMS, (4, 4, 4, 4), (4, 3)).build(iv))
    rows = []
    for d, blk in enumerate([c.self_] + [x for mu in range(4) for x in (c.fwd[mu], c.bwd[mu])]):
        m = blk[0, 0, 0, 0]
        for i in range(m.shape[0]):
            for j in range(m.shape[1]):
                rows.append((d, i, j, m[i, j].real, m[i, j].imag))
    _write("coarse_op_site0_8x8x8x8.txt",
           ["Galerkin coarse operator D_c = P^dagger D P (Sec. 3, Eq. 3.2) at coarse site 0: direction d",
            "(0 self, 1 + 2 mu forward, 2 + 2 mu backward), row i, column j; 4^4 aggregates x chirality,",
            "N = 4 test vectors synth.test_vector_draw(dims, 4, 303), orthonormalised per aggregate", inputs,
            "columns: d i j Re Im"], rows)
    ev = free_spectrum((2, 2, 2, 2), 0.1)
    uniq = {}
    for e in ev:
        key = (round(e.real, 12), round(e.imag, 12))
        uniq[key] = uniq.get(key, 0) + 1
    _write("free_spectrum_2x2x2x2.txt",
           ["eigenvalues of D at U = 1 on the periodic 2^4 lattice, m0 = 0.1 (the clover term vanishes): closed",
            "form m0 + sum_mu (1 - cos p_mu) +- i sqrt(sum_mu sin^2 p_mu), p_mu = pi n_mu",
            "columns: Re Im multiplicity"], [(k[0], k[1], n) for k, n in sorted(uniq.items())])


if __name__ == "__main__":
    main()
