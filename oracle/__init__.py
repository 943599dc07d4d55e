"""Plain FP64 CPU oracle of the SAP-multilevel solver (Frommer, Kahl, Krieg,
Leder, Rottmann, "Aggregation-based Multilevel Methods for Lattice QCD").

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously correct
restatement of the method against which the CUDA library is checked.  Only the
test-suite, the smoke check and the benchmark's CPU-baseline leg may import it;
the library itself never does, and shares no code with it (the two meet only
in the seeded input generators of the separate ``synth`` package, which hold
none of the method's arithmetic).

Everything is numpy complex128 on canonical arrays:
spinor fields (..., Lt, Lz, Ly, Lx, 4, 3), gauge fields
(Lt, Lz, Ly, Lx, 4, 3, 3), coarse fields (..., cLt, cLz, cLy, cLx, 2N).

Modules and the passages they follow:

* ``dirac``       -- D = D(U) + m, clover-improved Wilson (Sec. 1, Eq. 1.1)
* ``sap``         -- block decomposition, block solvers B_i, red-black
                     Schwarz (Sec. 2, Eq. 2.1, Algorithm 1)
* ``aggregation`` -- aggregation interpolation P, R = P^dagger, local
                     orthonormalisation (Sec. 3, Fig. 3 and the formula for
                     P e_j beside it)
* ``coarse``      -- Petrov-Galerkin coarse operator D_c = P^dagger D P as a
                     nearest-neighbour stencil (Sec. 3, Eq. 3.2 and the text on
                     its sparsity)
* ``krylov``      -- GMRES with a fixed iteration count and restarted
                     flexible GMRES (Sec. 2 and Sec. 4)
* ``mg``          -- the multilevel cycle, bootstrap set-up part 1 and the
                     outer solve (Sec. 3, Sec. 4)

Where the paper leaves a choice open the reading taken is stated in the
docstring of the function that makes it.
"""
