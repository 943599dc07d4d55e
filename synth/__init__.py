"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This package holds input generation only: a counter-based random number
generator, random SU(3) gauge fields U = exp(i eps H), random spinors, Z2 noise
and point sources, random gauge transformations, and the named workload
configurations.  It contains none of the solver's arithmetic (no Dirac
operator, no Schwarz sweep, no aggregation), so that the oracle and the CUDA
path can both consume the same inputs without sharing method code.

Array conventions (canonical layout, used everywhere outside the CUDA
library's internal blocked layout):

* lattice dims ``(Lx, Ly, Lz, Lt)``, x fastest; site index
  ``((t*Lz + z)*Ly + y)*Lx + x``;
* a spinor field is a complex128 array of shape ``(Lt, Lz, Ly, Lx, 4, 3)``
  ([site][spin][colour]);
* a gauge field is a complex128 array of shape ``(Lt, Lz, Ly, Lx, 4, 3, 3)``
  ([site][mu][row][col]) holding the forward links U_mu(x), mu = x, y, z, t.
"""

from .rng import splitmix64, counter_u64, uniform_pm1, uniform_open01, gaussian
from .fields import (
    random_gauge_field,
    unit_gauge_field,
    random_su3,
    random_gauge_rotation,
    random_spinor,
    uniform_spinor,
    z2_spinor,
    point_sources,
    test_vector_draw,
    gauge_transform,
    spinor_shape,
    gauge_shape,
)
from .configs import WORKLOADS, workload

__all__ = [
    "splitmix64", "counter_u64", "uniform_pm1", "uniform_open01", "gaussian",
    "random_gauge_field", "unit_gauge_field", "random_su3", "random_gauge_rotation", "random_spinor",
    "uniform_spinor", "z2_spinor", "point_sources", "test_vector_draw",
    "gauge_transform", "spinor_shape", "gauge_shape", "WORKLOADS", "workload",
]
