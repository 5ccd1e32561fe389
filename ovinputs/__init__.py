"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module draws gauge fields, sources and gauge transformations. It holds
none of the method's arithmetic (no Dirac operator, no Krylov step, no sign
function), so both sides may import it without sharing any computation.

Conventions (fixed for the whole project):
  * lattice dims (Lx, Ly, Lz, Lt); site = x + Lx*(y + Ly*(z + Lz*t)), x fastest.
  * gauge field: complex128 array [V][4][3][3], direction index 0..3 = x,y,z,t,
    U[site, nu, a, b] = (U_nu(site))_{ab}.
  * spinor: complex128 vector of n = 12*V entries, index 12*site + 3*spin + colour.
  * draws are site-major, then direction, from numpy's PCG64 generator.
"""
from .gen import (  # noqa: F401
    lattice_volume,
    complex_gaussian,
    haar_su3,
    near_unit_su3,
    gauge_field,
    gaussian_source,
    point_source,
    point_sources_12,
    gauge_rotation,
    round_links_fp32,
    problem_batch_48,
    training_problems,
    training_problems_rough,
    training_problems_large,
    problem_source,
)
