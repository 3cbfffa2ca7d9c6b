"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This package generates patterns (band, block arrow, Erdos-Renyi, 2D/3D grids
with a geometric nested-dissection ordering) and random values on a given
pattern.  It holds none of the barrier arithmetic: no factorisation, no
inverse, no projection of an inverse.  Random numbers come from
``numpy.random.default_rng(seed)`` (PCG64).
"""
from .patterns import (band, arrow, erdos_renyi, grid2d, grid3d, nested_dissection, nd_options, grid_dims, batch_mix,
                       permute, lower_csc_from_pairs, pattern_hash)
from .values import (diag_dominant, uniform_sym, projected_gram, grid_perturbed,
                     planted_factor, random_dense_lower)
