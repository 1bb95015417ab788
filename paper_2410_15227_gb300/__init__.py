"""GB300 (sm_103a) library for the pseudo-particle Exact mapping of
Lau, Petkova & Bonnell (2024): tree build, pseudo-particle selection and
smoothing lengths, Voronoi grid, particle-cell pairs, analytic mapping of
the M4 kernel onto the cells and the inverse mapping.

The compute path is ``libexactmap.so`` (C ABI in ``include/exactmap.h``);
``api`` binds it with the same call names.  ``inputs`` draws the seeded
synthetic workloads.  ``partition`` holds the host logic of the spatial split
over ranks.  Importing this package does not load the library; the
first call into ``api`` does, and fails loudly if it has not been built.
"""

__all__ = ["api", "inputs", "build", "partition"]
