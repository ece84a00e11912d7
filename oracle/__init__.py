"""CPU oracle for the hull-detection path (SC, MSC, SM) -- test infrastructure.

Only the test suite, the smoke check (`__graft_entry__.smoke`) and the
benchmark's CPU-baseline / reference arm may import this package.  The CUDA
library never calls it, and it never calls the CUDA library.

Parity status of each function (what pins it; tests under tests/ -m "not gpu"):
  cordic_table            exact big-integer series; pinned by atan/K closed
                          forms and libm cos/sin error bounds.
  grid_endpoints          pinned against float64 geometry within its error bound.
  voxel_set               pinned against the per-voxel slab test (an independent
                          statement) on small grids, closed forms (axis-aligned
                          rows, lattice diagonals) and the count identity.
  accumulate              pinned by sum identities and single-history sets.
  msc_decide / sm_decide  pinned by hand-built volumes (tests/golden) and the
                          definition's special cases.
  Tables 1-2 voxel counts: parity unpinned (the paper's phantom and data are
                          not available).
"""
from .oracle import *  # noqa: F401,F403
