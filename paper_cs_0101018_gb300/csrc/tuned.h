// tuned.h -- the engine's shape-keyed partition, as measured by
// paper_cs_0101018_gb300/tune.py (which rewrites this file).
//
// kTunedGroups: for grids of `dim` dimensions with n_tiles in [tiles_lo,
// tiles_hi], the tiles per group (the reduction unit) that gave the fastest
// lone solve among the sizes at least the floor the batch allows.
// kTunedItemTiles: the tiles per work item of a launch with more groups
// than the resident CTAs can take at once (batches, serving).
// Measured on NVIDIA GB300, 2026-12-04: mixed precision,
// tau_rel 1e-6, median of 5 solves (ms) for 1 / 2 / 4 tiles per group:
//   2-D side    32 (      1 tiles): 1.233 / 1.228 / 1.233  (fastest: 2)
//   2-D side    48 (      2 tiles): 1.268 / 1.563 / 1.566  (fastest: 1)
//   2-D side    64 (      2 tiles): 1.476 / 1.894 / 1.887  (fastest: 1)
//   2-D side    96 (      6 tiles): 1.542 / 1.887 / 2.232  (fastest: 1)
//   2-D side   128 (      8 tiles): 1.504 / 1.770 / 2.472  (fastest: 1)
//   2-D side   192 (     18 tiles): 1.614 / 1.942 / 2.582  (fastest: 1)
//   2-D side   256 (     32 tiles): 1.636 / 2.029 / 2.719  (fastest: 1)
//   2-D side   384 (     72 tiles): 1.902 / 2.363 / 3.305  (fastest: 1)
//   2-D side   512 (    128 tiles): 1.959 / 2.342 / 3.239  (fastest: 1)
//   2-D side   768 (    288 tiles): 2.263 / 2.654 / 3.488  (fastest: 1)
//   2-D side  1024 (    512 tiles): 2.898 / 2.904 / 3.701  (fastest: 1)
//   2-D side  1536 (   1152 tiles): 4.417 / 4.416 / 4.217  (fastest: 4)
//   3-D side    12 (     12 tiles): 2.393 / 2.993 / 4.333  (fastest: 1)
//   3-D side    16 (     16 tiles): 2.278 / 2.806 / 3.924  (fastest: 1)
//   3-D side    24 (     24 tiles): 2.258 / 2.866 / 4.062  (fastest: 1)
//   3-D side    32 (     32 tiles): 2.263 / 2.989 / 4.298  (fastest: 1)
//   3-D side    48 (     96 tiles): 2.904 / 3.720 / 5.539  (fastest: 1)
//   3-D side    64 (    128 tiles): 2.511 / 3.163 / 4.586  (fastest: 1)
//   3-D side    96 (    576 tiles): 4.878 / 4.777 / 6.522  (fastest: 2)
//   3-D side   128 (   1024 tiles): 7.912 / 7.903 / 7.760  (fastest: 4)
// 512-QP batch (best of 3, ms) with groups of at least 1 / 2 / 4 tiles: 272.2 / 228.5 / 226.4  -> at least 2 (within 2 % of the coarsest)
// 512-QP batch (best of 3, ms) for 2 / 4 / 8 tiles per item: 270.6 / 228.5 / 228.6  -> 4
#pragma once

namespace gpcg {

struct TunedGroup {
  int dim, tiles_lo, tiles_hi, group_tiles;
};

constexpr TunedGroup kTunedGroups[] = {
    {2, 1, 1, 2},
    {2, 2, 3, 4},
    {2, 4, 768, 2},
    {2, 769, 1 << 30, 4},
    {3, 1, 768, 2},
    {3, 769, 1 << 30, 4},
};
constexpr int kTunedItemTiles = 4;

}  // namespace gpcg
