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
//   2-D side    32 (      1 tiles): 1.128 / 1.131 / 1.129  (fastest: 1)
//   2-D side    48 (      2 tiles): 1.000 / 1.264 / 1.269  (fastest: 1)
//   2-D side    64 (      2 tiles): 1.263 / 1.663 / 1.660  (fastest: 1)
//   2-D side    96 (      6 tiles): 1.217 / 1.535 / 1.899  (fastest: 1)
//   2-D side   128 (      8 tiles): 1.255 / 1.591 / 2.304  (fastest: 1)
//   2-D side   192 (     18 tiles): 1.306 / 1.674 / 2.377  (fastest: 1)
//   2-D side   256 (     32 tiles): 1.328 / 1.707 / 2.466  (fastest: 1)
//   2-D side   384 (     72 tiles): 1.576 / 2.004 / 2.926  (fastest: 1)
//   2-D side   512 (    128 tiles): 1.761 / 2.020 / 2.881  (fastest: 1)
//   2-D side   768 (    288 tiles): 2.057 / 2.379 / 3.190  (fastest: 1)
//   2-D side  1024 (    512 tiles): 2.666 / 2.706 / 3.401  (fastest: 1)
//   2-D side  1536 (   1152 tiles): 4.084 / 4.085 / 3.909  (fastest: 4)
//   3-D side    12 (     12 tiles): 1.449 / 2.045 / 3.164  (fastest: 1)
//   3-D side    16 (     16 tiles): 1.446 / 2.046 / 3.246  (fastest: 1)
//   3-D side    24 (     24 tiles): 1.533 / 2.188 / 3.467  (fastest: 1)
//   3-D side    32 (     32 tiles): 1.538 / 2.200 / 3.531  (fastest: 1)
//   3-D side    48 (     96 tiles): 1.937 / 2.653 / 4.220  (fastest: 1)
//   3-D side    64 (    128 tiles): 1.859 / 2.447 / 3.815  (fastest: 1)
//   3-D side    96 (    576 tiles): 3.936 / 3.935 / 5.600  (fastest: 2)
//   3-D side   128 (   1024 tiles): 6.442 / 6.445 / 6.414  (fastest: 4)
// 512-QP batch (best of 3, ms) with groups of at least 1 / 2 / 4 tiles: 268.6 / 223.3 / 220.4  -> at least 2 (within 2 % of the coarsest)
// 512-QP batch (best of 3, ms) for 2 / 4 / 8 tiles per item: 266.0 / 223.2 / 223.1  -> 8
#pragma once

namespace gpcg {

struct TunedGroup {
  int dim, tiles_lo, tiles_hi, group_tiles;
};

constexpr TunedGroup kTunedGroups[] = {
    {2, 1, 1, 4},
    {2, 2, 768, 2},
    {2, 769, 1 << 30, 4},
    {3, 1, 768, 2},
    {3, 769, 1 << 30, 4},
};
constexpr int kTunedItemTiles = 8;

}  // namespace gpcg
