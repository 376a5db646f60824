// engine.h -- data shared by the host driver and the device passes of the
// GPCG engine.  Internal to libgpcg.so (the public ABI is include/gpcg.h).
//
// Layout in device memory (one problem):
//   every per-point array is stored with a padded row pitch px (a multiple of
//   8 elements, so each row starts on a 64-byte boundary for FP64 and 32-byte
//   for FP32); point (ix, iy, iz) lives at ix + px*(iy + ny*iz).  Pad columns
//   ix >= nx hold zeros and are never read as neighbours.
//   The free set is a bitmask: bit (ix & 31) of word (iy + ny*iz)*mw + ix/32
//   is 1 when the point is free; mw = ceil(px/32) rounded up to a multiple of
//   4 words, so that mask rows are 16-byte strides TMA can stage.
//
// One engine pass = one launch of the pass kernel over the tile table of all
// live instances.  Each CTA processes one 64 x 32 tile of one instance, writes
// its partial sums to a fixed slot, and the last CTA of an instance to finish
// reduces that instance's partials in a fixed order and advances the
// instance's GPCG state machine (Sec. 3, Algorithm GPCG).  Results therefore
// depend only on the instance itself, never on what else shares the launch.
#pragma once

#include <cstdint>

namespace gpcg {

constexpr int kTX = 64;          // tile width (columns): 32 lanes x 2 points
constexpr int kRY = 4;           // rows per warp
constexpr int kWarps = 8;        // warps per CTA
constexpr int kTY = kRY * kWarps;  // tile height (rows)
constexpr int kThreads = 32 * kWarps;
constexpr int kNRed = 8;         // partial sums per tile: 4 FP64 sums, 3 counts, 1 spare
constexpr int kMinBlocks = 2;    // resident CTAs per SM the pass kernel is compiled for

// The groups of an instance are consecutive ranges of its tiles; they depend
// only on its shape (about group_tiles tiles each, chosen per shape by the
// tuned table, at most kMaxGroups groups), and each group has one
// partial-sum slot, so the order of every sum is fixed by the shape.  A work
// item of a launch is a run of up to kMaxSpan consecutive groups of one
// instance (DevInst.span, the launch's choice): coarser items for crowded
// launches, one group per item for a lone solve, the same sums either way.
constexpr int kMaxGroups = 304;
constexpr int kMaxSpan = 2;

// TMA staging: a work item is streamed through shared memory in chunks of
// 64 columns by 8-32 rows, kStages stages deep (the next chunk is in flight
// while one is computed).  Two CTAs of the pass kernel fit on one SM.
constexpr int kStages = 2;
constexpr int kStageBytes = 45568;   // one stage: the largest layout (45056) + the mask box
constexpr int kMaskBox = 512;        // 4 words x 32 rows, at the end of every stage
constexpr int kOffMask = kStageBytes - kMaskBox;
constexpr int kDynSmem = kStages * kStageBytes + 128 + 8 * kStages;

// Tensor maps of an instance (one CUtensorMap, 128 bytes, each).  With c the
// CG_B chunk (32 rows FP32, 16 FP64) and a the CG_A chunk (32 / 16 rows):
// H = halo box (64+2h) x (c+2) starting at (x0-h, y0-1); D = 64 x c;
// CX = (64+h) x c from x0-h; CY = 64 x (c+1) from y0-1; W, R, P, AP are
// 64 x a boxes over the (nx, ny*nz) row space.
//
// The mixed-phase gradient-projection passes of a 2-D instance stage 16-row
// chunks (census, trial; their band boxes are the fused pass's FD, FCX, FCY)
// and 32-row chunks (alpha0): G18 = FP32 halo box 72 x 18 from (x0-4, y0-1);
// G34 = FP32 halo box 72 x 34; the interior boxes are 64 x 16.
//
// The fused CG pass (2-D) stages f-row chunks (16 FP32, 8 FP64): FRH, FPH,
// FAPH = halo boxes (64+2h) x (f+2) of r, p, Ap; FW, FD = 64 x f; FCX =
// (64+h) x f; FCY = 64 x (f+1); FDIH = halo box of 1/diag (Jacobi).  r, p
// and Ap are double-buffered (index pcur: the current vectors), so each map
// of them comes in two.  ADI = 64 x a box of 1/diag for P_CG_A.  FZH, FQH:
// halo boxes of z = M^-1 r and q = M^-1 Ap under the tile preconditioner
// (encoded when its vectors are first needed).
enum TMap : int {
  M32_RH0 = 0, M32_RH1, M32_PH0, M32_PH1, M32_D, M32_CX, M32_CY, M32_W, M32_R0, M32_R1, M32_P0,
  M32_P1, M32_AP0, M32_AP1, M32_FRH0, M32_FRH1, M32_FPH0, M32_FPH1, M32_FAPH0, M32_FAPH1, M32_FW,
  M32_FD, M32_FCX, M32_FCY, M32_FDIH, M32_ADI, M32_FZH0, M32_FZH1, M32_FQH0, M32_FQH1,
  M64_RH0, M64_RH1, M64_PH0, M64_PH1, M64_D, M64_CX, M64_CY, M64_W, M64_R0, M64_R1, M64_P0,
  M64_P1, M64_AP0, M64_AP1, M64_FRH0, M64_FRH1, M64_FPH0, M64_FPH1, M64_FAPH0, M64_FAPH1, M64_FW,
  M64_FD, M64_FCX, M64_FCY, M64_FDIH, M64_ADI, M64_FZH0, M64_FZH1, M64_FQH0, M64_FQH1,
  MG_X32H0, MG_X32H1, MG_L32H, MG_U32H, MG_G32H0, MG_G32H1, MG_W32H,  // G18
  MG_PGH0, MG_PGH1,                                                  // G34
  MG_L32, MG_U32, MG_B32,                                            // 64 x 16
  // the trial along -g with alpha0 at the trial point: halo-2 boxes 72 x 20
  // from (x0-4, y-2) of x32[2], l32, u32, g32[2]; 72 x 18 from (x0-4, y-1) of
  // b32 and the FP32 diag, cx; 72 x 19 from (x0-4, y-2) of the FP32 cy
  MG_X2H0, MG_X2H1, MG_L2H, MG_U2H, MG_G2H0, MG_G2H1, MG_B18, MG_D18, MG_CX18, MG_CY19,
  M_MASK0, M_MASK1,  // free-set words of mask[0], mask[1]: box 4 words x 32 rows
  M_MASKH0, M_MASKH1,  // the same words, box 8 words x 18 rows (staged first CG step)
  // the staged FP64 GP passes (FEAT_F64 kernels): halo boxes 68 x 10 from
  // (x0-2, y-1) of x[2], g[2], l, u, w (FP64), and b as a 64 x 8 box
  MF_X0, MF_X1, MF_G0, MF_G1, MF_L, MF_U, MF_W, MF_B,
  // the fused CG step of 3-D grids (FP32, 8-row chunks of one plane): halo
  // boxes 72 x 10 from (x0-4, row-1) of r[2], p[2], Ap[2]; 64 x 8 boxes of w
  // and diag; 68 x 8 of cx from x0-4; 64 x 9 of cy from row-1; 64 x 8 boxes of
  // cz and of r[2], p[2], Ap[2] (taken at the rows of the planes below and
  // above: row -+ ny)
  M3_RH0, M3_RH1, M3_PH0, M3_PH1, M3_APH0, M3_APH1, M3_W, M3_D, M3_CX, M3_CY, M3_CZ,
  M3_R0, M3_R1, M3_P0, M3_P1, M3_AP0, M3_AP1,
  M_COUNT
};
constexpr int kGpMaps = M_MASK0 - MG_X32H0;  // the GP maps (make_gp_maps encodes them)
constexpr int kCgMaps = M64_RH0 - M32_RH0;  // maps of one precision's CG passes
constexpr int kCgBase = M32_FZH0 - M32_RH0;  // of which make_maps encodes the first kCgBase
constexpr int kTileMaps = kCgMaps - kCgBase;  // and the tile preconditioner's the rest
constexpr int k3dMaps = M3_AP1 - M3_RH0 + 1;  // the 3-D fused step's maps

enum Pass : int {
  P_NONE = 0,
  P_START = 1,     // x = P[x0]
  P_CENSUS = 2,    // g = Ax + b, free mask, |A|, |B|, ||pg||^2, q
  P_GP_ALPHA = 3,  // <pg,pg>, <pg, A pg> for alpha0 (Eq. bqpls)
  P_TRIAL = 4,     // trial point P[x + alpha*dir] with gradient and census
  P_CG_B = 5,      // p = -r + beta p; Ap = A_FF p; <p, Ap>
  P_CG_A = 6,      // w += alpha p; r += alpha Ap; ||r||^2
  P_CG_F = 7,      // fused CG step (staged; 3-D: FP32 only): r += alpha Ap, w += alpha p,
                   // p = -r + beta p, Ap = A_FF p; ||r||^2, <p,Ap>, <r,Ap>, ||Ap||^2
  P_CG_Z = 8,      // first step of a tile-preconditioned CG phase: r = g_F,
                   // z = M^-1 r, <r, z>; p, Ap, q = M^-1 Ap and w set to 0
  // explicit reduced system (option extract, Sec. 4's extraction of A_k):
  P_RX_COUNT = 9,  // free points per group -> group offsets of the compact numbering
  P_RX_MAP = 10,   // compact index of every free point, r_0 = g_F (compact), w = 0
  P_RX_BUILD = 11, // rows of A_FF in compact numbering; z_0, rho_0; p, Ap, w = 0
  P_RCG = 12,      // fused CG step on the compact system
  P_RW = 13,       // w (full length) = the compact w_{j+1}, before the search
};

// Neighbour slots of a row of the explicit reduced system: x-1, x+1, y-1,
// y+1 (, z-1, z+1); a slot whose neighbour is outside the free set holds the
// row's own compact index and a zero coupling.
constexpr int kMaxNb = 6;

// Optional pass families, compiled into their own instantiations of the
// pass kernel so that the default kernel carries none of their code.
enum Feature : int { FEAT_TILE = 1, FEAT_EXT = 2, FEAT_F64 = 4, FEAT_3D = 8 };

// Preconditioners of the CG phase (Opts.precond; the public gpcg_precond).
enum Precond : int { PC_NONE = 0, PC_JACOBI = 1, PC_TILE = 2 };

// The tile preconditioner's blocks: 64 x 8 points of one xy-plane, starting
// at multiples of 64 in x and 8 in y.
constexpr int kBlkX = 64;
constexpr int kBlkY = 8;

enum Dir : int { D_NEG_G = 0, D_W64 = 1, D_W32 = 2, D_ZERO = 3 };

// Purpose of a P_CENSUS pass.
enum CensusMode : int {
  CM_INIT = 0,    // at x0: sets tau
  CM_FINAL = 1,   // at the returned point: refreshes the statistics, ends the solve
  CM_REFINE = 2,  // first FP64 census after the mixed phase met tau: closing FP64 CG
  CM_RESUME = 3,  // first FP64 census after the mixed phase stalled: continue in FP64
};

// Status values mirror gpcg_status.
enum Status : int {
  S_OK = 0,
  S_NUMERIC = 3,
  S_MAXIT = 7,
  S_LINESEARCH = 8,
  S_TIMEOUT = 9,
  S_RUNNING = 10,
};

struct Opts {
  double tau_abs, tau_rel, eta1, eta2, mu, eta2_shrink, eta2_floor, eta2_refine;
  double c;
  int max_outer, max_gp, max_cg, max_ls;
  int mixed, refine, use_x0, precond;  // precond: a Precond value
  int extract, pad_o;  // extract: the CG phase runs on the explicit reduced system
};

// Mutable per-instance state, owned by the finalizer of each pass.
struct Ctl {
  int pass, status, done, cur, pcur, cg32, first_cg, dir;
  int trial_gp, refining, refined, continue_cg, hold;
  int x32_live;      // mixed phase: the iterate lives in x32; the next FP64 census rebuilds x
  int outer_iters, gp_j, ls_i, cg_j, gp_iters, cg_iters, ls_trials, refine_cg_iters;
  int passes;
  int gp32;          // mixed phase: census / GP / search passes stream FP32 (see kernels)
  unsigned arrive;
  int census_mode;   // CM_* : what the next P_CENSUS is for
  int stall;         // mixed phase: outer iterates without progress of ||pg||
  int slow;          // mixed phase: consecutive iterates on an unchanged face without
                     // a halving of ||pg|| (the FP32 noise floor)
  int fp64_gp;       // mixed precision: GP steps taken in FP64 after the FP32 phase
  int cg_finish;     // the pending P_CG_A only completes w before the search
  int m;             // explicit reduced system: free points of the current phase
  int pad_m;
  double best_pg2;   // mixed phase: smallest ||pg||^2 seen
  double search_pg2; // mixed phase: ||pg||^2 after the previous outer iterate
  double alpha0, alpha, beta, rr, dmax, cdmax, eta2, tau, pg0;
  double pg2, nA, nB, xgb, gF2;  // census of the current iterate
  double alg_bytes;              // algorithmic HBM bytes of all passes so far
  double mixed_nA;               // |A| at the first FP64 census after the FP32 phase (-1: none)
  double red[kNRed];             // reduced sums of the latest pass
};

struct DevInst {
  int dim, nx, ny, nz, px, mw, tiles_x, tiles_y, n_tiles, kc;
  int n_groups, span;      // groups of the instance; groups per work item of this launch
  long long n, plane;
  double* part;            // [2][kNRed][n_groups] group partial sums of this instance
                           // (slot-major; the cooperative kernel alternates the two)
  const void* tmaps;       // M_COUNT CUtensorMaps in device memory (64-byte aligned)
  int tma64, tma32;        // the FP64 / FP32 CG maps are valid
  int tma_gp, tma_mask;    // the mixed-phase GP maps / the mask maps are valid
  int tma_f64gp;           // the FP64 alpha0 maps are valid
  int tma3;                // the 3-D fused step's maps (FP32) are valid, and this launch's
                           // kernel has the step (FEAT_3D; the host clears it otherwise)
  const double *diag, *cx, *cy, *cz, *b, *l, *u, *x0;
  const float *diag32, *cx32, *cy32, *cz32;
  const double* dinv;      // 1/diag (0 in pad columns): the point-Jacobi preconditioner
  const float* dinv32;
  int tma_tile;            // bit 0 / bit 1: the FP64 / FP32 tile-preconditioner maps are valid
  int pad_t;
  double *z64[2], *q64[2];  // tile preconditioner: z = M^-1 r, q = M^-1 Ap (index pcur)
  float *z32[2], *q32[2];
  // explicit reduced system (capacity n): compact index of each point (padded
  // layout, -1 off the free set), point of each compact index, group offsets,
  // neighbour slots [kMaxNb][n]; per precision the rows (diagonal, couplings
  // [kMaxNb][n], 1/diagonal) and the compact CG vectors (r, p, Ap by pcur)
  int *cidx, *fidx, *goff, *rnb;
  double *rd64, *rv64, *rdi64, *rc64[2], *pc64[2], *apc64[2], *wc64;
  float *rd32, *rv32, *rdi32, *rc32[2], *pc32[2], *apc32[2], *wc32;
  int rx64, rx32;          // the FP64 / FP32 compact arrays exist
  double *x[2], *g[2];
  unsigned* mask[2];
  double *r64[2], *w64, *p64[2], *Ap64[2];  // r, p, Ap double-buffered (index pcur)
  float *r32[2], *w32, *p32[2], *Ap32[2];
  float *x32[2], *g32[2], *b32, *l32, *u32;  // FP32 iterate and copies of the mixed phase
  float* pg32[2];          // mixed phase: grad_Omega q at x[k] (FP32), read by alpha0
  Opts opt;
};

struct EngineArgs {
  const DevInst* insts;
  Ctl* ctl;
  const int2* tiles;      // (instance slot, group) work items of the launch
  int n_work;             // number of work items
  int* queue;             // next work item (dynamic scheduling; reset by the last CTA)
  unsigned* exits;        // CTAs that found the queue empty
  int* live;              // instances not yet done
  unsigned* npass;        // passes so far (block 0 increments)
  int* err;               // bit 0: a copy's bounded wait gave up; bit 1: the pass is not in
                          // this instantiation; bit 2: the grid barrier's bounded wait gave up
  unsigned pass_cap;      // passes after which the loop (condition) ends
  unsigned long long cond;  // cudaGraphConditionalHandle, 0 when not in a WHILE graph
  unsigned* gbar;           // arrivals at the cooperative kernel's grid barrier (zero before
                            // its launch); unused by the other launches
};

}  // namespace gpcg
