// gpcg_resident.cu -- GPCG for QPs small enough to live in one CTA's shared
// memory (about 1e3 points): the whole solve (Sec. 3, Algorithm GPCG) runs
// inside one thread block, every pass of the engine becoming a block-level
// phase between barriers.  The engine pays a launch, a first copy and a
// grid-wide reduction for every pass; at this size those fixed costs are the
// whole solve, so here every vector stays in shared memory and the
// reductions are block reductions.  The scalar control (FP64 on GB300: slow
// and long-latency) runs in the controlling warp alone, which receives the
// reduced sums and hands its decisions (a code, an index, the step lengths)
// to the block through shared memory.  A batch launches one CTA per small
// instance.
//
// The arithmetic follows Algorithm GPCG step by step: the gradient
// projection phase (Eq. next-y with alpha0 of Eq. bqpls and the sufficient
// decrease of Eq. gplsstop, stopped by Eq. pgstop1 / pgstop2), the CG phase on
// the face (Eq. cg2, stopped by Eq. cgstop1), the projected search (Eq.
// cglsstop2) and the switch of Eq. cgstop3, with the termination test of Eq.
// bqp_approximate_sol; the readings of the paper are those of the engine.  In
// mixed precision an FP32 phase (FP32 iterate in the FP32 box, FP32 vectors
// and bands, each thread's few terms summed in FP32 and the block reduction
// carried in float-float) precedes the FP64 phase, with the same hand-over
// rules as the engine.
#include <cuda_runtime.h>

#include <cstdint>

#include "engine.h"

namespace gpcg {
namespace {

constexpr int kRT = 256;              // threads of the resident CTA
constexpr int kRWarps = kRT / 32;
constexpr int kRPts = 8;              // points per thread at most (n <= 2048)
constexpr int kRMaxN = kRT * kRPts;
constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------- compensated FP32 sums --
// A float-float accumulator: hi + lo carries a sum with about twice the FP32
// precision (the two-sum of Knuth at every addition), converted to FP64 once
// per reduction.
struct F2 {
  float hi, lo;
};

__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);
  const float lo = e + a.lo + b.lo;
  const float hi = s + lo;
  return F2{hi, lo - (hi - s)};
}

// Per-thread partial sums of one phase: FP64 terms in FP64, FP32 terms in
// float-float.
template <class T>
struct Sum;
template <>
struct Sum<double> {
  double v = 0.0;
  __device__ void fma(double a, double b) { v = ::fma(a, b, v); }
  __device__ void add(double a) { v += a; }
};
// A thread adds its few terms (at most kRPts) in FP32; the block reduction
// carries the sums in float-float from there on (as the engine folds a
// chunk's FP32 sums into its float-float accumulators).
template <>
struct Sum<float> {
  float v = 0.0f;
  __device__ void fma(float a, float b) { v = fmaf(a, b, v); }
  __device__ void add(float a) { v += a; }
};

// Scratch of the block reductions: per warp partials of up to 4 sums and 3
// counts, in two sets used in turn (a warp may start the next reduction
// while another still reads the previous one; the set after that is only
// written after a barrier that every reader has passed).
constexpr int kRSums = 4, kRCnts = 3;
struct Red {
  double* part;  // [2][kRSums][kRWarps] (FP32 phases: hi, lo as a float pair)
  int* ipart;    // [2][kRCnts][kRWarps]
  int flip;      // the set of the next reduction (the same in every thread)
};

// Block reduction of K sums and M integer counts in a fixed order: each warp
// reduces by butterfly and writes its partials; after the barrier the
// controlling warp (warp 0) reduces the kRWarps partials by butterfly (IEEE
// addition is commutative, so every lane ends with the same bits).  Only
// warp 0 receives the totals; its decisions reach the block through
// decide().
template <int K, int M>
__device__ __forceinline__ void block_reduce(Sum<double> (&s)[K], int (&c)[M], Red& R,
                                             double (&tot)[K], int (&cnt)[M]) {
  static_assert(K <= kRSums && M <= kRCnts, "reduction scratch");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* P = R.part + R.flip * kRSums * kRWarps;
  int* Q = R.ipart + R.flip * kRCnts * kRWarps;
  R.flip ^= 1;
  double v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = s[k].v;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] += __shfl_xor_sync(kFull, v[k], off);
  }
  int w[M];
#pragma unroll
  for (int m = 0; m < M; ++m) w[m] = __reduce_add_sync(kFull, c[m]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) P[k * kRWarps + warp] = v[k];
#pragma unroll
    for (int m = 0; m < M; ++m) Q[m * kRWarps + warp] = w[m];
  }
  __syncthreads();
  if (warp != 0) return;  // the controlling warp reduces the warps' partials
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = lane < kRWarps ? P[k * kRWarps + lane] : 0.0;
#pragma unroll
  for (int off = kRWarps / 2; off > 0; off >>= 1) {
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] += __shfl_xor_sync(kFull, v[k], off);
  }
#pragma unroll
  for (int k = 0; k < K; ++k) tot[k] = v[k];
#pragma unroll
  for (int m = 0; m < M; ++m) cnt[m] = __reduce_add_sync(kFull, lane < kRWarps ? Q[m * kRWarps + lane] : 0);
}

// The FP32 phases: each warp adds its lanes' FP32 sums (a few terms each)
// by an FP32 butterfly, and the controlling warp adds the warps' sums in
// float-float (the engine likewise folds short FP32 sums into float-float
// accumulators); tot receives hi + lo in FP64, or in FP32 for the FP32 CG
// steps, whose step lengths are FP32 (TT = float).
template <int K, int M, class TT>
__device__ __forceinline__ void block_reduce(Sum<float> (&s)[K], int (&c)[M], Red& R,
                                             TT (&tot)[K], int (&cnt)[M]) {
  static_assert(K <= kRSums && M <= kRCnts, "reduction scratch");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2* P = reinterpret_cast<float2*>(R.part) + R.flip * kRSums * kRWarps;
  int* Q = R.ipart + R.flip * kRCnts * kRWarps;
  R.flip ^= 1;
  float u[K];
#pragma unroll
  for (int k = 0; k < K; ++k) u[k] = s[k].v;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int k = 0; k < K; ++k) u[k] += __shfl_xor_sync(kFull, u[k], off);
  }
  int w[M];
#pragma unroll
  for (int m = 0; m < M; ++m) w[m] = __reduce_add_sync(kFull, c[m]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) P[k * kRWarps + warp] = make_float2(u[k], 0.0f);
#pragma unroll
    for (int m = 0; m < M; ++m) Q[m * kRWarps + warp] = w[m];
  }
  __syncthreads();
  if (warp != 0) return;  // the controlling warp reduces the warps' partials
  F2 v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float2 t = lane < kRWarps ? P[k * kRWarps + lane] : make_float2(0.0f, 0.0f);
    v[k] = F2{t.x, t.y};
  }
#pragma unroll
  for (int off = kRWarps / 2; off > 0; off >>= 1) {
#pragma unroll
    for (int k = 0; k < K; ++k)
      v[k] = f2_add(v[k], F2{__shfl_xor_sync(kFull, v[k].hi, off),
                             __shfl_xor_sync(kFull, v[k].lo, off)});
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if constexpr (sizeof(TT) == 4) tot[k] = v[k].hi + v[k].lo;
    else tot[k] = (double)v[k].hi + (double)v[k].lo;
  }
#pragma unroll
  for (int m = 0; m < M; ++m) cnt[m] = __reduce_add_sync(kFull, lane < kRWarps ? Q[m * kRWarps + lane] : 0);
}

// ------------------------------------------------------ point operations --

template <class T>
__device__ __forceinline__ T mid3(T l, T u, T x) {  // P[x] = mid(l, u, x), Sec. 3
  return x < l ? l : (x > u ? u : x);
}

// Component of the projected gradient (Eq. proj-gradient); a fixed variable
// (l = u) has component 0.
template <class T>
__device__ __forceinline__ T pg_comp(T x, T g, T l, T u) {
  const bool al = x == l, au = x == u;
  if (al && au) return T(0);
  if (al) return g < T(0) ? g : T(0);
  if (au) return g > T(0) ? g : T(0);
  return g;
}

template <class T>
__device__ __forceinline__ bool is_binding(T x, T g, T l, T u) {
  return (x == l && g >= T(0)) || (x == u && g <= T(0));
}

// The arrays of one precision in shared memory, compact row-major layout
// (point i = ix + nx*(iy + ny*iz)): the problem (bands, b, l, u, 1/diag for
// point Jacobi) and the work vectors.
template <class T>
struct Vecs {
  T *d, *cx, *cy, *cz, *b, *l, *u, *dinv;
  T *x, *g, *xt, *gt, *w, *r, *p, *ap;
};

// What a thread owns: points i_k = tid + k*kRT, and for each its
// neighbours present in the grid (bits: west, east, south, north, below,
// above).
struct Own {
  int n, nx, plane, dim;
  unsigned nb[kRPts];
  __device__ bool has(int k) const { return (int)threadIdx.x + k * kRT < n; }
  __device__ int idx(int k) const { return (int)threadIdx.x + k * kRT; }
};

// Row i of A a (Sec. 2), terms in the order diagonal, west, east, south,
// north, below, above.
// A neighbour outside the grid takes the row's own index and a zero
// coupling, so that every load is unconditional and the loads of a thread's
// points issue together (the term adds 0 x a[i], exactly 0 for the finite
// vectors of the solver).
template <class T>
__device__ __forceinline__ T arow(const Vecs<T>& V, const Own& O, int i, unsigned nb, const T* a) {
  const bool hw = nb & 1u, he = nb & 2u, hs = nb & 4u, hn = nb & 8u;
  const int iw = hw ? i - 1 : i, ie = he ? i + 1 : i;
  const int is = hs ? i - O.nx : i, in = hn ? i + O.nx : i;
  const T cw = V.cx[iw], ce = V.cx[i], cs = V.cy[is], cn = V.cy[i];
  T v = V.d[i] * a[i];
  v = fma(hw ? cw : T(0), a[iw], v);
  v = fma(he ? ce : T(0), a[ie], v);
  v = fma(hs ? cs : T(0), a[is], v);
  v = fma(hn ? cn : T(0), a[in], v);
  if (O.dim == 3) {
    const bool hd = nb & 16u, hu = nb & 32u;
    const int id = hd ? i - O.plane : i, iu = hu ? i + O.plane : i;
    const T cd = V.cz[id], cu = V.cz[i];
    v = fma(hd ? cd : T(0), a[id], v);
    v = fma(hu ? cu : T(0), a[iu], v);
  }
  return v;
}


// The solver's state.  The integer counters advance identically in every
// thread (they follow the broadcast decisions).  The FP64 scalars (tau,
// ||pg||^2, eta2, the running maxima of the stop tests, ...) are kept and
// used by the controlling warp only: GB300 runs FP64 at a small fraction of
// the FP32 rate, and the scalar logic repeated by every warp of the block
// would cost more than the vector work of a small problem.
struct RState {
  int status;
  int outer, gp, cg, ls, refine_cg, fp64_gp, continue_cg, refining, stall, slow;
  unsigned sweeps, sweep_cap;
  int bflip;  // the broadcast slot of the next decision
  double pg0, tau, pg2, xgb, nA, nB, eta2, best_pg2, search_pg2, mixed_nA;
};

// A decision of the controlling warp: what happens next, and the step
// lengths the other threads need (in both precisions, so that no thread
// converts them itself).
struct Bc {
  int code, ia;
  double a, b;
  float fa, fb;
};

__device__ __forceinline__ Bc mk(int code, double a = 0.0, double b = 0.0) {
  return Bc{code, 0, a, b, (float)a, (float)b};
}
// A decision whose step lengths are FP32 only (the FP32 CG steps).
__device__ __forceinline__ Bc mkf(int code, float a, float b) {
  return Bc{code, 0, 0.0, 0.0, a, b};
}

// Runs f in the controlling warp and publishes its result to the block.
// Two slots are used in turn: a slot is rewritten two decisions later, after
// a barrier every reader of its previous value has passed.
template <class F>
__device__ __forceinline__ Bc decide(Bc* bc, RState& S, F f) {
  Bc* slot = bc + S.bflip;
  S.bflip ^= 1;
  if ((threadIdx.x >> 5) == 0) {
    const Bc d = f();
    if ((threadIdx.x & 31) == 0) *slot = d;
  }
  __syncthreads();
  return *slot;
}

// Result of a census or an accepted trial at the current iterate.
struct Census {
  double pg2, xgb;
  int nA, nB;
};

// Census of x (Sec. 2): g = A x + b, ||grad_Omega q||^2, <x, g + b> = 2 (q - c),
// |A(x)| and |B(x)|.
template <class T>
__device__ Census census(const Vecs<T>& V, const Own& O, Red& R) {
  Sum<T> s[2];
  int c[2] = {0, 0};
#pragma unroll
  for (int k = 0; k < kRPts; ++k) {
    if (!O.has(k)) continue;
    const int i = O.idx(k);
    const T x = V.x[i], l = V.l[i], u = V.u[i];
    const T g = arow(V, O, i, O.nb[k], V.x) + V.b[i];
    V.g[i] = g;
    const T pg = pg_comp(x, g, l, u);
    s[0].fma(pg, pg);
    s[1].fma(x, g + V.b[i]);
    c[0] += (x == l || x == u);
    c[1] += is_binding(x, g, l, u);
  }
  double t[2];
  int n[2];
  block_reduce(s, c, R, t, n);
  return Census{t[0], t[1], n[0], n[1]};
}

// <g_Omega, g_Omega> and <g_Omega, A g_Omega> at x (Eq. bqpls); g_Omega is
// kept in p.
template <class T>
__device__ void alpha0_sums(const Vecs<T>& V, const Own& O, Red& R, double& gg,
                            double& gAg) {
#pragma unroll
  for (int k = 0; k < kRPts; ++k) {
    if (!O.has(k)) continue;
    const int i = O.idx(k);
    V.p[i] = pg_comp(V.x[i], V.g[i], V.l[i], V.u[i]);
  }
  __syncthreads();
  Sum<T> s[2];
  int c[1] = {0}, n[1];
#pragma unroll
  for (int k = 0; k < kRPts; ++k) {
    if (!O.has(k)) continue;
    const int i = O.idx(k);
    const T pg = V.p[i];
    s[0].fma(pg, pg);
    s[1].fma(pg, arow(V, O, i, O.nb[k], V.p));
  }
  double t[2];
  block_reduce(s, c, R, t, n);
  gg = t[0];
  gAg = t[1];
}

// A trial point xt = P[x + alpha d] (d = -g when dir is null, else dir) with
// its gradient gt = A xt + b and what the tests need: <g, s> and
// <s, g + gt> (s = xt - x; q(xt) - q(x) = <s, g + gt> / 2, exact for a
// quadratic), and the census of xt with the number of points whose active
// status differs from x's (Eq. pgstop1).
struct Trial {
  double gs, sgg;
  Census cs;
  int ndiff;
};

template <class T, class TD>
__device__ Trial trial(const Vecs<T>& V, const Own& O, Red& R, T alpha, const TD* dir) {
#pragma unroll
  for (int k = 0; k < kRPts; ++k) {
    if (!O.has(k)) continue;
    const int i = O.idx(k);
    const T d = dir ? (T)dir[i] : -V.g[i];
    V.xt[i] = mid3(V.l[i], V.u[i], fma(alpha, d, V.x[i]));
  }
  __syncthreads();
  Sum<T> s[4];
  int c[3] = {0, 0, 0};
#pragma unroll
  for (int k = 0; k < kRPts; ++k) {
    if (!O.has(k)) continue;
    const int i = O.idx(k);
    const T xt = V.xt[i], x = V.x[i], l = V.l[i], u = V.u[i], g = V.g[i];
    const T gt = arow(V, O, i, O.nb[k], V.xt) + V.b[i];
    V.gt[i] = gt;
    const T st = xt - x;
    s[0].fma(g, st);
    s[1].fma(st, g + gt);
    const T pg = pg_comp(xt, gt, l, u);
    s[2].fma(pg, pg);
    s[3].fma(xt, gt + V.b[i]);
    const bool at = xt == l || xt == u, ax = x == l || x == u;
    c[0] += at;
    c[1] += is_binding(xt, gt, l, u);
    c[2] += at != ax;
  }
  double t[4];
  int n[3];
  block_reduce(s, c, R, t, n);
  return Trial{t[0], t[1], Census{t[2], t[3], n[0], n[1]}, n[2]};
}


// One more sweep over the instance; false once the sweep cap is reached
// (every thread counts the same sweeps).
__device__ __forceinline__ bool sweep(RState& S) {
  if (++S.sweeps > S.sweep_cap) {
    S.status = S_TIMEOUT;
    return false;
  }
  return true;
}

enum { R_GO = 0, R_CONVERGED = 1, R_FAIL = 2, R_SWITCH = 3 };

// Decision codes.  D_NEXT: reject the trial (or go on), with the next step;
// D_ACCEPT: accept the trial and go on (ia: Eq. cgstop3 held after a
// projected search); D_ACC_STOP: accept, the gradient projection phase ends;
// D_ACC_CONV / D_ACC_SWITCH: accept, then tau is met / the FP32 phase ends;
// D_FAIL, D_SWITCH: a failure (or the end of the FP32 phase) without
// accepting; D_EMPTY: the CG phase takes no step.
enum { D_NEXT = 0, D_ACCEPT, D_ACC_STOP, D_ACC_CONV, D_ACC_SWITCH, D_FAIL, D_SWITCH, D_EMPTY };

template <class T>
__device__ __forceinline__ T step_a(const Bc& d);
template <>
__device__ __forceinline__ float step_a<float>(const Bc& d) { return d.fa; }
template <>
__device__ __forceinline__ double step_a<double>(const Bc& d) { return d.a; }
template <class T>
__device__ __forceinline__ T step_b(const Bc& d);
template <>
__device__ __forceinline__ float step_b<float>(const Bc& d) { return d.fb; }
template <>
__device__ __forceinline__ double step_b<double>(const Bc& d) { return d.b; }

// Make the trial the iterate (every thread swaps the same pointers).
template <class T>
__device__ __forceinline__ void swap_trial(Vecs<T>& V) {
  T* q = V.x;
  V.x = V.xt;
  V.xt = q;
  q = V.g;
  V.g = V.gt;
  V.gt = q;
}

// The controlling warp's copy of the census of the new iterate.
__device__ __forceinline__ void take_census(RState& S, const Census& c) {
  S.pg2 = c.pg2;
  S.xgb = c.xgb;
  S.nA = c.nA;
  S.nB = c.nB;
}

// The gradient projection phase from y_0 = x (Eq. next-y, bqpls, gplsstop),
// ended by Eq. pgstop1, pgstop2 or max_gp.  R_GO: go on to the CG phase.
template <class T>
__device__ int gp_phase(Vecs<T>& V, const Own& O, Red& R, Bc* bc, const Opts& o, RState& S,
                        bool fp32) {
  int j = 0;
  double dmax = 0.0;  // controlling warp
  for (;;) {
    if (!sweep(S)) return R_FAIL;
    double gg = 0.0, gAg = 0.0;
    alpha0_sums(V, O, R, gg, gAg);
    const Bc a0 = decide(bc, S, [&] {
      if (!(gAg > 0.0) || !isfinite(gg)) return mk(D_FAIL);
      return mk(D_NEXT, gg / gAg);  // Eq. bqpls
    });
    if (a0.code == D_FAIL) {
      S.status = S_NUMERIC;
      return R_FAIL;
    }
    Bc step = a0;
    for (int ls_i = 0;;) {
      if (!sweep(S)) return R_FAIL;
      const Trial t = trial<T, T>(V, O, R, step_a<T>(step), (const T*)nullptr);
      S.ls++;
      const Bc d = decide(bc, S, [&] {
        const double dq = 0.5 * t.sgg;  // q(y_t) - q(y_j)
        if (dq <= o.mu * t.gs) {         // Eq. gplsstop
          take_census(S, t.cs);
          const double dec = -dq;
          if (sqrt(S.pg2) <= S.tau) return mk(D_ACC_CONV);
          const bool stop = t.ndiff == 0 ||                          // Eq. pgstop1
                            (j + 1 >= 2 && dec <= o.eta1 * dmax) ||  // Eq. pgstop2
                            j + 1 >= o.max_gp;
          if (dec > dmax) dmax = dec;
          return mk(stop ? D_ACC_STOP : D_ACCEPT);
        }
        // the FP32 gradient may be too coarse for the test: go on in FP64
        if (ls_i + 1 > o.max_ls) return mk(fp32 ? D_SWITCH : D_FAIL);
        return mk(D_NEXT, ldexp(a0.a, -(ls_i + 1)));
      });
      if (d.code == D_NEXT) {
        ++ls_i;
        step = d;
        continue;
      }
      if (d.code == D_FAIL) {
        S.status = S_LINESEARCH;
        return R_FAIL;
      }
      if (d.code == D_SWITCH) return R_SWITCH;
      swap_trial(V);
      S.gp++;
      ++j;
      if (o.mixed && !fp32) S.fp64_gp++;
      if (d.code == D_ACC_CONV) return R_CONVERGED;
      if (d.code == D_ACC_STOP) return R_GO;
      break;  // the next gradient projection step
    }
  }
}

// CG on the reduced system of the current face (Eq. cg2), from w = 0, with
// z = M^-1 r (M = I, or diag(A_k) for point Jacobi), ended by Eq. cgstop1,
// r = 0 or max_cg.  The CG vectors are in precision TC; r_0 = g_F is taken
// from the iterate's gradient.  Each step takes one block reduction, with
// the recurrences of the engine's fused step: step j forms r_j, w_j,
// p_j = -z_j + beta p_{j-1} and A_k p_j, and sums rho_j = <r_j, z_j>,
// <p_j, A_k p_j>, <z_j, A_k p_j> and <A_k p_j, M^-1 A_k p_j>;
// alpha_j = rho_j / <p_j, A_k p_j> and beta_j = rho_{j+1} / rho_j with
// rho_{j+1} = rho_j + 2 alpha_j <z_j, A_k p_j> + alpha_j^2 <A_k p_j, M^-1 A_k p_j>
// (the same as the textbook recurrences in exact arithmetic; a predicted
// rho_{j+1} <= 0 ends the phase as r = 0 does).  The decrease of q_k in step
// j is alpha_j rho_j / 2.  *empty: no step was taken (w = 0).
template <class T, class TC>
__device__ bool cg_phase(const Vecs<T>& V, Vecs<TC>& C, const Own& O, Red& R, Bc* bc,
                         const Opts& o, RState& S, bool* empty) {
  const bool jac = o.precond == PC_JACOBI;
  bool fr[kRPts];
#pragma unroll
  for (int k = 0; k < kRPts; ++k) {
    fr[k] = false;
    if (!O.has(k)) continue;
    const int i = O.idx(k);
    fr[k] = !(V.x[i] == V.l[i] || V.x[i] == V.u[i]);
    const TC r = fr[k] ? (TC)V.g[i] : TC(0);
    C.r[i] = r;
    C.p[i] = -(jac ? r * C.dinv[i] : r);
    C.w[i] = TC(0);
  }
  double cdmax = 0.0;  // controlling warp
  float cdmaxf = 0.0f;  // (FP32 steps)
  const float eta2f = (float)S.eta2;
  TC alpha = TC(0), beta = TC(0);
  *empty = o.max_cg < 1;
  if (*empty) return true;
  for (int j = 0;; ++j) {
    if (!sweep(S)) return false;
    if (j > 0) {
      // r_j, w_j and p_j from step j-1
#pragma unroll
      for (int k = 0; k < kRPts; ++k) {
        if (!O.has(k)) continue;
        const int i = O.idx(k);
        const TC r = fma(alpha, C.ap[i], C.r[i]);
        C.r[i] = r;
        C.w[i] = fma(alpha, C.p[i], C.w[i]);
        C.p[i] = fma(beta, C.p[i], -(jac ? r * C.dinv[i] : r));
      }
    }
    __syncthreads();  // p_j complete before its product
    Sum<TC> a[4];
    int c[1] = {0}, n[1] = {0};
#pragma unroll
    for (int k = 0; k < kRPts; ++k) {
      if (!O.has(k)) continue;
      const int i = O.idx(k);
      const TC ap = fr[k] ? arow(C, O, i, O.nb[k], C.p) : TC(0);
      C.ap[i] = ap;
      const TC r = C.r[i];
      const TC z = jac ? r * C.dinv[i] : r;
      a[0].fma(r, z);
      a[1].fma(C.p[i], ap);
      a[2].fma(z, ap);
      a[3].fma(ap, jac ? ap * C.dinv[i] : ap);
    }
    Bc d;
    if constexpr (sizeof(TC) == 4) {
      // FP32 steps: the step lengths are FP32 numbers, and so is their
      // control (an FP64 division alone takes over a thousand cycles on
      // GB300, at every step of a latency-bound solve)
      float t[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      block_reduce(a, c, R, t, n);
      d = decide(bc, S, [&] {
        const float rho = t[0], pAp = t[1];
        if (j == 0 && !(rho > 0.0f)) return mk(D_EMPTY);  // r = g_F vanished
        if (!(pAp > 0.0f)) return mk(D_FAIL);
        const float al = rho / pAp, inv_rho = 1.0f / rho;
        const float rho_next = fmaf(al * al, t[3], fmaf(2.0f * al, t[2], rho));
        const float delta = 0.5f * al * rho;  // q_k(w_j) - q_k(w_{j+1})
        const bool stop = (j >= 1 && delta <= eta2f * cdmaxf) ||  // Eq. cgstop1 (steps 2, 3, ...)
                          rho_next <= 0.0f || j + 1 >= o.max_cg;
        if (delta > cdmaxf) cdmaxf = delta;
        return mkf(stop ? D_ACC_STOP : D_NEXT, al, stop ? 0.0f : rho_next * inv_rho);
      });
    } else {
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    block_reduce(a, c, R, t, n);
    d = decide(bc, S, [&] {
      const double rho = t[0], pAp = t[1];
      if (j == 0 && !(rho > 0.0)) return mk(D_EMPTY);  // r = g_F vanished
      if (!(pAp > 0.0)) return mk(D_FAIL);
      // 1/rho is formed beside alpha (two independent divisions), so that
      // beta costs one multiplication after rho_{j+1}: a dependent FP64
      // operation takes tens of cycles on GB300
      const double al = rho / pAp, inv_rho = 1.0 / rho;
      const double rho_next = fma(al * al, t[3], fma(2.0 * al, t[2], rho));
      const double delta = 0.5 * al * rho;  // q_k(w_j) - q_k(w_{j+1})
      const bool stop = (j >= 1 && delta <= S.eta2 * cdmax) ||  // Eq. cgstop1 (steps 2, 3, ...)
                        rho_next <= 0.0 || j + 1 >= o.max_cg;
      if (delta > cdmax) cdmax = delta;
      return mk(stop ? D_ACC_STOP : D_NEXT, al, stop ? 0.0 : rho_next * inv_rho);
    });
    }
    if (d.code == D_EMPTY) {
      *empty = true;
      return true;
    }
    if (d.code == D_FAIL) {
      S.status = S_NUMERIC;
      return false;
    }
    S.cg++;
    if (S.refining) S.refine_cg++;
    alpha = step_a<TC>(d);
    beta = step_b<TC>(d);
    if (d.code == D_ACC_STOP) {
      // w_{j+1} = w_j + alpha_j p_j, the direction of the projected search
#pragma unroll
      for (int k = 0; k < kRPts; ++k) {
        if (!O.has(k)) continue;
        const int i = O.idx(k);
        C.w[i] = fma(alpha, C.p[i], C.w[i]);
      }
      return true;
    }
  }
}

// The projected search along d = Z w (Eq. cglsstop2): x_t = P[x + alpha d],
// alpha = 1, 1/2, ... (0 after an empty CG phase), then the tests of the
// outer iterate: tau, the end of the FP32 phase (five iterates without a 2 %
// decrease of ||pg||^2, or two in a row on an unchanged face that do not
// halve ||pg||: the FP32 noise floor), and Eq. cgstop3 (S.continue_cg).
template <class T, class TD>
__device__ int search(Vecs<T>& V, const Own& O, Red& R, Bc* bc, const Opts& o, RState& S,
                      const TD* w, bool empty, bool fp32) {
  Bc step = mk(D_NEXT, empty ? 0.0 : 1.0);
  for (int ls_i = 0;;) {
    if (!sweep(S)) return R_FAIL;
    const Trial t = trial<T, TD>(V, O, R, step_a<T>(step), w);
    S.ls++;
    const Bc d = decide(bc, S, [&] {
      if (0.5 * t.sgg <= o.mu * t.gs) {
        take_census(S, t.cs);
        if (sqrt(S.pg2) <= S.tau) return mk(D_ACC_CONV);
        if (fp32) {
          const bool face_kept = S.nB == S.nA;
          const bool halved = S.pg2 < 0.25 * S.search_pg2;
          S.search_pg2 = S.pg2;
          S.slow = (face_kept && !halved) ? S.slow + 1 : 0;
          if (S.pg2 < 0.98 * S.best_pg2) {
            S.best_pg2 = S.pg2;
            S.stall = 0;
          } else {
            ++S.stall;
          }
          if (S.stall >= 5 || S.slow >= 2) return mk(D_ACC_SWITCH);
        }
        Bc r = mk(D_ACCEPT);
        if (S.nB == S.nA) {  // Eq. cgstop3: B(x) = A(x)
          S.eta2 = fmax(S.eta2 * o.eta2_shrink, o.eta2_floor);
          r.ia = 1;
        } else {
          S.eta2 = o.eta2;
          r.ia = 0;
        }
        return r;
      }
      if (ls_i + 1 > o.max_ls) return mk(fp32 ? D_SWITCH : D_FAIL);
      return mk(D_NEXT, empty ? 0.0 : ldexp(1.0, -(ls_i + 1)));
    });
    if (d.code == D_NEXT) {
      ++ls_i;
      step = d;
      continue;
    }
    if (d.code == D_FAIL) {
      S.status = S_LINESEARCH;
      return R_FAIL;
    }
    if (d.code == D_SWITCH) return R_SWITCH;
    swap_trial(V);
    S.refining = 0;
    if (d.code == D_ACC_CONV) return R_CONVERGED;
    if (d.code == D_ACC_SWITCH) return R_SWITCH;
    S.continue_cg = d.ia;
    return R_GO;
  }
}

// Outer iterates of Algorithm GPCG in precision T (CG phases in TC) from the
// current iterate.  enter_cg: start with the CG phase of an outer iterate
// already counted (the closing CG phase after the FP32 phase).  fp32: the
// FP32 phase.
template <class T, class TC>
__device__ int gpcg_loop(Vecs<T>& V, Vecs<TC>& C, const Own& O, Red& R, Bc* bc, const Opts& o,
                         RState& S, bool fp32, bool enter_cg) {
  for (bool skip = enter_cg;; skip = false) {
    if (!skip) {
      if (S.outer >= o.max_outer) {
        S.status = S_MAXIT;
        return R_FAIL;
      }
      S.outer++;
      if (!S.continue_cg) {
        const int r = gp_phase(V, O, R, bc, o, S, fp32);
        if (r != R_GO) return r;
      }
    }
    bool empty = false;
    if (!cg_phase(V, C, O, R, bc, o, S, &empty)) return R_FAIL;
    const int r = search<T, TC>(V, O, R, bc, o, S, C.w, empty, fp32);
    if (r != R_GO) return r;
  }
}

// Shared-memory layout: the reductions' scratch, then 16-byte aligned arrays
// of n values: the FP64 problem and work vectors, and with mixed precision
// the same in FP32.
constexpr size_t kHeadRed = 1920;  // the reductions' partials (1,408 bytes at 16 warps)
constexpr size_t kHead = 2048;     // ... then the two broadcast slots
static_assert(sizeof(double) * 2 * kRSums * kRWarps + sizeof(int) * 2 * kRCnts * kRWarps <=
                  kHeadRed,
              "reduction scratch");
static_assert(kHeadRed + 2 * sizeof(Bc) <= kHead, "broadcast slots");

__host__ __device__ inline int n_arrays(int dim, bool jac) { return 14 + (dim == 3) + (jac ? 1 : 0); }

__host__ __device__ inline size_t smem_bytes(int dim, long long n, bool mixed, bool jac) {
  const size_t a = (size_t)n_arrays(dim, jac);
  size_t b = kHead + a * 8 * (size_t)((n + 1) / 2 * 2);
  if (mixed) b += a * 4 * (size_t)((n + 3) / 4 * 4);
  return b;
}

template <class T>
__device__ Vecs<T> carve(unsigned char*& cur, int n, int dim, bool jac) {
  const size_t step = sizeof(T) * (size_t)(sizeof(T) == 8 ? (n + 1) / 2 * 2 : (n + 3) / 4 * 4);
  auto take = [&]() {
    T* a = reinterpret_cast<T*>(cur);
    cur += step;
    return a;
  };
  Vecs<T> V;
  V.d = take();
  V.cx = take();
  V.cy = take();
  V.cz = dim == 3 ? take() : nullptr;
  V.b = take();
  V.l = take();
  V.u = take();
  V.dinv = jac ? take() : nullptr;
  V.x = take();
  V.g = take();
  V.xt = take();
  V.gt = take();
  V.w = take();
  V.r = take();
  V.p = take();
  V.ap = take();
  return V;
}

// x from the FP32 iterate: the FP64 bound where x32 sits at its FP32 bound
// (the FP32 projection returns the bound itself), else P[x32] in FP64.
__device__ void rebuild_x(Vecs<double>& V, const Vecs<float>& F, int n) {
  for (int i = threadIdx.x; i < n; i += kRT) {
    const float xf = F.x[i];
    V.x[i] = xf == F.l[i] ? V.l[i] : (xf == F.u[i] ? V.u[i] : mid3(V.l[i], V.u[i], (double)xf));
  }
  __syncthreads();
}

// One CTA solves instance ids[blockIdx.x] of the table entirely in shared
// memory and leaves x, g, the free-set words and its control block as the
// engine would.
__global__ void __launch_bounds__(kRT, 1)
    resident_kernel(const DevInst* __restrict__ insts, const int* __restrict__ ids, Ctl* ctl,
                    unsigned sweep_cap) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int slot = ids[blockIdx.x];
  const DevInst& I = insts[slot];
  const Opts o = I.opt;
  const int n = (int)I.n, nx = I.nx, ny = I.ny, nz = I.nz, px = I.px, dim = I.dim;
  const bool jac = o.precond == PC_JACOBI, mixed = o.mixed != 0;
  const int tid = threadIdx.x;

  Red R;
  R.part = reinterpret_cast<double*>(sm);
  R.ipart = reinterpret_cast<int*>(sm + sizeof(double) * 2 * kRSums * kRWarps);
  R.flip = 0;
  unsigned char* cur = sm + kHead;
  Vecs<double> V = carve<double>(cur, n, dim, jac);
  Vecs<float> F{};
  if (mixed) F = carve<float>(cur, n, dim, jac);

  Own O;
  O.n = n;
  O.nx = nx;
  O.plane = nx * ny;
  O.dim = dim;
#pragma unroll
  for (int k = 0; k < kRPts; ++k) {
    const int i = tid + k * kRT;
    const int ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
    unsigned m = 0;
    if (ix > 0) m |= 1u;
    if (ix + 1 < nx) m |= 2u;
    if (iy > 0) m |= 4u;
    if (iy + 1 < ny) m |= 8u;
    if (dim == 3 && iz > 0) m |= 16u;
    if (dim == 3 && iz + 1 < nz) m |= 32u;
    O.nb[k] = m;
  }

  // the problem from the padded global arrays; x = P[x0], x0 the given start
  // or l, falling back to u then 0 where a bound is infinite
  for (int i = tid; i < n; i += kRT) {
    const int ix = i % nx, row = i / nx;
    const long long ip = (long long)row * px + ix;
    const double d = I.diag[ip], cx = I.cx[ip], cy = I.cy[ip], b = I.b[ip], l = I.l[ip],
                 u = I.u[ip];
    V.d[i] = d;
    V.cx[i] = cx;
    V.cy[i] = cy;
    V.b[i] = b;
    V.l[i] = l;
    V.u[i] = u;
    if (dim == 3) V.cz[i] = I.cz[ip];
    if (jac) V.dinv[i] = I.dinv[ip];
    const double s = o.use_x0 ? I.x0[ip] : (isfinite(l) ? l : (isfinite(u) ? u : 0.0));
    const double x = mid3(l, u, s);
    V.x[i] = x;
    if (mixed) {
      F.d[i] = (float)d;
      F.cx[i] = (float)cx;
      F.cy[i] = (float)cy;
      F.b[i] = (float)b;
      F.l[i] = (float)l;
      F.u[i] = (float)u;
      if (dim == 3) F.cz[i] = (float)V.cz[i];
      if (jac) F.dinv[i] = (float)V.dinv[i];
      F.x[i] = (float)x;
    }
  }
  __syncthreads();

  Bc* bc = reinterpret_cast<Bc*>(sm + kHeadRed);
  RState S{};
  S.status = S_RUNNING;
  S.sweep_cap = sweep_cap;
  S.mixed_nA = -1.0;
  S.eta2 = o.eta2;
  bool x32_live = mixed;
  int res = R_FAIL;
  // the census at x0 sets tau (Eq. bqp_approximate_sol, relative to ||pg(x0)||)
  const Census c0 = mixed ? census(F, O, R) : census(V, O, R);
  const Bc d0 = decide(bc, S, [&] {
    take_census(S, c0);
    S.best_pg2 = S.search_pg2 = S.pg2;
    S.pg0 = sqrt(S.pg2);
    S.tau = fmax(o.tau_abs, o.tau_rel * S.pg0);
    if (!isfinite(S.pg2)) return mk(D_FAIL);
    return mk(S.pg0 <= S.tau ? D_ACC_CONV : D_NEXT);
  });
  if (d0.code == D_FAIL) {
    S.status = S_NUMERIC;
  } else if (d0.code == D_ACC_CONV) {
    res = R_CONVERGED;
  } else if (!mixed) {
    res = gpcg_loop<double, double>(V, V, O, R, bc, o, S, false, false);
  } else {
    res = gpcg_loop<float, float>(F, F, O, R, bc, o, S, true, false);
    if (res == R_CONVERGED || res == R_SWITCH) {
      // hand over to FP64: a census at x rebuilt from x32, then the closing
      // CG phase on that face (refine) or GPCG in FP64
      const bool refine = res == R_CONVERGED && o.refine != 0;
      rebuild_x(V, F, n);
      x32_live = false;
      const Census ch = census(V, O, R);
      const Bc dh = decide(bc, S, [&] {
        take_census(S, ch);
        S.mixed_nA = S.nA;
        if (refine) {
          S.eta2 = o.eta2_refine;
          return mk(D_NEXT);
        }
        if (!isfinite(S.pg2)) return mk(D_FAIL);
        if (sqrt(S.pg2) <= S.tau) return mk(D_ACC_CONV);
        S.eta2 = o.eta2;
        return mk(D_NEXT);
      });
      if (dh.code == D_FAIL) {
        S.status = S_NUMERIC;
        res = R_FAIL;
      } else if (dh.code == D_ACC_CONV) {
        res = R_CONVERGED;
      } else {
        S.refining = refine ? 1 : 0;
        S.continue_cg = refine ? 1 : 0;
        if (refine) S.outer++;
        res = o.refine == 2 ? gpcg_loop<double, float>(V, F, O, R, bc, o, S, false, refine)
                            : gpcg_loop<double, double>(V, V, O, R, bc, o, S, false, refine);
      }
    }
  }
  if (res == R_CONVERGED) S.status = S_OK;
  // statistics at the returned point: an FP64 census (rebuilding x when the
  // FP32 iterate was still live)
  if (x32_live) rebuild_x(V, F, n);
  const Census cf = census(V, O, R);
  if (tid == 0) take_census(S, cf);

  double* xo = I.x[0];
  double* go = I.g[0];
  for (int i = tid; i < n; i += kRT) {
    const int ix = i % nx, row = i / nx;
    const long long ip = (long long)row * px + ix;
    xo[ip] = V.x[i];
    go[ip] = V.g[i];
  }
  // free-set words of x: bit (ix & 31) of word row*mw + ix/32
  const int rows = ny * nz, mw = I.mw;
  for (int wd = tid; wd < rows * mw; wd += kRT) {
    const int row = wd / mw, c0w = 32 * (wd - row * mw);
    unsigned bits = 0u;
    for (int bt = 0; bt < 32 && c0w + bt < nx; ++bt) {
      const int i = row * nx + c0w + bt;
      if (!(V.x[i] == V.l[i] || V.x[i] == V.u[i])) bits |= 1u << bt;
    }
    I.mask[0][(long long)row * mw + wd - row * mw] = bits;
  }
  if (tid == 0) {
    Ctl C{};
    C.pass = P_NONE;
    C.done = 1;
    C.status = S.status;
    C.outer_iters = S.outer;
    C.gp_iters = S.gp;
    C.cg_iters = S.cg;
    C.ls_trials = S.ls;
    C.refine_cg_iters = S.refine_cg;
    C.fp64_gp = S.fp64_gp;
    C.passes = 1;
    C.pg2 = S.pg2;
    C.xgb = S.xgb;
    C.nA = S.nA;
    C.nB = S.nB;
    C.tau = S.tau;
    C.pg0 = S.pg0;
    C.eta2 = S.eta2;
    C.mixed_nA = S.mixed_nA;
    C.alg_bytes = (double)n * (8.0 * (I.kc + 3 + (jac ? 1 : 0) + (o.use_x0 ? 1 : 0)) + 16.0) +
                  4.0 * rows * mw;
    ctl[slot] = C;
  }
}

}  // namespace

// Shared-memory bytes of the resident solve of an instance (0 when it does
// not fit: more than 2048 points or more than the CTA's shared memory).
size_t resident_smem(int dim, long long n, bool mixed, bool jacobi) {
  if (n < 1 || n > kRMaxN) return 0;
  const size_t b = smem_bytes(dim, n, mixed, jacobi);
  return b <= (size_t)227 * 1024 ? b : 0;
}

// Launch the resident solver for `count` instances of the descriptor table
// (their slots in ids), one CTA each, with the largest shared-memory size
// among them.
cudaError_t launch_resident(const DevInst* insts, const int* ids, Ctl* ctl, int count,
                            size_t smem, unsigned sweep_cap, cudaStream_t s) {
  cudaError_t e =
      cudaFuncSetAttribute(resident_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  resident_kernel<<<count, kRT, smem, s>>>(insts, ids, ctl, sweep_cap);
  return cudaGetLastError();
}

}  // namespace gpcg
