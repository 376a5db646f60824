// pass_engine.cuh -- the GPCG engine's pass kernel and its device code.
//
// Included by the translation units that instantiate the pass kernel: one
// per feature set (gpcg_kernels.cu: the default passes; gpcg_pass_tile.cu:
// with the tile preconditioner; gpcg_pass_rx.cu: with the explicit reduced
// system; gpcg_pass_f64.cu, gpcg_pass_3d.cu), so that the default kernel
// carries none of the optional code, and by gpcg_coop.cu and
// gpcg_coop_f64.cu, which instantiate the cooperative kernel (GPCG_COOP).
//
// One kernel, pass_kernel, runs every pass of Algorithm GPCG (Sec. 3 of
// Benson, McInnes & More) for every live instance.  The grid is persistent
// (two CTAs per SM); CTAs take work items -- one or two groups of 64x32
// tiles of one instance -- perform the pass the instance's state machine
// asks for, and deposit each group's partial sums in the group's own slot.
// The last CTA to finish an instance's groups reduces its slots in a fixed
// order and runs the state-machine transition (finalize below), so an
// instance's arithmetic depends only on the instance, never on the schedule
// or on the other instances in the launch.  The cooperative kernel,
// pass_kernel_coop, runs all passes of one instance in one launch: every
// CTA reduces the slots and runs the transition after a grid barrier.
//
// Stencil passes stream each operand once: a warp walks down its 64-column
// strip keeping the operand of rows y-1, y, y+1 in registers; east/west
// neighbours come from the adjacent lane by shuffle (lanes 0 and 31 load the
// point beyond the strip), and the planes above/below of a 3-D grid are
// loaded directly.  The operand is computed from its inputs on the fly (for
// example p = -r + beta*p in the CG pass, or P[x + alpha*d] in a trial), so no
// pass writes a vector that another CTA of the same launch reads.
//
// GB300 executes FP64 at a small fraction of its FP32 rate, so FP64 work is
// kept to the arithmetic the method needs: comparisons against the bounds and
// sign tests are done on the IEEE bit patterns with integer instructions, the
// FP32 passes accumulate their dot products with error-free transformations
// in FP32 (Ogita, Rump & Oishi, "Accurate sum and dot product", SISC 2005,
// algorithm Dot2) and convert to FP64 once per thread and tile, and the
// per-tile reduction runs through shared memory with one warp.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "engine.h"

// GPCG_COOP = 1: the translation unit instantiates the cooperative pass
// kernel, which runs pass after pass of one solve in a single launch (see
// pass_kernel).  A vector written by one pass and read by the next is then
// written and read within one launch, so every load of engine data takes the
// coherent path: no read-only-cache loads and no restrict-qualified pointers
// (which allow the compiler to use that cache); both promise data constant
// for the launch's lifetime.  The other translation units keep both.
#ifndef GPCG_COOP
#define GPCG_COOP 0
#endif
#if GPCG_COOP
#define GPCG_RESTRICT
#else
#define GPCG_RESTRICT __restrict__
#endif

namespace gpcg {
// internal linkage: every translation unit that includes this header has its
// own copy of the device code and instantiates the pass kernel it needs
namespace {

#define FULL_MASK 0xffffffffu

// A load of engine data: the read-only cache path in a kernel that runs one
// pass per launch, the L1-cached coherent path in the cooperative kernel
// (whose grid barrier orders it after the previous pass's stores).
template <class T>
__device__ __forceinline__ T ldro(const T* p) {
#if GPCG_COOP
  return __ldca(p);
#else
  return __ldg(p);
#endif
}

// ------------------------------------------------- FP64 tests on the bits --
// Inputs are checked to be NaN-free when a problem is created, so every value
// reaching these helpers is a number.

__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

// Integer key with the order of the doubles (-0 sorts just below +0).
__device__ __forceinline__ long long dkey(double x) {
  const long long b = dbits(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

// a == b as numbers (+0 == -0).
__device__ __forceinline__ bool deq(double a, double b) {
  const long long x = dbits(a), y = dbits(b);
  return x == y || ((x | y) << 1) == 0;
}

constexpr long long kNegZero = (long long)0x8000000000000000ULL;
__device__ __forceinline__ bool dge0(double a) {
  const long long x = dbits(a);
  return x >= 0 || x == kNegZero;
}
__device__ __forceinline__ bool dle0(double a) { return dbits(a) <= 0; }
__device__ __forceinline__ bool dlt0(double a) {
  const long long x = dbits(a);
  return x < 0 && x != kNegZero;
}
__device__ __forceinline__ bool dgt0(double a) { return dbits(a) > 0; }

// median of {l, u, x} for l <= u: the projection P of Sec. 3; returns l or u
// bit for bit when x lies outside [l, u]
__device__ __forceinline__ double mid3(double l, double u, double x) {
  const long long kx = dkey(x);
  if (kx < dkey(l)) return l;
  if (kx > dkey(u)) return u;
  return x;
}

// Projected gradient component, Eq. proj-gradient; a fixed variable
// (l == u) has component 0.
__device__ __forceinline__ double pg_comp(double x, double g, double l, double u) {
  const bool al = deq(x, l), au = deq(x, u);
  if (al && au) return 0.0;
  if (al) return dlt0(g) ? g : 0.0;
  if (au) return dgt0(g) ? g : 0.0;
  return g;
}

// FP32 projection and projected gradient of the mixed phase (the exact FP64
// versions above decide the active set; these only feed FP32 products).
__device__ __forceinline__ float mid3f(float l, float u, float x) { return fminf(fmaxf(x, l), u); }

__device__ __forceinline__ float pg_compf(bool al, bool au, float g) {
  if (al && au) return 0.0f;
  if (al) return g < 0.0f ? g : 0.0f;
  if (au) return g > 0.0f ? g : 0.0f;
  return g;
}

// ---------------------------------------------- FP32 compensated dot (Dot2) --

struct FF {
  float hi, lo;
};

// s += a*b with the product error (TwoProduct by FMA) and the addition error
// (TwoSum) accumulated in s.lo.
__device__ __forceinline__ void ff_fma(FF& s, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float pe = __fmaf_rn(a, b, -p);
  const float t = __fadd_rn(s.hi, p);
  const float z = __fsub_rn(t, s.hi);
  const float e = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, z)), __fsub_rn(p, z));
  s.hi = t;
  s.lo = __fadd_rn(s.lo, __fadd_rn(pe, e));
}

__device__ __forceinline__ double ff_val(const FF& s) { return (double)s.hi + (double)s.lo; }

// a + b in float-float arithmetic (TwoSum of the high parts, then a fast
// renormalisation).
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float z = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, z)), __fsub_rn(b.hi, z));
  const float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), e);
  const float hi = __fadd_rn(s, lo);
  return FF{hi, __fsub_rn(lo, __fsub_rn(hi, s))};
}

// Add a thread's FP32 partial of one chunk to its float-float accumulator.
__device__ __forceinline__ void ff_acc(FF& a, float v) { a = ff_add(a, FF{v, 0.0f}); }

// ------------------------------------------------------- TMA and mbarrier --

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// Add `bytes` to the transaction count of the barrier's current phase
// without arriving (for copies issued beside an arrive.expect_tx).
__device__ __forceinline__ void mbar_expect_only(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Wait for phase `parity` of the barrier; gives up after a bounded number of
// polls (returns false) so that a lost copy can never hang the GPU.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  for (int it = 0; it < (1 << 20); ++it) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Grid barrier of the cooperative pass kernel, run by thread 0 of each block
// after a block barrier (so the block's global stores precede it).  Every
// block of a cooperative launch is resident, so no block waits for one that
// cannot run.  The fence before the arrival publishes the block's stores; the
// acquire load and the fence after the wait make the other blocks' stores
// visible to this block's loads, and the proxy fence to its tensor copies.
// Returns false (the arrivals did not come) after a bounded number of polls.
__device__ __forceinline__ bool grid_barrier(unsigned* ctr, unsigned target) {
  __threadfence();
  atomicAdd(ctr, 1u);
  bool ok = false;
  for (int it = 0; it < (1 << 22); ++it) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
    if (v >= target) {
      ok = true;
      break;
    }
    if (it >= 64) __nanosleep(100);
  }
  __threadfence();
  asm volatile("fence.proxy.async.global;" ::: "memory");
  return ok;
}

// 2-D tiled bulk tensor copy global -> shared, completing on `bar`.  The x
// coordinate is always a multiple of 16 bytes; y may be -1 or beyond the
// last row (the unit fills zeros there).
__device__ __forceinline__ void tma_load2d(unsigned dst, const void* map, int x, int y,
                                           unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// The tensor maps live in global memory written by the host; make the TMA
// unit's view of them current before first use in this CTA.
__device__ __forceinline__ void tmap_acquire(const void* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                   (unsigned long long)map)
               : "memory");
}

// --------------------------------------------------------- memory helpers --

__device__ __forceinline__ void ld2(const double* GPCG_RESTRICT p, long long i, bool v0, bool v1,
                                    double o[2]) {
  if (v1) {
    const double2 t = ldro(reinterpret_cast<const double2*>(p + i));
    o[0] = t.x;
    o[1] = t.y;
  } else {
    o[0] = v0 ? ldro(p + i) : 0.0;
    o[1] = 0.0;
  }
}

__device__ __forceinline__ void ld2(const float* GPCG_RESTRICT p, long long i, bool v0, bool v1,
                                    float o[2]) {
  if (v1) {
    const float2 t = ldro(reinterpret_cast<const float2*>(p + i));
    o[0] = t.x;
    o[1] = t.y;
  } else {
    o[0] = v0 ? ldro(p + i) : 0.0f;
    o[1] = 0.0f;
  }
}

__device__ __forceinline__ void st2(double* p, long long i, bool v0, bool v1, double a, double b) {
  if (v1) {
    *reinterpret_cast<double2*>(p + i) = make_double2(a, b);
  } else if (v0) {
    p[i] = a;
  }
}

__device__ __forceinline__ void st2(float* p, long long i, bool v0, bool v1, float a, float b) {
  if (v1) {
    *reinterpret_cast<float2*>(p + i) = make_float2(a, b);
  } else if (v0) {
    p[i] = a;
  }
}

// Spread the low 16 bits of v to the even bit positions of a 32-bit word.
__device__ __forceinline__ unsigned spread16(unsigned v) {
  v &= 0xffffu;
  v = (v | (v << 8)) & 0x00ff00ffu;
  v = (v | (v << 4)) & 0x0f0f0f0fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}

// Per-thread partial results of a pass: up to 4 FP64 sums and 3 counts.
struct Acc {
  double s[4];
  int c[3];
};

// What a tile needs from the instance's control block (read once per tile).
struct Snap {
  int pass, cur, pcur, cg32, first_cg, dir, gp32, x32_live;
  int m, pad;  // explicit reduced system: free points of the phase
  double alpha, beta;
};

__device__ __forceinline__ long long row_index(const DevInst& I, int y, int z) {
  return (long long)z * I.ny + y;
}

__device__ __forceinline__ bool row_ok(const DevInst& I, int y, int z) {
  return y >= 0 && y < I.ny && z >= 0 && z < I.nz;
}

__device__ __forceinline__ long long pidx(const DevInst& I, int y, int z, int col) {
  return (long long)z * I.plane + (long long)y * I.px + col;
}

// The two free bits of this lane's points (e0, e0+1) in row (y, z).
__device__ __forceinline__ unsigned my_free_bits(const DevInst& I, const unsigned* GPCG_RESTRICT m,
                                                 int y, int z, int e0) {
  const unsigned w = ldro(m + row_index(I, y, z) * I.mw + (e0 >> 5));
  return (w >> (e0 & 31)) & 3u;
}

__device__ __forceinline__ bool free_bit(const DevInst& I, const unsigned* GPCG_RESTRICT m, int y,
                                         int z, int col) {
  const unsigned w = ldro(m + row_index(I, y, z) * I.mw + (col >> 5));
  return (w >> (col & 31)) & 1u;
}

// Write the free bits of a warp's 64-column strip (two words) for row (y,z);
// returns, for lanes 0 and 16, the number of bits that differ from `old`
// (nullptr: 0).
__device__ __forceinline__ int write_mask(const DevInst& I, unsigned* m, const unsigned* old,
                                          int y, int z, int x0, int lane, bool f0, bool f1) {
  const unsigned b0 = __ballot_sync(FULL_MASK, f0);
  const unsigned b1 = __ballot_sync(FULL_MASK, f1);
  int diff = 0;
  if ((lane & 15) == 0) {
    const int h = lane >> 4;
    const int wcol = (x0 >> 5) + h;
    if (wcol < I.mw) {
      const unsigned word = spread16(b0 >> (16 * h)) | (spread16(b1 >> (16 * h)) << 1);
      const long long wi = row_index(I, y, z) * I.mw + wcol;
      m[wi] = word;
      if (old) diff = __popc(word ^ ldro(old + wi));
    }
  }
  return diff;
}

// ---------------------------------------------------------- stencil sweep --
//
// Op supplies the operand v of the pass at any point (operand_row for the
// lane's two points of a row, operand_at for one point) and consumes, for
// each row of the strip, v and (A v) at the lane's two points (output).

template <class Op>
__device__ __forceinline__ void stencil_tile(const DevInst& I, const Op& op, int x0, int y0, int z,
                                             Acc& acc) {
  using T = typename Op::T;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ya = y0 + warp * kRY;
  if (ya >= I.ny) return;  // warp-uniform
  const int yb = min(ya + kRY, I.ny);
  const int e0 = x0 + 2 * lane;
  const bool v0 = e0 < I.nx, v1 = e0 + 1 < I.nx;
  const long long zb = (long long)z * I.plane;
  const T* GPCG_RESTRICT diag = op.diag();
  const T* GPCG_RESTRICT cx = op.cx();
  const T* GPCG_RESTRICT cy = op.cy();
  const T* GPCG_RESTRICT cz = op.cz();

  T vm[2], vc[2], vn[2], cs[2];
  op.operand_row(ya - 1, z, e0, v0, v1, vm);
  op.operand_row(ya, z, e0, v0, v1, vc);
  if (ya > 0) {
    ld2(cy, zb + (long long)(ya - 1) * I.px + e0, v0, v1, cs);
  } else {
    cs[0] = cs[1] = T(0);
  }
#pragma unroll 1
  for (int y = ya; y < yb; ++y) {
    op.operand_row(y + 1, z, e0, v0, v1, vn);
    const long long i = zb + (long long)y * I.px + e0;
    T d[2], ce[2], cn[2];
    ld2(diag, i, v0, v1, d);
    ld2(cx, i, v0, v1, ce);
    ld2(cy, i, v0, v1, cn);
    T vw = __shfl_up_sync(FULL_MASK, vc[1], 1);
    T cw = __shfl_up_sync(FULL_MASK, ce[1], 1);
    T ve = __shfl_down_sync(FULL_MASK, vc[0], 1);
    if (lane == 0) {
      const bool has = v0 && e0 > 0;
      vw = has ? op.operand_at(i - 1, y, z, e0 - 1) : T(0);
      cw = has ? ldro(cx + i - 1) : T(0);
    }
    if (lane == 31) ve = (e0 + 2 < I.nx) ? op.operand_at(i + 2, y, z, e0 + 2) : T(0);
    T av[2];
    // row sums in the order diag, west, east, south, north (, down, up)
    av[0] = d[0] * vc[0];
    av[0] = fma(cw, vw, av[0]);
    av[0] = fma(ce[0], vc[1], av[0]);
    av[0] = fma(cs[0], vm[0], av[0]);
    av[0] = fma(cn[0], vn[0], av[0]);
    av[1] = d[1] * vc[1];
    av[1] = fma(ce[0], vc[0], av[1]);
    av[1] = fma(ce[1], ve, av[1]);
    av[1] = fma(cs[1], vm[1], av[1]);
    av[1] = fma(cn[1], vn[1], av[1]);
    if (I.dim == 3) {
      T vd[2], vu[2], czd[2], czu[2];
      op.operand_row(y, z - 1, e0, v0, v1, vd);
      op.operand_row(y, z + 1, e0, v0, v1, vu);
      if (z > 0) {
        ld2(cz, i - I.plane, v0, v1, czd);
      } else {
        czd[0] = czd[1] = T(0);
      }
      ld2(cz, i, v0, v1, czu);
      av[0] = fma(czd[0], vd[0], av[0]);
      av[0] = fma(czu[0], vu[0], av[0]);
      av[1] = fma(czd[1], vd[1], av[1]);
      av[1] = fma(czu[1], vu[1], av[1]);
    }
    op.output(y, z, i, x0, e0, lane, v0, v1, vc, av, acc);
    vm[0] = vc[0];
    vm[1] = vc[1];
    vc[0] = vn[0];
    vc[1] = vn[1];
    cs[0] = cn[0];
    cs[1] = cn[1];
  }
}

// P_CENSUS: operand x; g = Ax + b and everything Sec. 2 defines at x:
// sums ||pg||^2 and <x, g + b> (= 2 (q - c)), counts |A(x)| and |B(x)|.
//
// After the mixed phase (x32 != nullptr) the iterate is rebuilt from the
// FP32 one first: a point on an FP32 bound goes to the FP64 bound, any other
// to P[x32] (the projection of Sec. 3 onto the FP64 box); x_out receives it.
struct OpCensus {
  using T = double;
  const DevInst& I;
  const double* GPCG_RESTRICT x;
  double* g_out;
  unsigned* m_out;
  const float* GPCG_RESTRICT x32;
  double* x_out;
  __device__ const double* diag() const { return I.diag; }
  __device__ const double* cx() const { return I.cx; }
  __device__ const double* cy() const { return I.cy; }
  __device__ const double* cz() const { return I.cz; }
  __device__ double rebuild(float xf, double l, double u, float lf, float uf) const {
    if (xf == lf) return l;
    if (xf == uf) return u;
    return mid3(l, u, (double)xf);
  }
  __device__ void operand_row(int y, int z, int e0, bool v0, bool v1, double o[2]) const {
    if (!row_ok(I, y, z)) {
      o[0] = o[1] = 0.0;
      return;
    }
    const long long i = pidx(I, y, z, e0);
    if (x32) {
      float xf[2], lf[2], uf[2];
      double l[2], u[2];
      ld2(x32, i, v0, v1, xf);
      ld2(I.l32, i, v0, v1, lf);
      ld2(I.u32, i, v0, v1, uf);
      ld2(I.l, i, v0, v1, l);
      ld2(I.u, i, v0, v1, u);
      o[0] = v0 ? rebuild(xf[0], l[0], u[0], lf[0], uf[0]) : 0.0;
      o[1] = v1 ? rebuild(xf[1], l[1], u[1], lf[1], uf[1]) : 0.0;
    } else {
      ld2(x, i, v0, v1, o);
    }
  }
  __device__ double operand_at(long long i, int, int, int) const {
    if (x32)
      return rebuild(ldro(x32 + i), ldro(I.l + i), ldro(I.u + i), ldro(I.l32 + i),
                     ldro(I.u32 + i));
    return ldro(x + i);
  }
  __device__ void output(int y, int z, long long i, int x0, int, int lane, bool v0, bool v1,
                         const double v[2], const double av[2], Acc& acc) const {
    double b[2], l[2], u[2], g[2];
    ld2(I.b, i, v0, v1, b);
    ld2(I.l, i, v0, v1, l);
    ld2(I.u, i, v0, v1, u);
    bool fr[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const bool ok = k == 0 ? v0 : v1;
      g[k] = av[k] + b[k];
      const bool al = deq(v[k], l[k]), au = deq(v[k], u[k]);
      const bool act = al || au;
      const bool bind = (al && dge0(g[k])) || (au && dle0(g[k]));
      fr[k] = ok && !act;
      if (ok) {
        const double pg = pg_comp(v[k], g[k], l[k], u[k]);
        acc.s[0] = fma(pg, pg, acc.s[0]);
        acc.s[1] = fma(v[k], g[k] + b[k], acc.s[1]);
        acc.c[0] += act;
        acc.c[1] += bind;
      }
    }
    st2(g_out, i, v0, v1, g[0], g[1]);
    if (x32) st2(x_out, i, v0, v1, v[0], v[1]);
    write_mask(I, m_out, nullptr, y, z, x0, lane, fr[0], fr[1]);
  }
};

// P_GP_ALPHA: operand pg = grad_Omega q(x); sums <pg,pg> and <pg, A pg>.
struct OpGpAlpha {
  using T = double;
  const DevInst& I;
  const double* GPCG_RESTRICT x;
  const double* GPCG_RESTRICT g;
  __device__ const double* diag() const { return I.diag; }
  __device__ const double* cx() const { return I.cx; }
  __device__ const double* cy() const { return I.cy; }
  __device__ const double* cz() const { return I.cz; }
  __device__ void operand_row(int y, int z, int e0, bool v0, bool v1, double o[2]) const {
    if (!row_ok(I, y, z)) {
      o[0] = o[1] = 0.0;
      return;
    }
    const long long i = pidx(I, y, z, e0);
    double xv[2], gv[2], l[2], u[2];
    ld2(x, i, v0, v1, xv);
    ld2(g, i, v0, v1, gv);
    ld2(I.l, i, v0, v1, l);
    ld2(I.u, i, v0, v1, u);
    o[0] = v0 ? pg_comp(xv[0], gv[0], l[0], u[0]) : 0.0;
    o[1] = v1 ? pg_comp(xv[1], gv[1], l[1], u[1]) : 0.0;
  }
  __device__ double operand_at(long long i, int, int, int) const {
    return pg_comp(ldro(x + i), ldro(g + i), ldro(I.l + i), ldro(I.u + i));
  }
  __device__ void output(int, int, long long, int, int, int, bool v0, bool v1, const double v[2],
                         const double av[2], Acc& acc) const {
    if (v0) {
      acc.s[0] = fma(v[0], v[0], acc.s[0]);
      acc.s[1] = fma(v[0], av[0], acc.s[1]);
    }
    if (v1) {
      acc.s[0] = fma(v[1], v[1], acc.s[0]);
      acc.s[1] = fma(v[1], av[1], acc.s[1]);
    }
  }
};

// P_TRIAL: operand xt = P[x + alpha*dir] (Eq. next-y with dir = -grad q, or
// the projected search along d with dir = w); gt = A xt + b; sums <g, s> and
// <s, gt> with s = xt - x (q(xt) - q(x) = 1/2 (<g,s> + <s,gt>) exactly for a
// quadratic) and ||grad_Omega q(xt)||^2; counts |A(xt)|, |B(xt)| and the
// number of points whose active/free status changed (Eq. pgstop1).
template <int DK>
struct OpTrial {
  using T = double;
  const DevInst& I;
  const double* GPCG_RESTRICT x;
  const double* GPCG_RESTRICT g;
  const double* GPCG_RESTRICT w64;
  const float* GPCG_RESTRICT w32;
  double alpha;
  double* xt_out;
  double* gt_out;
  unsigned* m_out;
  const unsigned* GPCG_RESTRICT m_old;
  __device__ const double* diag() const { return I.diag; }
  __device__ const double* cx() const { return I.cx; }
  __device__ const double* cy() const { return I.cy; }
  __device__ const double* cz() const { return I.cz; }
  __device__ void dir2(long long i, bool v0, bool v1, double d[2]) const {
    if (DK == D_NEG_G) {
      ld2(g, i, v0, v1, d);
      d[0] = -d[0];
      d[1] = -d[1];
    } else if (DK == D_W64) {
      ld2(w64, i, v0, v1, d);
    } else {
      float f[2];
      ld2(w32, i, v0, v1, f);
      d[0] = (double)f[0];
      d[1] = (double)f[1];
    }
  }
  __device__ void operand_row(int y, int z, int e0, bool v0, bool v1, double o[2]) const {
    if (!row_ok(I, y, z)) {
      o[0] = o[1] = 0.0;
      return;
    }
    const long long i = pidx(I, y, z, e0);
    double xv[2], d[2], l[2], u[2];
    ld2(x, i, v0, v1, xv);
    dir2(i, v0, v1, d);
    ld2(I.l, i, v0, v1, l);
    ld2(I.u, i, v0, v1, u);
    o[0] = v0 ? mid3(l[0], u[0], fma(alpha, d[0], xv[0])) : 0.0;
    o[1] = v1 ? mid3(l[1], u[1], fma(alpha, d[1], xv[1])) : 0.0;
  }
  __device__ double operand_at(long long i, int, int, int) const {
    double dv;
    if (DK == D_NEG_G) dv = -ldro(g + i);
    else if (DK == D_W64) dv = ldro(w64 + i);
    else dv = (double)ldro(w32 + i);
    return mid3(ldro(I.l + i), ldro(I.u + i), fma(alpha, dv, ldro(x + i)));
  }
  __device__ void output(int y, int z, long long i, int x0, int, int lane, bool v0, bool v1,
                         const double v[2], const double av[2], Acc& acc) const {
    double xv[2], gv[2], b[2], l[2], u[2], gt[2];
    ld2(x, i, v0, v1, xv);
    ld2(g, i, v0, v1, gv);
    ld2(I.b, i, v0, v1, b);
    ld2(I.l, i, v0, v1, l);
    ld2(I.u, i, v0, v1, u);
    bool fr[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const bool ok = k == 0 ? v0 : v1;
      gt[k] = av[k] + b[k];
      const bool al = deq(v[k], l[k]), au = deq(v[k], u[k]);
      const bool act = al || au;
      const bool bind = (al && dge0(gt[k])) || (au && dle0(gt[k]));
      fr[k] = ok && !act;
      if (ok) {
        const double s = v[k] - xv[k];
        acc.s[0] = fma(gv[k], s, acc.s[0]);
        acc.s[1] = fma(s, gt[k], acc.s[1]);
        const double pg = pg_comp(v[k], gt[k], l[k], u[k]);
        acc.s[2] = fma(pg, pg, acc.s[2]);
        acc.c[0] += act;
        acc.c[1] += bind;
      }
    }
    st2(xt_out, i, v0, v1, v[0], v[1]);
    st2(gt_out, i, v0, v1, gt[0], gt[1]);
    acc.c[2] += write_mask(I, m_out, m_old, y, z, x0, lane, fr[0], fr[1]);
  }
};


// ------------------------------------------------- mixed-phase FP32 passes --
//
// In the mixed phase the census, the alpha0 pass and the trials work on the
// FP32 iterate x32, kept on the FP32 box [l32, u32] by the FP32 projection
// (which returns the bound itself when it clamps): a point is active when x32
// equals l32 or u32.  The FP32 stencil is applied to FP32 operands and the
// gradient is kept in FP32; sums use the compensated FP32 accumulator.  The
// first FP64 census after the phase rebuilds the FP64 iterate (OpCensus).

// P_CENSUS (mixed): operand x32; g32 = A32 x32 + b32, pg32; |A|, |B|,
// ||pg||^2.
struct OpCensus32 {
  using T = float;
  const DevInst& I;
  const float* GPCG_RESTRICT x32;
  float* g_out;
  float* pg_out;
  unsigned* m_out;
  FF* ff;  // [1]: ||pg||^2
  __device__ const float* diag() const { return I.diag32; }
  __device__ const float* cx() const { return I.cx32; }
  __device__ const float* cy() const { return I.cy32; }
  __device__ const float* cz() const { return I.cz32; }
  __device__ void operand_row(int y, int z, int e0, bool v0, bool v1, float o[2]) const {
    if (!row_ok(I, y, z)) {
      o[0] = o[1] = 0.0f;
      return;
    }
    ld2(x32, pidx(I, y, z, e0), v0, v1, o);
  }
  __device__ float operand_at(long long i, int, int, int) const { return ldro(x32 + i); }
  __device__ void output(int y, int z, long long i, int x0, int, int lane, bool v0, bool v1,
                         const float v[2], const float av[2], Acc& acc) const {
    float l[2], u[2], b[2], g[2], pg[2];
    ld2(I.l32, i, v0, v1, l);
    ld2(I.u32, i, v0, v1, u);
    ld2(I.b32, i, v0, v1, b);
    bool fr[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const bool ok = k == 0 ? v0 : v1;
      g[k] = av[k] + b[k];
      const bool al = v[k] == l[k], au = v[k] == u[k];
      const bool act = al || au;
      fr[k] = ok && !act;
      pg[k] = pg_compf(al, au, g[k]);
      if (ok) {
        ff_fma(ff[0], pg[k], pg[k]);
        acc.c[0] += act;
        acc.c[1] += (al && g[k] >= 0.0f) || (au && g[k] <= 0.0f);
      }
    }
    st2(g_out, i, v0, v1, g[0], g[1]);
    st2(pg_out, i, v0, v1, pg[0], pg[1]);
    write_mask(I, m_out, nullptr, y, z, x0, lane, fr[0], fr[1]);
  }
};

// P_GP_ALPHA (mixed): operand pg32 (written by the census or the accepted
// trial at x); <pg,pg>, <pg, A32 pg>.
struct OpGpAlpha32 {
  using T = float;
  const DevInst& I;
  const float* GPCG_RESTRICT pg32;
  FF* ff;  // [2]
  __device__ const float* diag() const { return I.diag32; }
  __device__ const float* cx() const { return I.cx32; }
  __device__ const float* cy() const { return I.cy32; }
  __device__ const float* cz() const { return I.cz32; }
  __device__ void operand_row(int y, int z, int e0, bool v0, bool v1, float o[2]) const {
    if (!row_ok(I, y, z)) {
      o[0] = o[1] = 0.0f;
      return;
    }
    ld2(pg32, pidx(I, y, z, e0), v0, v1, o);
  }
  __device__ float operand_at(long long i, int, int, int) const { return ldro(pg32 + i); }
  __device__ void output(int, int, long long, int, int, int, bool v0, bool v1, const float v[2],
                         const float av[2], Acc&) const {
    if (v0) {
      ff_fma(ff[0], v[0], v[0]);
      ff_fma(ff[1], v[0], av[0]);
    }
    if (v1) {
      ff_fma(ff[0], v[1], v[1]);
      ff_fma(ff[1], v[1], av[1]);
    }
  }
};

// P_TRIAL (mixed): operand xt32 = P[x32 + alpha d] on the FP32 box;
// g32t = A32 xt32 + b32, the status of xt32, pg32; <g, s>, <s, gt>,
// ||pg||^2 with s = xt32 - x32.
template <int DK>
struct OpTrial32 {
  using T = float;
  const DevInst& I;
  const float* GPCG_RESTRICT x32;
  const float* GPCG_RESTRICT g32;
  const float* GPCG_RESTRICT w32;
  float alpha;
  float* xt32_out;
  float* gt_out;
  float* pg_out;
  unsigned* m_out;
  const unsigned* GPCG_RESTRICT m_old;
  FF* ff;  // [3]: <g,s>, <s,gt>, ||pg||^2
  __device__ const float* diag() const { return I.diag32; }
  __device__ const float* cx() const { return I.cx32; }
  __device__ const float* cy() const { return I.cy32; }
  __device__ const float* cz() const { return I.cz32; }
  __device__ float dir_at(long long i) const {
    return DK == D_NEG_G ? -ldro(g32 + i) : ldro(w32 + i);
  }
  __device__ void operand_row(int y, int z, int e0, bool v0, bool v1, float o[2]) const {
    if (!row_ok(I, y, z)) {
      o[0] = o[1] = 0.0f;
      return;
    }
    const long long i = pidx(I, y, z, e0);
    float xv[2], l[2], u[2], d[2];
    ld2(x32, i, v0, v1, xv);
    ld2(I.l32, i, v0, v1, l);
    ld2(I.u32, i, v0, v1, u);
    if (DK == D_NEG_G) {
      ld2(g32, i, v0, v1, d);
      d[0] = -d[0];
      d[1] = -d[1];
    } else {
      ld2(w32, i, v0, v1, d);
    }
    o[0] = v0 ? mid3f(l[0], u[0], fmaf(alpha, d[0], xv[0])) : 0.0f;
    o[1] = v1 ? mid3f(l[1], u[1], fmaf(alpha, d[1], xv[1])) : 0.0f;
  }
  __device__ float operand_at(long long i, int, int, int) const {
    return mid3f(ldro(I.l32 + i), ldro(I.u32 + i), fmaf(alpha, dir_at(i), ldro(x32 + i)));
  }
  __device__ void output(int y, int z, long long i, int x0, int, int lane, bool v0, bool v1,
                         const float v[2], const float av[2], Acc& acc) const {
    float xv[2], l[2], u[2], g[2], b[2], gt[2], pg[2];
    ld2(x32, i, v0, v1, xv);
    ld2(I.l32, i, v0, v1, l);
    ld2(I.u32, i, v0, v1, u);
    ld2(g32, i, v0, v1, g);
    ld2(I.b32, i, v0, v1, b);
    bool fr[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const bool ok = k == 0 ? v0 : v1;
      gt[k] = av[k] + b[k];
      const bool al = v[k] == l[k], au = v[k] == u[k];
      const bool act = al || au;
      fr[k] = ok && !act;
      pg[k] = pg_compf(al, au, gt[k]);
      if (ok) {
        const float sk = v[k] - xv[k];
        ff_fma(ff[0], g[k], sk);
        ff_fma(ff[1], sk, gt[k]);
        ff_fma(ff[2], pg[k], pg[k]);
        acc.c[0] += act;
        acc.c[1] += (al && gt[k] >= 0.0f) || (au && gt[k] <= 0.0f);
      }
    }
    st2(xt32_out, i, v0, v1, v[0], v[1]);
    st2(gt_out, i, v0, v1, gt[0], gt[1]);
    st2(pg_out, i, v0, v1, pg[0], pg[1]);
    acc.c[2] += write_mask(I, m_out, m_old, y, z, x0, lane, fr[0], fr[1]);
  }
};

// The first CG step's r_0 = g_F and M^-1 Ap under point Jacobi, out of line:
// it runs once per CG phase and, inlined, raises the register pressure of the
// whole sweep.
template <class T>
__device__ __noinline__ void first_step_jacobi(const float* GPCG_RESTRICT g32,
                                               const double* GPCG_RESTRICT g,
                                               const T* GPCG_RESTRICT dinv, long long i, bool v0,
                                               bool v1, unsigned fb, T* rv, T* da) {
  T di[2];
  ld2(dinv, i, v0, v1, di);
  double gv[2];
  if (g32) {
    float gf[2];
    ld2(g32, i, v0, v1, gf);
    gv[0] = gf[0];
    gv[1] = gf[1];
  } else {
    ld2(g, i, v0, v1, gv);
  }
  rv[0] = (fb & 1u) ? (T)gv[0] : T(0);
  rv[1] = (fb & 2u) ? (T)gv[1] : T(0);
  da[0] *= di[0];
  da[1] *= di[1];
}

// P_CG_B: operand p = -r + beta*p_old (FIRST: p = -g on the free set), the
// masked product Ap = Z Z' A Z Z' p of Eq. cg2 and <p, Ap> (FIRST: also
// ||r||^2 for r = g_F).  TV is the streamed precision (double, or float in the
// mixed CG, whose sums use the compensated FP32 accumulator).
template <class TV, bool FIRST, bool JAC = false>
struct OpCgB {
  using T = TV;
  static constexpr bool kF32 = sizeof(TV) == 4;
  const DevInst& I;
  const T* GPCG_RESTRICT r;
  const T* GPCG_RESTRICT p_old;
  const double* GPCG_RESTRICT g;
  const unsigned* GPCG_RESTRICT m;
  T beta;
  const float* GPCG_RESTRICT g32;  // mixed phase: the gradient is FP32 (FIRST)
  T* p_out;
  T* ap_out;
  T* r_out;
  T* w_out;
  const T* bd;
  const T* bx;
  const T* by;
  const T* bz;
  FF* ff;  // [3] FP32 accumulators (kF32)
  const T* GPCG_RESTRICT dinv;  // 1/diag (point Jacobi, z = r / diag), or nullptr
  __device__ const T* diag() const { return bd; }
  __device__ const T* cx() const { return bx; }
  __device__ const T* cy() const { return by; }
  __device__ const T* cz() const { return bz; }
  __device__ void operand_row(int y, int z, int e0, bool v0, bool v1, T o[2]) const {
    if (!row_ok(I, y, z)) {
      o[0] = o[1] = T(0);
      return;
    }
    const long long i = pidx(I, y, z, e0);
    if (FIRST) {
      double gv[2];
      if (g32) {
        float gf[2];
        ld2(g32, i, v0, v1, gf);
        gv[0] = gf[0];
        gv[1] = gf[1];
      } else {
        ld2(g, i, v0, v1, gv);
      }
      const unsigned fb = (v0 ? my_free_bits(I, m, y, z, e0) : 0u);
      T zv[2] = {(T)gv[0], (T)gv[1]};
      if (JAC) {
        T di[2];
        ld2(dinv, i, v0, v1, di);
        zv[0] *= di[0];
        zv[1] *= di[1];
      }
      o[0] = (fb & 1u) ? -zv[0] : T(0);
      o[1] = (fb & 2u) ? -zv[1] : T(0);
    } else {
      T rv[2], pv[2];
      ld2(r, i, v0, v1, rv);
      ld2(p_old, i, v0, v1, pv);
      if (JAC) {
        T di[2];
        ld2(dinv, i, v0, v1, di);
        rv[0] *= di[0];
        rv[1] *= di[1];
      }
      o[0] = fma(beta, pv[0], -rv[0]);
      o[1] = fma(beta, pv[1], -rv[1]);
    }
  }
  __device__ T operand_at(long long i, int y, int z, int col) const {
    const T di = JAC ? ldro(dinv + i) : T(1);
    if (FIRST) {
      if (!free_bit(I, m, y, z, col)) return T(0);
      return -(g32 ? (T)ldro(g32 + i) : (T)ldro(g + i)) * di;
    } else {
      return fma(beta, ldro(p_old + i), -ldro(r + i) * di);
    }
  }
  __device__ void output(int y, int z, long long i, int, int e0, int, bool v0, bool v1,
                         const T v[2], const T av[2], Acc& acc) const {
    const unsigned fb = v0 ? my_free_bits(I, m, y, z, e0) : 0u;
    const T a0 = (fb & 1u) ? av[0] : T(0);
    const T a1 = (fb & 2u) ? av[1] : T(0);
    st2(ap_out, i, v0, v1, a0, a1);
    st2(p_out, i, v0, v1, v[0], v[1]);
    if (kF32) {
      ff_fma(ff[0], (float)v[0], (float)a0);
      ff_fma(ff[0], (float)v[1], (float)a1);
    } else {
      acc.s[0] = fma((double)v[0], (double)a0, acc.s[0]);
      acc.s[0] = fma((double)v[1], (double)a1, acc.s[0]);
    }
    if (FIRST) {
      // r = g_F (v = -z = -M^-1 r); rho = <r, z>; <Ap, M^-1 Ap> (the fused
      // steps predict rho_1 from them)
      T rv[2] = {-v[0], -v[1]}, da[2] = {a0, a1};
      if (JAC) first_step_jacobi<T>(g32, g, dinv, i, v0, v1, fb, rv, da);
      st2(r_out, i, v0, v1, rv[0], rv[1]);
      st2(w_out, i, v0, v1, T(0), T(0));
      if (kF32) {
        ff_fma(ff[1], (float)rv[0], -(float)v[0]);
        ff_fma(ff[1], (float)rv[1], -(float)v[1]);
        ff_fma(ff[2], (float)a0, (float)da[0]);
        ff_fma(ff[2], (float)a1, (float)da[1]);
      } else {
        acc.s[1] = fma((double)rv[0], -(double)v[0], acc.s[1]);
        acc.s[1] = fma((double)rv[1], -(double)v[1], acc.s[1]);
        acc.s[2] = fma((double)a0, (double)da[0], acc.s[2]);
        acc.s[2] = fma((double)a1, (double)da[1], acc.s[2]);
      }
    }
  }
};

// ---------------------------------------------------------- pointwise passes

// P_CG_A: w += alpha p, r_out = r + alpha Ap, <r_out, M^-1 r_out> (M = I or
// diag(A) with dinv).
template <class T, bool JAC>
__device__ __forceinline__ void cg_a_tile(const DevInst& I, T* w, const T* GPCG_RESTRICT r,
                                          T* r_out, const T* GPCG_RESTRICT p,
                                          const T* GPCG_RESTRICT ap, const T* GPCG_RESTRICT dinv,
                                          double alpha, int x0, int y0, int z, Acc& acc,
                                          FF* ffs) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ya = y0 + warp * kRY;
  if (ya >= I.ny) return;
  const int yb = min(ya + kRY, I.ny);
  const int e0 = x0 + 2 * lane;
  const bool v0 = e0 < I.nx, v1 = e0 + 1 < I.nx;
  if (!v0) return;
  const T a = (T)alpha;
  FF& ff = ffs[0];
  for (int y = ya; y < yb; ++y) {
    const long long i = pidx(I, y, z, e0);
    T wv[2], rv[2], pv[2], av[2];
    ld2(w, i, v0, v1, wv);
    ld2(r, i, v0, v1, rv);
    ld2(p, i, v0, v1, pv);
    ld2(ap, i, v0, v1, av);
    wv[0] = fma(a, pv[0], wv[0]);
    wv[1] = fma(a, pv[1], wv[1]);
    rv[0] = fma(a, av[0], rv[0]);
    rv[1] = fma(a, av[1], rv[1]);
    st2(w, i, v0, v1, wv[0], wv[1]);
    st2(r_out, i, v0, v1, rv[0], rv[1]);
    T zv[2] = {rv[0], rv[1]};  // z = M^-1 r (point Jacobi) or r
    if (JAC) {
      T di[2];
      ld2(dinv, i, v0, v1, di);
      zv[0] *= di[0];
      zv[1] *= di[1];
    }
    if (sizeof(T) == 4) {
      ff_fma(ff, (float)rv[0], (float)zv[0]);
      ff_fma(ff, (float)rv[1], (float)zv[1]);
    } else {
      acc.s[0] = fma((double)rv[0], (double)zv[0], acc.s[0]);
      acc.s[0] = fma((double)rv[1], (double)zv[1], acc.s[0]);
    }
  }
}

// P_START: x = P[x0], x0 the given start or the default l -> u -> 0.
__device__ __forceinline__ void start_tile(const DevInst& I, double* x, float* x32, int x0, int y0,
                                           int z) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ya = y0 + warp * kRY;
  if (ya >= I.ny) return;
  const int yb = min(ya + kRY, I.ny);
  const int e0 = x0 + 2 * lane;
  const bool v0 = e0 < I.nx, v1 = e0 + 1 < I.nx;
  if (!v0) return;
  for (int y = ya; y < yb; ++y) {
    const long long i = pidx(I, y, z, e0);
    double l[2], u[2], s[2];
    ld2(I.l, i, v0, v1, l);
    ld2(I.u, i, v0, v1, u);
    if (I.opt.use_x0) {
      ld2(I.x0, i, v0, v1, s);
    } else {
#pragma unroll
      for (int k = 0; k < 2; ++k) s[k] = isfinite(l[k]) ? l[k] : (isfinite(u[k]) ? u[k] : 0.0);
    }
    const double a = mid3(l[0], u[0], s[0]), b = mid3(l[1], u[1], s[1]);
    st2(x, i, v0, v1, a, b);
    if (x32) st2(x32, i, v0, v1, (float)a, (float)b);
  }
}

// ------------------------------------------------- tile preconditioner --
//
// M of the tile preconditioner (the analogue of the block Jacobi with one
// block per processor of Sec. 6): one block per 64 x 8 tile of an xy-plane,
// couplings between tiles dropped; each block solved approximately by one
// symmetric zebra line Gauss-Seidel sweep on the free set -- the x-lines of
// the tile's even rows, then its odd rows, then its even rows, each solved
// exactly with the current values of the lines above and below on the
// right-hand side.  Per tile M = (D + L) D^-1 (D + U), D the line
// tridiagonals, L and U the couplings between lines in the order (even
// rows, odd rows); M is symmetric positive definite.  A warp holds a line
// (lane l: columns 2l and 2l+1).  M^-1 is applied in FP32 in every phase: it
// only shapes the search directions, which stay in the phase's precision.

// One line of a tile: b0, b1 the diagonal of the lane's points (1 off the
// free set), cw the coupling of column 2l-1 to 2l, cm of 2l to 2l+1 (0 unless
// both points are free; cw = 0 on lane 0, the tile's edge), cn / cs the
// couplings of the two points to the row above / below inside the tile.
struct TileLine {
  float b0, b1, cw, cm, cn0, cn1, cs0, cs1;
};

// Solve the warp's line system
//   cw x[2l-1] + b0 x[2l] + cm x[2l+1] = d0,  cm x[2l] + b1 x[2l+1] + ce x[2l+2] = d1,
// ce = the next lane's cw (0 on lane 31).  Each lane eliminates its even
// point and its east neighbour's, which leaves one equation per lane in
// u_l = x[2l+1]; parallel cyclic reduction (Hockney) then removes the
// couplings at distance 1, 2, 4, 8, 16 by shuffles, after which each u_l
// stands alone; last the even points are recovered.  The system is a
// principal submatrix of A (symmetric positive definite), so no pivot vanishes.
// The reciprocals are the hardware's approximate ones (__fdividef, within 2
// ulp): M^-1 stays a fixed operator, which is all the recurrences need.
__device__ __forceinline__ void line_solve(float b0, float b1, float cw, float cm, float d0,
                                           float d1, float& x0, float& x1) {
  const int lane = threadIdx.x & 31;
  const float ie = __fdividef(1.0f, b0);
  float ce = __shfl_down_sync(FULL_MASK, cw, 1);
  const float ie_n = __shfl_down_sync(FULL_MASK, ie, 1);
  const float d0_n = __shfl_down_sync(FULL_MASK, d0, 1);
  const float cm_n = __shfl_down_sync(FULL_MASK, cm, 1);
  if (lane == 31) ce = 0.0f;
  float a = -cm * cw * ie;
  float b = b1 - cm * cm * ie - ce * ce * ie_n;
  float c = -ce * cm_n * ie_n;
  float d = d1 - cm * d0 * ie - ce * d0_n * ie_n;
#pragma unroll
  for (int s = 1; s < 32; s <<= 1) {
    const float ib = __fdividef(1.0f, b);
    float am = __shfl_up_sync(FULL_MASK, a, s), cmm = __shfl_up_sync(FULL_MASK, c, s);
    float dm = __shfl_up_sync(FULL_MASK, d, s), ibm = __shfl_up_sync(FULL_MASK, ib, s);
    float ap = __shfl_down_sync(FULL_MASK, a, s), cp = __shfl_down_sync(FULL_MASK, c, s);
    float dp = __shfl_down_sync(FULL_MASK, d, s), ibp = __shfl_down_sync(FULL_MASK, ib, s);
    if (lane < s) am = cmm = dm = ibm = 0.0f;
    if (lane + s >= 32) ap = cp = dp = ibp = 0.0f;
    const float k1 = a * ibm, k2 = c * ibp;
    a = -k1 * am;
    c = -k2 * cp;
    b = b - k1 * cmm - k2 * ap;
    d = d - k1 * dm - k2 * dp;
  }
  const float u = __fdividef(d, b);
  float um = __shfl_up_sync(FULL_MASK, u, 1);
  if (lane == 0) um = 0.0f;
  x1 = u;
  x0 = (d0 - cw * um - cm * u) * ie;
}

// The zebra sweep over the chunk rows r0 .. r0+RPW-1 a warp holds (all warps
// of the CTA take part; the chunk starts on a multiple of 8 rows, so the
// parity of a chunk row is that of the grid row).  `scr`: a CTA buffer of
// (chunk rows) x `pitch` floats through which the lines see their
// neighbours; each warp writes only the rows it holds.  d: the right-hand
// side (0 off the free set); x: M^-1 d on the warp's rows.
template <int RPW>
__device__ __forceinline__ void zebra_sweep(const TileLine (&L)[RPW], const float (&d)[RPW][2],
                                            int r0, float* scr, int pitch, float (&x)[RPW][2]) {
  const int c = 2 * (threadIdx.x & 31);
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    if (((r0 + k) & 1) == 0) {
      line_solve(L[k].b0, L[k].b1, L[k].cw, L[k].cm, d[k][0], d[k][1], x[k][0], x[k][1]);
      *reinterpret_cast<float2*>(scr + (r0 + k) * pitch + c) = make_float2(x[k][0], x[k][1]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int h = 1; h >= 0; --h) {  // odd rows, then even rows again
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
      const int row = r0 + k;
      if ((row & 1) != h) continue;
      float e0 = d[k][0], e1 = d[k][1];
      if ((row & (kBlkY - 1)) != 0) {
        const float2 v = *reinterpret_cast<const float2*>(scr + (row - 1) * pitch + c);
        e0 -= L[k].cn0 * v.x;
        e1 -= L[k].cn1 * v.y;
      }
      if ((row & (kBlkY - 1)) != kBlkY - 1) {
        const float2 v = *reinterpret_cast<const float2*>(scr + (row + 1) * pitch + c);
        e0 -= L[k].cs0 * v.x;
        e1 -= L[k].cs1 * v.y;
      }
      line_solve(L[k].b0, L[k].b1, L[k].cw, L[k].cm, e0, e1, x[k][0], x[k][1]);
      if (h == 1)
        *reinterpret_cast<float2*>(scr + row * pitch + c) = make_float2(x[k][0], x[k][1]);
    }
    if (h == 1) __syncthreads();
  }
}

// The line of row `row` (a chunk row) from its coefficients: dg = the two
// diagonal entries, xw / xm = the couplings of columns 2l-1|2l and 2l|2l+1,
// yn / ys = the couplings to the rows above / below; f = the free bits of the
// lane's points in this row, fa / fb in the rows above / below.
__device__ __forceinline__ TileLine tile_line(int row, float dg0, float dg1, float xw, float xm,
                                              float yn0, float yn1, float ys0, float ys1,
                                              unsigned f, unsigned fa, unsigned fb) {
  const int lane = threadIdx.x & 31;
  const unsigned fw = __shfl_up_sync(FULL_MASK, f >> 1, 1) & 1u;  // column 2l-1
  const bool f0 = f & 1u, f1 = (f >> 1) & 1u;
  const bool top = (row & (kBlkY - 1)) == 0, bot = (row & (kBlkY - 1)) == kBlkY - 1;
  TileLine L;
  L.b0 = f0 ? dg0 : 1.0f;
  L.b1 = f1 ? dg1 : 1.0f;
  L.cw = (lane > 0 && f0 && fw) ? xw : 0.0f;
  L.cm = (f0 && f1) ? xm : 0.0f;
  L.cn0 = (!top && f0 && (fa & 1u)) ? yn0 : 0.0f;
  L.cn1 = (!top && f1 && (fa & 2u)) ? yn1 : 0.0f;
  L.cs0 = (!bot && f0 && (fb & 1u)) ? ys0 : 0.0f;
  L.cs1 = (!bot && f1 && (fb & 2u)) ? ys1 : 0.0f;
  return L;
}

// P_CG_Z on one 64 x 32 tile (register path, four rows per warp): the first
// step of a tile-preconditioned CG phase: r_0 = g_F, z_0 = M^-1 r_0 and
// rho_0 = <r_0, z_0>; p, Ap, q (buffer pcur) and w are set to 0, so that the
// first fused step, run with alpha = beta = 0, forms p_0 = -z_0 and Ap_0.
// The exchange buffer is the first TMA stage (no copy is in flight in a
// register pass).
template <class T>
__device__ void cg_z_tile(const DevInst& I, const Snap& S, int x0, int y0, int z,
                          float* scr, Acc& acc, FF* ffs) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = warp * kRY;
  const int e0 = x0 + 2 * lane;
  const bool v0 = e0 < I.nx, v1 = e0 + 1 < I.nx;
  const bool f32 = sizeof(T) == 4;
  const T* bd = f32 ? (const T*)I.diag32 : (const T*)I.diag;
  const T* bx = f32 ? (const T*)I.cx32 : (const T*)I.cx;
  const T* by = f32 ? (const T*)I.cy32 : (const T*)I.cy;
  const unsigned* m = I.mask[S.cur];
  auto bits = [&](int y) -> unsigned {
    return (v0 && y >= 0 && y < I.ny) ? my_free_bits(I, m, y, z, e0) : 0u;
  };
  TileLine L[kRY];
  float d[kRY][2], x[kRY][2];
  T rv[kRY][2];
#pragma unroll
  for (int k = 0; k < kRY; ++k) {
    const int y = y0 + r0 + k;
    const bool ok = y < I.ny && v0;
    const unsigned f = ok ? bits(y) : 0u;
    T dg[2] = {T(1), T(1)}, xm[2] = {T(0), T(0)}, yn[2] = {T(0), T(0)}, ys[2] = {T(0), T(0)};
    double gv[2] = {0.0, 0.0};
    if (ok) {
      const long long i = pidx(I, y, z, e0);
      ld2(bd, i, v0, v1, dg);
      ld2(bx, i, v0, v1, xm);
      if (y > 0) ld2(by, i - I.px, v0, v1, yn);
      ld2(by, i, v0, v1, ys);
      if (S.gp32) {
        float gf[2];
        ld2(I.g32[S.cur], i, v0, v1, gf);
        gv[0] = gf[0];
        gv[1] = gf[1];
      } else {
        ld2(I.g[S.cur], i, v0, v1, gv);
      }
    }
    // coupling of column 2l-1 to 2l: the west lane's cx of its second point
    const float xw = __shfl_up_sync(FULL_MASK, (float)xm[1], 1);
    L[k] = tile_line(r0 + k, (float)dg[0], (float)dg[1], xw, (float)xm[0], (float)yn[0],
                     (float)yn[1], (float)ys[0], (float)ys[1], f, ok ? bits(y - 1) : 0u,
                     ok ? bits(y + 1) : 0u);
    rv[k][0] = (f & 1u) ? (T)gv[0] : T(0);
    rv[k][1] = (f & 2u) ? (T)gv[1] : T(0);
    d[k][0] = (float)rv[k][0];
    d[k][1] = (float)rv[k][1];
  }
  zebra_sweep<kRY>(L, d, r0, scr, 64, x);
  const int pc = S.pcur;
  T* r_out = f32 ? (T*)I.r32[pc] : (T*)I.r64[pc];
  T* z_out = f32 ? (T*)I.z32[pc] : (T*)I.z64[pc];
  T* p_out = f32 ? (T*)I.p32[pc] : (T*)I.p64[pc];
  T* ap_out = f32 ? (T*)I.Ap32[pc] : (T*)I.Ap64[pc];
  T* q_out = f32 ? (T*)I.q32[pc] : (T*)I.q64[pc];
  T* w_out = f32 ? (T*)I.w32 : (T*)I.w64;
  float s32 = 0.0f;
#pragma unroll
  for (int k = 0; k < kRY; ++k) {
    const int y = y0 + r0 + k;
    if (y >= I.ny || !v0) continue;
    const long long i = pidx(I, y, z, e0);
    const T z0 = (T)x[k][0], z1 = (T)x[k][1];
    st2(r_out, i, v0, v1, rv[k][0], rv[k][1]);
    st2(z_out, i, v0, v1, z0, z1);
    st2(p_out, i, v0, v1, T(0), T(0));
    st2(ap_out, i, v0, v1, T(0), T(0));
    st2(q_out, i, v0, v1, T(0), T(0));
    st2(w_out, i, v0, v1, T(0), T(0));
    if (f32) {
      s32 = fmaf((float)rv[k][0], (float)z0, s32);
      s32 = fmaf((float)rv[k][1], (float)z1, s32);
    } else {
      acc.s[0] = fma((double)rv[k][0], (double)z0, acc.s[0]);
      acc.s[0] = fma((double)rv[k][1], (double)z1, acc.s[0]);
    }
  }
  if (f32) ff_acc(ffs[0], s32);
  __syncthreads();  // the exchange buffer is free again
}

// ----------------------------------------------- explicit reduced system --
//
// The paper's design extracts A_k = Z' A Z (Sec. 4) into its own matrix;
// here that is an option beside the bitmask: the free points get a compact
// numbering (tiles in order, rows within a tile, columns within a row, the
// groups' ranges concatenated), A_FF is stored in that numbering as rows of
// a diagonal and 2*dim neighbour slots (compact index and coupling), and the
// CG phase runs on compact vectors.  It pays when few points are free: a CG
// step then touches m entries instead of streaming all n.

// Exclusive prefix sum of v over the CTA in thread order; `total` receives
// the sum.  All threads must call it (two block barriers).
__device__ __forceinline__ int cta_excl_scan(int v, int* s_warp, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(FULL_MASK, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  int before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const int t = s_warp[w];
    before += w < warp ? t : 0;
    all += t;
  }
  __syncthreads();
  total = all;
  return before + x - v;
}

// The free bits of the lane's two points of row (y, z) (0 past the grid).
__device__ __forceinline__ unsigned rx_bits(const DevInst& I, const Snap& S, int y, int z,
                                            int e0) {
  if (y >= I.ny || e0 >= I.nx) return 0u;
  const unsigned b = my_free_bits(I, I.mask[S.cur], y, z, e0);
  return e0 + 1 < I.nx ? b : (b & 1u);
}

// P_RX_COUNT on one tile: the number of free points (a count of the pass).
__device__ __forceinline__ void rx_count_tile(const DevInst& I, const Snap& S, int x0, int y0,
                                              int z, Acc& acc) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e0 = x0 + 2 * lane;
#pragma unroll
  for (int k = 0; k < kRY; ++k) acc.c[0] += __popc(rx_bits(I, S, y0 + warp * kRY + k, z, e0));
}

// The passes of the explicit reduced system run out of line: they are not
// the hot path of the default solve and, inlined, would raise the register
// and stack use of the whole pass kernel.

// P_RX_MAP over a group's tiles: compact indices from the group's offset
// (written by P_RX_COUNT's last group), fidx, r_0 = g_F in compact order, and
// the full-length w set to 0 (the search direction is scattered into it).
template <class T>
__device__ __noinline__ void rx_map_group(const DevInst& I, const Snap& S, int grp, int t_lo, int t_hi,
                             int* s_warp) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool f32 = sizeof(T) == 4;
  T* rc = f32 ? (T*)I.rc32[S.pcur] : (T*)I.rc64[S.pcur];
  T* wf = f32 ? (T*)I.w32 : (T*)I.w64;
  const unsigned lt = (1u << lane) - 1u;
  int base = __ldcg(I.goff + grp);
  for (int tile = t_lo; tile < t_hi; ++tile) {
    const int rest = tile / I.tiles_x;
    const int x0 = (tile % I.tiles_x) * kTX, y0 = (rest % I.tiles_y) * kTY, z = rest / I.tiles_y;
    const int e0 = x0 + 2 * lane;
    const bool v0 = e0 < I.nx, v1 = e0 + 1 < I.nx;
    const int ya = y0 + warp * kRY;
    unsigned fb[kRY], b0[kRY], b1[kRY];
    int wtot = 0;
#pragma unroll
    for (int k = 0; k < kRY; ++k) {
      fb[k] = rx_bits(I, S, ya + k, z, e0);
      b0[k] = __ballot_sync(FULL_MASK, fb[k] & 1u);
      b1[k] = __ballot_sync(FULL_MASK, (fb[k] >> 1) & 1u);
      wtot += __popc(b0[k]) + __popc(b1[k]);
    }
    int tile_tot;
    const int wo = __shfl_sync(FULL_MASK, cta_excl_scan(lane == 0 ? wtot : 0, s_warp, tile_tot), 0);
    int off = base + wo;
#pragma unroll
    for (int k = 0; k < kRY; ++k) {
      const int y = ya + k;
      const int k0 = off + __popc(b0[k] & lt) + __popc(b1[k] & lt);
      const int k1 = k0 + (int)(fb[k] & 1u);
      if (y < I.ny && v0) {
        const long long i = pidx(I, y, z, e0);
        I.cidx[i] = (fb[k] & 1u) ? k0 : -1;
        if (v1) I.cidx[i + 1] = (fb[k] & 2u) ? k1 : -1;
        st2(wf, i, v0, v1, T(0), T(0));
        double gv[2] = {0.0, 0.0};
        if (S.gp32) {
          float gf[2];
          ld2(I.g32[S.cur], i, v0, v1, gf);
          gv[0] = gf[0];
          gv[1] = gf[1];
        } else {
          ld2(I.g[S.cur], i, v0, v1, gv);
        }
        if (fb[k] & 1u) {
          I.fidx[k0] = (int)i;
          rc[k0] = (T)gv[0];
        }
        if (fb[k] & 2u) {
          I.fidx[k1] = (int)(i + 1);
          rc[k1] = (T)gv[1];
        }
      }
      off += __popc(b0[k]) + __popc(b1[k]);
    }
    base += tile_tot;
  }
}

// P_RX_BUILD on one tile: the rows of A_FF of its free points in compact
// numbering, 1/diagonal, and the first CG step's state: z_0 = M^-1 r_0 (M = I
// or the diagonal), rho_0 = <r_0, z_0> (sum 0); compact p, Ap, w = 0 so that
// the first fused step, run with alpha = beta = 0, forms p_0 and Ap_0.
template <class T, bool JAC>
__device__ __noinline__ void rx_build_tile(const DevInst& I, const Snap& S, int x0, int y0, int z, Acc& acc,
                              FF* ffs) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool f32 = sizeof(T) == 4;
  const T* bd = f32 ? (const T*)I.diag32 : (const T*)I.diag;
  const T* bx = f32 ? (const T*)I.cx32 : (const T*)I.cx;
  const T* by = f32 ? (const T*)I.cy32 : (const T*)I.cy;
  const T* bz = f32 ? (const T*)I.cz32 : (const T*)I.cz;
  const T* dv = f32 ? (const T*)I.dinv32 : (const T*)I.dinv;
  T* rd = f32 ? (T*)I.rd32 : (T*)I.rd64;
  T* rv = f32 ? (T*)I.rv32 : (T*)I.rv64;
  T* rdi = f32 ? (T*)I.rdi32 : (T*)I.rdi64;
  const T* rc = f32 ? (const T*)I.rc32[S.pcur] : (const T*)I.rc64[S.pcur];
  T* pcv = f32 ? (T*)I.pc32[S.pcur] : (T*)I.pc64[S.pcur];
  T* apc = f32 ? (T*)I.apc32[S.pcur] : (T*)I.apc64[S.pcur];
  T* wc = f32 ? (T*)I.wc32 : (T*)I.wc64;
  const long long st = I.n;
  float s32 = 0.0f;
  for (int k = 0; k < kRY; ++k) {
    const int y = y0 + warp * kRY + k;
    if (y >= I.ny) break;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int x = x0 + 2 * lane + h;
      if (x >= I.nx) continue;
      const long long i = pidx(I, y, z, x);
      const int c = __ldcg(I.cidx + i);
      if (c < 0) continue;
      int nb[kMaxNb];
      T val[kMaxNb];
      auto slot = [&](int j, bool has, long long o, T cpl) {
        const int q = has ? __ldcg(I.cidx + i + o) : -1;
        nb[j] = q >= 0 ? q : c;
        val[j] = q >= 0 ? cpl : T(0);
      };
      slot(0, x > 0, -1, x > 0 ? bx[i - 1] : T(0));
      slot(1, x + 1 < I.nx, 1, bx[i]);
      slot(2, y > 0, -(long long)I.px, y > 0 ? by[i - I.px] : T(0));
      slot(3, y + 1 < I.ny, I.px, by[i]);
      if (I.dim == 3) {
        slot(4, z > 0, -I.plane, z > 0 ? bz[i - I.plane] : T(0));
        slot(5, z + 1 < I.nz, I.plane, bz[i]);
      }
      const int nn = 2 * I.dim;
      for (int j = 0; j < nn; ++j) {
        I.rnb[j * st + c] = nb[j];
        rv[j * st + c] = val[j];
      }
      rd[c] = bd[i];
      const T di = dv[i];
      rdi[c] = di;
      pcv[c] = T(0);
      apc[c] = T(0);
      wc[c] = T(0);
      const T r = rc[c];
      const T zz = JAC ? r * di : r;
      if (f32) s32 = fmaf((float)r, (float)zz, s32);
      else acc.s[0] = fma((double)r, (double)zz, acc.s[0]);
    }
  }
  if (f32) ff_acc(ffs[0], s32);
}

// P_RCG over compact indices [lo, hi): the fused CG step of P_CG_F on the
// compact system, with the neighbours' p_j formed from their old r, Ap, p.
template <class T, bool JAC>
__device__ __noinline__ void rcg_range(const DevInst& I, const Snap& S, long long lo, long long hi, Acc& acc,
                          FF* ffs) {
  const bool f32 = sizeof(T) == 4;
  const int pc = S.pcur;
  const T* GPCG_RESTRICT r = f32 ? (const T*)I.rc32[pc] : (const T*)I.rc64[pc];
  const T* GPCG_RESTRICT p = f32 ? (const T*)I.pc32[pc] : (const T*)I.pc64[pc];
  const T* GPCG_RESTRICT ap = f32 ? (const T*)I.apc32[pc] : (const T*)I.apc64[pc];
  const T* GPCG_RESTRICT rd = f32 ? (const T*)I.rd32 : (const T*)I.rd64;
  const T* GPCG_RESTRICT rv = f32 ? (const T*)I.rv32 : (const T*)I.rv64;
  const T* GPCG_RESTRICT di = f32 ? (const T*)I.rdi32 : (const T*)I.rdi64;
  T* r_o = f32 ? (T*)I.rc32[pc ^ 1] : (T*)I.rc64[pc ^ 1];
  T* p_o = f32 ? (T*)I.pc32[pc ^ 1] : (T*)I.pc64[pc ^ 1];
  T* ap_o = f32 ? (T*)I.apc32[pc ^ 1] : (T*)I.apc64[pc ^ 1];
  T* w = f32 ? (T*)I.wc32 : (T*)I.wc64;
  const int* GPCG_RESTRICT rnb = I.rnb;
  const long long st = I.n;
  const int nn = 2 * I.dim;
  const T a = (T)S.alpha, b = (T)S.beta;
  for (long long k = lo + threadIdx.x; k < hi; k += kThreads) {
    const T pk = p[k];
    const T rn = fma(a, ap[k], r[k]);
    const T zn = JAC ? rn * di[k] : rn;
    const T pn = fma(b, pk, -zn);
    w[k] = fma(a, pk, w[k]);
    T y = rd[k] * pn;
    for (int j = 0; j < nn; ++j) {
      const int q = ldro(rnb + j * st + k);
      const T rq = fma(a, ap[q], r[q]);
      const T pq = fma(b, p[q], -(JAC ? rq * di[q] : rq));
      y = fma(rv[j * st + k], pq, y);
    }
    r_o[k] = rn;
    p_o[k] = pn;
    ap_o[k] = y;
    const T dy = JAC ? y * di[k] : y;
    if (f32) {
      ff_fma(ffs[0], (float)rn, (float)zn);
      ff_fma(ffs[1], (float)pn, (float)y);
      ff_fma(ffs[2], (float)zn, (float)y);
      ff_fma(ffs[3], (float)y, (float)dy);
    } else {
      acc.s[0] = fma((double)rn, (double)zn, acc.s[0]);
      acc.s[1] = fma((double)pn, (double)y, acc.s[1]);
      acc.s[2] = fma((double)zn, (double)y, acc.s[2]);
      acc.s[3] = fma((double)y, (double)dy, acc.s[3]);
    }
  }
}

// P_RW over compact indices [lo, hi): w_{j+1} = w_j + alpha_j p_j scattered
// into the full-length w (zero elsewhere since P_RX_MAP).
template <class T>
__device__ __noinline__ void rw_range(const DevInst& I, const Snap& S, long long lo, long long hi) {
  const bool f32 = sizeof(T) == 4;
  const T* p = f32 ? (const T*)I.pc32[S.pcur] : (const T*)I.pc64[S.pcur];
  const T* wc = f32 ? (const T*)I.wc32 : (const T*)I.wc64;
  T* wf = f32 ? (T*)I.w32 : (T*)I.w64;
  const T a = (T)S.alpha;
  for (long long k = lo + threadIdx.x; k < hi; k += kThreads)
    wf[ldro(I.fidx + k)] = fma(a, p[k], wc[k]);
}

// ---------------------------------------------------------------- control --

__device__ double pass_bytes(const DevInst& I, const Ctl& C, int pass) {
  // algorithmic HBM bytes of one pass per valid point: every array the pass
  // must read or write, once (documented per pass in the design notes)
  const double kc = (double)I.kc;
  const double sv = C.cg32 ? 4.0 : 8.0;
  const double pj = I.opt.precond == PC_JACOBI ? sv : 0.0;
  double per = 0.0;
  switch (pass) {
    case P_START: per = 24.0 + (I.opt.use_x0 ? 8.0 : 0.0) + (I.x32[0] ? 4.0 : 0.0); break;
    case P_CENSUS:
      per = C.gp32 ? 4.0 * kc + 24.125 : 8.0 * kc + 40.0 + 0.125 + (C.x32_live ? 20.0 : 0.0);
      break;
    case P_GP_ALPHA: per = C.gp32 ? 4.0 * kc + 4.0 : 8.0 * kc + 32.0; break;
    case P_TRIAL:
      if (C.gp32)
        per = 4.0 * kc + 32.25 + (C.dir == D_W32 ? 4.0 : 0.0);
      else
        per = 8.0 * kc + 56.0 + 0.25 + (C.dir == D_W64 ? 8.0 : (C.dir == D_W32 ? 4.0 : 0.0));
      break;
    case P_CG_B:  // (+ 1/diag with point Jacobi)
      per = sv * kc + (C.first_cg ? (C.gp32 ? 4.0 : 8.0) + 4.0 * sv : 4.0 * sv) + 0.125 + pj;
      break;
    case P_CG_A: per = 6.0 * sv + pj; break;
    case P_CG_F:  // tile preconditioner: z, q, p, r, Ap, w read and written
      per = sv * kc + (I.opt.precond == PC_TILE ? 12.0 * sv : 8.0 * sv + pj) + 0.125;
      break;
    case P_CG_Z: per = (C.gp32 ? 4.0 : 8.0) + 3.0 * sv + 6.0 * sv + 0.125; break;
    case P_RX_COUNT: per = 0.125; break;
    case P_RX_MAP:  // mask, cidx and w for every point; g, fidx, r for the free ones
      return (0.125 + 4.0 + sv) * (double)I.n + ((C.gp32 ? 4.0 : 8.0) + 4.0 + sv) * (double)C.m;
    case P_RX_BUILD: {  // cidx of every point; bands, 1/diag, r in; rows, p, Ap, w out
      const double nn = 2.0 * I.dim;
      return 4.0 * (double)I.n +
             (sv * kc + sv + sv + (1.0 + nn) * sv + 4.0 * nn + sv + 3.0 * sv) * (double)C.m;
    }
    case P_RCG: {  // r, p, Ap, w in and out; the row (and 1/diag)
      const double nn = 2.0 * I.dim;
      return (8.0 * sv + (1.0 + nn) * sv + 4.0 * nn + pj) * (double)C.m;
    }
    case P_RW: return (4.0 + 3.0 * sv) * (double)C.m;
    default: break;
  }
  return per * (double)I.n;
}

// End the solve with `status`: one final census pass refreshes g, the active
// and binding counts, ||pg|| and q at the returned point.
__device__ void set_done(Ctl& C, int status) {
  C.status = status;
  C.census_mode = CM_FINAL;
  C.gp32 = 0;
  C.pass = P_CENSUS;
}

// Leave the mixed phase: everything from here on is FP64, starting with an
// FP64 census of the current iterate.
__device__ void switch_fp64(Ctl& C, int mode) {
  C.gp32 = 0;
  C.refined = 1;
  C.census_mode = mode;
  C.pass = P_CENSUS;
}

__device__ void start_search(Ctl& C, int dir) {
  C.dir = dir;
  C.alpha = dir == D_ZERO ? 0.0 : 1.0;
  C.ls_i = 0;
  C.trial_gp = 0;
  C.pass = P_TRIAL;
}

// Whether the instance's CG phase runs fused steps (P_CG_F): 2-D grids whose
// tensor maps of the CG precision are valid (and, under the tile preconditioner, its maps).
__device__ __forceinline__ bool cg_fused(const DevInst& I, const Ctl& C) {
  if (I.tmaps == nullptr) return false;
  // 3-D: the FP32 step without a preconditioner (its stage has no room for
  // FP64 boxes or for 1/diag of three planes)
  if (I.dim == 3) return C.cg32 && I.tma3 && I.opt.precond == PC_NONE;
  if (I.dim != 2 || !(C.cg32 ? I.tma32 : I.tma64)) return false;
  return I.opt.precond != PC_TILE || ((I.tma_tile >> (C.cg32 ? 1 : 0)) & 1);
}

// Start a CG phase on the face of the current iterate (Eq. cg, cg2), w0 = 0.
__device__ void begin_cg(const DevInst& I, Ctl& C) {
  // mixed precision: FP32 streams in the FP32 phase; after it, FP64 CG (refine
  // 1) or FP32 correction CG on the FP64 gradient (refine 2)
  C.cg32 = (I.opt.mixed && (!C.refined || I.opt.refine == 2)) ? 1 : 0;
  C.cg_j = 0;
  C.cdmax = 0.0;
  C.cg_finish = 0;
  if (I.opt.max_cg >= 1 && I.opt.extract) {
    C.first_cg = 0;
    C.beta = 0.0;
    C.pass = P_RX_COUNT;
  } else if (I.opt.max_cg >= 1 && I.opt.precond == PC_TILE && cg_fused(I, C)) {
    C.first_cg = 0;
    C.beta = 0.0;
    C.pass = P_CG_Z;
  } else if (I.opt.max_cg >= 1) {
    C.first_cg = 1;
    C.beta = 0.0;
    C.pass = P_CG_B;
  } else {
    start_search(C, D_ZERO);
  }
}

// Start outer iterate k (Algorithm GPCG): gradient projection unless the
// previous iterate satisfied Eq. cgstop3.
__device__ void begin_outer(const DevInst& I, Ctl& C) {
  if (C.outer_iters >= I.opt.max_outer) {
    set_done(C, S_MAXIT);
    return;
  }
  C.outer_iters++;
  if (!C.continue_cg) {
    C.gp_j = 0;
    C.dmax = 0.0;
    C.pass = P_GP_ALPHA;
  } else {
    begin_cg(I, C);
  }
}

// ||grad_Omega q|| <= tau held.  In mixed precision the first time this
// happens starts the closing FP64 CG phase on the identified face.
__device__ void on_converged(const DevInst& I, Ctl& C, int* live) {
  if (C.gp32) {
    // the FP32-streamed estimate met tau: certify in FP64 and, with refine,
    // run the closing FP64 CG phase on the identified face
    switch_fp64(C, I.opt.refine ? CM_REFINE : CM_RESUME);
  } else if (I.opt.mixed && I.opt.refine && !C.refined) {
    C.refined = 1;
    C.refining = 1;
    C.continue_cg = 1;
    C.eta2 = I.opt.eta2_refine;
    C.outer_iters++;
    begin_cg(I, C);
  } else {
    // the accepted FP64 trial already gave g, ||pg||, |A| and |B| at the
    // returned point, and q by its decrease: done without a final census
    C.status = S_OK;
    C.census_mode = CM_INIT;
    C.pass = P_NONE;
    C.done = 1;
    atomicSub(live, 1);
  }
}


// After alpha_j of a fused phase is known (C.rr = rho_j = <r_j, z_j>, z =
// M^-1 r): the CG bookkeeping and Eq. cgstop1 of step j (decrease
// alpha_j rho_j / 2), with rho_{j+1} = <r_j + alpha Ap_j, M^-1 (r_j + alpha Ap_j)>
// = rho_j + 2 alpha_j <z_j,Ap_j> + alpha_j^2 <Ap_j,M^-1 Ap_j> (its sums come
// from the pass that formed Ap_j); then either the next fused step or a last
// P_CG_A that completes w_{j+1} before the projected search.
__device__ void cg_advance(const DevInst& I, Ctl& C, double zAp, double ApMAp) {
  const Opts& o = I.opt;
  const double rr_next = C.rr + 2.0 * C.alpha * zAp + C.alpha * C.alpha * ApMAp;
  C.cg_j++;
  C.cg_iters++;
  if (C.refining) C.refine_cg_iters++;
  const double delta = 0.5 * C.alpha * C.rr;  // q_k(w_j) - q_k(w_{j+1})
  const bool stop = (C.cg_j >= 2 && delta <= C.eta2 * C.cdmax) ||  // Eq. cgstop1
                    rr_next <= 0.0 || C.cg_j >= o.max_cg;
  if (delta > C.cdmax) C.cdmax = delta;
  if (stop) {
    C.cg_finish = 1;
    C.pass = I.opt.extract ? P_RW : P_CG_A;
  } else {
    C.beta = rr_next / C.rr;
    C.rr = rr_next;
    C.pass = I.opt.extract ? P_RCG : P_CG_F;
  }
}

// The next gradient projection step (Eq. next-y) from <g_Omega, g_Omega> and
// <g_Omega, A g_Omega> at the current iterate: alpha0 = the exact minimiser
// along -grad_Omega q (Eq. bqpls), then trials alpha0, alpha0/2, ...
__device__ void gp_step(Ctl& C, double gg, double gAg) {
  if (!(gAg > 0.0) || !isfinite(gg)) {
    set_done(C, S_NUMERIC);
    return;
  }
  C.alpha0 = gg / gAg;
  C.alpha = C.alpha0;
  C.ls_i = 0;
  C.dir = D_NEG_G;
  C.trial_gp = 1;
  C.pass = P_TRIAL;
}

// Whether the instance's mixed-phase GP passes are staged (then a trial along
// -g also forms alpha0 at its trial point).
__device__ __forceinline__ bool staged_gp32(const DevInst& I, const Ctl& C) {
  return C.gp32 && I.dim == 2 && I.tma_gp && I.tma32 && I.tma_mask;
}

__device__ void finalize(const DevInst& I, Ctl& C, const double* red, int* live) {
  for (int k = 0; k < kNRed; ++k) C.red[k] = red[k];
  if (C.hold) return;  // standalone timing/test launch: leave the state alone
  const Opts& o = I.opt;
  C.passes++;
  C.alg_bytes += pass_bytes(I, C, C.pass);
  switch (C.pass) {
    case P_START:
      C.x32_live = C.gp32;  // the mixed phase moves the FP32 iterate only
      C.pass = P_CENSUS;
      break;
    case P_CENSUS: {
      if (!C.gp32) C.x32_live = 0;  // an FP64 census rebuilt x from x32
      C.pg2 = red[0];
      C.xgb = red[1];
      C.nA = red[4];
      C.nB = red[5];
      if ((C.census_mode == CM_REFINE || C.census_mode == CM_RESUME) && C.mixed_nA < 0.0)
        C.mixed_nA = C.nA;  // the face the FP32 phase handed over
      if (C.census_mode == CM_FINAL) {
        C.pass = P_NONE;
        C.done = 1;
        atomicSub(live, 1);
        break;
      }
      if (C.census_mode == CM_REFINE) {  // closing FP64 CG phase on this face
        C.census_mode = CM_INIT;
        C.refining = 1;
        C.continue_cg = 1;
        C.eta2 = o.eta2_refine;
        C.outer_iters++;
        begin_cg(I, C);
        break;
      }
      if (C.census_mode == CM_RESUME) {  // continue GPCG in FP64
        C.census_mode = CM_INIT;
        if (!isfinite(C.pg2)) {
          set_done(C, S_NUMERIC);
        } else if (sqrt(C.pg2) <= C.tau) {
          set_done(C, S_OK);
        } else {
          C.eta2 = o.eta2;
          C.continue_cg = 0;
          begin_outer(I, C);
        }
        break;
      }
      C.best_pg2 = C.pg2;
      C.search_pg2 = C.pg2;
      C.stall = 0;
      C.slow = 0;
      C.pg0 = sqrt(C.pg2);
      C.tau = fmax(o.tau_abs, o.tau_rel * C.pg0);
      C.eta2 = o.eta2;
      C.continue_cg = 0;
      if (!isfinite(C.pg2)) {
        set_done(C, S_NUMERIC);
      } else if (C.pg0 <= C.tau) {
        set_done(C, S_OK);
      } else {
        begin_outer(I, C);
      }
      break;
    }
    case P_GP_ALPHA:
      gp_step(C, red[0], red[1]);
      break;
    case P_TRIAL: {
      C.ls_trials++;
      const double gs = red[0];
      const double dq = 0.5 * (red[0] + red[1]);  // q(xt) - q(x)
      if (dq <= o.mu * gs) {                     // Eq. gplsstop / cglsstop2
        C.cur ^= 1;
        C.pg2 = red[2];
        C.nA = red[4];
        C.nB = red[5];
        // <x, g + b> = 2 (q(x) - c) moves by 2 (q(xt) - q(x)) = <s, g + gt>,
        // exact for a quadratic (every FP64 census sets it afresh)
        C.xgb += 2.0 * dq;
        const double pgn = sqrt(C.pg2);
        if (C.trial_gp) {
          C.gp_iters++;
          C.gp_j++;
          if (o.mixed && !C.gp32) C.fp64_gp++;
          const double dec = -dq;
          const bool same = red[6] == 0.0;  // Eq. pgstop1
          if (pgn <= C.tau) {
            on_converged(I, C, live);
            break;
          }
          const bool stop = same || (C.gp_j >= 2 && dec <= o.eta1 * C.dmax) ||  // Eq. pgstop2
                            (C.gp_j >= o.max_gp);
          if (dec > C.dmax) C.dmax = dec;
          if (stop) {
            begin_cg(I, C);
          } else if (staged_gp32(I, C)) {
            gp_step(C, red[2], red[3]);  // the trial formed alpha0 at the new iterate
          } else {
            C.pass = P_GP_ALPHA;
          }
        } else {
          C.refining = 0;
          if (pgn <= C.tau) {
            on_converged(I, C, live);
            break;
          }
          if (C.gp32) {
            // mixed phase: leave it when ||pg|| stops improving -- five
            // iterates without a 2 % decrease of ||pg||^2, or two in a row on
            // an unchanged face (Eq. cgstop3 holds) that do not halve ||pg||:
            // there CG runs on a fixed system and only FP32 noise stops it
            const bool face_kept = C.nB == C.nA;
            const bool halved = C.pg2 < 0.25 * C.search_pg2;
            C.search_pg2 = C.pg2;
            C.slow = (face_kept && !halved) ? C.slow + 1 : 0;
            if (C.pg2 < 0.98 * C.best_pg2) {
              C.best_pg2 = C.pg2;
              C.stall = 0;
            } else {
              ++C.stall;
            }
            if (C.stall >= 5 || C.slow >= 2) {
              switch_fp64(C, CM_RESUME);
              break;
            }
          }
          if (C.nB == C.nA) {  // Eq. cgstop3: B(x) = A(x)
            C.eta2 = fmax(C.eta2 * o.eta2_shrink, o.eta2_floor);
            C.continue_cg = 1;
          } else {
            C.eta2 = o.eta2;
            C.continue_cg = 0;
          }
          begin_outer(I, C);
        }
      } else {
        C.ls_i++;
        if (C.ls_i > o.max_ls) {
          // in the mixed phase the FP32 gradient may be too coarse for the
          // sufficient-decrease test: continue in FP64 instead of failing
          if (C.gp32) switch_fp64(C, CM_RESUME);
          else set_done(C, S_LINESEARCH);
          break;
        }
        if (C.dir != D_ZERO) C.alpha = ldexp(C.trial_gp ? C.alpha0 : 1.0, -C.ls_i);
      }
      break;
    }
    case P_CG_B: {
      if (C.first_cg) {
        C.rr = red[1];
        C.first_cg = 0;
        if (!(C.rr > 0.0)) {  // r = g_F vanished: no CG step (w stays 0)
          C.pcur ^= 1;
          start_search(C, D_ZERO);
          break;
        }
      }
      const double pAp = red[0];
      if (!(pAp > 0.0)) {
        set_done(C, S_NUMERIC);
        break;
      }
      C.alpha = C.rr / pAp;
      C.pcur ^= 1;
      if (cg_fused(I, C)) {
        // first step of a fused phase: z_0 = -p_0, so <z_0, Ap_0> = -<p_0, Ap_0>
        cg_advance(I, C, -pAp, red[2]);
      } else {
        C.pass = P_CG_A;
      }
      break;
    }
    case P_CG_Z: {
      const double rz = red[0];  // rho_0 = <r_0, M^-1 r_0>
      if (!isfinite(rz)) {
        set_done(C, S_NUMERIC);
      } else if (!(rz > 0.0)) {  // r = g_F vanished: no CG step (w stays 0)
        start_search(C, D_ZERO);
      } else {
        // the first fused step, with alpha = beta = 0, forms p_0 and Ap_0
        C.rr = rz;
        C.alpha = 0.0;
        C.beta = 0.0;
        C.pass = P_CG_F;
      }
      break;
    }
    case P_RX_COUNT:
      C.m = (int)red[4];  // the group offsets were written by this pass's last group
      if (C.m == 0) start_search(C, D_ZERO);  // no free variable: w = 0
      else C.pass = P_RX_MAP;
      break;
    case P_RX_MAP:
      C.pass = P_RX_BUILD;
      break;
    case P_RX_BUILD: {
      const double rz = red[0];  // rho_0 = <r_0, M^-1 r_0>
      if (!isfinite(rz)) {
        set_done(C, S_NUMERIC);
      } else if (!(rz > 0.0)) {  // r = g_F vanished: no CG step (w stays 0)
        start_search(C, D_ZERO);
      } else {
        C.rr = rz;
        C.alpha = 0.0;
        C.beta = 0.0;
        C.pass = P_RCG;
      }
      break;
    }
    case P_RW:
      C.cg_finish = 0;
      start_search(C, C.cg32 ? D_W32 : D_W64);
      break;
    case P_RCG:
    case P_CG_F: {
      C.rr = red[0];  // ||r_j||^2 of the stored r_j
      const double pAp = red[1];
      if (!(pAp > 0.0)) {
        set_done(C, S_NUMERIC);
        break;
      }
      C.alpha = C.rr / pAp;
      C.pcur ^= 1;
      cg_advance(I, C, red[2], red[3]);
      break;
    }
    case P_CG_A: {
      if (C.cg_finish) {  // w of the last fused step is complete: search along it
        C.cg_finish = 0;
        start_search(C, C.cg32 ? D_W32 : D_W64);
        break;
      }
      const double rr_new = red[0];
      C.cg_j++;
      C.cg_iters++;
      if (C.refining) C.refine_cg_iters++;
      const double delta = 0.5 * C.alpha * C.rr;  // q_k(w_{j-1}) - q_k(w_j)
      const bool stop = (C.cg_j >= 2 && delta <= C.eta2 * C.cdmax) ||  // Eq. cgstop1
                        rr_new == 0.0 || C.cg_j >= o.max_cg;
      if (delta > C.cdmax) C.cdmax = delta;
      if (stop) {
        start_search(C, C.cg32 ? D_W32 : D_W64);
      } else {
        C.beta = rr_new / C.rr;
        C.rr = rr_new;
        C.pass = P_CG_B;
      }
      break;
    }
    default:
      break;
  }
}


// ------------------------------------------------------- TMA-staged CG --
//
// The two CG passes of a 2-D instance (and the pointwise CG pass of any
// instance) stream a work item through shared memory with the tensor memory
// accelerator, kStages stages deep: the next kStages-1 chunks are in flight
// while chunk k is computed.  Stage layout (each array 128-byte aligned),
// T = float (h = 4) or double (h = 2):
//   P_CG_B (c = 32 rows FP32, 16 FP64): R (64+2h)x(c+2) from (x0-h, y-1) |
//           P likewise | D 64xc | CX (64+h)xc from x0-h | CY 64x(c+1) from y-1
//   P_CG_A (a = 32 rows FP32, 16 FP64): W | R | P | AP, 64xa each
// Out-of-range rows and columns arrive as zeros, which is exactly the
// operand and coupling outside the grid.

__host__ __device__ constexpr int align128(int b) { return (b + 127) / 128 * 128; }

template <class T>
struct ChunkGeo {
  static constexpr int H = 16 / (int)sizeof(T);
  static constexpr int CH = sizeof(T) == 4 ? 32 : 16;     // CG_B rows per chunk
  static constexpr int CH_A = sizeof(T) == 4 ? 32 : 16;  // CG_A rows per chunk
  static constexpr int BW = 64 + 2 * H;
  static constexpr int SZ_H = align128((CH + 2) * BW * (int)sizeof(T));
  static constexpr int OFF_R = 0;
  static constexpr int OFF_P = SZ_H;
  static constexpr int OFF_D = 2 * SZ_H;
  static constexpr int OFF_CX = OFF_D + 64 * CH * (int)sizeof(T);
  static constexpr int OFF_CY = OFF_CX + align128((64 + H) * CH * (int)sizeof(T));
  static constexpr int END_B = OFF_CY + align128(64 * (CH + 1) * (int)sizeof(T));
  static constexpr unsigned TX_B =
      (2 * (CH + 2) * BW + 64 * CH + (64 + H) * CH + 64 * (CH + 1)) * sizeof(T);
  static constexpr int SZ_A = 64 * CH_A * (int)sizeof(T);
  static constexpr unsigned TX_A = 4 * SZ_A;
  static constexpr int MB = sizeof(T) == 4 ? M32_RH0 : M64_RH0;  // first map of the precision
};
static_assert(ChunkGeo<float>::END_B <= kOffMask && ChunkGeo<double>::END_B <= kOffMask,
              "stage layout");
static_assert(5 * ChunkGeo<float>::SZ_A <= kOffMask &&
                  5 * ChunkGeo<double>::SZ_A <= kOffMask,
              "stage layout (W, R, P, AP and, with point Jacobi, 1/diag)");

__device__ __forceinline__ const void* tmap(const DevInst& I, int k) {
  return reinterpret_cast<const char*>(I.tmaps) + 128 * k;
}

template <class T>
__device__ __forceinline__ void issue_cgb(const DevInst& I, int pcur, int x0, int yc,
                                          unsigned st, unsigned bar) {
  using G = ChunkGeo<T>;
  constexpr int o = -M32_RH0;  // map offsets within a precision's block
  mbar_expect(bar, G::TX_B);
  // r of this step was written by P_CG_A into r[pcur^1]
  tma_load2d(st + G::OFF_R, tmap(I, G::MB + o + M32_RH0 + (pcur ^ 1)), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_P, tmap(I, G::MB + o + M32_PH0 + pcur), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_D, tmap(I, G::MB + o + M32_D), x0, yc, bar);
  tma_load2d(st + G::OFF_CX, tmap(I, G::MB + o + M32_CX), x0 - G::H, yc, bar);
  tma_load2d(st + G::OFF_CY, tmap(I, G::MB + o + M32_CY), x0, yc - 1, bar);
}

template <class T>
__device__ __forceinline__ void issue_cga(const DevInst& I, int pcur, int x0, int row,
                                          unsigned st, unsigned bar) {
  using G = ChunkGeo<T>;
  constexpr int o = -M32_RH0;
  mbar_expect(bar, G::TX_A + (I.opt.precond == PC_JACOBI ? G::SZ_A : 0));
  if (I.opt.precond == PC_JACOBI)
    tma_load2d(st + 4 * G::SZ_A, tmap(I, G::MB + o + M32_ADI), x0, row, bar);
  tma_load2d(st + 0 * G::SZ_A, tmap(I, G::MB + o + M32_W), x0, row, bar);
  tma_load2d(st + 1 * G::SZ_A, tmap(I, G::MB + o + M32_R0 + pcur), x0, row, bar);
  tma_load2d(st + 2 * G::SZ_A, tmap(I, G::MB + o + M32_P0 + pcur), x0, row, bar);
  tma_load2d(st + 3 * G::SZ_A, tmap(I, G::MB + o + M32_AP0 + pcur), x0, row, bar);
}

// P_CG_B (not the first step of a phase) on one staged chunk of a 2-D grid:
// p = -r + beta p_old over the halo'd box (in place), then Ap = Z Z' A Z Z' p
// and <p, Ap> for the chunk's interior.
template <class T>
__device__ __forceinline__ void cgb_chunk(const DevInst& I, unsigned char* st, int x0, int yc,
                                          int rows, T beta, const unsigned* fbits, T* p_out,
                                          T* ap_out, Acc& acc, FF& ff) {
  using G = ChunkGeo<T>;
  T* R = reinterpret_cast<T*>(st + G::OFF_R);
  const T* P = reinterpret_cast<const T*>(st + G::OFF_P);
  const T* D = reinterpret_cast<const T*>(st + G::OFF_D);
  const T* CX = reinterpret_cast<const T*>(st + G::OFF_CX);
  const T* CY = reinterpret_cast<const T*>(st + G::OFF_CY);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < (G::CH + 2) * G::BW; e += kThreads) R[e] = fma(beta, P[e], -R[e]);
  __syncthreads();
  constexpr int RPW = G::CH / kWarps;
  const int c = 2 * lane;
  const int e0 = x0 + c;
  const bool v0 = e0 < I.nx, v1 = e0 + 1 < I.nx;
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    const int ry = warp * RPW + k;
    const int y = yc + ry;
    if (ry >= rows || y >= I.ny || !v0) break;
    const T* Rr = R + (ry + 1) * G::BW + G::H + c;
    const T vc0 = Rr[0], vc1 = Rr[1];
    const T vw = Rr[-1], ve = Rr[2];
    const T vs0 = Rr[-G::BW], vs1 = Rr[1 - G::BW];
    const T vn0 = Rr[G::BW], vn1 = Rr[G::BW + 1];
    const T* Dr = D + ry * 64 + c;
    const T* Xr = CX + ry * (64 + G::H) + G::H + c;
    const T* Ys = CY + ry * 64 + c;
    const T* Yn = CY + (ry + 1) * 64 + c;
    T a0 = Dr[0] * vc0;
    a0 = fma(Xr[-1], vw, a0);
    a0 = fma(Xr[0], vc1, a0);
    a0 = fma(Ys[0], vs0, a0);
    a0 = fma(Yn[0], vn0, a0);
    T a1 = Dr[1] * vc1;
    a1 = fma(Xr[0], vc0, a1);
    a1 = fma(Xr[1], ve, a1);
    a1 = fma(Ys[1], vs1, a1);
    a1 = fma(Yn[1], vn1, a1);
    const unsigned fb = fbits[k] & 3u;
    a0 = (fb & 1u) ? a0 : T(0);
    a1 = (fb & 2u) ? a1 : T(0);
    const long long i = (long long)y * I.px + e0;
    st2(ap_out, i, v0, v1, a0, a1);
    st2(p_out, i, v0, v1, vc0, vc1);
    if (sizeof(T) == 4) {
      ff_fma(ff, (float)vc0, (float)a0);
      ff_fma(ff, (float)vc1, (float)a1);
    } else {
      acc.s[0] = fma((double)vc0, (double)a0, acc.s[0]);
      acc.s[0] = fma((double)vc1, (double)a1, acc.s[0]);
    }
  }
}

// P_CG_A on one staged chunk: w += alpha p, r' = r + alpha Ap (into `r`, the
// other buffer), <r', M^-1 r'> (M = I, or diag(A) from the staged 1/diag).  `row` is the chunk's first row in the (ny*nz) row
// space, `ylim` the number of rows of the chunk that lie inside the plane.
template <class T, bool JAC>
__device__ __forceinline__ void cga_chunk(const DevInst& I, const unsigned char* st, int x0,
                                          int row, int ylim, T alpha, T* w, T* r, Acc& acc,
                                          FF& ff) {
  using G = ChunkGeo<T>;
  const T* W = reinterpret_cast<const T*>(st + 0 * G::SZ_A);
  const T* R = reinterpret_cast<const T*>(st + 1 * G::SZ_A);
  const T* P = reinterpret_cast<const T*>(st + 2 * G::SZ_A);
  const T* AP = reinterpret_cast<const T*>(st + 3 * G::SZ_A);
  const T* DI = reinterpret_cast<const T*>(st + 4 * G::SZ_A);  // 1/diag (point Jacobi)
  constexpr bool jac = JAC;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int RPW = G::CH_A / kWarps;
  const int c = 2 * lane;
  const int e0 = x0 + c;
  const bool v0 = e0 < I.nx, v1 = e0 + 1 < I.nx;
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    const int ry = warp * RPW + k;
    if (ry >= ylim || !v0) break;
    const int o = ry * 64 + c;
    const T w0 = fma(alpha, P[o], W[o]), w1 = fma(alpha, P[o + 1], W[o + 1]);
    const T r0 = fma(alpha, AP[o], R[o]), r1 = fma(alpha, AP[o + 1], R[o + 1]);
    const T z0 = jac ? r0 * DI[o] : r0, z1 = jac ? r1 * DI[o + 1] : r1;
    const long long i = (long long)(row + ry) * I.px + e0;
    st2(w, i, v0, v1, w0, w1);
    st2(r, i, v0, v1, r0, r1);
    if (sizeof(T) == 4) {
      ff_fma(ff, (float)r0, (float)z0);
      ff_fma(ff, (float)r1, (float)z1);
    } else {
      acc.s[0] = fma((double)r0, (double)z0, acc.s[0]);
      acc.s[0] = fma((double)r1, (double)z1, acc.s[0]);
    }
  }
}

// ------------------------------------------------------- fused CG step --
//
// P_CG_F on a 2-D instance: one pass per CG step j >= 1 (Algorithm GPCG's
// CG phase on the reduced system, Eq. cg2).  With alpha = alpha_{j-1} and
// beta = beta_{j-1} over the halo box of the chunk, in place in the stage:
//   r_j = r_{j-1} + alpha Ap_{j-1},  z_j = M^-1 r_j,  p_j = -z_j + beta p_{j-1}
// (M = I, or diag(A) for point Jacobi, Sec. 6), at the chunk's points also
// w_j = w_{j-1} + alpha p_{j-1}; then Ap_j = Z Z' A Z Z' p_j and the sums
// rho_j = <r_j,z_j>, <p_j,Ap_j>, <z_j,Ap_j>, <Ap_j,M^-1 Ap_j> (from which the
// finalizer takes alpha_j and rho_{j+1}).
// r, p and Ap are read from buffer pcur and written to pcur^1.  Stage layout,
// T = float (f = 16 rows, h = 4) or double (f = 8, h = 2): R | P | AP, each
// (64+2h) x (f+2) from (x0-h, y-1) | W 64 x f | D 64 x f | CX (64+h) x f from
// x0-h | CY 64 x (f+1) from y-1.
template <class T>
struct GeoF {
  static constexpr int H = 16 / (int)sizeof(T);
  static constexpr int CH = sizeof(T) == 4 ? 16 : 8;
  static constexpr int BW = 64 + 2 * H;
  static constexpr int SZ_H = align128((CH + 2) * BW * (int)sizeof(T));
  static constexpr int SZ_I = 64 * CH * (int)sizeof(T);
  static constexpr int OFF_R = 0, OFF_P = SZ_H, OFF_AP = 2 * SZ_H, OFF_W = 3 * SZ_H;
  static constexpr int OFF_D = OFF_W + SZ_I, OFF_CX = OFF_D + SZ_I;
  static constexpr int OFF_CY = OFF_CX + align128((64 + H) * CH * (int)sizeof(T));
  static constexpr int OFF_DI = OFF_CY + align128(64 * (CH + 1) * (int)sizeof(T));  // 1/diag
  static constexpr int END = OFF_DI + SZ_H;
  static constexpr unsigned TX =
      (3 * (CH + 2) * BW + 2 * 64 * CH + (64 + H) * CH + 64 * (CH + 1)) * sizeof(T);
  static constexpr unsigned TX_DI = (CH + 2) * BW * sizeof(T);
  static constexpr int MB = sizeof(T) == 4 ? M32_RH0 : M64_RH0;
};
static_assert(GeoF<float>::END <= kOffMask && GeoF<double>::END <= kOffMask,
              "stage layout");

template <class T>
__device__ __forceinline__ void issue_cgf(const DevInst& I, int pcur, int x0, int yc,
                                          unsigned st, unsigned bar) {
  using G = GeoF<T>;
  constexpr int o = G::MB - M32_RH0;
  mbar_expect(bar, G::TX + (I.opt.precond == PC_JACOBI ? G::TX_DI : 0u));
  if (I.opt.precond == PC_JACOBI)
    tma_load2d(st + G::OFF_DI, tmap(I, o + M32_FDIH), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_R, tmap(I, o + M32_FRH0 + pcur), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_P, tmap(I, o + M32_FPH0 + pcur), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_AP, tmap(I, o + M32_FAPH0 + pcur), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_W, tmap(I, o + M32_FW), x0, yc, bar);
  tma_load2d(st + G::OFF_D, tmap(I, o + M32_FD), x0, yc, bar);
  tma_load2d(st + G::OFF_CX, tmap(I, o + M32_FCX), x0 - G::H, yc, bar);
  tma_load2d(st + G::OFF_CY, tmap(I, o + M32_FCY), x0, yc - 1, bar);
}

// The fused CG step on a 3-D grid (FP32): 8-row chunks of one plane, one row
// per warp.  Stage layout: RH | PH | APH (72 x 10 from (x0-4, row-1)) | W | D
// (64 x 8) | CX (68 x 8 from x0-4) | CY (64 x 9 from row-1) | CZD | CZU (cz of
// the plane below and of this plane) | RD | RU | PD | PU | APD | APU (r, p, Ap
// of the planes below and above), all 64 x 8 unless stated.  In the row space
// (nx, ny*nz) of the maps, the halo rows of a plane's first and last chunk
// rows are rows of the neighbouring planes; their couplings cy are zero (the
// last row of every plane has none), so they contribute nothing.  The planes
// below the first and above the last are out of range: zero-filled.
struct GeoF3 {
  static constexpr int H = 4, CH = 8, BW = 64 + 2 * H;
  static constexpr int SZ_H = align128((CH + 2) * BW * 4);
  static constexpr int SZ_I = 64 * CH * 4;
  static constexpr int OFF_R = 0, OFF_P = SZ_H, OFF_AP = 2 * SZ_H;
  static constexpr int OFF_W = 3 * SZ_H, OFF_D = OFF_W + SZ_I, OFF_CX = OFF_D + SZ_I;
  static constexpr int OFF_CY = OFF_CX + align128((64 + H) * CH * 4);
  static constexpr int OFF_CZD = OFF_CY + align128(64 * (CH + 1) * 4);
  static constexpr int OFF_CZU = OFF_CZD + SZ_I;
  static constexpr int OFF_RD = OFF_CZU + SZ_I, OFF_RU = OFF_RD + SZ_I;
  static constexpr int OFF_PD = OFF_RU + SZ_I, OFF_PU = OFF_PD + SZ_I;
  static constexpr int OFF_APD = OFF_PU + SZ_I, OFF_APU = OFF_APD + SZ_I;
  static constexpr int END = OFF_APU + SZ_I;
  static constexpr unsigned TX =
      (3 * (CH + 2) * BW + 2 * 64 * CH + (64 + H) * CH + 64 * (CH + 1) + 8 * 64 * CH) * 4;
};
static_assert(GeoF3::END <= kOffMask && GeoF3::CH == kWarps, "stage layout (one row per warp)");

// row: the chunk's first row in the row space (z * ny + yc).
__device__ __forceinline__ void issue_cgf3(const DevInst& I, int pcur, int x0, int row,
                                           unsigned st, unsigned bar) {
  using G = GeoF3;
  const int dn = row - I.ny, up = row + I.ny;
  mbar_expect(bar, G::TX);
  tma_load2d(st + G::OFF_R, tmap(I, M3_RH0 + pcur), x0 - G::H, row - 1, bar);
  tma_load2d(st + G::OFF_P, tmap(I, M3_PH0 + pcur), x0 - G::H, row - 1, bar);
  tma_load2d(st + G::OFF_AP, tmap(I, M3_APH0 + pcur), x0 - G::H, row - 1, bar);
  tma_load2d(st + G::OFF_W, tmap(I, M3_W), x0, row, bar);
  tma_load2d(st + G::OFF_D, tmap(I, M3_D), x0, row, bar);
  tma_load2d(st + G::OFF_CX, tmap(I, M3_CX), x0 - G::H, row, bar);
  tma_load2d(st + G::OFF_CY, tmap(I, M3_CY), x0, row - 1, bar);
  tma_load2d(st + G::OFF_CZD, tmap(I, M3_CZ), x0, dn, bar);
  tma_load2d(st + G::OFF_CZU, tmap(I, M3_CZ), x0, row, bar);
  tma_load2d(st + G::OFF_RD, tmap(I, M3_R0 + pcur), x0, dn, bar);
  tma_load2d(st + G::OFF_RU, tmap(I, M3_R0 + pcur), x0, up, bar);
  tma_load2d(st + G::OFF_PD, tmap(I, M3_P0 + pcur), x0, dn, bar);
  tma_load2d(st + G::OFF_PU, tmap(I, M3_P0 + pcur), x0, up, bar);
  tma_load2d(st + G::OFF_APD, tmap(I, M3_AP0 + pcur), x0, dn, bar);
  tma_load2d(st + G::OFF_APU, tmap(I, M3_AP0 + pcur), x0, up, bar);
}

// P_CG_F on one staged chunk of a 3-D grid (FP32): the 2-D step's arithmetic
// (sums [0] ||r_j||^2, [1] <p_j,Ap_j>, [2] <r_j,Ap_j>, [3] ||Ap_j||^2) with
// the couplings to the planes below and above, whose p_j each lane forms at
// its two points from their staged r, p, Ap.  row0: the chunk's first row in
// the row space; yc: in its plane.
__device__ __forceinline__ void cgf3_chunk(const DevInst& I, const unsigned char* st, int x0,
                                           int row0, int yc, int rows, float alpha, float beta,
                                           const unsigned* fbits, float* w, float* r_out,
                                           float* p_out, float* ap_out, FF* ff) {
  using G = GeoF3;
  const float* R = reinterpret_cast<const float*>(st + G::OFF_R);
  const float* P = reinterpret_cast<const float*>(st + G::OFF_P);
  const float* AP = reinterpret_cast<const float*>(st + G::OFF_AP);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ylim = min(rows, I.ny - yc);
  const int ry = warp;
  if (ry >= ylim) return;  // warp-uniform
  const int c = 2 * lane;
  const int e0 = x0 + c;
  const bool v0 = e0 < I.nx, v1 = e0 + 1 < I.nx;
  // rows ry-1, ry, ry+1 of the chunk (box rows ry .. ry+2)
  float pn[3][2], rn[2], po[2];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int b = (ry + q) * G::BW + G::H + c;
    const float2 rv = *reinterpret_cast<const float2*>(R + b);
    const float2 pv = *reinterpret_cast<const float2*>(P + b);
    const float2 av = *reinterpret_cast<const float2*>(AP + b);
    const float ra = fmaf(alpha, av.x, rv.x), rb = fmaf(alpha, av.y, rv.y);
    pn[q][0] = fmaf(beta, pv.x, -ra);
    pn[q][1] = fmaf(beta, pv.y, -rb);
    if (q == 1) {
      rn[0] = ra;
      rn[1] = rb;
      po[0] = pv.x;
      po[1] = pv.y;
    }
  }
  float pw = __shfl_up_sync(FULL_MASK, pn[1][1], 1);
  float pe = __shfl_down_sync(FULL_MASK, pn[1][0], 1);
  {
    const int b = (ry + 1) * G::BW + G::H + c;
    if (lane == 0) pw = fmaf(beta, P[b - 1], -fmaf(alpha, AP[b - 1], R[b - 1]));
    if (lane == 31) pe = fmaf(beta, P[b + 2], -fmaf(alpha, AP[b + 2], R[b + 2]));
  }
  // p_j of the planes below (d) and above (u) at the lane's points
  const int bi = ry * 64 + c;
  auto plane_p = [&](int o_r, int o_p, int o_a, float out[2]) {
    const float2 rv = *reinterpret_cast<const float2*>(st + o_r + 4 * bi);
    const float2 pv = *reinterpret_cast<const float2*>(st + o_p + 4 * bi);
    const float2 av = *reinterpret_cast<const float2*>(st + o_a + 4 * bi);
    out[0] = fmaf(beta, pv.x, -fmaf(alpha, av.x, rv.x));
    out[1] = fmaf(beta, pv.y, -fmaf(alpha, av.y, rv.y));
  };
  float pd[2], pu[2];
  plane_p(G::OFF_RD, G::OFF_PD, G::OFF_APD, pd);
  plane_p(G::OFF_RU, G::OFF_PU, G::OFF_APU, pu);
  const float* Dr = reinterpret_cast<const float*>(st + G::OFF_D) + bi;
  const float* Xr = reinterpret_cast<const float*>(st + G::OFF_CX) + ry * (64 + G::H) + G::H + c;
  const float* Ys = reinterpret_cast<const float*>(st + G::OFF_CY) + bi;
  const float* Yn = Ys + 64;
  const float* Zd = reinterpret_cast<const float*>(st + G::OFF_CZD) + bi;
  const float* Zu = reinterpret_cast<const float*>(st + G::OFF_CZU) + bi;
  // diag, west, east, south, north, down, up (the order of the register sweep)
  float a0 = Dr[0] * pn[1][0];
  a0 = fmaf(Xr[-1], pw, a0);
  a0 = fmaf(Xr[0], pn[1][1], a0);
  a0 = fmaf(Ys[0], pn[0][0], a0);
  a0 = fmaf(Yn[0], pn[2][0], a0);
  a0 = fmaf(Zd[0], pd[0], a0);
  a0 = fmaf(Zu[0], pu[0], a0);
  float a1 = Dr[1] * pn[1][1];
  a1 = fmaf(Xr[0], pn[1][0], a1);
  a1 = fmaf(Xr[1], pe, a1);
  a1 = fmaf(Ys[1], pn[0][1], a1);
  a1 = fmaf(Yn[1], pn[2][1], a1);
  a1 = fmaf(Zd[1], pd[1], a1);
  a1 = fmaf(Zu[1], pu[1], a1);
  const unsigned fb = fbits[0] & 3u;
  a0 = (fb & 1u) ? a0 : 0.0f;
  a1 = (fb & 2u) ? a1 : 0.0f;
  const float2 wv = *reinterpret_cast<const float2*>(st + G::OFF_W + 4 * bi);
  const long long i = (long long)(row0 + ry) * I.px + e0;
  st2(w, i, v0, v1, fmaf(alpha, po[0], wv.x), fmaf(alpha, po[1], wv.y));
  st2(r_out, i, v0, v1, rn[0], rn[1]);
  st2(p_out, i, v0, v1, pn[1][0], pn[1][1]);
  st2(ap_out, i, v0, v1, a0, a1);
  // points past nx hold zeros (the boxes are zero-filled there)
  float s_rr = rn[0] * rn[0];
  s_rr = fmaf(rn[1], rn[1], s_rr);
  float s_pap = pn[1][0] * a0;
  s_pap = fmaf(pn[1][1], a1, s_pap);
  float s_rap = rn[0] * a0;
  s_rap = fmaf(rn[1], a1, s_rap);
  float s_apap = a0 * a0;
  s_apap = fmaf(a1, a1, s_apap);
  ff_acc(ff[0], s_rr);
  ff_acc(ff[1], s_pap);
  ff_acc(ff[2], s_rap);
  ff_acc(ff[3], s_apap);
}

// P_CG_F, FP64 (one row per warp): r_j and p_j are formed once per element
// of the halo box, in place in the stage, then a block barrier; recomputing
// them per warp would triple the FP64 work, the bound of this pass.
template <bool JAC>
__device__ __forceinline__ void cgf_chunk_box(const DevInst& I, unsigned char* st, int x0, int yc,
                                              int rows, double alpha, double beta,
                                              const unsigned* fbits, double* w, double* r_out,
                                              double* p_out, double* ap_out, Acc& acc) {
  using G = GeoF<double>;
  double* R = reinterpret_cast<double*>(st + G::OFF_R);
  double* P = reinterpret_cast<double*>(st + G::OFF_P);
  const double* AP = reinterpret_cast<const double*>(st + G::OFF_AP);
  const double* W = reinterpret_cast<const double*>(st + G::OFF_W);
  const double* D = reinterpret_cast<const double*>(st + G::OFF_D);
  const double* CX = reinterpret_cast<const double*>(st + G::OFF_CX);
  const double* CY = reinterpret_cast<const double*>(st + G::OFF_CY);
  const double* DI = reinterpret_cast<const double*>(st + G::OFF_DI);
  constexpr bool jac = JAC;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ylim = min(rows, I.ny - yc);
  double s_rr = 0.0;
  for (int e = tid; e < (G::CH + 2) * G::BW; e += kThreads) {
    const int br = e / G::BW, bc = e - br * G::BW;
    const double pold = P[e];
    const double rn = fma(alpha, AP[e], R[e]);
    const double zn = jac ? rn * DI[e] : rn;  // z = M^-1 r
    const double pn = fma(beta, pold, -zn);
    R[e] = zn;  // the stage keeps z for <z, Ap>
    P[e] = pn;
    const int ry = br - 1, col = bc - G::H;
    if (ry >= 0 && ry < ylim && col >= 0 && col < 64 && x0 + col < I.nx) {
      const long long i = (long long)(yc + ry) * I.px + x0 + col;
      w[i] = fma(alpha, pold, W[ry * 64 + col]);
      r_out[i] = rn;
      p_out[i] = pn;
      s_rr = fma(rn, zn, s_rr);
    }
  }
  acc.s[0] += s_rr;
  __syncthreads();
  static_assert(G::CH == kWarps, "one row per warp");
  const int ry = warp;
  const int c = 2 * lane;
  const int e0 = x0 + c;
  const bool v0 = e0 < I.nx, v1 = e0 + 1 < I.nx;
  if (ry >= ylim || !v0) return;
  const double* Pr = P + (ry + 1) * G::BW + G::H + c;
  const double* Rr = R + (ry + 1) * G::BW + G::H + c;
  const double vc0 = Pr[0], vc1 = Pr[1];
  const double* Dr = D + ry * 64 + c;
  const double* Xr = CX + ry * (64 + G::H) + G::H + c;
  const double* Ys = CY + ry * 64 + c;
  const double* Yn = CY + (ry + 1) * 64 + c;
  double a0 = Dr[0] * vc0;
  a0 = fma(Xr[-1], Pr[-1], a0);
  a0 = fma(Xr[0], vc1, a0);
  a0 = fma(Ys[0], Pr[-G::BW], a0);
  a0 = fma(Yn[0], Pr[G::BW], a0);
  double a1 = Dr[1] * vc1;
  a1 = fma(Xr[0], vc0, a1);
  a1 = fma(Xr[1], Pr[2], a1);
  a1 = fma(Ys[1], Pr[1 - G::BW], a1);
  a1 = fma(Yn[1], Pr[G::BW + 1], a1);
  const unsigned fb = fbits[0] & 3u;
  a0 = (fb & 1u) ? a0 : 0.0;
  a1 = (fb & 2u) ? a1 : 0.0;
  st2(ap_out, (long long)(yc + ry) * I.px + e0, v0, v1, a0, a1);
  const double z0 = Rr[0], z1 = Rr[1];
  const double* Dr2 = DI + (ry + 1) * G::BW + G::H + c;
  const double da0 = jac ? a0 * Dr2[0] : a0, da1 = jac ? a1 * Dr2[1] : a1;
  acc.s[1] = fma(vc0, a0, fma(vc1, a1, acc.s[1]));
  acc.s[2] = fma(z0, a0, fma(z1, a1, acc.s[2]));
  acc.s[3] = fma(a0, da0, fma(a1, da1, acc.s[3]));
}

template <class T>
struct V2;
template <>
struct V2<float> {
  using type = float2;
};
template <>
struct V2<double> {
  using type = double2;
};


// P_CG_F on one staged chunk (rows yc .. yc+rows-1).  Sums: [0] ||r_j||^2,
// [1] <p_j,Ap_j>, [2] <r_j,Ap_j>, [3] ||Ap_j||^2.  Each warp forms r_j and p_j
// for its rows and the rows above and below from the staged r, p, Ap (west
// and east neighbours by shuffles), so no block barrier is needed.  For
// T = float a thread sums its few terms of the chunk in FP32 and adds that to
// its float-float accumulator once per chunk.
template <class T, bool JAC>
__device__ __forceinline__ void cgf_chunk(const DevInst& I, const unsigned char* st, int x0,
                                          int yc, int rows, T alpha, T beta, const unsigned* fbits,
                                          T* w, T* r_out, T* p_out, T* ap_out, Acc& acc, FF* ff) {
  using G = GeoF<T>;
  using T2 = typename V2<T>::type;
  constexpr int RPW = G::CH / kWarps;
  const T* R = reinterpret_cast<const T*>(st + G::OFF_R);
  const T* P = reinterpret_cast<const T*>(st + G::OFF_P);
  const T* AP = reinterpret_cast<const T*>(st + G::OFF_AP);
  const T* W = reinterpret_cast<const T*>(st + G::OFF_W);
  const T* D = reinterpret_cast<const T*>(st + G::OFF_D);
  const T* CX = reinterpret_cast<const T*>(st + G::OFF_CX);
  const T* CY = reinterpret_cast<const T*>(st + G::OFF_CY);
  const T* DI = reinterpret_cast<const T*>(st + G::OFF_DI);  // 1/diag (point Jacobi)
  constexpr bool jac = JAC;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ylim = min(rows, I.ny - yc);
  const int r0 = warp * RPW;  // first chunk row of this warp
  if (r0 >= ylim) return;     // warp-uniform
  const int c = 2 * lane;
  const int e0 = x0 + c;
  const bool v0 = e0 < I.nx, v1 = e0 + 1 < I.nx;
  // window q = 0 .. RPW+1 is chunk row r0-1+q (box row r0+q); z = M^-1 r
  T pn[RPW + 2][2], rn[RPW][2], po[RPW][2], pw[RPW], pe[RPW];
#pragma unroll
  for (int q = 0; q < RPW + 2; ++q) {
    const int b = (r0 + q) * G::BW + G::H + c;
    const T2 rv = *reinterpret_cast<const T2*>(R + b);
    const T2 pv = *reinterpret_cast<const T2*>(P + b);
    const T2 av = *reinterpret_cast<const T2*>(AP + b);
    T2 dv;
    dv.x = T(1);
    dv.y = T(1);
    if (jac) dv = *reinterpret_cast<const T2*>(DI + b);
    const T ra = fma(alpha, av.x, rv.x), rb = fma(alpha, av.y, rv.y);
    const T za = ra * dv.x, zb = rb * dv.y;
    pn[q][0] = fma(beta, pv.x, -za);
    pn[q][1] = fma(beta, pv.y, -zb);
    if (q >= 1 && q <= RPW) {
      rn[q - 1][0] = ra;
      rn[q - 1][1] = rb;
      po[q - 1][0] = pv.x;
      po[q - 1][1] = pv.y;
    }
  }
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    pw[k] = __shfl_up_sync(FULL_MASK, pn[k + 1][1], 1);
    pe[k] = __shfl_down_sync(FULL_MASK, pn[k + 1][0], 1);
    const int b = (r0 + k + 1) * G::BW + G::H + c;
    if (lane == 0)
      pw[k] = fma(beta, P[b - 1], -fma(alpha, AP[b - 1], R[b - 1]) * (jac ? DI[b - 1] : T(1)));
    if (lane == 31)
      pe[k] = fma(beta, P[b + 2], -fma(alpha, AP[b + 2], R[b + 2]) * (jac ? DI[b + 2] : T(1)));
  }
  T s_rr = T(0), s_pap = T(0), s_rap = T(0), s_apap = T(0);
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    const int ry = r0 + k;
    if (ry >= ylim) break;
    const int q = k + 1;
    const T* Dr = D + ry * 64 + c;
    const T* Xr = CX + ry * (64 + G::H) + G::H + c;
    const T* Ys = CY + ry * 64 + c;
    const T* Yn = CY + (ry + 1) * 64 + c;
    // diag, west, east, south, north (the order of the register sweep)
    T a0 = Dr[0] * pn[q][0];
    a0 = fma(Xr[-1], pw[k], a0);
    a0 = fma(Xr[0], pn[q][1], a0);
    a0 = fma(Ys[0], pn[q - 1][0], a0);
    a0 = fma(Yn[0], pn[q + 1][0], a0);
    T a1 = Dr[1] * pn[q][1];
    a1 = fma(Xr[0], pn[q][0], a1);
    a1 = fma(Xr[1], pe[k], a1);
    a1 = fma(Ys[1], pn[q - 1][1], a1);
    a1 = fma(Yn[1], pn[q + 1][1], a1);
    const unsigned fb = fbits[k] & 3u;
    a0 = (fb & 1u) ? a0 : T(0);
    a1 = (fb & 2u) ? a1 : T(0);
    const T2 wv = *reinterpret_cast<const T2*>(W + ry * 64 + c);
    const long long i = (long long)(yc + ry) * I.px + e0;
    st2(w, i, v0, v1, fma(alpha, po[k][0], wv.x), fma(alpha, po[k][1], wv.y));
    st2(r_out, i, v0, v1, rn[k][0], rn[k][1]);
    st2(p_out, i, v0, v1, pn[q][0], pn[q][1]);
    st2(ap_out, i, v0, v1, a0, a1);
    // points past nx hold zeros (the boxes are zero-filled there)
    T d0 = T(1), d1 = T(1);
    if (jac) {
      const T2 dv = *reinterpret_cast<const T2*>(DI + (ry + 1) * G::BW + G::H + c);
      d0 = dv.x;
      d1 = dv.y;
    }
    const T z0 = rn[k][0] * d0, z1 = rn[k][1] * d1;
    s_rr = fma(rn[k][0], z0, s_rr);
    s_rr = fma(rn[k][1], z1, s_rr);
    s_pap = fma(pn[q][0], a0, s_pap);
    s_pap = fma(pn[q][1], a1, s_pap);
    s_rap = fma(z0, a0, s_rap);
    s_rap = fma(z1, a1, s_rap);
    s_apap = fma(a0, a0 * d0, s_apap);
    s_apap = fma(a1, a1 * d1, s_apap);
  }
  if (sizeof(T) == 4) {
    ff_acc(ff[0], (float)s_rr);
    ff_acc(ff[1], (float)s_pap);
    ff_acc(ff[2], (float)s_rap);
    ff_acc(ff[3], (float)s_apap);
  } else {
    acc.s[0] += (double)s_rr;
    acc.s[1] += (double)s_pap;
    acc.s[2] += (double)s_rap;
    acc.s[3] += (double)s_apap;
  }
}

// P_CG_F under the tile preconditioner (2-D): the same CG step with
// z = M^-1 r carried by its own recurrence, so that M^-1 is applied once per
// step, to Ap, inside the chunk:
//   r_j = r_{j-1} + alpha Ap_{j-1},  z_j = z_{j-1} + alpha q_{j-1}  (q = M^-1 Ap),
//   w_j = w_{j-1} + alpha p_{j-1},  p_j = -z_j + beta p_{j-1},
//   Ap_j = Z Z' A Z Z' p_j,  q_j = M^-1 Ap_j  (the zebra sweep over the chunk's
//   8-row tiles), sums <r_j,z_j>, <p_j,Ap_j>, <z_j,Ap_j>, <Ap_j,q_j>.
// The first step of a phase runs with alpha = beta = 0 on the vectors P_CG_Z
// left.  z, q, p, r, Ap are read from buffer pcur and written to pcur^1.
// Stage layout (T = float: f = 16 rows, h = 4; double: f = 8, h = 2): ZH | QH
// | PH | RH | APH, each (64+2h) x (f+2) from (x0-h, y-1) | W 64 x f | D 64 x f |
// CX (64+h) x f from x0-h | CY 64 x (f+1) from y-1.  Once a warp has read its
// rows of W, those rows of the W box become its rows of the sweep's exchange
// buffer (no other warp reads them).
template <class T>
struct GeoT {
  static constexpr int H = 16 / (int)sizeof(T);
  static constexpr int CH = GeoF<T>::CH;
  static constexpr int BW = 64 + 2 * H;
  static constexpr int SZ_H = align128((CH + 2) * BW * (int)sizeof(T));
  static constexpr int SZ_I = 64 * CH * (int)sizeof(T);
  static constexpr int OFF_Z = 0, OFF_Q = SZ_H, OFF_P = 2 * SZ_H, OFF_R = 3 * SZ_H;
  static constexpr int OFF_AP = 4 * SZ_H, OFF_W = 5 * SZ_H;
  static constexpr int OFF_D = OFF_W + SZ_I, OFF_CX = OFF_D + SZ_I;
  static constexpr int OFF_CY = OFF_CX + align128((64 + H) * CH * (int)sizeof(T));
  static constexpr int END = OFF_CY + align128(64 * (CH + 1) * (int)sizeof(T));
  static constexpr unsigned TX =
      (5 * (CH + 2) * BW + 2 * 64 * CH + (64 + H) * CH + 64 * (CH + 1)) * sizeof(T);
  static constexpr int PITCH = 64 * (int)sizeof(T) / 4;  // exchange row pitch (floats)
  static constexpr int MB = sizeof(T) == 4 ? M32_RH0 : M64_RH0;
};
static_assert(GeoT<float>::END <= kOffMask && GeoT<double>::END <= kOffMask, "stage layout");
static_assert(GeoT<float>::CH % kBlkY == 0 && GeoT<double>::CH % kBlkY == 0 &&
                  kTX == kBlkX && kTY % kBlkY == 0,
              "chunks and tiles hold whole preconditioner blocks");

template <class T>
__device__ __forceinline__ void issue_cgt(const DevInst& I, int pcur, int x0, int yc,
                                          unsigned st, unsigned bar) {
  using G = GeoT<T>;
  constexpr int o = G::MB - M32_RH0;
  mbar_expect(bar, G::TX);
  tma_load2d(st + G::OFF_Z, tmap(I, o + M32_FZH0 + pcur), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_Q, tmap(I, o + M32_FQH0 + pcur), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_P, tmap(I, o + M32_FPH0 + pcur), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_R, tmap(I, o + M32_FRH0 + pcur), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_AP, tmap(I, o + M32_FAPH0 + pcur), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_W, tmap(I, o + M32_FW), x0, yc, bar);
  tma_load2d(st + G::OFF_D, tmap(I, o + M32_FD), x0, yc, bar);
  tma_load2d(st + G::OFF_CX, tmap(I, o + M32_FCX), x0 - G::H, yc, bar);
  tma_load2d(st + G::OFF_CY, tmap(I, o + M32_FCY), x0, yc - 1, bar);
}

// The free bits of this lane's two columns in chunk row `row` of the staged
// mask box (0 outside the box's rows).
__device__ __forceinline__ unsigned stage_row_bits(const unsigned char* st, int x0, int row) {
  if (row < 0 || row >= 32) return 0u;
  const unsigned* M = reinterpret_cast<const unsigned*>(st + kOffMask);
  const int lane = threadIdx.x & 31;
  return (M[row * 4 + ((x0 >> 5) & 3) + (lane >> 4)] >> ((2 * lane) & 31)) & 3u;
}

template <class T>
__device__ __forceinline__ void cgt_chunk(const DevInst& I, unsigned char* st, int x0, int yc,
                                          int rows, T alpha, T beta, const unsigned* fbits,
                                          T* w, T* r_out, T* z_out, T* p_out, T* ap_out,
                                          T* q_out, Acc& acc, FF* ff) {
  using G = GeoT<T>;
  using T2 = typename V2<T>::type;
  constexpr int RPW = G::CH / kWarps;
  const T* Z = reinterpret_cast<const T*>(st + G::OFF_Z);
  const T* Q = reinterpret_cast<const T*>(st + G::OFF_Q);
  const T* P = reinterpret_cast<const T*>(st + G::OFF_P);
  const T* R = reinterpret_cast<const T*>(st + G::OFF_R);
  const T* AP = reinterpret_cast<const T*>(st + G::OFF_AP);
  const T* W = reinterpret_cast<const T*>(st + G::OFF_W);
  const T* D = reinterpret_cast<const T*>(st + G::OFF_D);
  const T* CX = reinterpret_cast<const T*>(st + G::OFF_CX);
  const T* CY = reinterpret_cast<const T*>(st + G::OFF_CY);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ylim = min(rows, I.ny - yc);
  const int r0 = warp * RPW;  // first chunk row of this warp
  const int c = 2 * lane;
  const int e0 = x0 + c;
  const bool v0 = e0 < I.nx, v1 = e0 + 1 < I.nx;
  // window q = 0 .. RPW+1 is chunk row r0-1+q (box row r0+q): z_j, p_j there
  T pn[RPW + 2][2], zn[RPW][2], rn[RPW][2], pw[RPW], pe[RPW];
#pragma unroll
  for (int q = 0; q < RPW + 2; ++q) {
    const int b = (r0 + q) * G::BW + G::H + c;
    const T2 zv = *reinterpret_cast<const T2*>(Z + b);
    const T2 qv = *reinterpret_cast<const T2*>(Q + b);
    const T2 pv = *reinterpret_cast<const T2*>(P + b);
    const T za = fma(alpha, qv.x, zv.x), zb = fma(alpha, qv.y, zv.y);
    pn[q][0] = fma(beta, pv.x, -za);
    pn[q][1] = fma(beta, pv.y, -zb);
    if (q >= 1 && q <= RPW) {
      const int k = q - 1, ry = r0 + k;
      zn[k][0] = za;
      zn[k][1] = zb;
      const T2 rv = *reinterpret_cast<const T2*>(R + b);
      const T2 av = *reinterpret_cast<const T2*>(AP + b);
      rn[k][0] = fma(alpha, av.x, rv.x);
      rn[k][1] = fma(alpha, av.y, rv.y);
      const T2 wv = *reinterpret_cast<const T2*>(W + ry * 64 + c);
      if (ry < ylim)
        st2(w, (long long)(yc + ry) * I.px + e0, v0, v1, fma(alpha, pv.x, wv.x),
            fma(alpha, pv.y, wv.y));
    }
  }
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    pw[k] = __shfl_up_sync(FULL_MASK, pn[k + 1][1], 1);
    pe[k] = __shfl_down_sync(FULL_MASK, pn[k + 1][0], 1);
    const int b = (r0 + k + 1) * G::BW + G::H + c;
    if (lane == 0) pw[k] = fma(beta, P[b - 1], -fma(alpha, Q[b - 1], Z[b - 1]));
    if (lane == 31) pe[k] = fma(beta, P[b + 2], -fma(alpha, Q[b + 2], Z[b + 2]));
  }
  TileLine L[RPW];
  float d[RPW][2], x[RPW][2];
  T ap[RPW][2];
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    const int ry = r0 + k;
    const int q = k + 1;
    const T* Dr = D + ry * 64 + c;
    const T* Xr = CX + ry * (64 + G::H) + G::H + c;
    const T* Ys = CY + ry * 64 + c;
    const T* Yn = CY + (ry + 1) * 64 + c;
    // diag, west, east, south, north (the order of the register sweep)
    T a0 = Dr[0] * pn[q][0];
    a0 = fma(Xr[-1], pw[k], a0);
    a0 = fma(Xr[0], pn[q][1], a0);
    a0 = fma(Ys[0], pn[q - 1][0], a0);
    a0 = fma(Yn[0], pn[q + 1][0], a0);
    T a1 = Dr[1] * pn[q][1];
    a1 = fma(Xr[0], pn[q][0], a1);
    a1 = fma(Xr[1], pe[k], a1);
    a1 = fma(Ys[1], pn[q - 1][1], a1);
    a1 = fma(Yn[1], pn[q + 1][1], a1);
    // rows past the grid arrive as zeros in the mask box: no free point
    const unsigned fb = fbits[k] & 3u;
    a0 = (fb & 1u) ? a0 : T(0);
    a1 = (fb & 2u) ? a1 : T(0);
    ap[k][0] = a0;
    ap[k][1] = a1;
    const float xw = __shfl_up_sync(FULL_MASK, (float)Xr[1], 1);
    L[k] = tile_line(ry, (float)Dr[0], (float)Dr[1], xw, (float)Xr[0], (float)Ys[0],
                     (float)Ys[1], (float)Yn[0], (float)Yn[1], fb,
                     stage_row_bits(st, x0, ry - 1), stage_row_bits(st, x0, ry + 1));
    d[k][0] = (float)a0;
    d[k][1] = (float)a1;
  }
  // every warp has read its rows of W (above): they now carry the sweep
  zebra_sweep<RPW>(L, d, r0, reinterpret_cast<float*>(st + G::OFF_W), G::PITCH, x);
  T s_rz = T(0), s_pap = T(0), s_zap = T(0), s_aq = T(0);
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    const int ry = r0 + k;
    if (ry >= ylim) break;
    const int q = k + 1;
    const T q0 = (T)x[k][0], q1 = (T)x[k][1];
    const long long i = (long long)(yc + ry) * I.px + e0;
    st2(r_out, i, v0, v1, rn[k][0], rn[k][1]);
    st2(z_out, i, v0, v1, zn[k][0], zn[k][1]);
    st2(p_out, i, v0, v1, pn[q][0], pn[q][1]);
    st2(ap_out, i, v0, v1, ap[k][0], ap[k][1]);
    st2(q_out, i, v0, v1, q0, q1);
    // points past nx hold zeros (the boxes are zero-filled there)
    s_rz = fma(rn[k][0], zn[k][0], s_rz);
    s_rz = fma(rn[k][1], zn[k][1], s_rz);
    s_pap = fma(pn[q][0], ap[k][0], s_pap);
    s_pap = fma(pn[q][1], ap[k][1], s_pap);
    s_zap = fma(zn[k][0], ap[k][0], s_zap);
    s_zap = fma(zn[k][1], ap[k][1], s_zap);
    s_aq = fma(ap[k][0], q0, s_aq);
    s_aq = fma(ap[k][1], q1, s_aq);
  }
  if (sizeof(T) == 4) {
    ff_acc(ff[0], (float)s_rz);
    ff_acc(ff[1], (float)s_pap);
    ff_acc(ff[2], (float)s_zap);
    ff_acc(ff[3], (float)s_aq);
  } else {
    acc.s[0] += (double)s_rz;
    acc.s[1] += (double)s_pap;
    acc.s[2] += (double)s_zap;
    acc.s[3] += (double)s_aq;
  }
}

// ------------------------------------ TMA-staged mixed-phase GP passes --
//
// In the mixed phase the iterate is x32, kept on the FP32 box [l32, u32]: a
// point is active when x32 equals l32 or u32 (bit for bit; the FP32
// projection returns the bound itself), and the first FP64 census after the
// phase rebuilds the FP64 iterate from it (see OpCensus).  The census and the
// trial of a 2-D instance stream 16-row chunks (two rows per warp).  Stage
// layout (boxes 128-byte aligned):
//   XH | LH | UH | DH | GH : FP32 72 x 18 from (x0-4, y-1): x32, l32, u32,
//                            the direction (g32 or w32), g32 (trial along w)
//   B : 64 x 16 (b32)   D : 64 x 16   CX : 68 x 16 from x0-4   CY : 64 x 17 from y-1
// The census loads XH, l32 and u32 as 64 x 16 boxes in the LH and UH slots,
// B and the bands.  The alpha0 pass streams 32-row chunks of pg32 through the
// R slot of the FP32 CG_B layout, with its D, CX and CY boxes.
struct GeoGP {
  static constexpr int CH = 16, H = 4, BW = 64 + 2 * H;
  static constexpr int RPW = CH / kWarps;
  static constexpr int SZ_H = align128((CH + 2) * BW * 4);
  static constexpr int SZ_32 = 64 * CH * 4;
  static constexpr int OFF_XH = 0, OFF_LH = SZ_H, OFF_UH = 2 * SZ_H, OFF_DH = 3 * SZ_H;
  static constexpr int OFF_GH = 4 * SZ_H;
  static constexpr int OFF_B = 5 * SZ_H, OFF_D = OFF_B + SZ_32;
  static constexpr int OFF_CX = OFF_D + SZ_32;
  static constexpr int OFF_CY = OFF_CX + align128((64 + H) * CH * 4);
  static constexpr int END = OFF_CY + align128(64 * (CH + 1) * 4);
  static constexpr unsigned TX_H = (CH + 2) * BW * 4;  // one halo box
  static constexpr unsigned TX_BANDS = SZ_32 + SZ_32 + (64 + H) * CH * 4 + 64 * (CH + 1) * 4;
};
static_assert(GeoGP::END <= kOffMask, "stage layout");
static_assert(GeoGP::CH == GeoF<float>::CH, "the GP passes use the fused pass's band maps");

// The trial along -g of the mixed phase also forms the next GP step's alpha0
// (Eq. bqpls) at the trial point, <pg, A32 pg> with pg its projected
// gradient, which needs pg one point around the chunk and so xt two: its
// stage (boxes 128-byte aligned) holds
//   X | L | U | G : FP32 72 x 20 from (x0-4, y-2): x32, l32, u32, g32
//   B | D | CX : 72 x 18 from (x0-4, y-1)    CY : 72 x 19 from (x0-4, y-2).
// The G box receives xt once the direction is used, the B box pg once b is.
struct GeoGA {
  static constexpr int CH = GeoGP::CH, H = 4, BW = 64 + 2 * H;
  static constexpr int RH = CH + 4, RB = CH + 2, RY = CH + 3;
  static constexpr int SZ_H = align128(RH * BW * 4), SZ_B = align128(RB * BW * 4);
  static constexpr int OFF_X = 0, OFF_L = SZ_H, OFF_U = 2 * SZ_H, OFF_G = 3 * SZ_H;
  static constexpr int OFF_B = 4 * SZ_H, OFF_D = OFF_B + SZ_B, OFF_CX = OFF_D + SZ_B;
  static constexpr int OFF_CY = OFF_CX + SZ_B;
  static constexpr int END = OFF_CY + align128(RY * BW * 4);
  static constexpr unsigned TX = (4 * RH * BW + 3 * RB * BW + RY * BW) * 4;
};
static_assert(GeoGA::END <= kOffMask, "stage layout");

// Whether the pass is the staged trial along -g that forms alpha0 (a trial
// along w, the projected search, streams the GeoGP layout).
__device__ __forceinline__ bool trial_alpha0(const Snap& S) {
  return S.pass == P_TRIAL && S.dir != D_W32;
}

// Whether the item's pass is a mixed-phase GP pass on the TMA path.
__device__ __forceinline__ bool gp_tma(const DevInst& I, const Snap& S) {
  return S.gp32 && I.dim == 2 && I.tma_gp && I.tma32 && I.tma_mask &&
         (S.pass == P_CENSUS || S.pass == P_GP_ALPHA || S.pass == P_TRIAL);
}

// Issue the chunk at rows yc.. of a mixed-phase GP pass.
__device__ __forceinline__ void issue_gp(const DevInst& I, const Snap& S, int x0, int yc,
                                         unsigned st, unsigned bar) {
  using G = GeoGP;
  const int cur = S.cur;
  if (S.pass == P_GP_ALPHA) {
    using F = ChunkGeo<float>;
    mbar_expect(bar, ((F::CH + 2) * F::BW + 64 * F::CH + (64 + F::H) * F::CH +
                      64 * (F::CH + 1)) * 4);
    tma_load2d(st + F::OFF_R, tmap(I, MG_PGH0 + cur), x0 - F::H, yc - 1, bar);
    tma_load2d(st + F::OFF_D, tmap(I, M32_D), x0, yc, bar);
    tma_load2d(st + F::OFF_CX, tmap(I, M32_CX), x0 - F::H, yc, bar);
    tma_load2d(st + F::OFF_CY, tmap(I, M32_CY), x0, yc - 1, bar);
    return;
  }
  if (trial_alpha0(S)) {
    using A = GeoGA;
    mbar_expect(bar, A::TX);
    tma_load2d(st + A::OFF_X, tmap(I, MG_X2H0 + cur), x0 - A::H, yc - 2, bar);
    tma_load2d(st + A::OFF_L, tmap(I, MG_L2H), x0 - A::H, yc - 2, bar);
    tma_load2d(st + A::OFF_U, tmap(I, MG_U2H), x0 - A::H, yc - 2, bar);
    tma_load2d(st + A::OFF_G, tmap(I, MG_G2H0 + cur), x0 - A::H, yc - 2, bar);
    tma_load2d(st + A::OFF_B, tmap(I, MG_B18), x0 - A::H, yc - 1, bar);
    tma_load2d(st + A::OFF_D, tmap(I, MG_D18), x0 - A::H, yc - 1, bar);
    tma_load2d(st + A::OFF_CX, tmap(I, MG_CX18), x0 - A::H, yc - 1, bar);
    tma_load2d(st + A::OFF_CY, tmap(I, MG_CY19), x0 - A::H, yc - 2, bar);
    return;
  }
  const bool along_w = S.pass == P_TRIAL && S.dir == D_W32;
  mbar_expect(bar, S.pass == P_TRIAL ? (along_w ? 5u : 4u) * G::TX_H + G::TX_BANDS
                                     : G::TX_H + 2 * G::SZ_32 + G::TX_BANDS);
  tma_load2d(st + G::OFF_XH, tmap(I, MG_X32H0 + cur), x0 - G::H, yc - 1, bar);
  if (S.pass == P_TRIAL) {
    tma_load2d(st + G::OFF_LH, tmap(I, MG_L32H), x0 - G::H, yc - 1, bar);
    tma_load2d(st + G::OFF_UH, tmap(I, MG_U32H), x0 - G::H, yc - 1, bar);
    tma_load2d(st + G::OFF_DH, tmap(I, along_w ? MG_W32H : MG_G32H0 + cur), x0 - G::H, yc - 1,
               bar);
    if (along_w) tma_load2d(st + G::OFF_GH, tmap(I, MG_G32H0 + cur), x0 - G::H, yc - 1, bar);
  } else {
    tma_load2d(st + G::OFF_LH, tmap(I, MG_L32), x0, yc, bar);
    tma_load2d(st + G::OFF_UH, tmap(I, MG_U32), x0, yc, bar);
  }
  tma_load2d(st + G::OFF_B, tmap(I, MG_B32), x0, yc, bar);
  tma_load2d(st + G::OFF_D, tmap(I, M32_FD), x0, yc, bar);
  tma_load2d(st + G::OFF_CX, tmap(I, M32_FCX), x0 - G::H, yc, bar);
  tma_load2d(st + G::OFF_CY, tmap(I, M32_FCY), x0, yc - 1, bar);
}

// In the staged GP passes lane `lane` of a warp owns columns lane and lane+32
// of each of its rows, so that shared-memory reads are unit-stride and a
// warp ballot is one word of the free-set bitmask.

// P_CENSUS (mixed) on one staged 16-row chunk: g32 = A32 x32 + b32, pg32,
// the free set and |A|, |B|, ||pg||^2 (as OpCensus32).  Points past nx
// arrive as zeros and contribute nothing.
__device__ __forceinline__ void census32_chunk(const DevInst& I, const unsigned char* st, int x0,
                                               int yc, int rows, float* g_out, float* pg_out,
                                               unsigned* m_out, Acc& acc, FF& ff) {
  using G = GeoGP;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float* XH = reinterpret_cast<const float*>(st + G::OFF_XH);
  const float* L = reinterpret_cast<const float*>(st + G::OFF_LH);  // 64 x 16
  const float* U = reinterpret_cast<const float*>(st + G::OFF_UH);
  const float* B = reinterpret_cast<const float*>(st + G::OFF_B);
  const float* D = reinterpret_cast<const float*>(st + G::OFF_D);
  const float* CX = reinterpret_cast<const float*>(st + G::OFF_CX);
  const float* CY = reinterpret_cast<const float*>(st + G::OFF_CY);
  float s_pg = 0.0f;
#pragma unroll
  for (int k = 0; k < G::RPW; ++k) {
    const int r = warp * G::RPW + k;
    const int y = yc + r;
    if (r >= rows || y >= I.ny) break;  // warp-uniform
    const long long row = (long long)y * I.px + x0;
    bool fr[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = lane + 32 * h;
      const bool ok = x0 + j < I.nx;
      const float* V = XH + (r + 1) * G::BW + G::H + j;
      const float* cx = CX + r * (64 + G::H) + G::H + j;
      // diag, west, east, south, north (the order of the register sweep)
      float a = D[r * 64 + j] * V[0];
      a = fmaf(cx[-1], V[-1], a);
      a = fmaf(cx[0], V[1], a);
      a = fmaf(CY[r * 64 + j], V[-G::BW], a);
      a = fmaf(CY[(r + 1) * 64 + j], V[G::BW], a);
      const float g = a + B[r * 64 + j];
      const bool al = V[0] == L[r * 64 + j], au = V[0] == U[r * 64 + j];
      const bool act = al || au;
      fr[h] = ok && !act;
      const float pg = pg_compf(al, au, g);
      s_pg = fmaf(pg, pg, s_pg);
      acc.c[0] += ok && act;
      acc.c[1] += ok && ((al && g >= 0.0f) || (au && g <= 0.0f));
      if (ok) {
        g_out[row + j] = g;
        pg_out[row + j] = pg;
      }
    }
    const unsigned w0 = __ballot_sync(FULL_MASK, fr[0]);
    const unsigned w1 = __ballot_sync(FULL_MASK, fr[1]);
    const int wc = (x0 >> 5) + lane;
    if (lane < 2 && wc < I.mw) m_out[(long long)y * I.mw + wc] = lane ? w1 : w0;
  }
  ff_acc(ff, s_pg);
}

// P_GP_ALPHA (mixed) on one staged chunk of up to 32 rows: <pg,pg>,
// <pg, A32 pg> over its first `rows` rows.
__device__ __forceinline__ void alpha32_chunk(const DevInst& I, const unsigned char* st, int yc,
                                              int rows, FF* ff) {
  using F = ChunkGeo<float>;
  constexpr int RPW = F::CH / kWarps;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float* PH = reinterpret_cast<const float*>(st + F::OFF_R);
  const float* D = reinterpret_cast<const float*>(st + F::OFF_D);
  const float* CX = reinterpret_cast<const float*>(st + F::OFF_CX);
  const float* CY = reinterpret_cast<const float*>(st + F::OFF_CY);
  float s_gg = 0.0f, s_gag = 0.0f;  // this chunk's terms, added once to ff
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    const int r = warp * RPW + k;
    if (r >= rows || yc + r >= I.ny) break;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = lane + 32 * h;
      const float* V = PH + (r + 1) * F::BW + F::H + j;
      const float* cx = CX + r * (64 + F::H) + F::H + j;
      float a = D[r * 64 + j] * V[0];
      a = fmaf(cx[-1], V[-1], a);
      a = fmaf(cx[0], V[1], a);
      a = fmaf(CY[r * 64 + j], V[-F::BW], a);
      a = fmaf(CY[(r + 1) * 64 + j], V[F::BW], a);
      s_gg = fmaf(V[0], V[0], s_gg);
      s_gag = fmaf(V[0], a, s_gag);
    }
  }
  ff_acc(ff[0], s_gg);
  ff_acc(ff[1], s_gag);
}

// P_TRIAL (mixed) on one staged 16-row chunk (as OpTrial32): each warp forms
// xt32 = P[x32 + alpha d] on the FP32 box for its rows and the rows above and
// below (west and east neighbours by shuffles), then g32t = A32 xt32 + b32,
// the status of xt32, pg32 and the sums <g,s>, <s,gt>, ||pg||^2 with
// s = xt32 - x32.  `fbits` holds the lane's bits of the current free set.
template <int DK>
__device__ __forceinline__ void trial32_chunk(const DevInst& I, const unsigned char* st, int x0,
                                              int yc, int rows, float alpha,
                                              const unsigned* fbits,
                                              float* xt_out, float* gt_out, float* pg_out,
                                              unsigned* m_out, Acc& acc, FF* ff) {
  using G = GeoGP;
  constexpr int RPW = G::RPW;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = warp * RPW;
  if (r0 >= rows || yc + r0 >= I.ny) return;  // warp-uniform
  const float* XH = reinterpret_cast<const float*>(st + G::OFF_XH);
  const float* LH = reinterpret_cast<const float*>(st + G::OFF_LH);
  const float* UH = reinterpret_cast<const float*>(st + G::OFF_UH);
  const float* DH = reinterpret_cast<const float*>(st + G::OFF_DH);
  const float* GH = reinterpret_cast<const float*>(st + (DK == D_W32 ? G::OFF_GH : G::OFF_DH));
  const float* B = reinterpret_cast<const float*>(st + G::OFF_B);
  const float* D = reinterpret_cast<const float*>(st + G::OFF_D);
  const float* CX = reinterpret_cast<const float*>(st + G::OFF_CX);
  const float* CY = reinterpret_cast<const float*>(st + G::OFF_CY);
  auto opnd = [&](int e) {
    const float d = DK == D_NEG_G ? -DH[e] : DH[e];
    return mid3f(LH[e], UH[e], fmaf(alpha, d, XH[e]));
  };
  // window q = 0 .. RPW+1 is chunk row r0-1+q (box row r0+q)
  float v[RPW + 2][2];
#pragma unroll
  for (int q = 0; q < RPW + 2; ++q) {
    const int b = (r0 + q) * G::BW + G::H + lane;
    v[q][0] = opnd(b);
    v[q][1] = opnd(b + 32);
  }
  float s_gs = 0.0f, s_sgt = 0.0f, s_pg = 0.0f;  // this chunk's terms, added once to ff
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    const int r = r0 + k;
    const int y = yc + r;
    if (r >= rows || y >= I.ny) break;  // warp-uniform: a chunk may hold 8 of the box's rows
    const int q = k + 1;
    const int b = (r + 1) * G::BW + G::H + lane;  // box index of column `lane` of row r
    // west and east neighbours across the 64 columns
    float vw[2], ve[2];
    vw[0] = __shfl_up_sync(FULL_MASK, v[q][0], 1);
    vw[1] = __shfl_up_sync(FULL_MASK, v[q][1], 1);
    ve[0] = __shfl_down_sync(FULL_MASK, v[q][0], 1);
    ve[1] = __shfl_down_sync(FULL_MASK, v[q][1], 1);
    const float col31 = __shfl_sync(FULL_MASK, v[q][0], 31);
    const float col32 = __shfl_sync(FULL_MASK, v[q][1], 0);
    if (lane == 0) {
      vw[0] = opnd(b - 1);
      vw[1] = col31;
    }
    if (lane == 31) {
      ve[0] = col32;
      ve[1] = opnd(b + 33);
    }
    const long long row = (long long)y * I.px + x0;
    bool fr[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = lane + 32 * h;
      const int e = b + 32 * h;
      const bool ok = x0 + j < I.nx;
      const float* cx = CX + r * (64 + G::H) + G::H + j;
      float a = D[r * 64 + j] * v[q][h];
      a = fmaf(cx[-1], vw[h], a);
      a = fmaf(cx[0], ve[h], a);
      a = fmaf(CY[r * 64 + j], v[q - 1][h], a);
      a = fmaf(CY[(r + 1) * 64 + j], v[q + 1][h], a);
      const float gt = a + B[r * 64 + j];
      const float xt = v[q][h];
      const float sk = xt - XH[e];
      const float g = GH[e];
      const bool al = xt == LH[e], au = xt == UH[e];
      const bool act = al || au;
      fr[h] = ok && !act;
      const float pg = pg_compf(al, au, gt);
      s_gs = fmaf(g, sk, s_gs);
      s_sgt = fmaf(sk, gt, s_sgt);
      s_pg = fmaf(pg, pg, s_pg);
      acc.c[0] += ok && act;
      acc.c[1] += ok && ((al && gt >= 0.0f) || (au && gt <= 0.0f));
      acc.c[2] += ok && (((fbits[k] >> h) & 1u) != (fr[h] ? 1u : 0u));
      if (ok) {
        xt_out[row + j] = xt;
        gt_out[row + j] = gt;
        pg_out[row + j] = pg;
      }
    }
    const unsigned w0 = __ballot_sync(FULL_MASK, fr[0]);
    const unsigned w1 = __ballot_sync(FULL_MASK, fr[1]);
    const int wc = (x0 >> 5) + lane;
    if (lane < 2 && wc < I.mw) m_out[(long long)y * I.mw + wc] = lane ? w1 : w0;
  }
  ff_acc(ff[0], s_gs);
  ff_acc(ff[1], s_sgt);
  ff_acc(ff[2], s_pg);
}

// P_TRIAL along -g (mixed) on one staged chunk of `rows` rows, with the next
// GP step's alpha0 terms at the trial point: (1) xt32 = P[x32 - alpha g32] on
// the whole 20 x 72 box, in place of g32 (with <g,s> at the chunk's points);
// (2) gt = A32 xt + b32 and pg at the chunk's points (the outputs, counts,
// free set, <s,gt> and ||pg||^2 of trial32_chunk, in the same arithmetic),
// then pg on the ring one point around them, each in place of b32; (3) the
// sum <pg, A32 pg> over the chunk's points (the terms of alpha32_chunk).
// Two block barriers; every thread calls it.
__device__ __forceinline__ void trial32a_chunk(const DevInst& I, unsigned char* st, int x0, int yc,
                                               int rows, float alpha, const unsigned* fbits,
                                               float* xt_out, float* gt_out, float* pg_out,
                                               unsigned* m_out, Acc& acc, FF* ff) {
  using G = GeoGA;
  constexpr int BW = G::BW, RPW = GeoGP::RPW;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float* X = reinterpret_cast<const float*>(st + G::OFF_X);
  const float* L = reinterpret_cast<const float*>(st + G::OFF_L);
  const float* U = reinterpret_cast<const float*>(st + G::OFF_U);
  float* XT = reinterpret_cast<float*>(st + G::OFF_G);  // g32, then xt
  float* PG = reinterpret_cast<float*>(st + G::OFF_B);  // b32, then pg
  const float* D = reinterpret_cast<const float*>(st + G::OFF_D);
  const float* CX = reinterpret_cast<const float*>(st + G::OFF_CX);
  const float* CY = reinterpret_cast<const float*>(st + G::OFF_CY);
  const int ylim = min(rows, I.ny - yc);  // the chunk's rows inside the grid
  // (1) xt on the box; <g, s> at the chunk's points
  float s_gs = 0.0f;
  for (int e = tid; e < G::RH * BW; e += kThreads) {
    const int br = e / BW, bc = e - br * BW;
    const float x = X[e], g = XT[e];
    const float xt = mid3f(L[e], U[e], fmaf(alpha, -g, x));
    const int r = br - 2, j = bc - G::H;
    if (r >= 0 && r < ylim && j >= 0 && j < 64) s_gs = fmaf(g, xt - x, s_gs);
    XT[e] = xt;
  }
  __syncthreads();
  // gt at chunk row r, column j (-1 <= r <= 16, -1 <= j <= 64): diag, west,
  // east, the row above, the row below (the order of the register sweep).
  // Band boxes start one row above the chunk, the CY box two.
  auto gt_at = [&](int r, int j) {
    const int e = (r + 2) * BW + G::H + j, b = (r + 1) * BW + G::H + j;
    float a = D[b] * XT[e];
    a = fmaf(CX[b - 1], XT[e - 1], a);
    a = fmaf(CX[b], XT[e + 1], a);
    a = fmaf(CY[b], XT[e - BW], a);
    a = fmaf(CY[b + BW], XT[e + BW], a);
    return a + PG[b];
  };
  // (2) the chunk's points: warp w holds rows 2w and 2w+1
  float s_sgt = 0.0f, s_pg = 0.0f;
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    const int r = warp * RPW + k;
    if (r >= ylim) break;  // warp-uniform
    const int y = yc + r;
    const long long row = (long long)y * I.px + x0;
    bool fr[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = lane + 32 * h;
      const bool ok = x0 + j < I.nx;
      const int e = (r + 2) * BW + G::H + j, b = (r + 1) * BW + G::H + j;
      const float gt = gt_at(r, j);
      const float xt = XT[e];
      const float sk = xt - X[e];
      const bool al = xt == L[e], au = xt == U[e];
      const bool act = al || au;
      fr[h] = ok && !act;
      const float pg = pg_compf(al, au, gt);
      PG[b] = pg;
      s_sgt = fmaf(sk, gt, s_sgt);
      s_pg = fmaf(pg, pg, s_pg);
      acc.c[0] += ok && act;
      acc.c[1] += ok && ((al && gt >= 0.0f) || (au && gt <= 0.0f));
      acc.c[2] += ok && (((fbits[k] >> h) & 1u) != (fr[h] ? 1u : 0u));
      if (ok) {
        xt_out[row + j] = xt;
        gt_out[row + j] = gt;
        pg_out[row + j] = pg;
      }
    }
    const unsigned w0 = __ballot_sync(FULL_MASK, fr[0]);
    const unsigned w1 = __ballot_sync(FULL_MASK, fr[1]);
    const int wc = (x0 >> 5) + lane;
    if (lane < 2 && wc < I.mw) m_out[(long long)y * I.mw + wc] = lane ? w1 : w0;
  }
  // the ring: rows -1 and ylim over columns -1..64, columns -1 and 64 of the
  // chunk's rows (points outside the grid arrive as zeros and give pg = 0)
  const int n_ring = 2 * (64 + 2) + 2 * ylim;
  for (int t = tid; t < n_ring; t += kThreads) {
    int r, j;
    if (t < 2 * (64 + 2)) {
      r = t < 64 + 2 ? -1 : ylim;
      j = t % (64 + 2) - 1;
    } else {
      r = (t - 2 * (64 + 2)) >> 1;
      j = (t & 1) ? 64 : -1;
    }
    const int e = (r + 2) * BW + G::H + j, b = (r + 1) * BW + G::H + j;
    const float gt = gt_at(r, j);
    const float xt = XT[e];
    PG[b] = pg_compf(xt == L[e], xt == U[e], gt);
  }
  __syncthreads();
  // (3) <pg, A32 pg> over the chunk's points
  float s_pap = 0.0f;
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    const int r = warp * RPW + k;
    if (r >= ylim) break;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int b = (r + 1) * BW + G::H + lane + 32 * h;
      const float v = PG[b];
      float a = D[b] * v;
      a = fmaf(CX[b - 1], PG[b - 1], a);
      a = fmaf(CX[b], PG[b + 1], a);
      a = fmaf(CY[b], PG[b - BW], a);
      a = fmaf(CY[b + BW], PG[b + BW], a);
      s_pap = fmaf(v, a, s_pap);
    }
  }
  ff_acc(ff[0], s_gs);
  ff_acc(ff[1], s_sgt);
  ff_acc(ff[2], s_pg);
  ff_acc(ff[3], s_pap);
}

// P_GP_ALPHA in FP64 (FEAT_F64 kernels, 2-D): <pg,pg> and <pg, A pg> over
// 8-row chunks.  Stage layout: X | G | L | U, FP64 halo boxes 68 x 10 from
// (x0-2, y-1) | D 64 x 8 | CX 66 x 8 from x0-2 | CY 64 x 9 from y-1 (the fused
// FP64 step's band boxes).  The projected gradient needs no FP64 arithmetic
// (its tests are on bit patterns); it is formed once per staged element, in
// place of g, then each warp applies the stencil to its row.
struct GeoA64 {
  static constexpr int CH = 8, H = 2, BW = 64 + 2 * H;
  static constexpr int SZ_H = align128((CH + 2) * BW * 8);
  static constexpr int OFF_X = 0, OFF_G = SZ_H, OFF_L = 2 * SZ_H, OFF_U = 3 * SZ_H;
  static constexpr int OFF_D = 4 * SZ_H, OFF_CX = OFF_D + 64 * CH * 8;
  static constexpr int OFF_CY = OFF_CX + align128((64 + H) * CH * 8);
  static constexpr int END = OFF_CY + align128(64 * (CH + 1) * 8);
  static constexpr unsigned TX =
      (4 * (CH + 2) * BW + 64 * CH + (64 + H) * CH + 64 * (CH + 1)) * 8;
};
static_assert(GeoA64::END <= kOffMask && GeoA64::CH == kWarps && GeoA64::CH == GeoF<double>::CH,
              "stage layout (one row per warp; the fused FP64 step's band maps)");

// Whether the item's pass is the staged FP64 alpha0 pass of a FEAT_F64 kernel.
template <int kFeat>
__device__ __forceinline__ bool alpha64_tma(const DevInst& I, const Snap& S) {
  return (kFeat & FEAT_F64) != 0 && S.pass == P_GP_ALPHA && !S.gp32 && I.dim == 2 &&
         I.tma_f64gp && I.tma64;
}

__device__ __forceinline__ void issue_alpha64(const DevInst& I, const Snap& S, int x0, int yc,
                                              unsigned st, unsigned bar) {
  using G = GeoA64;
  const int cur = S.cur;
  mbar_expect(bar, G::TX);
  tma_load2d(st + G::OFF_X, tmap(I, MF_X0 + cur), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_G, tmap(I, MF_G0 + cur), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_L, tmap(I, MF_L), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_U, tmap(I, MF_U), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_D, tmap(I, M64_FD), x0, yc, bar);
  tma_load2d(st + G::OFF_CX, tmap(I, M64_FCX), x0 - G::H, yc, bar);
  tma_load2d(st + G::OFF_CY, tmap(I, M64_FCY), x0, yc - 1, bar);
}

__device__ __forceinline__ void alpha64_chunk(const DevInst& I, unsigned char* st, int x0, int yc,
                                              int rows, Acc& acc) {
  using G = GeoA64;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double* X = reinterpret_cast<const double*>(st + G::OFF_X);
  double* PG = reinterpret_cast<double*>(st + G::OFF_G);  // g, then pg
  const double* L = reinterpret_cast<const double*>(st + G::OFF_L);
  const double* U = reinterpret_cast<const double*>(st + G::OFF_U);
  const double* D = reinterpret_cast<const double*>(st + G::OFF_D);
  const double* CX = reinterpret_cast<const double*>(st + G::OFF_CX);
  const double* CY = reinterpret_cast<const double*>(st + G::OFF_CY);
  // points outside the grid arrive as zeros: l = u = x, pg = 0
  for (int e = tid; e < (G::CH + 2) * G::BW; e += kThreads) PG[e] = pg_comp(X[e], PG[e], L[e], U[e]);
  __syncthreads();
  const int ry = warp;
  const int c = 2 * lane;
  const int e0 = x0 + c;
  const bool v0 = e0 < I.nx, v1 = e0 + 1 < I.nx;
  if (ry >= min(rows, I.ny - yc) || !v0) return;
  const double* Pr = PG + (ry + 1) * G::BW + G::H + c;
  const double* Dr = D + ry * 64 + c;
  const double* Xr = CX + ry * (64 + G::H) + G::H + c;
  const double* Ys = CY + ry * 64 + c;
  const double* Yn = CY + (ry + 1) * 64 + c;
  // diag, west, east, south, north (the order of the register sweep)
  double a0 = Dr[0] * Pr[0];
  a0 = fma(Xr[-1], Pr[-1], a0);
  a0 = fma(Xr[0], Pr[1], a0);
  a0 = fma(Ys[0], Pr[-G::BW], a0);
  a0 = fma(Yn[0], Pr[G::BW], a0);
  acc.s[0] = fma(Pr[0], Pr[0], acc.s[0]);
  acc.s[1] = fma(Pr[0], a0, acc.s[1]);
  if (v1) {
    double a1 = Dr[1] * Pr[1];
    a1 = fma(Xr[0], Pr[0], a1);
    a1 = fma(Xr[1], Pr[2], a1);
    a1 = fma(Ys[1], Pr[1 - G::BW], a1);
    a1 = fma(Yn[1], Pr[G::BW + 1], a1);
    acc.s[0] = fma(Pr[1], Pr[1], acc.s[0]);
    acc.s[1] = fma(Pr[1], a1, acc.s[1]);
  }
}

// P_TRIAL in FP64 (FEAT_F64 kernels, 2-D; along -g, or along an FP64 w):
// the trial of OpTrial on 8-row chunks.  Stage layout: X | L | U | DH (g, or
// w) | GH (g, along w) FP64 halo boxes 68 x 10 from (x0-2, y-1) | B 64 x 8 |
// D 64 x 8 | CX 66 x 8 from x0-2 | CY 64 x 9 from y-1.  xt = P[x + alpha d]
// is formed once per staged element, in place of the direction, with <g, s>
// summed first at the chunk's points; then each warp forms gt = A xt + b,
// the status of xt, the sums and the outputs of its row.
struct GeoT64 {
  static constexpr int CH = 8, H = 2, BW = 64 + 2 * H;
  static constexpr int SZ_H = align128((CH + 2) * BW * 8), SZ_I = 64 * CH * 8;
  static constexpr int OFF_X = 0, OFF_L = SZ_H, OFF_U = 2 * SZ_H, OFF_DH = 3 * SZ_H;
  static constexpr int OFF_GH = 4 * SZ_H, OFF_B = 5 * SZ_H, OFF_D = OFF_B + SZ_I;
  static constexpr int OFF_CX = OFF_D + SZ_I;
  static constexpr int OFF_CY = OFF_CX + align128((64 + H) * CH * 8);
  static constexpr int END = OFF_CY + align128(64 * (CH + 1) * 8);
  static constexpr unsigned TX_H = (CH + 2) * BW * 8;
  static constexpr unsigned TX_REST = (2 * 64 * CH + (64 + H) * CH + 64 * (CH + 1)) * 8;
};
static_assert(GeoT64::END <= kOffMask && GeoT64::CH == kWarps, "stage layout (one row per warp)");

template <int kFeat>
__device__ __forceinline__ bool trial64_tma(const DevInst& I, const Snap& S) {
  return (kFeat & FEAT_F64) != 0 && S.pass == P_TRIAL && !S.gp32 && S.dir != D_W32 &&
         I.dim == 2 && I.tma_f64gp && I.tma64;
}

__device__ __forceinline__ void issue_trial64(const DevInst& I, const Snap& S, int x0, int yc,
                                              unsigned st, unsigned bar) {
  using G = GeoT64;
  const int cur = S.cur;
  const bool along_w = S.dir == D_W64;
  mbar_expect(bar, (along_w ? 5u : 4u) * G::TX_H + G::TX_REST);
  tma_load2d(st + G::OFF_X, tmap(I, MF_X0 + cur), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_L, tmap(I, MF_L), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_U, tmap(I, MF_U), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_DH, tmap(I, along_w ? MF_W : MF_G0 + cur), x0 - G::H, yc - 1, bar);
  if (along_w) tma_load2d(st + G::OFF_GH, tmap(I, MF_G0 + cur), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_B, tmap(I, MF_B), x0, yc, bar);
  tma_load2d(st + G::OFF_D, tmap(I, M64_FD), x0, yc, bar);
  tma_load2d(st + G::OFF_CX, tmap(I, M64_FCX), x0 - G::H, yc, bar);
  tma_load2d(st + G::OFF_CY, tmap(I, M64_FCY), x0, yc - 1, bar);
}

template <int DK>
__device__ __forceinline__ void trial64_chunk(const DevInst& I, unsigned char* st, int x0, int yc,
                                              int rows, double alpha, double* xt_out,
                                              double* gt_out, unsigned* m_out,
                                              const unsigned* m_old, Acc& acc) {
  using G = GeoT64;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double* X = reinterpret_cast<const double*>(st + G::OFF_X);
  const double* L = reinterpret_cast<const double*>(st + G::OFF_L);
  const double* U = reinterpret_cast<const double*>(st + G::OFF_U);
  double* XT = reinterpret_cast<double*>(st + G::OFF_DH);  // direction, then xt
  const double* GH = reinterpret_cast<const double*>(st + (DK == D_W64 ? G::OFF_GH : G::OFF_DH));
  const double* B = reinterpret_cast<const double*>(st + G::OFF_B);
  const double* D = reinterpret_cast<const double*>(st + G::OFF_D);
  const double* CX = reinterpret_cast<const double*>(st + G::OFF_CX);
  const double* CY = reinterpret_cast<const double*>(st + G::OFF_CY);
  const int ylim = min(rows, I.ny - yc);
  // xt on the box (zeros outside the grid give xt = 0); <g, s> at the chunk's points
  double s_gs = 0.0;
  for (int e = tid; e < (G::CH + 2) * G::BW; e += kThreads) {
    const int br = e / G::BW, bc = e - br * G::BW;
    const int r = br - 1, j = bc - G::H;
    const double x = X[e], g = GH[e];
    const double d = DK == D_W64 ? XT[e] : -g;
    const double xt = mid3(L[e], U[e], fma(alpha, d, x));
    if (r >= 0 && r < ylim && j >= 0 && j < 64 && x0 + j < I.nx) s_gs = fma(g, xt - x, s_gs);
    XT[e] = xt;
  }
  acc.s[0] += s_gs;
  __syncthreads();
  const int ry = warp;
  if (ry >= ylim) return;  // warp-uniform
  const int c = 2 * lane;
  const int e0 = x0 + c;
  const bool v0 = e0 < I.nx, v1 = e0 + 1 < I.nx;
  const int b = (ry + 1) * G::BW + G::H + c;
  const double* Pr = XT + b;
  const double* Dr = D + ry * 64 + c;
  const double* Xr = CX + ry * (64 + G::H) + G::H + c;
  const double* Ys = CY + ry * 64 + c;
  const double* Yn = CY + (ry + 1) * 64 + c;
  // diag, west, east, south, north (the order of the register sweep)
  double a[2];
  a[0] = Dr[0] * Pr[0];
  a[0] = fma(Xr[-1], Pr[-1], a[0]);
  a[0] = fma(Xr[0], Pr[1], a[0]);
  a[0] = fma(Ys[0], Pr[-G::BW], a[0]);
  a[0] = fma(Yn[0], Pr[G::BW], a[0]);
  a[1] = Dr[1] * Pr[1];
  a[1] = fma(Xr[0], Pr[0], a[1]);
  a[1] = fma(Xr[1], Pr[2], a[1]);
  a[1] = fma(Ys[1], Pr[1 - G::BW], a[1]);
  a[1] = fma(Yn[1], Pr[G::BW + 1], a[1]);
  bool fr[2];
  double gt[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const bool ok = k == 0 ? v0 : v1;
    const int e = b + k;
    const double v = Pr[k];
    gt[k] = a[k] + B[ry * 64 + c + k];
    const bool al = deq(v, L[e]), au = deq(v, U[e]);
    const bool act = al || au;
    const bool bind = (al && dge0(gt[k])) || (au && dle0(gt[k]));
    fr[k] = ok && !act;
    if (ok) {
      const double sk = v - X[e];
      acc.s[1] = fma(sk, gt[k], acc.s[1]);
      const double pg = pg_comp(v, gt[k], L[e], U[e]);
      acc.s[2] = fma(pg, pg, acc.s[2]);
      acc.c[0] += act;
      acc.c[1] += bind;
    }
  }
  const long long i = (long long)(yc + ry) * I.px + e0;
  if (v0) {
    st2(xt_out, i, v0, v1, Pr[0], Pr[1]);
    st2(gt_out, i, v0, v1, gt[0], gt[1]);
  }
  acc.c[2] += write_mask(I, m_out, m_old, yc + ry, 0, x0, lane, fr[0], fr[1]);
}

// The first CG step of a mixed-phase CG phase (P_CG_B with first_cg: FP32
// CG, FP32 gradient, 2-D, no preconditioner or point Jacobi), staged: the
// operand p_0 = -z_F (z = g, or g / diag) needs the free bits of the halo
// points, taken from a mask box 8 words wide (from word ((x0/32) - 1)
// rounded down to a multiple of 4, so that it covers columns x0-4 .. x0+67)
// and 18 rows high from y-1.  Stage layout: G (g32, 72 x 18 from (x0-4,
// y-1)) | M (8 x 18 words) | D 64 x 16 | CX 68 x 16 from x0-4 | CY 64 x 17
// from y-1 (the fused step's band maps) | DI (1/diag, 72 x 18 from (x0-4,
// y-1); point Jacobi only).
struct GeoB0 {
  static constexpr int CH = 16, H = 4, BW = 64 + 2 * H, MW = 8;
  static constexpr int OFF_G = 0, OFF_M = align128((CH + 2) * BW * 4);
  static constexpr int OFF_D = OFF_M + align128(MW * (CH + 2) * 4);
  static constexpr int OFF_CX = OFF_D + 64 * CH * 4;
  static constexpr int OFF_CY = OFF_CX + align128((64 + H) * CH * 4);
  static constexpr int OFF_DI = OFF_CY + align128(64 * (CH + 1) * 4);
  static constexpr int END = OFF_DI + align128((CH + 2) * BW * 4);
  static constexpr unsigned TX =
      ((CH + 2) * BW + MW * (CH + 2) + 64 * CH + (64 + H) * CH + 64 * (CH + 1)) * 4;
  static constexpr unsigned TX_DI = (CH + 2) * BW * 4;
};
static_assert(GeoB0::END <= kOffMask && GeoB0::CH == GeoF<float>::CH && GeoB0::H == GeoGP::H,
              "stage layout (the fused FP32 step's band maps, the GP passes' g32 maps)");

__device__ __forceinline__ bool first_staged(const DevInst& I, const Snap& S) {
  return S.pass == P_CG_B && S.first_cg && S.cg32 && S.gp32 && I.dim == 2 &&
         (I.opt.precond == PC_NONE || I.opt.precond == PC_JACOBI) && I.tma32 && I.tma_gp &&
         I.tma_mask;
}

// The mask box's first word column for a chunk at column x0 (a multiple of
// 4 words, 16 bytes; negative at the grid's west edge, where the box is
// zero-filled).
__device__ __forceinline__ int first_mask_word(int x0) { return ((x0 >> 5) - 1) & ~3; }

__device__ __forceinline__ void issue_cgb0(const DevInst& I, int cur, int x0, int yc, unsigned st,
                                           unsigned bar) {
  using G = GeoB0;
  const bool jac = I.opt.precond == PC_JACOBI;
  mbar_expect(bar, G::TX + (jac ? G::TX_DI : 0u));
  if (jac) tma_load2d(st + G::OFF_DI, tmap(I, M32_FDIH), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_G, tmap(I, MG_G32H0 + cur), x0 - G::H, yc - 1, bar);
  tma_load2d(st + G::OFF_M, tmap(I, M_MASKH0 + cur), first_mask_word(x0), yc - 1, bar);
  tma_load2d(st + G::OFF_D, tmap(I, M32_FD), x0, yc, bar);
  tma_load2d(st + G::OFF_CX, tmap(I, M32_FCX), x0 - G::H, yc, bar);
  tma_load2d(st + G::OFF_CY, tmap(I, M32_FCY), x0, yc - 1, bar);
}

// The staged first step on one chunk (warp w: rows 2w, 2w+1): p_0 = -z on
// the free set (0 elsewhere; z = g, or g / diag under point Jacobi), Ap_0 =
// Z Z' A Z Z' p_0 (the stencil in the order of the register sweep), r_0 =
// g_F, w = 0; sums <p_0, Ap_0>, rho_0 = <r_0, z_0> and <Ap_0, M^-1 Ap_0>,
// the sums of P_CG_B's first step.
template <bool JAC>
__device__ __forceinline__ void cgb0_chunk(const DevInst& I, const unsigned char* st, int x0,
                                           int yc, int rows, float* p_out, float* ap_out,
                                           float* r_out, float* w, FF* ff) {
  using G = GeoB0;
  const float* DI = reinterpret_cast<const float*>(st + G::OFF_DI);
  constexpr int RPW = G::CH / kWarps;
  const float* GS = reinterpret_cast<const float*>(st + G::OFF_G);
  const unsigned* M = reinterpret_cast<const unsigned*>(st + G::OFF_M);
  const float* D = reinterpret_cast<const float*>(st + G::OFF_D);
  const float* CX = reinterpret_cast<const float*>(st + G::OFF_CX);
  const float* CY = reinterpret_cast<const float*>(st + G::OFF_CY);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ylim = min(rows, I.ny - yc);
  const int r0 = warp * RPW;  // first chunk row of this warp
  if (r0 >= ylim) return;     // warp-uniform
  const int c = 2 * lane;
  const int e0 = x0 + c;
  const bool v0 = e0 < I.nx, v1 = e0 + 1 < I.nx;
  const int wx = first_mask_word(x0);
  // the free bit of column col (x0-4 <= col < x0+68) in box row br
  auto free_at = [&](int br, int col) {
    return (M[br * G::MW + ((col >> 5) - wx)] >> (col & 31)) & 1u;
  };
  // window q = 0 .. RPW+1 is chunk row r0-1+q (box row r0+q)
  float pn[RPW + 2][2], pw[RPW], pe[RPW];
#pragma unroll
  for (int q = 0; q < RPW + 2; ++q) {
    const int br = r0 + q;
    float2 gv = *reinterpret_cast<const float2*>(GS + br * G::BW + G::H + c);
    if (JAC) {
      const float2 dv = *reinterpret_cast<const float2*>(DI + br * G::BW + G::H + c);
      gv.x *= dv.x;
      gv.y *= dv.y;
    }
    const unsigned wd = M[br * G::MW + ((e0 >> 5) - wx)] >> (e0 & 31);
    pn[q][0] = (wd & 1u) ? -gv.x : 0.0f;
    pn[q][1] = (wd & 2u) ? -gv.y : 0.0f;
  }
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    pw[k] = __shfl_up_sync(FULL_MASK, pn[k + 1][1], 1);
    pe[k] = __shfl_down_sync(FULL_MASK, pn[k + 1][0], 1);
    const int br = r0 + k + 1, b = br * G::BW + G::H;
    if (lane == 0) pw[k] = free_at(br, x0 - 1) ? -GS[b - 1] * (JAC ? DI[b - 1] : 1.0f) : 0.0f;
    if (lane == 31) pe[k] = free_at(br, x0 + 64) ? -GS[b + 64] * (JAC ? DI[b + 64] : 1.0f) : 0.0f;
  }
  float s_pap = 0.0f, s_rr = 0.0f, s_apap = 0.0f;
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    const int ry = r0 + k;
    if (ry >= ylim) break;
    const int q = k + 1;
    const float* Dr = D + ry * 64 + c;
    const float* Xr = CX + ry * (64 + G::H) + G::H + c;
    const float* Ys = CY + ry * 64 + c;
    const float* Yn = CY + (ry + 1) * 64 + c;
    // diag, west, east, south, north (the order of the register sweep)
    float a0 = Dr[0] * pn[q][0];
    a0 = fmaf(Xr[-1], pw[k], a0);
    a0 = fmaf(Xr[0], pn[q][1], a0);
    a0 = fmaf(Ys[0], pn[q - 1][0], a0);
    a0 = fmaf(Yn[0], pn[q + 1][0], a0);
    float a1 = Dr[1] * pn[q][1];
    a1 = fmaf(Xr[0], pn[q][0], a1);
    a1 = fmaf(Xr[1], pe[k], a1);
    a1 = fmaf(Ys[1], pn[q - 1][1], a1);
    a1 = fmaf(Yn[1], pn[q + 1][1], a1);
    const unsigned wd = M[(ry + 1) * G::MW + ((e0 >> 5) - wx)] >> (e0 & 31);
    a0 = (wd & 1u) ? a0 : 0.0f;
    a1 = (wd & 2u) ? a1 : 0.0f;
    const long long i = (long long)(yc + ry) * I.px + e0;
    // r_0 = g_F (under point Jacobi g_F, not z_F) and M^-1 Ap_0
    float r0v = -pn[q][0], r1v = -pn[q][1], d0 = 1.0f, d1 = 1.0f;
    if (JAC) {
      const float2 gv = *reinterpret_cast<const float2*>(GS + (ry + 1) * G::BW + G::H + c);
      const float2 dv = *reinterpret_cast<const float2*>(DI + (ry + 1) * G::BW + G::H + c);
      r0v = (wd & 1u) ? gv.x : 0.0f;
      r1v = (wd & 2u) ? gv.y : 0.0f;
      d0 = dv.x;
      d1 = dv.y;
    }
    st2(p_out, i, v0, v1, pn[q][0], pn[q][1]);
    st2(ap_out, i, v0, v1, a0, a1);
    st2(r_out, i, v0, v1, r0v, r1v);
    st2(w, i, v0, v1, 0.0f, 0.0f);
    // points past nx hold zeros (the boxes are zero-filled there)
    s_pap = fmaf(pn[q][0], a0, s_pap);
    s_pap = fmaf(pn[q][1], a1, s_pap);
    s_rr = fmaf(r0v, -pn[q][0], s_rr);
    s_rr = fmaf(r1v, -pn[q][1], s_rr);
    s_apap = fmaf(a0, a0 * d0, s_apap);
    s_apap = fmaf(a1, a1 * d1, s_apap);
  }
  ff_acc(ff[0], s_pap);
  ff_acc(ff[1], s_rr);
  ff_acc(ff[2], s_apap);
}

// Whether the item's pass runs through the TMA pipeline.
template <int kFeat>
__device__ __forceinline__ bool tma_pass(const DevInst& I, const Snap& S) {
  if (gp_tma(I, S)) return true;
  if (alpha64_tma<kFeat>(I, S) || trial64_tma<kFeat>(I, S)) return true;
  if (S.pass == P_CG_F) return true;  // scheduled only for instances with the maps
  if (first_staged(I, S)) return true;
  if (S.pass != P_CG_A && S.pass != P_CG_B) return false;
  if (!I.tma_mask) return false;
  const int ok = S.cg32 ? I.tma32 : I.tma64;
  if (!ok) return false;
  if (S.pass == P_CG_A) return true;
  return S.pass == P_CG_B && !S.first_cg && I.dim == 2;
}

// Rows per chunk of the item's TMA pass.
__device__ __forceinline__ int chunk_rows(const DevInst& I, const Snap& S, bool gp) {
  if (gp) return S.pass == P_GP_ALPHA ? ChunkGeo<float>::CH : GeoGP::CH;
  if (S.pass == P_GP_ALPHA) return GeoA64::CH;  // the staged FP64 GP passes
  if (S.pass == P_TRIAL) return GeoT64::CH;
  if (S.pass == P_CG_A) return S.cg32 ? ChunkGeo<float>::CH_A : ChunkGeo<double>::CH_A;
  if (S.pass == P_CG_F && I.dim == 3) return GeoF3::CH;
  if (S.pass == P_CG_F) return S.cg32 ? GeoF<float>::CH : GeoF<double>::CH;
  if (S.pass == P_CG_B && S.first_cg) return GeoB0::CH;  // (staged only as first_staged)
  return S.cg32 ? ChunkGeo<float>::CH : ChunkGeo<double>::CH;
}

// A chunk of a TMA pass: rows yc .. yc+(rows & (kEndG0-1))-1 (a multiple of
// 8, at most the pass's chunk height) of the tile at column x0 of plane z;
// bit kEndG0 of `rows` marks the last chunk of the first group of a
// two-group work item (the group's sums are set aside after it).
constexpr int kEndG0 = 1 << 8;
struct Chunk {
  int x0, yc, z, rows;
};

// Walks the 8-row strips of a work item's groups [g0, g1) (g1 - g0 <=
// kMaxSpan = 2) in chunks: a chunk starts at the current strip and takes up
// to ch/8 strips without leaving its tile or its group, so that every group
// is cut into the same chunks whatever the item.  Group g covers the strips
// [g * S / n_groups, (g+1) * S / n_groups), S = 4 n_tiles; tile coordinates
// are divided out once, at the item's first strip.
struct Walk {
  int u, u_hi, gend, ch8, tx, ty, z, s;
  __device__ Walk(const DevInst& I, int g0, int g1, int ch) : ch8(ch >> 3) {
    static_assert(kMaxSpan == 2, "a work item ends at most one group before its own end");
    const long long strips = (long long)I.n_tiles * (kTY / 8);
    u = (int)((long long)g0 * strips / I.n_groups);
    gend = (int)((long long)(g0 + 1) * strips / I.n_groups);
    u_hi = g1 == g0 + 1 ? gend : (int)((long long)g1 * strips / I.n_groups);
    const int t = u >> 2, rest = t / I.tiles_x;
    s = u & 3;
    tx = t - rest * I.tiles_x;
    ty = rest % I.tiles_y;
    z = rest / I.tiles_y;
  }
  __device__ bool done() const { return u >= u_hi; }
  __device__ Chunk take(const DevInst& I) {
    const int k = min(min(ch8, 4 - s), gend - u);
    Chunk c{tx * kTX, ty * kTY + 8 * s, z, 8 * k};
    u += k;
    if (u == gend && u < u_hi) {
      c.rows |= kEndG0;
      gend = u_hi;
    }
    s += k;
    if (s == 4) {
      s = 0;
      if (++tx == I.tiles_x) {
        tx = 0;
        if (++ty == I.tiles_y) {
          ty = 0;
          ++z;
        }
      }
    }
    return c;
  }
};

// The free-set bits of this lane for each of its rows of a chunk, read from
// the staged mask box (4 words x 32 rows from word (x0/32) rounded down to a
// multiple of 4).  `gp`: bit h is column lane+32h (the GP passes); otherwise
// bits 0 and 1 are columns 2*lane and 2*lane+1.
__device__ __forceinline__ void stage_bits(const unsigned char* st, int x0, int rpw, bool gp,
                                           unsigned fbits[4]) {
  const unsigned* M = reinterpret_cast<const unsigned*>(st + kOffMask);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int off = (x0 >> 5) & 3;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (k >= rpw) break;
    const unsigned* row = M + (warp * rpw + k) * 4 + off;
    if (gp) {
      fbits[k] = ((row[0] >> lane) & 1u) | (((row[1] >> lane) & 1u) << 1);
    } else {
      fbits[k] = row[lane >> 4] >> ((2 * lane) & 31);
    }
  }
}

// Issue a chunk of the item's pass into a stage; `mask`: also the chunk's
// free-set words of mask[S.cur].
template <int kFeat>
__device__ __forceinline__ void issue_chunk(const DevInst& I, const Snap& S, bool gp,
                                            const Chunk& c, unsigned st, unsigned bar,
                                            bool mask) {
  if (mask) {
    mbar_expect_only(bar, kMaskBox);
    tma_load2d(st + kOffMask, tmap(I, M_MASK0 + S.cur), (c.x0 >> 5) & ~3, c.z * I.ny + c.yc, bar);
  }
  if (gp) {
    issue_gp(I, S, c.x0, c.yc, st, bar);
  } else if (S.pass == P_GP_ALPHA) {
    if constexpr ((kFeat & FEAT_F64) != 0) issue_alpha64(I, S, c.x0, c.yc, st, bar);
  } else if (S.pass == P_TRIAL) {
    if constexpr ((kFeat & FEAT_F64) != 0) issue_trial64(I, S, c.x0, c.yc, st, bar);
  } else if (S.pass == P_CG_F && I.opt.precond == PC_TILE) {
    if constexpr ((kFeat & FEAT_TILE) != 0) {
      if (S.cg32) issue_cgt<float>(I, S.pcur, c.x0, c.yc, st, bar);
      else issue_cgt<double>(I, S.pcur, c.x0, c.yc, st, bar);
    }
  } else if (S.pass == P_CG_F && I.dim == 3) {
    // FP32 only, and only scheduled in a FEAT_3D kernel (cg_fused)
    if constexpr ((kFeat & FEAT_3D) != 0) issue_cgf3(I, S.pcur, c.x0, c.z * I.ny + c.yc, st, bar);
  } else if (S.pass == P_CG_F) {
    if (S.cg32) issue_cgf<float>(I, S.pcur, c.x0, c.yc, st, bar);
    else issue_cgf<double>(I, S.pcur, c.x0, c.yc, st, bar);
  } else if (S.pass == P_CG_B && S.first_cg) {
    issue_cgb0(I, S.cur, c.x0, c.yc, st, bar);  // (staged only as first_staged)
  } else if (S.cg32) {
    if (S.pass == P_CG_B) issue_cgb<float>(I, S.pcur, c.x0, c.yc, st, bar);
    else issue_cga<float>(I, S.pcur, c.x0, c.z * I.ny + c.yc, st, bar);
  } else {
    if (S.pass == P_CG_B) issue_cgb<double>(I, S.pcur, c.x0, c.yc, st, bar);
    else issue_cga<double>(I, S.pcur, c.x0, c.z * I.ny + c.yc, st, bar);
  }
}

// Compute a staged chunk of the item's pass.
template <int kFeat>
__device__ __forceinline__ void run_chunk(const DevInst& I, const Snap& S, bool gp,
                                          unsigned char* st, const Chunk& cf,
                                          const unsigned* fbits, Acc& acc, FF* ffs) {
  const Chunk c{cf.x0, cf.yc, cf.z, cf.rows & (kEndG0 - 1)};
  const int cur = S.cur;
  if (gp) {
    if (S.pass == P_CENSUS) {
      census32_chunk(I, st, c.x0, c.yc, c.rows, I.g32[cur], I.pg32[cur], I.mask[cur], acc,
                     ffs[0]);
    } else if (S.pass == P_GP_ALPHA) {
      alpha32_chunk(I, st, c.yc, c.rows, ffs);
    } else {
      const float al = S.dir == D_ZERO ? 0.0f : (float)S.alpha;
      if (S.dir == D_W32)
        trial32_chunk<D_W32>(I, st, c.x0, c.yc, c.rows, al, fbits, I.x32[cur ^ 1],
                             I.g32[cur ^ 1], I.pg32[cur ^ 1], I.mask[cur ^ 1], acc, ffs);
      else
        trial32a_chunk(I, st, c.x0, c.yc, c.rows, al, fbits, I.x32[cur ^ 1], I.g32[cur ^ 1],
                       I.pg32[cur ^ 1], I.mask[cur ^ 1], acc, ffs);
    }
  } else if (S.pass == P_GP_ALPHA) {
    if constexpr ((kFeat & FEAT_F64) != 0) alpha64_chunk(I, st, c.x0, c.yc, c.rows, acc);
  } else if (S.pass == P_TRIAL) {
    if constexpr ((kFeat & FEAT_F64) != 0) {
      const double al = S.dir == D_ZERO ? 0.0 : S.alpha;
      if (S.dir == D_W64)
        trial64_chunk<D_W64>(I, st, c.x0, c.yc, c.rows, al, I.x[cur ^ 1], I.g[cur ^ 1],
                             I.mask[cur ^ 1], I.mask[cur], acc);
      else
        trial64_chunk<D_NEG_G>(I, st, c.x0, c.yc, c.rows, al, I.x[cur ^ 1], I.g[cur ^ 1],
                               I.mask[cur ^ 1], I.mask[cur], acc);
    }
  } else if (S.pass == P_CG_F && I.opt.precond == PC_TILE) {
    if constexpr ((kFeat & FEAT_TILE) != 0) {
      const int q = S.pcur ^ 1;
      if (S.cg32)
        cgt_chunk<float>(I, st, c.x0, c.yc, c.rows, (float)S.alpha, (float)S.beta, fbits, I.w32,
                         I.r32[q], I.z32[q], I.p32[q], I.Ap32[q], I.q32[q], acc, ffs);
      else
        cgt_chunk<double>(I, st, c.x0, c.yc, c.rows, S.alpha, S.beta, fbits, I.w64, I.r64[q],
                          I.z64[q], I.p64[q], I.Ap64[q], I.q64[q], acc, ffs);
    }
  } else if (S.pass == P_CG_F && I.dim == 3) {
    if constexpr ((kFeat & FEAT_3D) != 0) {
      const int q = S.pcur ^ 1;
      cgf3_chunk(I, st, c.x0, c.z * I.ny + c.yc, c.yc, c.rows, (float)S.alpha, (float)S.beta,
                 fbits, I.w32, I.r32[q], I.p32[q], I.Ap32[q], ffs);
    }
  } else if (S.pass == P_CG_F) {
    const int q = S.pcur ^ 1;
    const bool jac = I.opt.precond == PC_JACOBI;
    if (S.cg32 && jac)
      cgf_chunk<float, true>(I, st, c.x0, c.yc, c.rows, (float)S.alpha, (float)S.beta, fbits,
                             I.w32, I.r32[q], I.p32[q], I.Ap32[q], acc, ffs);
    else if (S.cg32)
      cgf_chunk<float, false>(I, st, c.x0, c.yc, c.rows, (float)S.alpha, (float)S.beta, fbits,
                              I.w32, I.r32[q], I.p32[q], I.Ap32[q], acc, ffs);
    else if (jac)
      cgf_chunk_box<true>(I, st, c.x0, c.yc, c.rows, S.alpha, S.beta, fbits, I.w64, I.r64[q],
                          I.p64[q], I.Ap64[q], acc);
    else
      cgf_chunk_box<false>(I, st, c.x0, c.yc, c.rows, S.alpha, S.beta, fbits, I.w64, I.r64[q],
                           I.p64[q], I.Ap64[q], acc);
  } else if (S.pass == P_CG_B && S.first_cg) {
    const int q = S.pcur ^ 1;
    if (I.opt.precond == PC_JACOBI)
      cgb0_chunk<true>(I, st, c.x0, c.yc, c.rows, I.p32[q], I.Ap32[q], I.r32[q], I.w32, ffs);
    else
      cgb0_chunk<false>(I, st, c.x0, c.yc, c.rows, I.p32[q], I.Ap32[q], I.r32[q], I.w32, ffs);
  } else if (S.pass == P_CG_B) {
    const int q = S.pcur ^ 1;
    if (S.cg32)
      cgb_chunk<float>(I, st, c.x0, c.yc, c.rows, (float)S.beta, fbits, I.p32[q], I.Ap32[q],
                       acc, ffs[0]);
    else
      cgb_chunk<double>(I, st, c.x0, c.yc, c.rows, S.beta, fbits, I.p64[q], I.Ap64[q], acc,
                        ffs[0]);
  } else {
    const int ylim = min(c.rows, I.ny - c.yc);
    const int q = S.pcur ^ 1;
    const int row = c.z * I.ny + c.yc;
    if (S.cg32 && I.opt.precond == PC_JACOBI)
      cga_chunk<float, true>(I, st, c.x0, row, ylim, (float)S.alpha, I.w32, I.r32[q], acc,
                             ffs[0]);
    else if (S.cg32)
      cga_chunk<float, false>(I, st, c.x0, row, ylim, (float)S.alpha, I.w32, I.r32[q], acc,
                              ffs[0]);
    else if (I.opt.precond == PC_JACOBI)
      cga_chunk<double, true>(I, st, c.x0, row, ylim, S.alpha, I.w64, I.r64[q], acc, ffs[0]);
    else
      cga_chunk<double, false>(I, st, c.x0, row, ylim, S.alpha, I.w64, I.r64[q], acc, ffs[0]);
  }
}

// ------------------------------------------------------------------ kernel --

// Number of FP64 sums each pass reduces.
__device__ __forceinline__ int n_sums(int pass, int first, int gp32) {
  switch (pass) {
    case P_CENSUS: return gp32 ? 1 : 2;
    case P_GP_ALPHA: return 2;
    case P_TRIAL: return 4;  // the staged trial along -g adds <pg, A pg> at the trial point
    case P_CG_B: return first ? 3 : 1;
    case P_CG_A: return 1;
    case P_CG_F: return 4;
    case P_CG_Z: return 1;
    case P_RX_BUILD: return 1;
    case P_RCG: return 4;
    default: return 0;
  }
}

template <int kFeat>
__device__ __forceinline__ void run_tile(const DevInst& I, const Snap& S, int x0, int y0, int z,
                                         Acc& acc, FF* ffs, float* scr) {
  const int cur = S.cur, pcur = S.pcur;
  switch (S.pass) {
    case P_START:
      start_tile(I, I.x[cur], I.x32[cur], x0, y0, z);
      break;
    case P_CENSUS: {
      if (S.gp32) {
        OpCensus32 op{I, I.x32[cur], I.g32[cur], I.pg32[cur], I.mask[cur], ffs};
        stencil_tile(I, op, x0, y0, z, acc);
      } else {
        // the first FP64 census after the mixed phase rebuilds x from x32
        OpCensus op{I, I.x[cur], I.g[cur], I.mask[cur], S.x32_live ? I.x32[cur] : nullptr,
                    I.x[cur]};
        stencil_tile(I, op, x0, y0, z, acc);
      }
      break;
    }
    case P_GP_ALPHA: {
      if (S.gp32) {
        OpGpAlpha32 op{I, I.pg32[cur], ffs};
        stencil_tile(I, op, x0, y0, z, acc);
      } else {
        OpGpAlpha op{I, I.x[cur], I.g[cur]};
        stencil_tile(I, op, x0, y0, z, acc);
      }
      break;
    }
    case P_TRIAL: {
      const double alpha = S.dir == D_ZERO ? 0.0 : S.alpha;
      if (S.gp32) {
        if (S.dir == D_W32) {
          OpTrial32<D_W32> op{I, I.x32[cur], I.g32[cur], I.w32, (float)alpha, I.x32[cur ^ 1],
                              I.g32[cur ^ 1], I.pg32[cur ^ 1], I.mask[cur ^ 1], I.mask[cur],
                              ffs};
          stencil_tile(I, op, x0, y0, z, acc);
        } else {
          OpTrial32<D_NEG_G> op{I, I.x32[cur], I.g32[cur], I.w32, (float)alpha, I.x32[cur ^ 1],
                                I.g32[cur ^ 1], I.pg32[cur ^ 1], I.mask[cur ^ 1], I.mask[cur],
                                ffs};
          stencil_tile(I, op, x0, y0, z, acc);
        }
      } else if (S.dir == D_W64) {
        OpTrial<D_W64> op{I, I.x[cur], I.g[cur], I.w64, I.w32, alpha, I.x[cur ^ 1],
                          I.g[cur ^ 1], I.mask[cur ^ 1], I.mask[cur]};
        stencil_tile(I, op, x0, y0, z, acc);
      } else if (S.dir == D_W32) {
        OpTrial<D_W32> op{I, I.x[cur], I.g[cur], I.w64, I.w32, alpha, I.x[cur ^ 1],
                          I.g[cur ^ 1], I.mask[cur ^ 1], I.mask[cur]};
        stencil_tile(I, op, x0, y0, z, acc);
      } else {
        OpTrial<D_NEG_G> op{I, I.x[cur], I.g[cur], I.w64, I.w32, alpha, I.x[cur ^ 1],
                            I.g[cur ^ 1], I.mask[cur ^ 1], I.mask[cur]};
        stencil_tile(I, op, x0, y0, z, acc);
      }
      break;
    }
    case P_CG_B: {
      const float* g32 = S.gp32 ? I.g32[cur] : nullptr;
      // point Jacobi (z = r / diag) runs in its own instantiations
      const bool jac = I.opt.precond == PC_JACOBI;
      if (S.cg32) {
        float* p_new = I.p32[pcur ^ 1];
        float* ap = I.Ap32[pcur ^ 1];
        float* r1 = I.r32[pcur ^ 1];
#define GPCG_CGB32(FIRST, JAC, BETA)                                                          \
  {                                                                                          \
    OpCgB<float, FIRST, JAC> op{I, r1, I.p32[pcur], I.g[cur], I.mask[cur], BETA, g32, p_new, \
                                ap, r1, I.w32, I.diag32, I.cx32, I.cy32, I.cz32, ffs,         \
                                I.dinv32};                                                   \
    stencil_tile(I, op, x0, y0, z, acc);                                                      \
  }
        if (S.first_cg && jac) GPCG_CGB32(true, true, 0.0f)
        else if (S.first_cg) GPCG_CGB32(true, false, 0.0f)
        else if (jac) GPCG_CGB32(false, true, (float)S.beta)
        else GPCG_CGB32(false, false, (float)S.beta)
#undef GPCG_CGB32
      } else {
        double* p_new = I.p64[pcur ^ 1];
        double* ap = I.Ap64[pcur ^ 1];
        double* r1 = I.r64[pcur ^ 1];
#define GPCG_CGB64(FIRST, JAC, BETA)                                                           \
  {                                                                                           \
    OpCgB<double, FIRST, JAC> op{I, r1, I.p64[pcur], I.g[cur], I.mask[cur], BETA, nullptr,     \
                                 p_new, ap, r1, I.w64, I.diag, I.cx, I.cy, I.cz, nullptr,     \
                                 I.dinv};                                                     \
    stencil_tile(I, op, x0, y0, z, acc);                                                       \
  }
        if (S.first_cg && jac) GPCG_CGB64(true, true, 0.0)
        else if (S.first_cg) GPCG_CGB64(true, false, 0.0)
        else if (jac) GPCG_CGB64(false, true, S.beta)
        else GPCG_CGB64(false, false, S.beta)
#undef GPCG_CGB64
      }
      break;
    }
    case P_RX_COUNT:
      if constexpr ((kFeat & FEAT_EXT) != 0) rx_count_tile(I, S, x0, y0, z, acc);
      break;
    case P_RX_BUILD:
      if constexpr ((kFeat & FEAT_EXT) != 0) {
        const bool jac = I.opt.precond == PC_JACOBI;
        if (S.cg32 && jac) rx_build_tile<float, true>(I, S, x0, y0, z, acc, ffs);
        else if (S.cg32) rx_build_tile<float, false>(I, S, x0, y0, z, acc, ffs);
        else if (jac) rx_build_tile<double, true>(I, S, x0, y0, z, acc, ffs);
        else rx_build_tile<double, false>(I, S, x0, y0, z, acc, ffs);
      }
      break;
    case P_CG_Z:
      if constexpr ((kFeat & FEAT_TILE) != 0) {
        if (S.cg32) cg_z_tile<float>(I, S, x0, y0, z, scr, acc, ffs);
        else cg_z_tile<double>(I, S, x0, y0, z, scr, acc, ffs);
      }
      break;
    case P_CG_A:
      if (S.cg32 && I.opt.precond == PC_JACOBI)
        cg_a_tile<float, true>(I, I.w32, I.r32[pcur], I.r32[pcur ^ 1], I.p32[pcur],
                               I.Ap32[pcur], I.dinv32, S.alpha, x0, y0, z, acc, ffs);
      else if (S.cg32)
        cg_a_tile<float, false>(I, I.w32, I.r32[pcur], I.r32[pcur ^ 1], I.p32[pcur],
                                I.Ap32[pcur], I.dinv32, S.alpha, x0, y0, z, acc, ffs);
      else if (I.opt.precond == PC_JACOBI)
        cg_a_tile<double, true>(I, I.w64, I.r64[pcur], I.r64[pcur ^ 1], I.p64[pcur],
                                I.Ap64[pcur], I.dinv, S.alpha, x0, y0, z, acc, ffs);
      else
        cg_a_tile<double, false>(I, I.w64, I.r64[pcur], I.r64[pcur ^ 1], I.p64[pcur],
                                 I.Ap64[pcur], I.dinv, S.alpha, x0, y0, z, acc, ffs);
      break;
    default:
      break;
  }
}

// Whether this instantiation has the code of the item's pass.
template <int kFeat>
__device__ __forceinline__ bool pass_supported(const DevInst& I, const Snap& S) {
  const bool tile = S.pass == P_CG_Z || (S.pass == P_CG_F && I.opt.precond == PC_TILE);
  const bool ext = S.pass >= P_RX_COUNT && S.pass <= P_RW;
  const bool f3 = S.pass == P_CG_F && I.dim == 3;
  return (!tile || (kFeat & FEAT_TILE) != 0) && (!ext || (kFeat & FEAT_EXT) != 0) &&
         (!f3 || (kFeat & FEAT_3D) != 0);
}

// The body of the pass kernels: pass_kernel runs one pass of every live
// instance per launch; pass_kernel_coop (GPCG_COOP) runs every pass of one
// instance in a cooperative launch.
//
// kCond: the launch belongs to a WHILE-conditional graph whose condition this
// kernel clears (a separate instantiation, because profilers cannot capture
// graph nodes able to set a condition).
//
// The cooperative kernel takes one work item per block, every block
// resident.  After a pass the blocks meet at a grid barrier instead of a
// kernel boundary; then every block reduces the group partials and runs the
// state machine on its own copy of the control block -- the same arithmetic
// in the same order, so the copies agree bit for bit and every block knows
// the next pass without a round trip to global memory -- and block 0 alone
// writes the control block back, counts the pass and counts the instance out
// when it is done.  The partials alternate between two slot arrays, so a
// block that starts the next pass never overwrites slots another block is
// still reducing.
template <bool kCond, int kFeat>
__device__ __forceinline__ void pass_body(const EngineArgs& E) {
  constexpr bool kCoop = GPCG_COOP != 0;
  __shared__ DevInst sI;
  __shared__ Snap sS;
  __shared__ Ctl sC;
  __shared__ int s_scan[kWarps];
  __shared__ double s_red[kNRed];
  // the threads' sums of the first group of a two-group work item (those of
  // an item's last group go to the first stage once the copies have landed)
  __shared__ double s_stash[4][kThreads];
  __shared__ int s_gcnt[kMaxSpan][3][kWarps];  // the warps' counts per group of the item
  __shared__ int s_t, s_inst, s_last;
  __shared__ int s_live;  // the cooperative kernel's blocks other than 0 count out here
  __shared__ int s_spec;  // cooperative kernel: chunks of the next pass issued ahead (< 0: dropped)
  extern __shared__ unsigned char dyn_smem[];
  static_assert(sizeof(DevInst) % 8 == 0 && sizeof(DevInst) / 8 <= kThreads, "descriptor copy");
  static_assert(sizeof(Ctl) % 8 == 0 && sizeof(Ctl) / 8 <= kThreads, "control block copy");
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // kStages TMA stages and their barriers, 128-byte aligned (offset from the
  // array itself, so that the compiler keeps every stage access in the
  // shared address space)
  unsigned char* stage0 = dyn_smem + ((128u - (smem_u32(dyn_smem) & 127u)) & 127u);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(stage0 + kStages * kStageBytes);

  if (tid == 0) {
    s_inst = -1;
    for (int k = 0; k < kStages; ++k) mbar_init(smem_u32(&bars[k]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // Static prologue, which may overlap the end of the previous pass (launched
  // as a programmatic dependent): the descriptor and tensor maps of the
  // first work item's instance.  Nothing the previous pass writes is read
  // before griddepcontrol.wait.
  if (blockIdx.x < (unsigned)E.n_work) {
    const int inst = __ldg(E.tiles + blockIdx.x).x;
    if (tid < (int)(sizeof(DevInst) / 8))
      reinterpret_cast<long long*>(&sI)[tid] =
          __ldg(reinterpret_cast<const long long*>(E.insts + inst) + tid);
    __syncthreads();
    if (tid == 0) s_inst = inst;
    if (sI.tmaps && tid < M_COUNT) tmap_acquire(tmap(sI, tid));
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // the next pass may start its own prologue as soon as SMs free up
  asm volatile("griddepcontrol.launch_dependents;" :::);
  if (!kCoop && blockIdx.x == 0 && tid == 0) {
    const unsigned np = atomicAdd(E.npass, 1u) + 1u;
    if (kCond && E.cond != 0ull && (*((volatile int*)E.live) <= 0 || np >= E.pass_cap)) {
      cudaGraphSetConditional((cudaGraphConditionalHandle)E.cond, 0u);
    }
  }
  int seq = 0;  // chunks of the TMA pipeline consumed so far (same in all threads)
  int pre = 0;  // chunks of this pass already issued by the previous one (cooperative kernel)

  for (int pi = 0;; ++pi) {  // passes of the launch (one unless cooperative)
    bool again = false;        // the cooperative kernel runs another pass
    for (int first = 1;; first = 0) {
      __syncthreads();  // the previous item's shared state is no longer read
      // the first item of a CTA is its own index; later ones are claimed (the
      // cooperative kernel has one item per block)
      if (tid == 0) {
        s_t = first ? (int)blockIdx.x : (kCoop ? E.n_work : (int)gridDim.x + atomicAdd(E.queue, 1));
        s_spec = 0;
      }
      __syncthreads();
      const int t = s_t;
      if (t >= E.n_work) break;
      const int2 tr = __ldg(E.tiles + t);
      if (tr.x != s_inst || first) {
        // a new instance (or the first item, whose descriptor the prologue
        // loaded): read the snapshot of its state, the control block in one
        // round trip (the finalizer's shared copy sC is free here); after the
        // cooperative kernel's first pass sC already holds the state
        const bool fresh = tr.x != s_inst;
        __syncthreads();  // everyone compared against the old s_inst
        if ((!kCoop || pi == 0) && tid < (int)(sizeof(Ctl) / 8))
          reinterpret_cast<long long*>(&sC)[tid] =
              __ldcg(reinterpret_cast<const long long*>(E.ctl + tr.x) + tid);
        __syncthreads();
        const bool skip = sC.pass == P_NONE;
        // a finished instance's groups are skipped without loading its descriptor
        if (fresh && !skip && tid < (int)(sizeof(DevInst) / 8))
          reinterpret_cast<long long*>(&sI)[tid] =
              __ldg(reinterpret_cast<const long long*>(E.insts + tr.x) + tid);
        if (tid == 0) {
          sS.pass = sC.pass;
          sS.cur = sC.cur;
          sS.pcur = sC.pcur;
          sS.cg32 = sC.cg32;
          sS.first_cg = sC.first_cg;
          sS.dir = sC.dir;
          sS.gp32 = sC.gp32;
          sS.x32_live = sC.x32_live;
          sS.m = sC.m;
          sS.alpha = sC.alpha;
          sS.beta = sC.beta;
          s_inst = tr.x;
        }
        __syncthreads();
        if (fresh && !skip && sI.tmaps && tid < M_COUNT) tmap_acquire(tmap(sI, tid));
      }
      const DevInst& I = sI;
      const Snap& S = sS;
      // this pass's group partials (the cooperative kernel alternates two arrays)
      double* const part = I.part + (kCoop && (pi & 1) ? (long long)I.n_groups * kNRed : 0LL);
      if (S.pass == P_NONE) continue;
      if (!pass_supported<kFeat>(I, S)) {
        // launched with the wrong instantiation: report it and leave the
        // instance unfinished (the engine stops at its pass cap)
        if (tid == 0) atomicOr(E.err, 2);
        continue;
      }

      Acc acc;
#pragma unroll
      for (int k = 0; k < 4; ++k) acc.s[k] = 0.0;
      acc.c[0] = acc.c[1] = acc.c[2] = 0;
      FF ffs[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
      // the work item: groups [grp, grp_end) of the instance (the partition
      // into groups depends on the shape only; how many groups an item spans
      // is the launch's choice, and every group keeps its own sums, so the
      // results do not depend on it)
      const int grp = tr.y;
      const int grp_end = min(grp + max(1, min(I.span, kMaxSpan)), I.n_groups);
      // group sums: FP32 passes carry float-float accumulators (FP64 adds are
      // slow and long-latency on GB300), the others FP64
      auto ff_pass = [&]() {
        return (S.pass == P_CG_A || S.pass == P_CG_B || S.pass == P_CG_F || S.pass == P_CG_Z ||
                S.pass == P_RX_BUILD || S.pass == P_RCG)
                   ? S.cg32 != 0
                   : (S.pass != P_START && S.gp32 != 0);
      };
      // the end of a group: every thread stores its sums for the group in
      // shared memory (float-float pairs packed in 8 bytes for the FP32
      // passes, plain stores that the compiler need not order against the
      // stages) and each warp its counts, then the accumulators restart.  No
      // barrier and no reduction here (a barrier inside the item would take
      // away the slack between warps that hides latency); the item's end
      // reduces every group in the same fixed order as a group alone, so each
      // group's sums do not depend on the item that holds it.
      auto stash = [&](double* dst, int gi) {
        const bool ffred = ff_pass();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const double v = ffred ? __hiloint2double(__float_as_int(ffs[k].hi),
                                                    __float_as_int(ffs[k].lo))
                                 : acc.s[k];
          asm volatile("st.shared.f64 [%0], %1;" ::"r"(smem_u32(dst + k * kThreads + tid)), "d"(v));
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int c = __reduce_add_sync(FULL_MASK, acc.c[k]);
          if (lane == 0) s_gcnt[gi][k][warp] = c;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          acc.s[k] = 0.0;
          ffs[k] = FF{0.f, 0.f};
        }
        acc.c[0] = acc.c[1] = acc.c[2] = 0;
      };
      const bool tma = tma_pass<kFeat>(I, S);
      if ((kFeat & FEAT_EXT) != 0 && (S.pass == P_RCG || S.pass == P_RW)) {
        if constexpr ((kFeat & FEAT_EXT) != 0) {
          // compact passes of the explicit reduced system: the group is a
          // range of compact indices (one group per item)
          const long long lo = (long long)grp * S.m / I.n_groups;
          const long long hi = (long long)(grp + 1) * S.m / I.n_groups;
          const bool jac = I.opt.precond == PC_JACOBI;
          if (S.pass == P_RW) {
            if (S.cg32) rw_range<float>(I, S, lo, hi);
            else rw_range<double>(I, S, lo, hi);
          } else if (S.cg32) {
            if (jac) rcg_range<float, true>(I, S, lo, hi, acc, ffs);
            else rcg_range<float, false>(I, S, lo, hi, acc, ffs);
          } else {
            if (jac) rcg_range<double, true>(I, S, lo, hi, acc, ffs);
            else rcg_range<double, false>(I, S, lo, hi, acc, ffs);
          }
        }
      } else if ((kFeat & FEAT_EXT) != 0 && S.pass == P_RX_MAP) {
        if constexpr ((kFeat & FEAT_EXT) != 0) {
          const int t_lo = (int)((long long)grp * I.n_tiles / I.n_groups);
          const int t_hi = (int)((long long)(grp + 1) * I.n_tiles / I.n_groups);
          if (S.cg32) rx_map_group<float>(I, S, grp, t_lo, t_hi, s_scan);
          else rx_map_group<double>(I, S, grp, t_lo, t_hi, s_scan);
        }
      } else if (!tma) {
        // register sweep: a group is a range of whole tiles
        for (int g = grp; g < grp_end; ++g) {
          const int t_lo = (int)((long long)g * I.n_tiles / I.n_groups);
          const int t_hi = (int)((long long)(g + 1) * I.n_tiles / I.n_groups);
          for (int tile = t_lo; tile < t_hi; ++tile) {
            const int rest = tile / I.tiles_x;
            run_tile<kFeat>(I, S, (tile % I.tiles_x) * kTX, (rest % I.tiles_y) * kTY,
                            rest / I.tiles_y, acc, ffs, reinterpret_cast<float*>(stage0));
          }
          if (g + 1 < grp_end) stash(&s_stash[0][0], 0);
        }
      } else {
        // TMA pipeline: a group is a range of 8-row strips (4 per tile), cut
        // into chunks of up to `ch` rows that stay inside one tile and one
        // group; the next kStages-1 chunks are in flight while chunk k is
        // computed (the stage refilled at the top of an iteration is the one
        // computed in the previous iteration), across the groups of the item.
        // Nothing is in flight between work items.
        constexpr int kDepth = kStages - 1;
        static_assert(kDepth == 1 || kDepth == 2, "prefetch depth");
        const bool gp = gp_tma(I, S);
        const bool want_bits = (S.pass == P_CG_B && !S.first_cg) || S.pass == P_CG_F ||
                               (gp && S.pass == P_TRIAL);
        const int ch = chunk_rows(I, S, gp);
        const int rpw = ch / kWarps;
        // chunks that write to their stage (and have block barriers inside)
        const bool writes_stage =
            gp ? trial_alpha0(S)
               : ((S.pass == P_CG_B && !S.first_cg) || S.pass == P_GP_ALPHA || S.pass == P_TRIAL ||
                  (S.pass == P_CG_F && (!S.cg32 || I.opt.precond == PC_TILE)));
        Walk wk(I, grp, grp_end, ch);
        // the current chunk and the next two (h1, h2: they exist)
        Chunk c0 = wk.take(I);
        const bool hh1 = !wk.done();
        Chunk c1 = hh1 ? wk.take(I) : c0;
        const bool hh2 = !wk.done();
        Chunk c2 = hh2 ? wk.take(I) : c0;
        bool h1 = hh1, h2 = hh2;
        auto stage = [&](int q) { return stage0 + (q % kStages) * kStageBytes; };
        auto bar = [&](int q) { return smem_u32(&bars[q % kStages]); };
        if (tid == 0 && pre == 0) {
          // order earlier generic writes to the stages before the copies
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          issue_chunk<kFeat>(I, S, gp, c0, smem_u32(stage(seq)), bar(seq), want_bits);
          if (kDepth == 2 && h1)
            issue_chunk<kFeat>(I, S, gp, c1, smem_u32(stage(seq + 1)), bar(seq + 1), want_bits);
        }
        pre = 0;  // (the previous pass issued exactly these chunks)
        unsigned fbits[4] = {0u, 0u, 0u, 0u};
        for (;;) {
          if (tid == 0 && (kDepth == 2 ? h2 : h1)) {
            if (writes_stage)
              asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (kDepth == 2)
              issue_chunk<kFeat>(I, S, gp, c2, smem_u32(stage(seq + 2)), bar(seq + 2), want_bits);
            else
              issue_chunk<kFeat>(I, S, gp, c1, smem_u32(stage(seq + 1)), bar(seq + 1), want_bits);
          }
          unsigned char* st = stage(seq);
          const bool ok = mbar_wait(bar(seq), (seq / kStages) & 1);
          bool failed;
          if (ok && want_bits) stage_bits(st, c0.x0, rpw, gp, fbits);
          if (writes_stage) {
            // the chunk has a barrier inside: agree on the wait first
            failed = __syncthreads_or(!ok);
            if (!failed) run_chunk<kFeat>(I, S, gp, st, c0, fbits, acc, ffs);
            __syncthreads();  // the stage may be refilled
          } else {
            // one barrier per chunk: every thread is done with the stage (which
            // may then be refilled) and no bounded wait gave up
            if (ok) run_chunk<kFeat>(I, S, gp, st, c0, fbits, acc, ffs);
            failed = __syncthreads_or(!ok);
          }
          if (c0.rows & kEndG0) stash(&s_stash[0][0], 0);
          if (failed) {
            // a copy never completed: record it, give the copies still in
            // flight a bounded chance to land, and leave; the engine's loop
            // then ends on its pass cap and the host reports the error
            if (tid == 0) {
              atomicOr(E.err, 1);
              if (h1) mbar_wait(bar(seq + 1), ((seq + 1) / kStages) & 1);
              if (kDepth == 2 && h2) mbar_wait(bar(seq + 2), ((seq + 2) / kStages) & 1);
            }
            return;
          }
          seq++;
          if (!h1) break;
          c0 = c1;
          c1 = c2;
          h1 = h2;
          h2 = !wk.done();
          if (h2) c2 = wk.take(I);
        }
      }
      // the item's end: the last group's sums go to the first stage, past the
      // zebra sweep's line buffer (a slow warp may still read that buffer; no
      // copy is in flight, and every thread has passed the last chunk's
      // barrier);
      // warp w reduces sum w & 3 of group w >> 2 (lane j adds the threads j,
      // j+32, ..., then a butterfly; float-float for the FP32 passes) and
      // writes it, with the group's counts summed in warp order, to the
      // group's partial slots (kNRed per group: 4 sums, 3 counts, a spare;
      // stored slot-major, [k][group], so that the finalizer's loads of one
      // slot over the groups are contiguous); thread 0 then advances the
      // instance's arrival counter by the item's groups
      const int nspan = grp_end - grp;
      constexpr int kScrBytes = kTY * kTX * (int)sizeof(float);  // the register sweep's line buffer
      double* last_sums = reinterpret_cast<double*>(stage0 + kScrBytes);
      stash(last_sums, nspan - 1);
      __syncthreads();
      {
        static_assert(kWarps == 4 * kMaxSpan, "one warp per sum of each group of an item");
        static_assert(kScrBytes + 4 * kThreads * 8 <= kStageBytes, "last group's sums in the first stage");
        const int gi = warp >> 2, k = warp & 3;
        if (gi < nspan) {
          const int ns = n_sums(S.pass, S.first_cg, S.gp32);
          const double* src = (gi == nspan - 1 ? last_sums : &s_stash[0][0]) + k * kThreads;
          double v = 0.0;
          if (k < ns) {
            if (ff_pass()) {
              auto ld = [&](int t) {
                const double d = src[t];
                return FF{__int_as_float(__double2hiint(d)), __int_as_float(__double2loint(d))};
              };
              FF a = ld(lane);
              for (int j = 1; j < kWarps; ++j) a = ff_add(a, ld(lane + 32 * j));
#pragma unroll
              for (int off = 16; off > 0; off >>= 1)
                a = ff_add(a, FF{__shfl_xor_sync(FULL_MASK, a.hi, off),
                                 __shfl_xor_sync(FULL_MASK, a.lo, off)});
              v = ff_val(a);
            } else {
              v = src[lane];
              for (int j = 1; j < kWarps; ++j) v += src[lane + 32 * j];
#pragma unroll
              for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL_MASK, v, off);
            }
          }
          double* P = part + grp + gi;
          const long long ng = I.n_groups;
          if (lane == 0) {
            P[k * ng] = v;
          } else if (lane == 1) {
            // the counts as integers in the slots' bits (k == 3: the spare)
            long long c = 0;
            if (k < 3)
              for (int w = 0; w < kWarps; ++w) c += s_gcnt[gi][k][w];
            P[(4 + k) * ng] = __longlong_as_double(c);
          }
        }
      }
      __syncthreads();
      if (tid == 0) {
        if (kCoop) {
          // every block reduces: wait for all of them (the grid's arrivals
          // accumulate over the launch's passes)
          if (grid_barrier(E.gbar, (unsigned)(pi + 1) * gridDim.x)) {
            s_last = 1;
          } else {
            atomicOr(E.err, 4);
            s_last = -1;
          }
        } else {
          __threadfence();  // the block's partial writes (ordered by the barrier) before the arrival
          const unsigned prev = atomicAdd(&E.ctl[tr.x].arrive, (unsigned)nspan);
          s_last = (prev + (unsigned)nspan == (unsigned)I.n_groups);
        }
      }
      __syncthreads();
      if (s_last < 0) return;  // the grid barrier gave up: nothing is in flight
      if (!s_last) continue;

      // last group of this instance: reduce the group slots in a fixed order
      // that depends on the shape only.  Warp k < 7 takes slot k: lane j loads
      // the slots of groups j, j+32, ... (all loads in flight at once; each
      // load of the warp reads 32 consecutive groups) and adds them in that
      // order, then a butterfly; the sums in FP64, the counts (integers in the
      // slots' bits) in integer arithmetic.  The last warp reads the control
      // block meanwhile (the cooperative kernel: issues the guessed next
      // pass's first chunks).  FP64 arithmetic is slow on GB300:
      // one FP64 add per group and slot, none for the counts.
      if (!kCoop && tid == 0) __threadfence();  // (the grid barrier has fenced)
      __syncthreads();
      if (kCoop && warp == kWarps - 1 && lane == 0 && S.pass == P_CG_F &&
          I.opt.precond != PC_TILE) {
        // cooperative kernel: the next pass's first chunks, issued now on the
        // guess that a fused CG step is followed by another (most are).  The
        // copies read what this pass wrote, which the grid barrier has
        // published, and none of the step's scalars, so their latency hides
        // behind this reduction and the state machine; a wrong guess only
        // lets them land and drops them.
        Snap nx = S;
        nx.pcur ^= 1;
        Walk w2(I, grp, grp_end, chunk_rows(I, nx, false));
        asm volatile("fence.proxy.async.global;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        int n = 0;
        for (; n < kStages - 1 && !w2.done(); ++n) {
          const int q = (seq + n) % kStages;
          issue_chunk<kFeat>(I, nx, false, w2.take(I), smem_u32(stage0 + q * kStageBytes),
                             smem_u32(&bars[q]), true);
        }
        s_spec = n;
      }
      long long* cg = reinterpret_cast<long long*>(E.ctl + tr.x);
      long long* cs = reinterpret_cast<long long*>(&sC);
      {
        static_assert(kWarps >= kNRed, "one warp per reduced slot and one for the control block");
        constexpr int kPer = (kMaxGroups + 31) / 32;
        if (warp == kWarps - 1) {
          // (the cooperative kernel's own copy is the state: block 0 may be
          // rewriting the global one already)
          if (!kCoop)
            for (int j = lane; j < (int)(sizeof(Ctl) / 8); j += 32) cs[j] = __ldcg(cg + j);
        } else if (warp < kNRed - 1) {
          const int k = warp;
          const double* P0 = part + (long long)k * I.n_groups;
          double v[kPer];
#pragma unroll
          for (int q = 0; q < kPer; ++q) {
            const int gi = lane + 32 * q;
            v[q] = gi < I.n_groups ? __ldcg(P0 + gi) : 0.0;
          }
          if (k < 4) {
            double t = v[0];
#pragma unroll
            for (int q = 1; q < kPer; ++q) t += v[q];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(FULL_MASK, t, off);
            if (lane == 0) s_red[k] = t;
          } else {
            int c = 0;  // at most n < 2^31 points
#pragma unroll
            for (int q = 0; q < kPer; ++q) c += (int)__double_as_longlong(v[q]);
            c = __reduce_add_sync(FULL_MASK, c);
            if (lane == 0) s_red[k] = (double)c;
          }
        }
      }
      __syncthreads();
      if ((kFeat & FEAT_EXT) != 0 && S.pass == P_RX_COUNT) {
        // the groups' offsets in the compact numbering (exclusive prefix sum
        // of their free counts, two groups per thread)
        static_assert(kMaxGroups <= 2 * kThreads, "two groups per thread");
        int t0, t1;
        const double* P0 = I.part + 4LL * I.n_groups;  // slot 4: the free counts
        const int c0 = tid < I.n_groups ? (int)__double_as_longlong(__ldcg(P0 + tid)) : 0;
        const int o0 = cta_excl_scan(c0, s_scan, t0);
        const int g1 = tid + kThreads;
        const int c1 = g1 < I.n_groups ? (int)__double_as_longlong(__ldcg(P0 + g1)) : 0;
        const int o1 = cta_excl_scan(c1, s_scan, t1);
        if (tid < I.n_groups) I.goff[tid] = o0;
        if (g1 < I.n_groups) I.goff[g1] = t0 + o1;
      }
      // the state machine runs on the shared copy of the control block (one
      // round trip in, one out, instead of dependent global accesses)
      if (tid == 0) {
        s_red[kNRed - 1] = 0.0;
        sC.arrive = 0u;
        finalize(I, sC, s_red, (!kCoop || blockIdx.x == 0) ? E.live : &s_live);
        if (kCoop && blockIdx.x == 0) atomicAdd(E.npass, 1u);
        if (kCoop && s_spec > 0) {
          // the guess holds when another fused step of this block's item
          // follows on the other buffers; else the issued chunks land and
          // their stages count as consumed
          const bool next = sC.pass != P_NONE && !sC.hold && (unsigned)(pi + 1) < E.pass_cap;
          if (!(next && sC.pass == P_CG_F && sC.pcur == (S.pcur ^ 1) && sC.cur == S.cur &&
                sC.cg32 == S.cg32)) {
            bool ok = true;
            for (int n = 0; n < s_spec; ++n)
              ok = mbar_wait(smem_u32(&bars[(seq + n) % kStages]), ((seq + n) / kStages) & 1) && ok;
            if (!ok) atomicOr(E.err, 1);
            s_spec = -s_spec;
          }
        }
      }
      __syncthreads();
      if ((!kCoop || blockIdx.x == 0) && tid < (int)(sizeof(Ctl) / 8)) __stcg(cg + tid, cs[tid]);
      if (kCoop) {
        // every block holds the same next state: run it, unless the instance
        // is done, the state is held (a standalone launch) or the pass cap is
        // reached
        again = sC.pass != P_NONE && !sC.hold && (unsigned)(pi + 1) < E.pass_cap;
        const int sp = s_spec;
        if (sp < 0) seq -= sp;  // dropped chunks
        pre = sp > 0 ? sp : 0;
        break;
      }
    }
    if (!again) break;
  }

  // the last CTA to leave resets the queue for the next launch
  if (tid == 0) {
    if (atomicAdd(E.exits, 1u) == gridDim.x - 1) {
      *E.queue = 0;
      *E.exits = 0u;
      if (kCoop) *E.gbar = 0u;
      __threadfence();
    }
  }
}

#if GPCG_COOP
template <int kFeat>
__global__ void __launch_bounds__(kThreads, kMinBlocks) pass_kernel_coop(EngineArgs E) {
  pass_body<false, kFeat>(E);
}
#else
template <bool kCond, int kFeat>
__global__ void __launch_bounds__(kThreads, kMinBlocks) pass_kernel(EngineArgs E) {
  pass_body<kCond, kFeat>(E);
}
#endif

}  // namespace
}  // namespace gpcg
