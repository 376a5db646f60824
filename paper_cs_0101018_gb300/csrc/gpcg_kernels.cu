// gpcg_kernels.cu -- device side of the GB300 GPCG engine: the default
// instantiation of the pass kernel (pass_engine.cuh), the standalone masked
// product, the set-up kernels and the host-side launch wrappers.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "pass_engine.cuh"

namespace gpcg {

// -------------------------------------------- standalone masked product --
//
// y = Z Z' A Z Z' p and <p_F, y> (Eq. cg2) for one 2-D instance, the
// operation of gpcg_masked_spmv: p (zero outside the free set) and the bands
// stream through shared memory with TMA in 64 x c chunks (c = 16 rows FP32,
// 8 FP64), four stages deep, three CTAs per SM; CTAs take chunks
// round-robin.  Each CTA adds its terms in a fixed order; the last CTA to
// finish adds the CTA partials in index order, so the sum does not depend on
// the schedule.  Stage layout: P (64+2h) x (c+2) from (x0-h, y-1) | D 64 x c |
// CX (64+h) x c from x0-h | CY 64 x (c+1) from y-1 -- the boxes of the fused
// CG pass's maps (p[0]).
constexpr int kMsStages = 4;
template <class T>
struct GeoMS {
  using G = GeoF<T>;
  static constexpr int H = G::H, CH = G::CH, BW = G::BW;
  static constexpr int OFF_P = 0, OFF_D = G::SZ_H;
  static constexpr int OFF_CX = OFF_D + 64 * CH * (int)sizeof(T);
  static constexpr int OFF_CY = OFF_CX + align128((64 + H) * CH * (int)sizeof(T));
  static constexpr int OFF_M = OFF_CY + align128(64 * (CH + 1) * (int)sizeof(T));  // mask box
  static constexpr int END = OFF_M + kMaskBox;
  static constexpr unsigned TX =
      ((CH + 2) * BW + 64 * CH + (64 + H) * CH + 64 * (CH + 1)) * sizeof(T) + kMaskBox;
};
constexpr int kMsStage = GeoMS<float>::END > GeoMS<double>::END ? GeoMS<float>::END : GeoMS<double>::END;
constexpr int kMsCtasPerSm = 3;  // the launch bounds below
constexpr int kMsSmem = kMsStages * kMsStage + 128 + 8 * kMsStages;

struct MsArgs {
  const void* tmaps;       // the instance's maps (CG_B boxes of p[0] and the bands)
  int mask;                // free-set words: mask[0] or mask[1] (map M_MASK0 + mask)
  void* y;                 // output, padded layout
  double* part;            // [gridDim.x] CTA partials
  unsigned* counter;       // CTAs done (the last one resets it)
  double* result;          // <p_F, y>
  int* err;                // a bounded wait gave up
  int nx, ny, px, mw, tiles_x, n_chunks;
};

template <class T>
__global__ void __launch_bounds__(kThreads, kMsCtasPerSm) mspmv_kernel(MsArgs A) {
  using G = GeoMS<T>;
  constexpr int RPW = G::CH / kWarps;
  extern __shared__ unsigned char dyn_smem[];
  __shared__ double s_part[kWarps];
  __shared__ int s_last;
  unsigned char* st0 = dyn_smem + ((128u - (smem_u32(dyn_smem) & 127u)) & 127u);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(st0 + kMsStages * kMsStage);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const char* maps = reinterpret_cast<const char*>(A.tmaps);
  constexpr int mb = sizeof(T) == 4 ? M32_RH0 : M64_RH0;
  const void* mP = maps + 128 * (mb + (M32_FPH0 - M32_RH0));
  const void* mD = maps + 128 * (mb + (M32_FD - M32_RH0));
  const void* mX = maps + 128 * (mb + (M32_FCX - M32_RH0));
  const void* mY = maps + 128 * (mb + (M32_FCY - M32_RH0));
  const void* mM = maps + 128 * (M_MASK0 + A.mask);
  if (tid == 0) {
    for (int k = 0; k < kMsStages; ++k) mbar_init(smem_u32(&bars[k]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    tmap_acquire(mP);
    tmap_acquire(mD);
    tmap_acquire(mX);
    tmap_acquire(mY);
    tmap_acquire(mM);
  }
  __syncthreads();
  const int G0 = (int)gridDim.x;
  const int my = (A.n_chunks - (int)blockIdx.x + G0 - 1) / G0;  // chunks of this CTA
  auto coords = [&](int k, int& x0, int& yc) {
    const int c = (int)blockIdx.x + k * G0;
    const int cy = c / A.tiles_x;
    x0 = (c - cy * A.tiles_x) * kTX;
    yc = cy * G::CH;
  };
  auto issue = [&](int k) {
    int x0, yc;
    coords(k, x0, yc);
    const unsigned st = smem_u32(st0 + (k % kMsStages) * kMsStage);
    const unsigned bar = smem_u32(&bars[k % kMsStages]);
    mbar_expect(bar, G::TX);
    tma_load2d(st + G::OFF_P, mP, x0 - G::H, yc - 1, bar);
    tma_load2d(st + G::OFF_D, mD, x0, yc, bar);
    tma_load2d(st + G::OFF_CX, mX, x0 - G::H, yc, bar);
    tma_load2d(st + G::OFF_CY, mY, x0, yc - 1, bar);
    tma_load2d(st + G::OFF_M, mM, (x0 >> 5) & ~3, yc, bar);
  };
  if (tid == 0)
    for (int k = 0; k < kMsStages - 1 && k < my; ++k) issue(k);
  // launched as a programmatic dependent of the previous product in the
  // stream (a different problem's): the next launch may start its own
  // prologue as this one's CTAs drain.  The operands and y are this launch's
  // own; only the CTA partials and the counter wait for the previous launch.
  asm volatile("griddepcontrol.launch_dependents;" :::);
  T sum = T(0);  // this thread's terms of the current chunk
  FF ffs{0.f, 0.f};
  double dsum = 0.0;
  T* y = reinterpret_cast<T*>(A.y);
  for (int k = 0; k < my; ++k) {
    if (tid == 0 && k + kMsStages - 1 < my) issue(k + kMsStages - 1);
    const unsigned char* st = st0 + (k % kMsStages) * kMsStage;
    const bool ok = mbar_wait(smem_u32(&bars[k % kMsStages]), (k / kMsStages) & 1);
    if (ok) {
      int x0, yc;
      coords(k, x0, yc);
      const T* P = reinterpret_cast<const T*>(st + G::OFF_P);
      const T* D = reinterpret_cast<const T*>(st + G::OFF_D);
      const T* CX = reinterpret_cast<const T*>(st + G::OFF_CX);
      const T* CY = reinterpret_cast<const T*>(st + G::OFF_CY);
      const int c = 2 * lane, e0 = x0 + c;
      const bool v0 = e0 < A.nx, v1 = e0 + 1 < A.nx;
      const unsigned* M = reinterpret_cast<const unsigned*>(st + G::OFF_M) + ((x0 >> 5) & 3);
      unsigned fb[RPW];
#pragma unroll
      for (int q = 0; q < RPW; ++q) fb[q] = M[(warp * RPW + q) * 4 + (lane >> 4)] >> (c & 31);
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        const int ry = warp * RPW + q;
        if (yc + ry >= A.ny || !v0) break;
        const T* Pr = P + (ry + 1) * G::BW + G::H + c;
        const T* Xr = CX + ry * (64 + G::H) + G::H + c;
        const T vc0 = Pr[0], vc1 = Pr[1];
        // diag, west, east, south, north (the order of the register sweep)
        T a0 = D[ry * 64 + c] * vc0;
        a0 = fma(Xr[-1], Pr[-1], a0);
        a0 = fma(Xr[0], vc1, a0);
        a0 = fma(CY[ry * 64 + c], Pr[-G::BW], a0);
        a0 = fma(CY[(ry + 1) * 64 + c], Pr[G::BW], a0);
        T a1 = D[ry * 64 + c + 1] * vc1;
        a1 = fma(Xr[0], vc0, a1);
        a1 = fma(Xr[1], Pr[2], a1);
        a1 = fma(CY[ry * 64 + c + 1], Pr[1 - G::BW], a1);
        a1 = fma(CY[(ry + 1) * 64 + c + 1], Pr[G::BW + 1], a1);
        a0 = (fb[q] & 1u) ? a0 : T(0);
        a1 = (fb[q] & 2u) ? a1 : T(0);
        st2(y, (long long)(yc + ry) * A.px + e0, v0, v1, a0, a1);
        sum = fma(vc0, a0, fma(vc1, a1, sum));
      }
      if (sizeof(T) == 4) ff_acc(ffs, (float)sum);
      else dsum += (double)sum;
      sum = T(0);
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(A.err, 1);
        for (int j = 1; j < kMsStages && k + j < my; ++j)
          mbar_wait(smem_u32(&bars[(k + j) % kMsStages]), ((k + j) / kMsStages) & 1);
      }
      return;
    }
  }
  // fixed-order CTA sum, then the last CTA adds the CTA partials in order
  // (after the previous launch in the stream has finished with its own)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  double v = sizeof(T) == 4 ? ff_val(ffs) : dsum;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL_MASK, v, off);
  if (lane == 0) s_part[warp] = v;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += s_part[w];
    A.part[blockIdx.x] = t;
    __threadfence();
    s_last = atomicAdd(A.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  if (tid == 0) __threadfence();
  __syncthreads();
  double t = 0.0;
  for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(A.part + b);
  if (warp == 0) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(FULL_MASK, t, off);
    if (lane == 0) {
      *A.result = t;
      *A.counter = 0u;
    }
  }
}

// Grid of the standalone masked product: the resident CTAs of the GPU, at
// most one per chunk.
// The shared-memory attribute and the occupancy are per device: each device
// gets its own entry, set once under a lock (the server's workers and the
// caller's threads may reach these functions at the same time).
constexpr int kMaxDevices = 64;

static int device_now() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = 0;
  return dev;
}

static int ms_grid(int n_chunks) {
  static std::mutex mu;
  static int cached[kMaxDevices] = {0};
  const int dev = device_now();
  int c;
  {
    std::lock_guard<std::mutex> g(mu);
    if (!cached[dev]) {
      int sms = 0, per = 0;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaFuncSetAttribute(mspmv_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kMsSmem);
      cudaFuncSetAttribute(mspmv_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kMsSmem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, mspmv_kernel<float>, kThreads, kMsSmem);
      cached[dev] = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
    }
    c = cached[dev];
  }
  return n_chunks < c ? (n_chunks > 0 ? n_chunks : 1) : c;
}

// Launch the standalone masked product of a 2-D instance whose CG maps are
// valid, with free-set words mask[mask]; `part` holds at least ms_max_ctas()
// doubles.
// With pdl the launch is a programmatic dependent of the stream's previous
// kernel (its CTAs may start while that kernel's last CTAs run); the caller
// guarantees that the previous kernel writes nothing this one reads.
cudaError_t launch_mspmv(const DevInst& I, bool f32, int mask, void* y, double* part,
                         unsigned* counter, double* result, int* err, cudaStream_t s, bool pdl) {
  const int ch = f32 ? GeoMS<float>::CH : GeoMS<double>::CH;
  MsArgs A{I.tmaps, mask, y, part, counter, result, err,
           I.nx, I.ny, I.px, I.mw, I.tiles_x, I.tiles_x * ((I.ny + ch - 1) / ch)};
  // in a stream of products each launch takes one CTA per SM (a third of
  // what the GPU holds at once): its CTAs wait for the previous launch only
  // before their CTA sums, so up to three consecutive products stream at the
  // same time and the copies of one cover the start and the tail of another
  int grid = ms_grid(A.n_chunks);
  if (pdl) grid = std::max(1, std::min(grid, ms_grid(1 << 30) / kMsCtasPerSm));
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kMsSmem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  if (f32) return cudaLaunchKernelEx(&cfg, mspmv_kernel<float>, A);
  return cudaLaunchKernelEx(&cfg, mspmv_kernel<double>, A);
}

int ms_max_ctas() { return ms_grid(1 << 30); }

// p restricted to the free set into pm (padded layout) and the free-set words.
template <class T>
__global__ void mspmv_setup_kernel(DevInst I, const uint8_t* __restrict__ fm,
                                   const double* __restrict__ pv, unsigned* mask, T* pm) {
  const long long rows = (long long)I.ny * I.nz;
  const long long total = rows * I.mw;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long row = t / I.mw;
    const int wcol = (int)(t % I.mw);
    const int iy = (int)(row % I.ny), iz = (int)(row / I.ny);
    unsigned word = 0;
    for (int b = 0; b < 32; ++b) {
      const int ix = wcol * 32 + b;
      if (ix >= I.px) break;
      const long long i = pidx(I, iy, iz, ix);
      T v = T(0);
      if (ix < I.nx) {
        const long long j = ((long long)iz * I.ny + iy) * I.nx + ix;
        if (fm[j]) {
          word |= 1u << b;
          v = (T)pv[j];
        }
      }
      pm[i] = v;
    }
    mask[t] = word;
  }
}

// ------------------------------------------------------- set-up kernels --

// Zero the couplings of the last point along each axis, fill missing bounds
// and check the input; flags: 1 = non-finite b / coupling / NaN bound,
// 2 = diag <= 0 or non-finite, 4 = empty box (l > u, l = +inf, u = -inf).
__global__ void prep_kernel(DevInst I, double* cx, double* cy, double* cz, double* l, double* u,
                            int fill_l, int fill_u, int* flags) {
  const long long total = (long long)I.nx * I.ny * I.nz;
  int f = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(t % I.nx);
    const long long r = t / I.nx;
    const int iy = (int)(r % I.ny);
    const int iz = (int)(r / I.ny);
    const long long i = pidx(I, iy, iz, ix);
    if (fill_l) l[i] = -INFINITY;
    if (fill_u) u[i] = INFINITY;
    if (ix == I.nx - 1) cx[i] = 0.0;
    if (iy == I.ny - 1) cy[i] = 0.0;
    if (I.dim == 3 && iz == I.nz - 1) cz[i] = 0.0;
    const double d = I.diag[i], b = I.b[i], lv = l[i], uv = u[i];
    if (!isfinite(b) || !isfinite(cx[i]) || !isfinite(cy[i]) ||
        (I.dim == 3 && !isfinite(cz[i])) || isnan(lv) || isnan(uv))
      f |= 1;
    if (!(d > 0.0) || !isfinite(d)) f |= 2;
    if (lv > uv || lv == INFINITY || uv == -INFINITY) f |= 4;
  }
  if (f) atomicOr(flags, f);
}

__global__ void to_float_kernel(const double* __restrict__ src, float* dst, long long count) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
       t += (long long)gridDim.x * blockDim.x)
    dst[t] = (float)src[t];
}

// 1/diag in FP64 and (rounded from it) FP32; pad columns (diag 0) get 0.
__global__ void recip_kernel(const double* __restrict__ d, double* out64, float* out32,
                             long long count) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
       t += (long long)gridDim.x * blockDim.x) {
    const double v = d[t] != 0.0 ? 1.0 / d[t] : 0.0;
    if (out64) out64[t] = v;
    if (out32) out32[t] = (float)v;
  }
}

// Byte mask (unpadded, one byte per point) -> bit mask; and a value array
// (unpadded FP64) -> -value on the free set in T (used by the masked
// product entry point: p = -r + 0 * p_old with r = -p_F).
template <class T>
__global__ void spmv_setup_kernel(DevInst I, const uint8_t* __restrict__ fm,
                                  const double* __restrict__ pv, unsigned* mask, T* r, T* pold) {
  const long long rows = (long long)I.ny * I.nz;
  const long long total = rows * I.mw;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long row = t / I.mw;
    const int wcol = (int)(t % I.mw);
    const int iy = (int)(row % I.ny), iz = (int)(row / I.ny);
    unsigned word = 0;
    for (int b = 0; b < 32; ++b) {
      const int ix = wcol * 32 + b;
      if (ix >= I.px) break;
      const long long i = pidx(I, iy, iz, ix);
      T rv = T(0);
      if (ix < I.nx) {
        const long long j = ((long long)iz * I.ny + iy) * I.nx + ix;
        if (fm[j]) {
          word |= 1u << b;
          rv = (T)(-pv[j]);
        }
      }
      r[i] = rv;
      pold[i] = T(0);
    }
    mask[t] = word;
  }
}

template __global__ void spmv_setup_kernel<double>(DevInst, const uint8_t*, const double*,
                                                   unsigned*, double*, double*);
template __global__ void spmv_setup_kernel<float>(DevInst, const uint8_t*, const double*,
                                                  unsigned*, float*, float*);

// Padded T array -> unpadded FP64 array.
template <class T>
__global__ void unpad_kernel(DevInst I, const T* __restrict__ src, double* dst) {
  const long long total = (long long)I.nx * I.ny * I.nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(t % I.nx);
    const long long r = t / I.nx;
    dst[t] = (double)src[pidx(I, (int)(r % I.ny), (int)(r / I.ny), ix)];
  }
}

template __global__ void unpad_kernel<double>(DevInst, const double*, double*);
template __global__ void unpad_kernel<float>(DevInst, const float*, double*);

// ---------------------------------------------------------- host wrappers --

namespace {  // the header's namespace
template __global__ void pass_kernel<true, 0>(EngineArgs);
template __global__ void pass_kernel<false, 0>(EngineArgs);
}  // namespace

// the instantiations with optional passes (their own translation units)
const void* pass_kernel_ptr_tile(bool cond);
const void* pass_kernel_ptr_rx(bool cond);
const void* pass_kernel_ptr_f64(bool cond);
const void* pass_kernel_ptr_3d(bool cond);
const void* pass_kernel_coop_ptr_a(int feat);
const void* pass_kernel_coop_ptr_b(int feat);

// The pass kernel for a feature set (0, FEAT_TILE, FEAT_EXT or FEAT_F64); `cond`: the
// instantiation that may clear a WHILE graph's condition.
const void* pass_kernel_ptr(bool cond, int feat) {
  if (feat == FEAT_TILE) return pass_kernel_ptr_tile(cond);
  if (feat == FEAT_EXT) return pass_kernel_ptr_rx(cond);
  if (feat == FEAT_F64) return pass_kernel_ptr_f64(cond);
  if (feat == FEAT_3D) return pass_kernel_ptr_3d(cond);
  return cond ? (const void*)pass_kernel<true, 0> : (const void*)pass_kernel<false, 0>;
}

// The cooperative pass kernel for a feature set (nullptr for the explicit
// reduced system, whose passes exchange group offsets through the finalizer).
const void* pass_kernel_coop_ptr(int feat) {
  if (feat == 0 || feat == FEAT_3D) return pass_kernel_coop_ptr_a(feat);
  if (feat == FEAT_F64 || feat == FEAT_TILE) return pass_kernel_coop_ptr_b(feat);
  return nullptr;
}

int pass_grid(int n_work) {
  // persistent grid: the resident CTAs of the whole GPU, at most one per item
  static std::mutex mu;
  static int cached[kMaxDevices] = {0};
  const int dev = device_now();
  int c;
  {
    std::lock_guard<std::mutex> g(mu);
    if (!cached[dev]) {
      int sms = 0, per = 0;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      for (int feat : {0, (int)FEAT_TILE, (int)FEAT_EXT, (int)FEAT_F64, (int)FEAT_3D}) {
        for (bool cond : {true, false})
          cudaFuncSetAttribute(pass_kernel_ptr(cond, feat),
                               cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmem);
        if (const void* k = pass_kernel_coop_ptr(feat))
          cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmem);
      }
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pass_kernel<false, 0>, kThreads,
                                                    kDynSmem);
      cached[dev] = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
    }
    c = cached[dev];
  }
  return n_work < c ? (n_work > 0 ? n_work : 1) : c;
}

cudaError_t launch_pass(const EngineArgs& E, int n_blocks, cudaStream_t s, int feat) {
  pass_grid(1);  // sets the shared-memory attribute once
  EngineArgs a = E;
  void* args[] = {&a};
  return cudaLaunchKernel(pass_kernel_ptr(false, feat), dim3(n_blocks), dim3(kThreads), args,
                          kDynSmem, s);
}

// One cooperative pass kernel at a time per device: two whose blocks were
// resident only in part could each wait at its grid barrier for blocks that
// the other keeps from running.  The caller holds this lock from the launch
// until the kernel has finished.
std::mutex& coop_mutex() {
  static std::mutex mu[kMaxDevices];
  return mu[device_now()];
}

// Every pass of one solve in one cooperative launch of n_blocks blocks (one
// work item each).  Fails without launching when the blocks cannot all be
// resident at once (cudaErrorCooperativeLaunchTooLarge) or the feature set
// has no cooperative kernel; the caller then runs the passes as launches.
cudaError_t launch_pass_coop(const EngineArgs& E, int n_blocks, cudaStream_t s, int feat) {
  pass_grid(1);  // sets the shared-memory attribute once
  const void* k = pass_kernel_coop_ptr(feat);
  if (k == nullptr || n_blocks != E.n_work) return cudaErrorInvalidValue;
  EngineArgs a = E;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel(k, dim3(n_blocks), dim3(kThreads), args, kDynSmem, s);
}

static int grid_for(long long work) {
  long long b = (work + 255) / 256;
  if (b < 1) b = 1;
  if (b > 8192) b = 8192;
  return (int)b;
}

cudaError_t launch_prep(const DevInst& I, double* cx, double* cy, double* cz, double* l, double* u,
                        int fill_l, int fill_u, int* flags, cudaStream_t s) {
  prep_kernel<<<grid_for(I.n), 256, 0, s>>>(I, cx, cy, cz, l, u, fill_l, fill_u, flags);
  return cudaGetLastError();
}

cudaError_t launch_to_float(const double* src, float* dst, long long count, cudaStream_t s) {
  to_float_kernel<<<grid_for(count), 256, 0, s>>>(src, dst, count);
  return cudaGetLastError();
}

cudaError_t launch_recip(const double* d, double* out64, float* out32, long long count,
                         cudaStream_t s) {
  recip_kernel<<<grid_for(count), 256, 0, s>>>(d, out64, out32, count);
  return cudaGetLastError();
}

cudaError_t launch_spmv_setup(const DevInst& I, const uint8_t* fm, const double* pv,
                              unsigned* mask, void* r, void* pold, bool f32, cudaStream_t s) {
  const long long work = (long long)I.ny * I.nz * I.mw;
  if (f32)
    spmv_setup_kernel<float><<<grid_for(work), 256, 0, s>>>(I, fm, pv, mask, (float*)r,
                                                            (float*)pold);
  else
    spmv_setup_kernel<double><<<grid_for(work), 256, 0, s>>>(I, fm, pv, mask, (double*)r,
                                                             (double*)pold);
  return cudaGetLastError();
}

cudaError_t launch_mspmv_setup(const DevInst& I, const uint8_t* fm, const double* pv,
                               unsigned* mask, void* pm, bool f32, cudaStream_t s) {
  const long long words = (long long)I.ny * I.nz * I.mw;
  const int grid = (int)std::min<long long>((words + 255) / 256, 4096);
  if (f32) mspmv_setup_kernel<float><<<grid, 256, 0, s>>>(I, fm, pv, mask, (float*)pm);
  else mspmv_setup_kernel<double><<<grid, 256, 0, s>>>(I, fm, pv, mask, (double*)pm);
  return cudaGetLastError();
}

cudaError_t launch_unpad(const DevInst& I, const void* src, bool f32, double* dst,
                         cudaStream_t s) {
  if (f32)
    unpad_kernel<float><<<grid_for(I.n), 256, 0, s>>>(I, (const float*)src, dst);
  else
    unpad_kernel<double><<<grid_for(I.n), 256, 0, s>>>(I, (const double*)src, dst);
  return cudaGetLastError();
}

}  // namespace gpcg
