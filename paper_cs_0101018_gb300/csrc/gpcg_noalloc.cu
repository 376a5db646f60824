// gpcg_noalloc.cu -- the masked stencil product y = Z Z' A Z Z' p with
// <p_F, y_F>, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: processes whose device memory is owned
// entirely by their own pool allocator, and latency-critical loops that cannot
// take the implicit device synchronisation that cudaMalloc / cudaFree may
// cause.  This entry point allocates nothing.  The caller passes every input
// and output; the only scratch (one partial sum per 64x32 tile, a completion
// counter and the final sum) lives in a file-scope __device__ array of fixed
// size, which every GPU that loads the library keeps until the process exits.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/gpcg.h"

namespace gpcg {
void set_last_error(const char* msg);  // gpcg_last_error() reports it
}

namespace {

constexpr int kTX = 64, kTY = 32, kThreads = 256;
constexpr int kMaxTiles = 4096;  // largest problem: 4096 tiles of 64x32 points (8.4e6 in 2-D)
constexpr size_t kCounterOff = sizeof(double) * kMaxTiles;
constexpr size_t kResultOff = kCounterOff + 256;
constexpr size_t kScratchBytes = kResultOff + 256;

// Scratch shared by every call on a device: the tile partials, the counter of
// finished tiles (zeroed by each call before its kernel) and the reduced sum.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct Geo {
  int dim, nx, ny, nz, tiles_x, tiles_y, n_tiles;
};

// One CTA per tile; each thread takes two columns and four rows of the tile.
// Rows of non-free points are zero and non-free points contribute nothing, so
// the result is the reduced Hessian of Eq. cg2 applied to the free part of p.
__global__ void __launch_bounds__(kThreads) noalloc_masked_spmv(
    Geo G, const double* __restrict__ diag, const double* __restrict__ cx,
    const double* __restrict__ cy, const double* __restrict__ cz, const uint8_t* __restrict__ fm,
    const double* __restrict__ p, double* y, unsigned char* scratch) {
  __shared__ double s_part[kThreads / 32];
  __shared__ int s_last;
  double* part = reinterpret_cast<double*>(scratch);
  unsigned* counter = reinterpret_cast<unsigned*>(scratch + kCounterOff);
  double* result = reinterpret_cast<double*>(scratch + kResultOff);
  const int tile = blockIdx.x;
  const int tx = tile % G.tiles_x, rest = tile / G.tiles_x;
  const int ty = rest % G.tiles_y, z = rest / G.tiles_y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long plane = (long long)G.nx * G.ny;
  auto pf = [&](long long j) { return fm[j] ? p[j] : 0.0; };  // p restricted to the free set
  double acc = 0.0;
  for (int k = 0; k < 4; ++k) {
    const int iy = ty * kTY + warp * 4 + k;
    if (iy >= G.ny) break;
    for (int h = 0; h < 2; ++h) {
      const int ix = tx * kTX + 2 * lane + h;
      if (ix >= G.nx) continue;
      const long long i = (long long)z * plane + (long long)iy * G.nx + ix;
      double v = 0.0;
      if (fm[i]) {
        v = diag[i] * p[i];
        if (ix > 0) v += cx[i - 1] * pf(i - 1);
        if (ix + 1 < G.nx) v += cx[i] * pf(i + 1);
        if (iy > 0) v += cy[i - G.nx] * pf(i - G.nx);
        if (iy + 1 < G.ny) v += cy[i] * pf(i + G.nx);
        if (G.dim == 3) {
          if (z > 0) v += cz[i - plane] * pf(i - plane);
          if (z + 1 < G.nz) v += cz[i] * pf(i + plane);
        }
        acc += p[i] * v;
      }
      y[i] = v;
    }
  }
  // fixed-order reduction: butterfly in each warp, warps in order
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) s_part[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += s_part[w];
    part[tile] = t;
    __threadfence();
    s_last = atomicAdd(counter, 1u) == (unsigned)(G.n_tiles - 1);
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  double t = 0.0;
  for (int j = 0; j < G.n_tiles; ++j) t += __ldcg(part + j);
  *result = t;
  *counter = 0u;
}

std::mutex g_mu;
void* g_addr[256] = {nullptr};  // device address of the scratch, per device

gpcg_status bad(gpcg_status s, const char* fmt, ...) {
  char msg[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof(msg), fmt, ap);
  va_end(ap);
  gpcg::set_last_error(msg);
  return s;
}

bool on_device(const void* q) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" gpcg_status gpcg_masked_spmv_noalloc(const gpcg_stencil* A, const uint8_t* free_mask,
                                                const double* p, double* y, double* pAp,
                                                void* cuda_stream) {
  if (!A || !free_mask || !p || !y) return bad(GPCG_ERR_ARG, "NULL argument");
  if (A->dim != 2 && A->dim != 3) return bad(GPCG_ERR_ARG, "dim must be 2 or 3");
  if (A->nx < 1 || A->ny < 1 || A->nz < 1 || (A->dim == 2 && A->nz != 1))
    return bad(GPCG_ERR_ARG, "bad grid size");
  if (!A->diag || !A->cx || !A->cy || (A->dim == 3 && !A->cz))
    return bad(GPCG_ERR_ARG, "missing stencil band");
  // each factor is bounded before the product is formed, so it cannot wrap
  const long long tiles_x = (A->nx + kTX - 1) / kTX, tiles_y = (A->ny + kTY - 1) / kTY;
  const bool huge = A->nx >= (1LL << 31) || A->ny >= (1LL << 31) || A->nz >= (1LL << 31) ||
                    tiles_x > kMaxTiles || tiles_y > kMaxTiles || A->nz > kMaxTiles;
  const long long n_tiles = huge ? (long long)kMaxTiles + 1 : tiles_x * tiles_y * A->nz;
  if (n_tiles < 1 || n_tiles > kMaxTiles)
    return bad(GPCG_ERR_ARG,
               "problem too large for the no-allocation entry point: %lld tiles of 64x32 points, "
               "at most %d",
               n_tiles, kMaxTiles);
  const void* arrays[] = {A->diag, A->cx, A->cy, free_mask, p, y};
  for (const void* q : arrays)
    if (!on_device(q)) return bad(GPCG_ERR_ARG, "every array must be a device pointer");
  if (A->dim == 3 && !on_device(A->cz)) return bad(GPCG_ERR_ARG, "cz must be a device pointer");
  // y is written while neighbouring CTAs still read p, the mask and the
  // bands: it must not overlap any input
  const long long n = A->nx * A->ny * A->nz;
  const uintptr_t y0 = (uintptr_t)y, y1 = y0 + sizeof(double) * (size_t)n;
  const void* inputs[] = {A->diag, A->cx, A->cy, A->dim == 3 ? A->cz : nullptr, p, free_mask};
  const size_t elem[] = {8, 8, 8, 8, 8, 1};
  for (int k = 0; k < 6; ++k) {
    if (!inputs[k]) continue;
    const uintptr_t a0 = (uintptr_t)inputs[k], a1 = a0 + elem[k] * (size_t)n;
    if (a0 < y1 && y0 < a1) return bad(GPCG_ERR_ARG, "y must not overlap an input array");
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (pAp) {
    // returning <p_F, y_F> waits for the stream, which a capture cannot do
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
      cudaGetLastError();
      return bad(GPCG_ERR_CUDA, "cudaStreamIsCapturing failed");
    }
    if (cs != cudaStreamCaptureStatusNone)
      return bad(GPCG_ERR_ARG, "pAp must be NULL while the stream is being captured");
  }

  // once per device, with that device current: the device address of the
  // scratch (the host-side name of the array is not a device address)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256)
    return bad(GPCG_ERR_CUDA, "no current CUDA device");
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess)
        return bad(GPCG_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      g_addr[dev] = ptr;
    }
    scratch = g_addr[dev];
  }
  cudaError_t e = cudaMemsetAsync((char*)scratch + kCounterOff, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return bad(GPCG_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  const Geo G{A->dim, (int)A->nx, (int)A->ny, (int)A->nz, (int)tiles_x, (int)tiles_y,
              (int)n_tiles};
  noalloc_masked_spmv<<<(unsigned)n_tiles, kThreads, 0, s>>>(
      G, A->diag, A->cx, A->cy, A->cz, free_mask, p, y, (unsigned char*)scratch);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return bad(GPCG_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
  if (pAp) {
    e = cudaMemcpyAsync(pAp, (char*)scratch + kResultOff, sizeof(double), cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bad(GPCG_ERR_CUDA, "result copy: %s", cudaGetErrorString(e));
  }
  return GPCG_OK;
}
