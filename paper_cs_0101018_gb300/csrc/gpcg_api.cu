// gpcg_api.cu -- host side of libgpcg.so: the C ABI of include/gpcg.h, device
// memory of each problem, the engine driver (CUDA graphs) and the
// continuous-batching server.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <string>
#include <vector>

#include "../../include/gpcg.h"
#include "engine.h"
#include "tuned.h"

namespace gpcg {
const void* pass_kernel_ptr(bool cond, int feat);
int pass_grid(int n_work);
cudaError_t launch_pass(const EngineArgs& E, int n_blocks, cudaStream_t s, int feat);
cudaError_t launch_pass_coop(const EngineArgs& E, int n_blocks, cudaStream_t s, int feat);
std::mutex& coop_mutex();
size_t resident_smem(int dim, long long n, bool mixed, bool jacobi);
cudaError_t launch_resident(const DevInst* insts, const int* ids, Ctl* ctl, int count,
                            size_t smem, unsigned sweep_cap, cudaStream_t s);
cudaError_t launch_prep(const DevInst& I, double* cx, double* cy, double* cz, double* l, double* u,
                        int fill_l, int fill_u, int* flags, cudaStream_t s);
cudaError_t launch_to_float(const double* src, float* dst, long long count, cudaStream_t s);
cudaError_t launch_recip(const double* d, double* out64, float* out32, long long count,
                         cudaStream_t s);
cudaError_t launch_spmv_setup(const DevInst& I, const uint8_t* fm, const double* pv,
                              unsigned* mask, void* r, void* pold, bool f32, cudaStream_t s);
cudaError_t launch_mspmv(const DevInst& I, bool f32, int mask, void* y, double* part,
                         unsigned* counter, double* result, int* err, cudaStream_t s,
                         bool pdl = false);
int ms_max_ctas();
cudaError_t launch_mspmv_setup(const DevInst& I, const uint8_t* fm, const double* pv,
                               unsigned* mask, void* pm, bool f32, cudaStream_t s);
cudaError_t launch_unpad(const DevInst& I, const void* src, bool f32, double* dst,
                         cudaStream_t s);
}  // namespace gpcg

using namespace gpcg;

// ------------------------------------------------------------------ errors --

static thread_local char g_err[512] = "";

static gpcg_status fail(gpcg_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(e_ == cudaErrorMemoryAllocation ? GPCG_ERR_OOM : GPCG_ERR_CUDA,      \
                  "%s failed: %s", #call, cudaGetErrorString(e_));                    \
  } while (0)

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

static unsigned env_pass_cap() {
  const char* s = getenv("GPCG_PASS_CAP");
  if (s && *s) return (unsigned)strtoul(s, nullptr, 10);
  return 4u * 1024u * 1024u;
}

static int env_engine_mode() {
  // 0: one WHILE-conditional CUDA graph per solve (default); 1: host-driven
  // loop of fixed-length graphs.
  const char* s = getenv("GPCG_ENGINE_MODE");
  return (s && *s) ? atoi(s) : 0;
}

static bool env_no_coop() {
  // GPCG_NO_COOP=1: a lone solve runs its passes as graph launches too
  const char* s = getenv("GPCG_NO_COOP");
  return s && *s && *s != '0';
}

static bool env_no_pdl() {
  // GPCG_NO_PDL=1: plain edges between the passes of a graph
  const char* s = getenv("GPCG_NO_PDL");
  return s && *s && *s != '0';
}

// ------------------------------------------------------------ problem --

struct Scratch {
  DevInst* d_insts = nullptr;
  Ctl* d_ctl = nullptr;
  int2* d_tiles = nullptr;
  int* d_live = nullptr;
  unsigned* d_npass = nullptr;
  int* d_queue = nullptr;  // [0] work queue head, [1] exit counter (zero between launches),
                           // [2] error flag of the bounded waits
  int* h_pin = nullptr;  // pinned: [0] live, [1] npass
  int* d_ids = nullptr;  // slots of the instances the resident solver takes
  int cap_inst = 0;
  long long cap_tiles = 0;
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;          // the graph gexec was instantiated from
  std::vector<cudaGraphNode_t> nodes;  // its pass nodes (plain graphs: updated in place)
  long long g_tiles = -1;
  int g_mode = -1;
  int g_steps = 0;
  bool g_pdl = false;      // the cached graph joins its passes by programmatic edges
  bool g_no_pdl = false;   // GPCG_NO_PDL when it was built
  int g_feat = -1;         // the feature set of its pass kernel (Feature bits)
  ~Scratch() { release(); }
  void release() {
    invalidate();
    for (void* d : {(void*)d_insts, (void*)d_ctl, (void*)d_tiles, (void*)d_live, (void*)d_npass,
                    (void*)d_queue, (void*)d_ids})
      if (d) cudaFree(d);
    d_ids = nullptr;
    if (h_pin) cudaFreeHost(h_pin);
    d_queue = nullptr;
    d_insts = nullptr;
    d_ctl = nullptr;
    d_tiles = nullptr;
    d_live = nullptr;
    d_npass = nullptr;
    h_pin = nullptr;
    cap_inst = 0;
    cap_tiles = 0;
    g_tiles = -1;
  }
  gpcg_status ensure(int n_inst, long long n_tiles) {
    if (!h_pin) {
      CK(cudaMallocHost(&h_pin, 4 * sizeof(int)));
      CK(cudaMalloc(&d_live, sizeof(int)));
      CK(cudaMalloc(&d_npass, sizeof(unsigned)));
      CK(cudaMalloc(&d_queue, 4 * sizeof(int)));
      CK(cudaMemset(d_queue, 0, 4 * sizeof(int)));
    }
    if (n_inst > cap_inst) {
      cudaFree(d_insts);
      cudaFree(d_ctl);
      cudaFree(d_ids);
      d_insts = nullptr;
      d_ctl = nullptr;
      d_ids = nullptr;
      CK(cudaMalloc(&d_insts, sizeof(DevInst) * n_inst));
      CK(cudaMalloc(&d_ctl, sizeof(Ctl) * n_inst));
      CK(cudaMalloc(&d_ids, sizeof(int) * n_inst));
      cap_inst = n_inst;
      invalidate();
    }
    if (n_tiles > cap_tiles) {
      cudaFree(d_tiles);
      d_tiles = nullptr;
      CK(cudaMalloc(&d_tiles, sizeof(int2) * n_tiles));
      cap_tiles = n_tiles;
      invalidate();
    }
    return GPCG_OK;
  }
  void invalidate() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    gexec = nullptr;
    graph = nullptr;
    nodes.clear();
    g_tiles = -1;
  }
};

struct gpcg_problem {
  int dim = 2, nx = 0, ny = 0, nz = 1, px = 0, mw = 0, kc = 3;
  long long n = 0, plane = 0, pn = 0, mwords = 0;
  int tiles_x = 0, tiles_y = 0, n_tiles = 0, n_groups = 0;
  double c = 0.0;
  void* arena64 = nullptr;
  size_t bytes64 = 0;
  void* arena32 = nullptr;
  size_t bytes32 = 0;
  void* arena_t64 = nullptr;  // tile preconditioner: z[2], q[2] in FP64, then in FP32
  void* arena_t32 = nullptr;
  void* arena_xi = nullptr;   // explicit reduced system: index arrays, then values
  void* arena_x64 = nullptr;
  void* arena_x32 = nullptr;
  double* ms_buf = nullptr;  // standalone masked product: CTA partials, result, counter, flag
  int* d_flags = nullptr;    // device-side input checks (a word in the FP64 arena)
  DevInst inst{};
  Scratch sc;
  Ctl last{};
  int last_path = 0;  // GPCG_PATH_ENGINE / GPCG_PATH_RESIDENT of the latest solve
  bool have = false;
  double lambda_min = 0.0;
  long long launches = 0;
  // A server's problems take their arenas from its stream-ordered pool, on
  // its side stream (no device-wide synchronisation at allocation or free).
  cudaMemPool_t pool = nullptr;
  cudaStream_t pstream = nullptr;
  CUtensorMap hmaps[M_COUNT];  // host copies of the tensor maps (their upload's source)
  // gpcg_problem_update_async: its copies end at up_ev; the device-side set-up
  // (device_init) runs on the stream of the next call that uses the data
  cudaEvent_t up_ev = nullptr;
  bool pending = false, fill_l = false, fill_u = false;
  bool bad = false;        // its data failed the value checks: no solve until an update
  int* h_flags = nullptr;  // pinned word: the input checks of that set-up
  ~gpcg_problem() {
    sc.release();
    void* arenas[] = {arena64, arena32, arena_t64, arena_t32, arena_xi, arena_x64, arena_x32};
    for (void* a : arenas)
      if (a) {
        if (pool) cudaFreeAsync(a, pstream);
        else cudaFree(a);
      }
    if (ms_buf) cudaFree(ms_buf);
    if (up_ev) cudaEventDestroy(up_ev);
    if (h_flags) cudaFreeHost(h_flags);
  }
};

// Device memory of a problem's arenas: from the owning server's pool when
// there is one, else cudaMalloc.
static cudaError_t dev_alloc(gpcg_problem* p, void** ptr, size_t bytes) {
  if (!p->pool) return cudaMalloc(ptr, bytes);
  cudaError_t e = cudaMallocFromPoolAsync(ptr, bytes, p->pool, p->pstream);
  // the arenas are carved in 256-byte steps for the tensor maps and vector
  // accesses: a base off that boundary is refused
  if (e == cudaSuccess && ((uintptr_t)*ptr & 255u) != 0) {
    cudaFreeAsync(*ptr, p->pstream);
    *ptr = nullptr;
    e = cudaErrorInvalidValue;
  }
  return e;
}

// Tiles per group of an instance from the tuned table (GPCG_GROUP_TILES
// overrides it, for the tuner's measurements).
static int group_tiles(int dim, int n_tiles) {
  const char* e = getenv("GPCG_GROUP_TILES");
  if (e && *e) return std::max(1, atoi(e));
  for (const TunedGroup& t : kTunedGroups)
    if (t.dim == dim && n_tiles >= t.tiles_lo && n_tiles <= t.tiles_hi)
      return std::max(1, t.group_tiles);
  return 4;
}

// Tiles per work item of a crowded launch (GPCG_ITEM_TILES overrides it).
static int item_tiles() {
  const char* e = getenv("GPCG_ITEM_TILES");
  if (e && *e) return std::max(1, atoi(e));
  return std::max(1, kTunedItemTiles);
}

// Groups per work item of problem p: one when the launch's groups fit the
// resident CTAs at once (a lone solve takes all the parallelism it can),
// else about item_tiles() tiles per item, the groups spread evenly over the
// instance's items (an instance's pass lasts as long as its longest item).
// The explicit reduced system's passes keep one group per item.
static int item_span(const gpcg_problem* p, long long launch_groups, bool extract) {
  if (extract || launch_groups <= (long long)pass_grid(1 << 30)) return 1;
  const int ng = std::max(1, p->n_groups);
  const double tiles_per_group = (double)p->n_tiles / (double)ng;
  const int target = std::min(std::max((int)std::lround((double)item_tiles() / tiles_per_group),
                                       1), kMaxSpan);
  const int items = (ng + target - 1) / target;
  return (ng + items - 1) / items;
}

static void geometry(int dim, long long nx, long long ny, long long nz, gpcg_problem* p) {
  p->dim = dim;
  p->nx = (int)nx;
  p->ny = (int)ny;
  p->nz = (int)nz;
  p->px = (int)((nx + 7) / 8 * 8);
  p->mw = ((p->px + 31) / 32 + 3) / 4 * 4;
  p->kc = dim == 3 ? 4 : 3;
  p->n = nx * ny * nz;
  p->plane = (long long)p->px * ny;
  p->pn = p->plane * nz;
  p->mwords = (long long)p->mw * ny * nz;
  p->tiles_x = (int)((nx + kTX - 1) / kTX);
  p->tiles_y = (int)((ny + kTY - 1) / kTY);
  p->n_tiles = p->tiles_x * p->tiles_y * (int)nz;
  const int gt = group_tiles(dim, p->n_tiles);
  p->n_groups = std::min((p->n_tiles + gt - 1) / gt, kMaxGroups);
}

// Bytes of the FP64 arena: kc bands, 1/diag, b, l, u, x[2], g[2], r[2], w,
// p[2], Ap[2], two masks, the group partials (two arrays: the cooperative
// kernel alternates them), the tensor maps and the word of the input checks.
static size_t arena64_bytes(const gpcg_problem* p) {
  const size_t vec = align256(sizeof(double) * (size_t)p->pn);
  const size_t msk = align256(sizeof(unsigned) * (size_t)p->mwords);
  const size_t part = align256(sizeof(double) * kNRed * 2 * (size_t)p->n_groups);
  const size_t maps = align256(sizeof(CUtensorMap) * M_COUNT);
  return (size_t)(p->kc + 15) * vec + 2 * msk + part + maps + 256;
}

// FP32 bands and 1/diag, the FP32 CG vectors r[2], w, p[2], Ap[2], and the
// FP32 arrays of the mixed phase x[2], g[2], b, l, u, pg[2].
static size_t arena32_bytes(const gpcg_problem* p) {
  const size_t vec = align256(sizeof(float) * (size_t)p->pn);
  return (size_t)(p->kc + 1 + 7 + 9) * vec;
}

// Bytes of the explicit reduced system: the index arrays (cidx over the padded
// layout, fidx, group offsets, 2*dim neighbour slots per point) and, per
// precision, the rows (diagonal, 2*dim couplings, 1/diagonal) and the compact
// vectors r[2], p[2], Ap[2], w.
static size_t arena_rx_index_bytes(const gpcg_problem* p) {
  return align256(sizeof(int) * (size_t)p->pn) + align256(sizeof(int) * (size_t)p->n) +
         align256(sizeof(int) * kMaxGroups) + align256(sizeof(int) * 2 * p->dim * (size_t)p->n);
}
static size_t arena_rx_value_bytes(const gpcg_problem* p, bool f32) {
  const size_t vec = align256((f32 ? sizeof(float) : sizeof(double)) * (size_t)p->n);
  return (size_t)(9 + 2 * p->dim) * vec;
}

// Bytes of the tile preconditioner's vectors of one precision: z[2], q[2].
static size_t arena_tile_bytes(const gpcg_problem* p, bool f32) {
  return 4 * align256((f32 ? sizeof(float) : sizeof(double)) * (size_t)p->pn);
}

static void carve64(gpcg_problem* p) {
  char* a = (char*)p->arena64;
  const size_t vec = align256(sizeof(double) * (size_t)p->pn);
  const size_t msk = align256(sizeof(unsigned) * (size_t)p->mwords);
  auto take = [&](size_t b) {
    char* r = a;
    a += b;
    return r;
  };
  DevInst& I = p->inst;
  I.dim = p->dim;
  I.nx = p->nx;
  I.ny = p->ny;
  I.nz = p->nz;
  I.px = p->px;
  I.mw = p->mw;
  I.tiles_x = p->tiles_x;
  I.tiles_y = p->tiles_y;
  I.n_tiles = p->n_tiles;
  I.n_groups = p->n_groups;
  I.kc = p->kc;
  I.n = p->n;
  I.plane = p->plane;
  I.diag = (double*)take(vec);
  I.cx = (double*)take(vec);
  I.cy = (double*)take(vec);
  I.cz = p->dim == 3 ? (double*)take(vec) : nullptr;
  I.dinv = (double*)take(vec);
  I.b = (double*)take(vec);
  I.l = (double*)take(vec);
  I.u = (double*)take(vec);
  for (int k = 0; k < 2; ++k) I.x[k] = (double*)take(vec);
  for (int k = 0; k < 2; ++k) I.g[k] = (double*)take(vec);
  for (int k = 0; k < 2; ++k) I.r64[k] = (double*)take(vec);
  I.w64 = (double*)take(vec);
  for (int k = 0; k < 2; ++k) I.p64[k] = (double*)take(vec);
  for (int k = 0; k < 2; ++k) I.Ap64[k] = (double*)take(vec);
  for (int k = 0; k < 2; ++k) I.mask[k] = (unsigned*)take(msk);
  I.part = (double*)take(align256(sizeof(double) * kNRed * 2 * (size_t)p->n_groups));
  I.tmaps = take(align256(sizeof(CUtensorMap) * M_COUNT));
  p->d_flags = (int*)take(256);
  I.tma64 = 0;
  I.tma32 = 0;
  I.tma_gp = 0;
  I.tma_mask = 0;
  I.tma3 = 0;
  I.x0 = I.r64[0];  // a given start point is staged in r (unused until CG starts)
}

// ----------------------------------------------------------- tensor maps --

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static bool have_encode() {
  static std::once_flag once;
  std::call_once(once, []() {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    else
      cudaGetLastError();
  });
  return g_encode != nullptr;
}

// One 2-D map over the padded array `base` seen as (nx columns, rows rows,
// row pitch px elements), with a bw x bh box; out-of-range boxes fill zeros.
static bool encode_map(CUtensorMap* m, bool f32, const void* base, const gpcg_problem* p, int bw,
                       int bh) {
  const size_t es = f32 ? 4 : 8;
  cuuint64_t dims[2] = {(cuuint64_t)p->nx, (cuuint64_t)p->ny * (cuuint64_t)p->nz};
  cuuint64_t strides[1] = {(cuuint64_t)p->px * es};
  cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
  cuuint32_t estr[2] = {1, 1};
  return g_encode(m, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                  const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Copy maps [b0, b0 + count) from the problem's host copies to its device
// area (ordered on s; the host copies live as long as the problem).
static bool put_maps(gpcg_problem* p, int b0, int count, cudaStream_t s) {
  char* dst = (char*)const_cast<void*>(p->inst.tmaps) + sizeof(CUtensorMap) * b0;
  return cudaMemcpyAsync(dst, &p->hmaps[b0], sizeof(CUtensorMap) * count, cudaMemcpyHostToDevice,
                         s) == cudaSuccess;
}

// Encode the maps of one precision (the box shapes of the CG stages, see the
// kernels) and copy them to the problem's device area.  Returns false (and
// leaves the TMA path off) when the driver cannot encode them.
static bool make_maps(gpcg_problem* p, bool f32, cudaStream_t s) {
  if (!have_encode()) return false;
  DevInst& I = p->inst;
  // h: halo columns; c: CG_B chunk rows; a: CG_A chunk rows; f: fused chunk rows
  const int h = f32 ? 4 : 2, c = f32 ? 32 : 16, a = f32 ? 32 : 16, f = f32 ? 16 : 8;
  const int b0 = f32 ? M32_RH0 : M64_RH0;
  auto v = [&](int k, const char* which) -> const void* {
    if (which[0] == 'r') return f32 ? (const void*)I.r32[k] : (const void*)I.r64[k];
    if (which[0] == 'p') return f32 ? (const void*)I.p32[k] : (const void*)I.p64[k];
    return f32 ? (const void*)I.Ap32[k] : (const void*)I.Ap64[k];
  };
  const void* d = f32 ? (const void*)I.diag32 : (const void*)I.diag;
  const void* cx = f32 ? (const void*)I.cx32 : (const void*)I.cx;
  const void* cy = f32 ? (const void*)I.cy32 : (const void*)I.cy;
  const void* w = f32 ? (const void*)I.w32 : (const void*)I.w64;
  const void* di = f32 ? (const void*)I.dinv32 : (const void*)I.dinv;
  CUtensorMap* m = &p->hmaps[b0];
  CUtensorMap* q = m;
  auto e = [&](const void* base, int bw, int bh) { return encode_map(q++, f32, base, p, bw, bh); };
  const bool ok =
      // CG_B: RH[2], PH[2], D, CX, CY
      e(v(0, "r"), 64 + 2 * h, c + 2) && e(v(1, "r"), 64 + 2 * h, c + 2) &&
      e(v(0, "p"), 64 + 2 * h, c + 2) && e(v(1, "p"), 64 + 2 * h, c + 2) && e(d, 64, c) &&
      e(cx, 64 + h, c) && e(cy, 64, c + 1) &&
      // CG_A: W, R[2], P[2], AP[2]
      e(w, 64, a) && e(v(0, "r"), 64, a) && e(v(1, "r"), 64, a) && e(v(0, "p"), 64, a) &&
      e(v(1, "p"), 64, a) && e(v(0, "A"), 64, a) && e(v(1, "A"), 64, a) &&
      // fused: FRH[2], FPH[2], FAPH[2], FW, FD, FCX, FCY
      e(v(0, "r"), 64 + 2 * h, f + 2) && e(v(1, "r"), 64 + 2 * h, f + 2) &&
      e(v(0, "p"), 64 + 2 * h, f + 2) && e(v(1, "p"), 64 + 2 * h, f + 2) &&
      e(v(0, "A"), 64 + 2 * h, f + 2) && e(v(1, "A"), 64 + 2 * h, f + 2) && e(w, 64, f) &&
      e(d, 64, f) && e(cx, 64 + h, f) && e(cy, 64, f + 1) &&
      // 1/diag: FDIH, ADI
      e(di, 64 + 2 * h, f + 2) && e(di, 64, a);
  return ok && q == m + kCgBase && put_maps(p, b0, kCgBase, s);
}

// Encode the maps of the 3-D fused CG step (FP32; box shapes of GeoF3 in the
// kernels) and copy them to the problem's device area.
static bool make_3d_maps(gpcg_problem* p, cudaStream_t s) {
  if (!have_encode() || p->dim != 3) return false;
  DevInst& I = p->inst;
  CUtensorMap* m = &p->hmaps[M3_RH0];
  CUtensorMap* q = m;
  auto e = [&](const float* a, int bw, int bh) { return encode_map(q++, true, a, p, bw, bh); };
  const bool ok = e(I.r32[0], 72, 10) && e(I.r32[1], 72, 10) && e(I.p32[0], 72, 10) &&
                  e(I.p32[1], 72, 10) && e(I.Ap32[0], 72, 10) && e(I.Ap32[1], 72, 10) &&
                  e(I.w32, 64, 8) && e(I.diag32, 64, 8) && e(I.cx32, 68, 8) &&
                  e(I.cy32, 64, 9) && e(I.cz32, 64, 8) && e(I.r32[0], 64, 8) &&
                  e(I.r32[1], 64, 8) && e(I.p32[0], 64, 8) && e(I.p32[1], 64, 8) &&
                  e(I.Ap32[0], 64, 8) && e(I.Ap32[1], 64, 8);
  return ok && q == m + k3dMaps && put_maps(p, M3_RH0, k3dMaps, s);
}

// Encode the maps of the mixed-phase gradient-projection passes (2-D only:
// their chunks take halo rows from the same plane).
static bool make_gp_maps(gpcg_problem* p, cudaStream_t s) {
  if (!have_encode() || p->dim != 2) return false;
  DevInst& I = p->inst;
  CUtensorMap* m = &p->hmaps[MG_X32H0];
  CUtensorMap* q = m;
  auto f32 = [&](const float* a, int bw, int bh) { return encode_map(q++, true, a, p, bw, bh); };
  bool ok = f32(I.x32[0], 72, 18) && f32(I.x32[1], 72, 18) && f32(I.l32, 72, 18) &&
            f32(I.u32, 72, 18) && f32(I.g32[0], 72, 18) && f32(I.g32[1], 72, 18) &&
            f32(I.w32, 72, 18) && f32(I.pg32[0], 72, 34) && f32(I.pg32[1], 72, 34) &&
            f32(I.l32, 64, 16) && f32(I.u32, 64, 16) && f32(I.b32, 64, 16) &&
            f32(I.x32[0], 72, 20) && f32(I.x32[1], 72, 20) && f32(I.l32, 72, 20) &&
            f32(I.u32, 72, 20) && f32(I.g32[0], 72, 20) && f32(I.g32[1], 72, 20) &&
            f32(I.b32, 72, 18) && f32(I.diag32, 72, 18) && f32(I.cx32, 72, 18) &&
            f32(I.cy32, 72, 19);
  return ok && q == m + kGpMaps && put_maps(p, MG_X32H0, kGpMaps, s);
}

// The free-set words as a 2-D u32 tensor (mw words x ny*nz rows): boxes 4 x 32
// (M_MASK0/1) and 8 x 18 (M_MASKH0/1, the staged first CG step's halo).
static bool make_mask_maps(gpcg_problem* p, cudaStream_t s) {
  if (!have_encode()) return false;
  static_assert(M_MASKH0 == M_MASK0 + 2, "mask maps in a row");
  DevInst& I = p->inst;
  CUtensorMap* m = &p->hmaps[M_MASK0];
  for (int k = 0; k < 4; ++k) {
    cuuint64_t dims[2] = {(cuuint64_t)p->mw, (cuuint64_t)p->ny * (cuuint64_t)p->nz};
    cuuint64_t strides[1] = {(cuuint64_t)p->mw * 4};
    cuuint32_t box[2] = {k < 2 ? 4u : 8u, k < 2 ? 32u : 18u};
    cuuint32_t estr[2] = {1, 1};
    if (g_encode(&m[k], CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, I.mask[k & 1], dims, strides, box,
                 estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                 CU_TENSOR_MAP_L2_PROMOTION_NONE,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return put_maps(p, M_MASK0, 4, s);
}

// Encode the tile preconditioner's maps of one precision: FZH[2], FQH[2],
// halo boxes of z and q like the fused CG step's FRH.
static bool make_tile_maps(gpcg_problem* p, bool f32, cudaStream_t s) {
  if (!have_encode()) return false;
  DevInst& I = p->inst;
  const int h = f32 ? 4 : 2, f = f32 ? 16 : 8;
  const void* zq[4] = {f32 ? (const void*)I.z32[0] : (const void*)I.z64[0],
                       f32 ? (const void*)I.z32[1] : (const void*)I.z64[1],
                       f32 ? (const void*)I.q32[0] : (const void*)I.q64[0],
                       f32 ? (const void*)I.q32[1] : (const void*)I.q64[1]};
  static_assert(kTileMaps == 4, "FZH[2], FQH[2]");
  const int b0 = (f32 ? M32_RH0 : M64_RH0) + kCgBase;
  for (int k = 0; k < 4; ++k)
    if (!encode_map(&p->hmaps[b0 + k], f32, zq[k], p, 64 + 2 * h, f + 2)) return false;
  return put_maps(p, b0, kTileMaps, s);
}

// Encode the staged FP64 GP passes' maps: halo boxes 68 x 10 of x[2], g[2], l,
// u, w; b as 64 x 8.
static bool make_f64gp_maps(gpcg_problem* p, cudaStream_t s) {
  if (!have_encode() || p->dim != 2) return false;
  DevInst& I = p->inst;
  const void* src[8] = {I.x[0], I.x[1], I.g[0], I.g[1], I.l, I.u, I.w64, I.b};
  static_assert(MF_B - MF_X0 == 7, "eight FP64 GP maps");
  for (int k = 0; k < 8; ++k)
    if (!encode_map(&p->hmaps[MF_X0 + k], false, src[k], p, k < 7 ? 68 : 64, k < 7 ? 10 : 8))
      return false;
  return put_maps(p, MF_X0, 8, s);
}

static bool tma_disabled() {
  const char* e = getenv("GPCG_NO_TMA");
  return e && *e && *e != '0';
}

// The FP32 copies of the bands, b, l, u and 1/diag in the mixed arena.
static gpcg_status convert32(gpcg_problem* p, cudaStream_t s) {
  DevInst& I = p->inst;
  CK(launch_to_float(I.b, (float*)I.b32, p->pn, s));
  CK(launch_to_float(I.l, (float*)I.l32, p->pn, s));
  CK(launch_to_float(I.u, (float*)I.u32, p->pn, s));
  CK(launch_to_float(I.diag, (float*)I.diag32, p->pn, s));
  CK(launch_to_float(I.cx, (float*)I.cx32, p->pn, s));
  CK(launch_to_float(I.cy, (float*)I.cy32, p->pn, s));
  if (I.cz32) CK(launch_to_float(I.cz, (float*)I.cz32, p->pn, s));
  CK(launch_recip(I.diag, nullptr, (float*)I.dinv32, p->pn, s));
  return GPCG_OK;
}

// init: zero the arena and fill the FP32 copies here (else device_init does,
// on the stream of the first solve).
static gpcg_status ensure_mixed(gpcg_problem* p, cudaStream_t s, bool init) {
  if (p->arena32) return GPCG_OK;
  const size_t bytes = arena32_bytes(p);
  CK(dev_alloc(p, &p->arena32, bytes));
  if (init) CK(cudaMemsetAsync(p->arena32, 0, bytes, s));
  p->bytes32 = bytes;
  char* a = (char*)p->arena32;
  const size_t vec = align256(sizeof(float) * (size_t)p->pn);
  auto take = [&]() {
    char* r = a;
    a += vec;
    return (float*)r;
  };
  DevInst& I = p->inst;
  float* d32 = take();
  float* dinv32 = take();
  float* x32 = take();
  float* y32 = take();
  float* z32 = p->dim == 3 ? take() : nullptr;
  for (int k = 0; k < 2; ++k) I.r32[k] = take();
  I.w32 = take();
  for (int k = 0; k < 2; ++k) I.p32[k] = take();
  for (int k = 0; k < 2; ++k) I.Ap32[k] = take();
  for (int k = 0; k < 2; ++k) I.x32[k] = take();
  for (int k = 0; k < 2; ++k) I.g32[k] = take();
  float* b32 = take();
  float* l32 = take();
  float* u32 = take();
  for (int k = 0; k < 2; ++k) I.pg32[k] = take();
  I.b32 = b32;
  I.l32 = l32;
  I.u32 = u32;
  I.diag32 = d32;
  I.cx32 = x32;
  I.cy32 = y32;
  I.cz32 = z32;
  I.dinv32 = dinv32;
  if (init) {
    gpcg_status st = convert32(p, s);
    if (st != GPCG_OK) return st;
  }
  I.tma32 = (I.tma_mask && make_maps(p, true, s)) ? 1 : 0;
  I.tma_gp = (I.tma_mask && make_gp_maps(p, s)) ? 1 : 0;
  I.tma3 = (I.tma32 && make_3d_maps(p, s)) ? 1 : 0;
  return GPCG_OK;
}

// The tile preconditioner's vectors and maps for the CG precisions of a
// solve (FP64 always; FP32 too in mixed precision), made on first use.  The
// vectors start at zero and stay finite: the first fused step of a phase
// multiplies them by alpha = beta = 0.
static gpcg_status ensure_tile(gpcg_problem* p, bool mixed, cudaStream_t s, bool init) {
  DevInst& I = p->inst;
  if (p->dim != 2)
    return fail(GPCG_ERR_ARG, "the tile preconditioner is for 2-D problems only");
  if (!I.tma64 || (mixed && !I.tma32))
    return fail(GPCG_ERR_ARG, "the tile preconditioner needs the TMA-staged path");
  for (int f32 = 0; f32 <= (mixed ? 1 : 0); ++f32) {
    void*& a = f32 ? p->arena_t32 : p->arena_t64;
    if (a) continue;
    const size_t bytes = arena_tile_bytes(p, f32);
    CK(dev_alloc(p, &a, bytes));
    if (init) CK(cudaMemsetAsync(a, 0, bytes, s));
    const size_t vec = bytes / 4;
    char* c = (char*)a;
    for (int k = 0; k < 2; ++k) {
      if (f32) {
        I.z32[k] = (float*)(c + k * vec);
        I.q32[k] = (float*)(c + (2 + k) * vec);
      } else {
        I.z64[k] = (double*)(c + k * vec);
        I.q64[k] = (double*)(c + (2 + k) * vec);
      }
    }
    if (!make_tile_maps(p, f32, s))
      return fail(GPCG_ERR_CUDA, "tensor maps of the tile preconditioner could not be encoded");
    I.tma_tile |= f32 ? 2 : 1;
  }
  return GPCG_OK;
}

// The explicit reduced system's arrays for the CG precisions of a solve,
// made on first use.
static gpcg_status ensure_extract(gpcg_problem* p, bool mixed, cudaStream_t s, bool init) {
  DevInst& I = p->inst;
  if (p->pn >= (1LL << 31))
    return fail(GPCG_ERR_ARG, "the explicit reduced system needs fewer than 2^31 points");
  if (!p->arena_xi) {
    const size_t bytes = arena_rx_index_bytes(p);
    CK(dev_alloc(p, &p->arena_xi, bytes));
    if (init) CK(cudaMemsetAsync(p->arena_xi, 0, bytes, s));
    char* a = (char*)p->arena_xi;
    I.cidx = (int*)a;
    a += align256(sizeof(int) * (size_t)p->pn);
    I.fidx = (int*)a;
    a += align256(sizeof(int) * (size_t)p->n);
    I.goff = (int*)a;
    a += align256(sizeof(int) * kMaxGroups);
    I.rnb = (int*)a;
  }
  for (int f32 = 0; f32 <= (mixed ? 1 : 0); ++f32) {
    void*& arena = f32 ? p->arena_x32 : p->arena_x64;
    if (arena) continue;
    const size_t bytes = arena_rx_value_bytes(p, f32);
    CK(dev_alloc(p, &arena, bytes));
    if (init) CK(cudaMemsetAsync(arena, 0, bytes, s));
    const size_t vec = align256((f32 ? sizeof(float) : sizeof(double)) * (size_t)p->n);
    char* a = (char*)arena;
    auto take = [&](size_t k) {
      char* r = a;
      a += k * vec;
      return r;
    };
    if (f32) {
      I.rd32 = (float*)take(1);
      I.rv32 = (float*)take(2 * p->dim);
      I.rdi32 = (float*)take(1);
      for (int k = 0; k < 2; ++k) I.rc32[k] = (float*)take(1);
      for (int k = 0; k < 2; ++k) I.pc32[k] = (float*)take(1);
      for (int k = 0; k < 2; ++k) I.apc32[k] = (float*)take(1);
      I.wc32 = (float*)take(1);
      I.rx32 = 1;
    } else {
      I.rd64 = (double*)take(1);
      I.rv64 = (double*)take(2 * p->dim);
      I.rdi64 = (double*)take(1);
      for (int k = 0; k < 2; ++k) I.rc64[k] = (double*)take(1);
      for (int k = 0; k < 2; ++k) I.pc64[k] = (double*)take(1);
      for (int k = 0; k < 2; ++k) I.apc64[k] = (double*)take(1);
      I.wc64 = (double*)take(1);
      I.rx64 = 1;
    }
  }
  return GPCG_OK;
}

static gpcg_status copy_in(const gpcg_problem* p, double* dst, const double* src, cudaStream_t s) {
  CK(cudaMemcpy2DAsync(dst, sizeof(double) * p->px, src, sizeof(double) * p->nx,
                       sizeof(double) * p->nx, (size_t)p->ny * p->nz, cudaMemcpyDefault, s));
  return GPCG_OK;
}

// Argument checks of a stencil problem (nothing is touched).
static gpcg_status check_problem(const gpcg_stencil* A, const double* b, double c) {
  if (!A || !b) return fail(GPCG_ERR_ARG, "A or b is NULL");
  if (A->dim != 2 && A->dim != 3) return fail(GPCG_ERR_ARG, "dim must be 2 or 3");
  if (A->nx < 1 || A->ny < 1 || A->nz < 1) return fail(GPCG_ERR_ARG, "grid sizes must be >= 1");
  if (A->dim == 2 && A->nz != 1) return fail(GPCG_ERR_ARG, "nz must be 1 when dim == 2");
  if (!A->diag || !A->cx || !A->cy || (A->dim == 3 && !A->cz))
    return fail(GPCG_ERR_ARG, "missing stencil band");
  // The padded point count px*ny*nz (px = nx rounded up to a multiple of 8)
  // must stay below 2^31, checked without forming a product that could wrap.
  constexpr long long kLim = 1LL << 31;
  if (A->nx > kLim - 9 || A->ny >= kLim || A->nz >= kLim)
    return fail(GPCG_ERR_ARG, "problem too large (n must be below 2^31)");
  const long long px = (A->nx + 7) / 8 * 8;
  if (A->ny > (kLim - 1) / px || A->nz > (kLim - 1) / (px * A->ny))
    return fail(GPCG_ERR_ARG, "problem too large (n must be below 2^31)");
  if (!std::isfinite(c)) return fail(GPCG_ERR_ARG, "c is not finite");
  return GPCG_OK;
}

// Enqueue on s the copies of the bands, b, l and u into the problem's FP64
// arrays and what the passes derive from them (couplings beyond the grid
// cleared, default bounds, 1/diag; the FP32 copies when the mixed arena
// exists), with the device-side checks of the values, whose result word is
// p->d_flags (see flags_status).  Nothing waits.
static gpcg_status upload_enqueue(gpcg_problem* p, const gpcg_stencil* A, const double* b,
                                  const double* l, const double* u, cudaStream_t s) {
  DevInst& I = p->inst;
  gpcg_status st;
  if ((st = copy_in(p, (double*)I.diag, A->diag, s)) != GPCG_OK) return st;
  if ((st = copy_in(p, (double*)I.cx, A->cx, s)) != GPCG_OK) return st;
  if ((st = copy_in(p, (double*)I.cy, A->cy, s)) != GPCG_OK) return st;
  if (A->dim == 3 && (st = copy_in(p, (double*)I.cz, A->cz, s)) != GPCG_OK) return st;
  if ((st = copy_in(p, (double*)I.b, b, s)) != GPCG_OK) return st;
  if (l && (st = copy_in(p, (double*)I.l, l, s)) != GPCG_OK) return st;
  if (u && (st = copy_in(p, (double*)I.u, u, s)) != GPCG_OK) return st;
  CK(cudaMemsetAsync(p->d_flags, 0, sizeof(int), s));
  CK(launch_prep(I, (double*)I.cx, (double*)I.cy, (double*)I.cz, (double*)I.l, (double*)I.u,
                 l == nullptr, u == nullptr, p->d_flags, s));
  CK(launch_recip(I.diag, (double*)I.dinv, nullptr, p->pn, s));
  if (p->arena32) return convert32(p, s);
  return GPCG_OK;
}

// Pinned staging of a server worker for transfers from and to pageable host
// memory: two buffers used in turn, each with the event of its last copy.
// The driver's own path for pageable memory stalls while a step's passes
// hold the GPU; staged, the CPU moves the bytes and the copy engines DMA them.
struct Stager {
  static constexpr size_t kBytes = 8u << 20;
  double* buf[2] = {nullptr, nullptr};
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int next = 0;
  cudaError_t init() {
    for (int k = 0; k < 2; ++k) {
      cudaError_t e = cudaMallocHost(&buf[k], kBytes);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  void release() {
    for (int k = 0; k < 2; ++k) {
      if (ev[k]) cudaEventSynchronize(ev[k]);
      if (ev[k]) cudaEventDestroy(ev[k]);
      if (buf[k]) cudaFreeHost(buf[k]);
      ev[k] = nullptr;
      buf[k] = nullptr;
    }
  }
};

static bool pageable(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeUnregistered;
}

// rows x nx values from host src (row length nx) into the device array dst
// (row pitch px): whole rows, padded with zeros to px, through the staging
// buffers.
static gpcg_status staged_in(Stager& sg, double* dst, const double* src, size_t nx, size_t px,
                             size_t rows, cudaStream_t s) {
  const size_t per = Stager::kBytes / (sizeof(double) * px);
  for (size_t r0 = 0; r0 < rows; r0 += per) {
    const size_t nr = std::min(per, rows - r0);
    const int k = sg.next;
    sg.next ^= 1;
    CK(cudaEventSynchronize(sg.ev[k]));  // its previous copy has left the buffer
    double* b = sg.buf[k];
    for (size_t i = 0; i < nr; ++i) {
      memcpy(b + i * px, src + (r0 + i) * nx, sizeof(double) * nx);
      if (px > nx) memset(b + i * px + nx, 0, sizeof(double) * (px - nx));
    }
    CK(cudaMemcpyAsync(dst + r0 * px, b, sizeof(double) * nr * px, cudaMemcpyHostToDevice, s));
    CK(cudaEventRecord(sg.ev[k], s));
  }
  return GPCG_OK;
}

// rows x nx values from the device array src (row pitch px) to host dst (row
// length nx) through the staging buffers.
static gpcg_status staged_out(Stager& sg, double* dst, const double* src, size_t nx, size_t px,
                              size_t rows, cudaStream_t s) {
  const size_t per = Stager::kBytes / (sizeof(double) * px);
  for (size_t r0 = 0; r0 < rows; r0 += per) {
    const size_t nr = std::min(per, rows - r0);
    double* b = sg.buf[0];
    CK(cudaEventSynchronize(sg.ev[0]));
    CK(cudaMemcpyAsync(b, src + r0 * px, sizeof(double) * nr * px, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (size_t i = 0; i < nr; ++i)
      memcpy(dst + (r0 + i) * nx, b + i * px, sizeof(double) * nx);
  }
  return GPCG_OK;
}

// One input array of a server's request: staged when it is pageable host
// memory (and a whole row fits a staging buffer), else copied directly.
static gpcg_status copy_in_served(const gpcg_problem* p, double* dst, const double* src,
                                  cudaStream_t s, Stager* sg) {
  if (sg && sizeof(double) * (size_t)p->px <= Stager::kBytes && pageable(src))
    return staged_in(*sg, dst, src, (size_t)p->nx, (size_t)p->px, (size_t)p->ny * p->nz, s);
  return copy_in(p, dst, src, s);
}

// Enqueue on s the copies of the bands, b, l and u into the problem's FP64
// arrays, nothing else (copy engines only; device_init derives the rest).
static gpcg_status upload_copies(gpcg_problem* p, const gpcg_stencil* A, const double* b,
                                 const double* l, const double* u, cudaStream_t s, Stager* sg) {
  DevInst& I = p->inst;
  gpcg_status st;
  if ((st = copy_in_served(p, (double*)I.diag, A->diag, s, sg)) != GPCG_OK) return st;
  if ((st = copy_in_served(p, (double*)I.cx, A->cx, s, sg)) != GPCG_OK) return st;
  if ((st = copy_in_served(p, (double*)I.cy, A->cy, s, sg)) != GPCG_OK) return st;
  if (A->dim == 3 && (st = copy_in_served(p, (double*)I.cz, A->cz, s, sg)) != GPCG_OK) return st;
  if ((st = copy_in_served(p, (double*)I.b, b, s, sg)) != GPCG_OK) return st;
  if (l && (st = copy_in_served(p, (double*)I.l, l, s, sg)) != GPCG_OK) return st;
  if (u && (st = copy_in_served(p, (double*)I.u, u, s, sg)) != GPCG_OK) return st;
  return GPCG_OK;
}

// The device-side set-up after upload_copies: everything upload_enqueue
// derives (default bounds, cleared couplings, checks, 1/diag, the FP32
// copies).  fresh: the arenas were allocated without initialisation, so
// first zero the pad columns of the input arrays, the work vectors, masks and
// partials (not the tensor maps), and the optional arenas.
static gpcg_status device_init(gpcg_problem* p, bool fill_l, bool fill_u, cudaStream_t s,
                               bool fresh = true) {
  DevInst& I = p->inst;
  if (fresh && p->px > p->nx) {
    double* in[7] = {(double*)I.diag, (double*)I.cx, (double*)I.cy, (double*)I.cz,
                     (double*)I.b, (double*)I.l, (double*)I.u};
    for (double* a : in)
      if (a)
        CK(cudaMemset2DAsync(a + p->nx, sizeof(double) * p->px, 0,
                             sizeof(double) * (p->px - p->nx), (size_t)p->ny * p->nz, s));
  }
  char* w0 = (char*)I.x[0];
  if (fresh) CK(cudaMemsetAsync(w0, 0, (size_t)((const char*)I.tmaps - w0), s));
  CK(cudaMemsetAsync(p->d_flags, 0, sizeof(int), s));
  CK(launch_prep(I, (double*)I.cx, (double*)I.cy, (double*)I.cz, (double*)I.l, (double*)I.u,
                 fill_l, fill_u, p->d_flags, s));
  CK(launch_recip(I.diag, (double*)I.dinv, nullptr, p->pn, s));
  if (p->arena32) {
    if (fresh) CK(cudaMemsetAsync(p->arena32, 0, p->bytes32, s));
    gpcg_status st = convert32(p, s);
    if (st != GPCG_OK) return st;
  }
  if (!fresh) return GPCG_OK;
  for (int f32 = 0; f32 < 2; ++f32) {
    void* a = f32 ? p->arena_t32 : p->arena_t64;
    if (a) CK(cudaMemsetAsync(a, 0, arena_tile_bytes(p, f32), s));
    void* x = f32 ? p->arena_x32 : p->arena_x64;
    if (x) CK(cudaMemsetAsync(x, 0, arena_rx_value_bytes(p, f32), s));
  }
  if (p->arena_xi) CK(cudaMemsetAsync(p->arena_xi, 0, arena_rx_index_bytes(p), s));
  return GPCG_OK;
}

// The status of the device-side input checks' result word.
static gpcg_status flags_status(int h_flags) {
  if (!h_flags) return GPCG_OK;
  if (h_flags & 1) return fail(GPCG_ERR_ARG, "non-finite b, coupling or NaN bound");
  if (h_flags & 2) return fail(GPCG_ERR_ARG, "diagonal entry <= 0 or not finite");
  return fail(GPCG_ERR_INFEASIBLE, "empty box: some l > u, l = +inf or u = -inf");
}

// upload_enqueue, then wait for it and report the checks.
static gpcg_status upload(gpcg_problem* p, const gpcg_stencil* A, const double* b,
                          const double* l, const double* u, cudaStream_t s) {
  gpcg_status st = upload_enqueue(p, A, b, l, u, s);
  int h_flags = 0;
  if (st == GPCG_OK) {
    CK(cudaMemcpyAsync(&h_flags, p->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return st != GPCG_OK ? st : flags_status(h_flags);
}

// A problem with its FP64 arena carved (zeroed on s unless zero is false:
// device_init then clears what the copies do not write) and nothing copied in.
static gpcg_status new_problem(const gpcg_stencil* A, double c, cudaMemPool_t pool,
                               cudaStream_t s, gpcg_problem** out, bool zero = true) {
  gpcg_problem* p = new gpcg_problem();
  geometry(A->dim, A->nx, A->ny, A->nz, p);
  p->c = c;
  p->pool = pool;
  p->pstream = s;
  p->bytes64 = arena64_bytes(p);
  cudaError_t e = dev_alloc(p, &p->arena64, p->bytes64);
  if (e != cudaSuccess) {
    const size_t bytes = p->bytes64;
    p->arena64 = nullptr;
    delete p;
    return fail(e == cudaErrorMemoryAllocation ? GPCG_ERR_OOM : GPCG_ERR_CUDA,
                "allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  carve64(p);
  e = zero ? cudaMemsetAsync(p->arena64, 0, p->bytes64, s) : cudaSuccess;
  if (e != cudaSuccess) {
    delete p;
    return fail(GPCG_ERR_CUDA, "memset: %s", cudaGetErrorString(e));
  }
  *out = p;
  return GPCG_OK;
}

// The TMA descriptors of the FP64 passes (the mask maps first: every staged
// pass reads the free set through them).
static void make_fp64_maps(gpcg_problem* p, cudaStream_t s) {
  p->inst.tma_mask = (!tma_disabled() && make_mask_maps(p, s)) ? 1 : 0;
  p->inst.tma64 = (p->inst.tma_mask && make_maps(p, false, s)) ? 1 : 0;
  p->inst.tma_f64gp = (p->inst.tma64 && make_f64gp_maps(p, s)) ? 1 : 0;
}

extern "C" gpcg_status gpcg_problem_create(const gpcg_stencil* A, const double* b,
                                           const double* l, const double* u, double c,
                                           gpcg_problem** out) {
  if (!out) return fail(GPCG_ERR_ARG, "out is NULL");
  *out = nullptr;
  gpcg_status st = check_problem(A, b, c);
  if (st != GPCG_OK) return st;
  gpcg_problem* p = nullptr;
  cudaStream_t s = 0;
  if ((st = new_problem(A, c, nullptr, s, &p)) != GPCG_OK) return st;
  if ((st = upload(p, A, b, l, u, s)) != GPCG_OK) {
    delete p;
    return st;
  }
  make_fp64_maps(p, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    delete p;
    return fail(GPCG_ERR_CUDA, "problem set-up failed");
  }
  *out = p;
  return GPCG_OK;
}

// Wait for a pending asynchronous update's copies (no device-side work).
static gpcg_status wait_pending_copies(gpcg_problem* p) {
  if (p->pending) CK(cudaEventSynchronize(p->up_ev));
  return GPCG_OK;
}

// A pending asynchronous update's device-side set-up, ordered on s after its
// copies; its input checks are read back into p->h_flags (valid once s has
// reached this point, see settle_status).
static gpcg_status settle(gpcg_problem* p, cudaStream_t s) {
  if (!p->pending) return GPCG_OK;
  p->pending = false;
  CK(cudaStreamWaitEvent(s, p->up_ev, 0));
  gpcg_status st = device_init(p, p->fill_l, p->fill_u, s, false);
  if (st != GPCG_OK) return st;
  *p->h_flags = 0;
  CK(cudaMemcpyAsync(p->h_flags, p->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  return GPCG_OK;
}

// The input checks of the last settled set-up, once its stream has been
// synchronised (GPCG_OK when there was none).
static gpcg_status settle_status(gpcg_problem* p) {
  if (!p->h_flags || *p->h_flags == 0) return GPCG_OK;
  const int f = *p->h_flags;
  *p->h_flags = 0;
  return flags_status(f);
}

// settle on the legacy stream, wait, and report the checks (the synchronous
// entry points other than the solves).
static gpcg_status settle_now(gpcg_problem* p) {
  if (p->bad) return fail(GPCG_ERR_ARG, "the problem's data failed the value checks");
  if (!p->pending) return GPCG_OK;
  gpcg_status st = settle(p, 0);
  if (st != GPCG_OK) return st;
  CK(cudaStreamSynchronize(0));
  st = settle_status(p);
  p->bad = st != GPCG_OK;
  return st;
}

extern "C" gpcg_status gpcg_problem_update(gpcg_problem* p, const gpcg_stencil* A,
                                           const double* b, const double* l, const double* u,
                                           double c) {
  if (!p) return fail(GPCG_ERR_ARG, "problem is NULL");
  gpcg_status st = check_problem(A, b, c);
  if (st != GPCG_OK) return st;
  if (A->dim != p->dim || A->nx != p->nx || A->ny != p->ny || A->nz != p->nz)
    return fail(GPCG_ERR_ARG, "the update's grid differs from the problem's");
  if ((st = wait_pending_copies(p)) != GPCG_OK) return st;
  p->pending = false;
  p->have = false;  // the previous result belongs to the old data
  st = upload(p, A, b, l, u, 0);
  p->bad = st != GPCG_OK;
  if (st != GPCG_OK) return st;
  p->c = c;
  return GPCG_OK;
}

extern "C" gpcg_status gpcg_problem_update_async(gpcg_problem* p, const gpcg_stencil* A,
                                                 const double* b, const double* l,
                                                 const double* u, double c, void* stream) {
  if (!p) return fail(GPCG_ERR_ARG, "problem is NULL");
  gpcg_status st = check_problem(A, b, c);
  if (st != GPCG_OK) return st;
  if (A->dim != p->dim || A->nx != p->nx || A->ny != p->ny || A->nz != p->nz)
    return fail(GPCG_ERR_ARG, "the update's grid differs from the problem's");
  if ((st = wait_pending_copies(p)) != GPCG_OK) return st;
  if (!p->up_ev) CK(cudaEventCreateWithFlags(&p->up_ev, cudaEventDisableTiming));
  if (!p->h_flags) {
    CK(cudaMallocHost(&p->h_flags, sizeof(int)));
    *p->h_flags = 0;
  }
  // every other entry point returns with its work on p complete, so nothing
  // in flight still reads the arrays these copies overwrite
  cudaStream_t s = (cudaStream_t)stream;
  p->have = false;
  if ((st = upload_copies(p, A, b, l, u, s, nullptr)) != GPCG_OK) return st;
  CK(cudaEventRecord(p->up_ev, s));
  p->pending = true;
  p->bad = false;
  p->fill_l = l == nullptr;
  p->fill_u = u == nullptr;
  p->c = c;
  return GPCG_OK;
}

extern "C" void gpcg_problem_destroy(gpcg_problem* p) { delete p; }

extern "C" int64_t gpcg_problem_size(const gpcg_problem* p) { return p ? p->n : 0; }

extern "C" void gpcg_default_options(gpcg_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->tau_abs = 0.0;
  o->tau_rel = 1e-8;
  o->eta1 = 0.1;
  o->eta2 = 0.05;
  o->mu = 0.01;
  o->eta2_shrink = 0.1;
  o->eta2_floor = 1e-12;
  o->max_outer = 10000;
  o->max_gp = 50;
  o->max_cg = 10000;
  o->max_ls = 60;
  o->precision = GPCG_FP64;
  o->refine = 2;
  o->x0 = nullptr;
  o->cuda_stream = nullptr;
  o->lambda_min = 0.0;
  o->precond = GPCG_PRECOND_NONE;
  o->cg_system = GPCG_CG_MASKED;
  o->path = GPCG_PATH_AUTO;
}

static gpcg_status check_options(const gpcg_options* o) {
  if (!o) return fail(GPCG_ERR_ARG, "options are NULL");
  if (!(o->tau_abs >= 0.0) || !(o->tau_rel >= 0.0)) return fail(GPCG_ERR_ARG, "bad tolerance");
  if (!(o->eta1 > 0.0 && o->eta1 < 1.0) || !(o->eta2 > 0.0 && o->eta2 < 1.0))
    return fail(GPCG_ERR_ARG, "eta1 and eta2 must lie in (0,1)");
  if (!(o->mu > 0.0 && o->mu < 0.5)) return fail(GPCG_ERR_ARG, "mu must lie in (0,1/2)");
  if (!(o->eta2_shrink > 0.0 && o->eta2_shrink <= 1.0) || !(o->eta2_floor >= 0.0))
    return fail(GPCG_ERR_ARG, "bad eta2_shrink / eta2_floor");
  if (o->max_outer < 1 || o->max_gp < 1 || o->max_cg < 0 || o->max_ls < 0)
    return fail(GPCG_ERR_ARG, "bad iteration caps");
  if (o->precision != GPCG_FP64 && o->precision != GPCG_MIXED)
    return fail(GPCG_ERR_ARG, "unknown precision");
  if (o->refine < 0 || o->refine > 2) return fail(GPCG_ERR_ARG, "refine must be 0, 1 or 2");
  if (o->precond != GPCG_PRECOND_NONE && o->precond != GPCG_PRECOND_JACOBI &&
      o->precond != GPCG_PRECOND_TILE)
    return fail(GPCG_ERR_ARG, "unknown preconditioner");
  if (o->cg_system != GPCG_CG_MASKED && o->cg_system != GPCG_CG_EXTRACTED)
    return fail(GPCG_ERR_ARG, "unknown CG system");
  if (o->cg_system == GPCG_CG_EXTRACTED && o->precond == GPCG_PRECOND_TILE)
    return fail(GPCG_ERR_ARG, "the tile preconditioner works on the masked system only");
  if (o->path != GPCG_PATH_AUTO && o->path != GPCG_PATH_ENGINE && o->path != GPCG_PATH_RESIDENT)
    return fail(GPCG_ERR_ARG, "unknown path");
  return GPCG_OK;
}

static Opts make_opts(const gpcg_options* o, double c, bool use_x0) {
  Opts r{};
  r.tau_abs = o->tau_abs;
  r.tau_rel = o->tau_rel;
  r.eta1 = o->eta1;
  r.eta2 = o->eta2;
  r.mu = o->mu;
  r.eta2_shrink = o->eta2_shrink;
  r.eta2_floor = o->eta2_floor;
  r.eta2_refine = std::max(o->eta2 * o->eta2_shrink, o->eta2_floor);
  r.c = c;
  r.max_outer = o->max_outer;
  r.max_gp = o->max_gp;
  r.max_cg = o->max_cg;
  r.max_ls = o->max_ls;
  r.mixed = o->precision == GPCG_MIXED;
  r.refine = o->refine;
  r.use_x0 = use_x0 ? 1 : 0;
  r.extract = o->cg_system == GPCG_CG_EXTRACTED ? 1 : 0;
  r.precond = o->precond == GPCG_PRECOND_JACOBI ? PC_JACOBI
              : o->precond == GPCG_PRECOND_TILE  ? PC_TILE
                                                 : PC_NONE;
  return r;
}

// The pass kernel instantiation a solve with these options needs; `any3d`:
// the launch has 3-D instances (a mixed solve without preconditioner then
// takes the kernel with the fused 3-D step).
static int feature_set(const gpcg_options* o, bool any3d) {
  if (o->precond == GPCG_PRECOND_TILE) return FEAT_TILE;
  if (o->cg_system == GPCG_CG_EXTRACTED) return FEAT_EXT;
  if (o->precision == GPCG_FP64) return FEAT_F64;
  if (any3d && o->precond == GPCG_PRECOND_NONE) return FEAT_3D;
  return 0;
}

static Ctl fresh_ctl() {
  Ctl C;
  memset(&C, 0, sizeof(C));
  C.pass = P_START;
  C.status = S_RUNNING;
  C.mixed_nA = -1.0;
  return C;
}

// ------------------------------------------------------------- engine --

// Build (or reuse) the executable graph for `tiles` CTAs per pass.
// mode 0: WHILE-conditional graph whose body is kBody passes; the pass kernel
// clears the condition once every instance is done or the pass cap is hit.
// mode 1: a plain graph of `steps` passes replayed by the host.
static constexpr int kBody = 16;

static gpcg_status get_graph(Scratch& sc, long long tiles, int mode, int steps, unsigned cap,
                             int feat) {
  const bool same = sc.gexec && sc.g_mode == mode && (mode == 0 || sc.g_steps == steps) &&
                    sc.g_no_pdl == env_no_pdl() && sc.g_feat == feat;
  if (same && sc.g_tiles == tiles) return GPCG_OK;
  if (same && mode == 1 && !sc.nodes.empty()) {
    // only the work items changed: set the pass nodes' grid and arguments in
    // the instantiated graph (no new instantiation)
    EngineArgs args{sc.d_insts, sc.d_ctl,  sc.d_tiles, (int)tiles, sc.d_queue, (unsigned*)(sc.d_queue + 1),
                    sc.d_live,   sc.d_npass, sc.d_queue + 2, cap, 0ull};
    void* kp[] = {&args};
    cudaKernelNodeParams k;
    memset(&k, 0, sizeof(k));
    k.func = const_cast<void*>(pass_kernel_ptr(false, feat));
    k.gridDim = dim3((unsigned)pass_grid((int)tiles));
    k.blockDim = dim3(kThreads);
    k.sharedMemBytes = kDynSmem;
    k.kernelParams = kp;
    bool ok = true;
    for (cudaGraphNode_t node : sc.nodes)
      if (cudaGraphExecKernelNodeSetParams(sc.gexec, node, &k) != cudaSuccess) {
        cudaGetLastError();
        ok = false;
        break;
      }
    if (ok) {
      sc.g_tiles = tiles;
      return GPCG_OK;
    }
  }
  sc.invalidate();
  EngineArgs args{sc.d_insts, sc.d_ctl,  sc.d_tiles, (int)tiles, sc.d_queue, (unsigned*)(sc.d_queue + 1),
                  sc.d_live,   sc.d_npass, sc.d_queue + 2, cap, 0ull};
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  cudaGraph_t body = g;
  int count = steps;
  gpcg_status st = GPCG_OK;
  if (mode == 0) {
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
      alignas(cudaGraphNodeParams) unsigned char cp_buf[sizeof(cudaGraphNodeParams)];
      memset(cp_buf, 0, sizeof(cp_buf));
      cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_buf);
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t cn;
      e = cudaGraphAddNode(&cn, g, nullptr, nullptr, 0, &cp);
      if (e == cudaSuccess) {
        body = cp.conditional.phGraph_out[0];
        args.cond = (unsigned long long)h;
        count = kBody;
      }
    }
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return fail(GPCG_ERR_CUDA, "conditional graph set-up failed: %s", cudaGetErrorString(e));
    }
  }
  void* kp[] = {&args};
  cudaKernelNodeParams k;
  memset(&k, 0, sizeof(k));
  k.func = const_cast<void*>(pass_kernel_ptr(mode == 0, feat));
  k.gridDim = dim3((unsigned)pass_grid((int)tiles));
  k.blockDim = dim3(kThreads);
  k.sharedMemBytes = kDynSmem;
  k.kernelParams = kp;
  // consecutive passes are joined by programmatic edges: the next pass's CTAs
  // start (and load their static descriptors) while the previous pass's
  // finalizer runs, and wait for its results in the kernel.  Plain edges are
  // used where the driver does not accept them.
  bool pdl = !env_no_pdl();
  cudaGraphNode_t prev = nullptr;
  for (int i = 0; i < count; ++i) {
    cudaGraphNode_t node;
    cudaError_t e = cudaErrorUnknown;
    if (prev && pdl) {
      alignas(cudaGraphNodeParams) unsigned char np_buf[sizeof(cudaGraphNodeParams)];
      memset(np_buf, 0, sizeof(np_buf));
      cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(np_buf);
      np.type = cudaGraphNodeTypeKernel;
      np.kernel.func = k.func;
      np.kernel.gridDim = k.gridDim;
      np.kernel.blockDim = k.blockDim;
      np.kernel.sharedMemBytes = k.sharedMemBytes;
      np.kernel.kernelParams = k.kernelParams;
      cudaGraphEdgeData ed;
      memset(&ed, 0, sizeof(ed));
      ed.from_port = cudaGraphKernelNodePortProgrammatic;
      ed.type = cudaGraphDependencyTypeProgrammatic;
      e = cudaGraphAddNode(&node, body, &prev, &ed, 1, &np);
      if (e != cudaSuccess) {
        cudaGetLastError();
        pdl = false;
      }
    }
    if (e != cudaSuccess)
      e = cudaGraphAddKernelNode(&node, body, prev ? &prev : nullptr, prev ? 1 : 0, &k);
    if (e != cudaSuccess) {
      st = fail(GPCG_ERR_CUDA, "cudaGraphAddKernelNode: %s", cudaGetErrorString(e));
      break;
    }
    prev = node;
    if (mode == 1) sc.nodes.push_back(node);
  }
  if (st == GPCG_OK) {
    cudaError_t e = cudaGraphInstantiate(&sc.gexec, g, 0);
    if (e != cudaSuccess) st = fail(GPCG_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  }
  sc.g_pdl = pdl;
  sc.g_no_pdl = env_no_pdl();
  sc.g_feat = feat;
  if (st != GPCG_OK) {
    cudaGraphDestroy(g);
    sc.gexec = nullptr;
    sc.nodes.clear();
    return st;
  }
  sc.graph = g;
  sc.g_tiles = tiles;
  sc.g_mode = mode;
  sc.g_steps = steps;
  return GPCG_OK;
}

// Run the engine until every instance in the scratch tables is done.
// coop: the launch's work items all belong to one instance and may run as
// one cooperative launch (*coop_used tells whether they did).
static gpcg_status run_engine(Scratch& sc, int n_live, long long tiles, cudaStream_t s,
                              int feat, bool coop, bool* coop_used) {
  const unsigned cap = env_pass_cap();
  const int mode = env_engine_mode();
  *coop_used = false;
  std::unique_lock<std::mutex> coop_lock;  // held until a cooperative kernel has finished
  sc.h_pin[0] = n_live;
  sc.h_pin[1] = 0;
  CK(cudaMemcpyAsync(sc.d_live, &sc.h_pin[0], sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(sc.d_npass, &sc.h_pin[1], sizeof(unsigned), cudaMemcpyHostToDevice, s));
  if (mode == 0 && coop && tiles > 0 && tiles <= (long long)pass_grid(1 << 30)) {
    // every pass in one launch: the counters (queue, exits, barrier) start
    // at zero; the pass cap keeps the barrier's running count below 2^32
    coop_lock = std::unique_lock<std::mutex>(coop_mutex());
    CK(cudaMemsetAsync(sc.d_queue, 0, 4 * sizeof(int), s));
    EngineArgs args{sc.d_insts, sc.d_ctl,  sc.d_tiles, (int)tiles, sc.d_queue, (unsigned*)(sc.d_queue + 1),
                    sc.d_live,   sc.d_npass, sc.d_queue + 2, cap, 0ull};
    args.gbar = (unsigned*)(sc.d_queue + 3);
    args.pass_cap = std::min<unsigned>(cap, 0xffffffffu / (unsigned)tiles - 1u);
    const cudaError_t e = launch_pass_coop(args, (int)tiles, s, feat);
    if (e == cudaSuccess) {
      *coop_used = true;
    } else {
      cudaGetLastError();  // not launched (no room for every block): run the graph below
      coop_lock.unlock();
    }
  }
  if (*coop_used) {
    CK(cudaMemcpyAsync(&sc.h_pin[0], sc.d_live, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&sc.h_pin[1], sc.d_npass, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  } else if (mode == 0) {
    gpcg_status st = get_graph(sc, tiles, 0, kBody, cap, feat);
    if (st != GPCG_OK) return st;
    CK(cudaGraphLaunch(sc.gexec, s));
    CK(cudaMemcpyAsync(&sc.h_pin[0], sc.d_live, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&sc.h_pin[1], sc.d_npass, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  } else {
    int steps = 8;
    unsigned done_passes = 0;
    for (;;) {
      gpcg_status st = get_graph(sc, tiles, 1, steps, cap, feat);
      if (st != GPCG_OK) return st;
      CK(cudaGraphLaunch(sc.gexec, s));
      CK(cudaMemcpyAsync(&sc.h_pin[0], sc.d_live, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(&sc.h_pin[1], sc.d_npass, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      done_passes += steps;
      if (sc.h_pin[0] == 0 || done_passes >= cap) break;
      steps = std::min(steps * 2, 256);
    }
  }
  CK(cudaMemcpyAsync(&sc.h_pin[2], sc.d_queue + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (sc.h_pin[2] != 0) {
    // blocks that gave up left without counting their exit: clear the queue,
    // exit and barrier counters with the error word for the next launch
    const int bits = sc.h_pin[2];
    cudaMemset(sc.d_queue, 0, 4 * sizeof(int));
    if (bits & 2) return fail(GPCG_ERR_CUDA, "a pass ran in a kernel without its code");
    return fail(GPCG_ERR_TIMEOUT, "a bounded wait %s gave up",
                (bits & 4) ? "at the grid barrier" : "for a TMA copy");
  }
  if (sc.h_pin[0] != 0) return fail(GPCG_ERR_TIMEOUT, "pass cap reached with live solves");
  return GPCG_OK;
}

// The arenas and tensor maps a solve with options o needs.  init = false
// leaves their device-side initialisation to device_init (a server's
// uploads: only copies run on the worker's stream).
static gpcg_status prepare_instance(gpcg_problem* p, const gpcg_options* o, cudaStream_t s,
                                    DevInst* out, bool init = true) {
  gpcg_status st;
  if (o->precision == GPCG_MIXED && (st = ensure_mixed(p, s, init)) != GPCG_OK) return st;
  if (o->precond == GPCG_PRECOND_TILE &&
      (st = ensure_tile(p, o->precision == GPCG_MIXED, s, init)) != GPCG_OK)
    return st;
  if (o->cg_system == GPCG_CG_EXTRACTED &&
      (st = ensure_extract(p, o->precision == GPCG_MIXED, s, init)) != GPCG_OK)
    return st;
  const bool use_x0 = o->x0 != nullptr;
  if (use_x0 && (st = copy_in(p, (double*)p->inst.x0, o->x0, s)) != GPCG_OK) return st;
  *out = p->inst;
  out->opt = make_opts(o, p->c, use_x0);
  return GPCG_OK;
}

static int to_status(int s) {
  switch (s) {
    case S_OK: return GPCG_OK;
    case S_NUMERIC: return GPCG_ERR_NUMERIC;
    case S_MAXIT: return GPCG_ERR_MAXIT;
    case S_LINESEARCH: return GPCG_ERR_LINESEARCH;
    case S_TIMEOUT: return GPCG_ERR_TIMEOUT;
    default: return GPCG_ERR_PENDING;
  }
}

// Shared-memory bytes of the resident solve of p under options o, 0 when
// that solver does not take it.
static size_t resident_fit(const gpcg_problem* p, const gpcg_options* o) {
  if (o->path == GPCG_PATH_ENGINE) return 0;
  if (o->precond == GPCG_PRECOND_TILE || o->cg_system != GPCG_CG_MASKED) return 0;
  return resident_smem(p->dim, p->n, o->precision == GPCG_MIXED,
                       o->precond == GPCG_PRECOND_JACOBI);
}

static gpcg_status solve_set(gpcg_problem* const* probs, int count, const gpcg_options* o,
                             Scratch& sc) {
  cudaStream_t s = (cudaStream_t)o->cuda_stream;
  // the problems the resident solver takes; the others go to the engine
  std::vector<int> res_ids;
  std::vector<char> resident(count, 0);
  size_t res_smem = 0;
  long long tiles = 0;
  for (int k = 0; k < count; ++k) {
    const size_t b = resident_fit(probs[k], o);
    if (b == 0 && o->path == GPCG_PATH_RESIDENT)
      return fail(GPCG_ERR_ARG, "problem %d does not fit the resident solver", k);
    if (b > 0) {
      resident[k] = 1;
      res_ids.push_back(k);
      res_smem = std::max(res_smem, b);
    } else {
      tiles += probs[k]->n_groups;
    }
  }
  const int n_eng = count - (int)res_ids.size();
  gpcg_status st = sc.ensure(count, std::max(tiles, 1LL));
  if (st != GPCG_OK) return st;
  std::vector<DevInst> insts(count);
  Ctl c0 = fresh_ctl();
  c0.gp32 = o->precision == GPCG_MIXED ? 1 : 0;  // the mixed phase streams FP32
  std::vector<Ctl> ctl(count, c0);
  std::vector<int2> table((size_t)tiles);
  long long t = 0;
  // pending asynchronous updates: their set-up, and their value checks
  // before anything runs on the data
  bool settled = false;
  for (int k = 0; k < count; ++k) {
    if (probs[k]->bad)
      return fail(GPCG_ERR_ARG, "problem %d: its data failed the value checks", k);
    settled |= probs[k]->pending;
    if ((st = settle(probs[k], s)) != GPCG_OK) return st;
  }
  if (settled) {
    CK(cudaStreamSynchronize(s));
    for (int k = 0; k < count; ++k)
      if ((st = settle_status(probs[k])) != GPCG_OK) {
        probs[k]->bad = true;
        return st;
      }
  }
  const bool extract = o->cg_system == GPCG_CG_EXTRACTED;
  bool any3d = false;
  for (int k = 0; k < count; ++k) any3d |= !resident[k] && probs[k]->dim == 3;
  const int feat = feature_set(o, any3d);
  for (int k = 0; k < count; ++k) {
    if ((st = prepare_instance(probs[k], o, s, &insts[k])) != GPCG_OK) return st;
    if (resident[k]) continue;
    if ((feat & FEAT_3D) == 0) insts[k].tma3 = 0;  // this launch's kernel lacks the 3-D step
    // work items of `span` consecutive groups (their sums stay per group)
    const int span = item_span(probs[k], tiles, extract);
    insts[k].span = span;
    for (int j = 0; j < probs[k]->n_groups; j += span) table[(size_t)t++] = make_int2(k, j);
  }
  tiles = t;  // work items of the launch
  CK(cudaMemcpyAsync(sc.d_insts, insts.data(), sizeof(DevInst) * count, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(sc.d_ctl, ctl.data(), sizeof(Ctl) * count, cudaMemcpyHostToDevice, s));
  if (tiles > 0)
    CK(cudaMemcpyAsync(sc.d_tiles, table.data(), sizeof(int2) * tiles, cudaMemcpyHostToDevice,
                       s));
  if (!res_ids.empty()) {
    CK(cudaMemcpyAsync(sc.d_ids, res_ids.data(), sizeof(int) * res_ids.size(),
                       cudaMemcpyHostToDevice, s));
    CK(launch_resident(sc.d_insts, sc.d_ids, sc.d_ctl, (int)res_ids.size(), res_smem,
                       env_pass_cap(), s));
  }
  gpcg_status run = GPCG_OK;
  sc.h_pin[1] = 0;
  // one engine instance: its passes may run in one cooperative launch
  const bool coop = n_eng == 1 && !extract && !env_no_coop();
  bool coop_used = false;
  if (n_eng > 0) run = run_engine(sc, n_eng, tiles, s, feat, coop, &coop_used);
  if (run != GPCG_OK && run != GPCG_ERR_TIMEOUT) return run;
  CK(cudaMemcpyAsync(ctl.data(), sc.d_ctl, sizeof(Ctl) * count, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  gpcg_status first_bad = GPCG_OK;
  for (int k = 0; k < count; ++k) {
    if (!ctl[k].done) ctl[k].status = S_TIMEOUT;
    probs[k]->launches = (resident[k] || coop_used) ? 1 : (unsigned)sc.h_pin[1];
    probs[k]->last_path = resident[k] ? GPCG_PATH_RESIDENT : GPCG_PATH_ENGINE;
    probs[k]->last = ctl[k];
    probs[k]->have = true;
    probs[k]->lambda_min = o->lambda_min;
    const gpcg_status sk = (gpcg_status)to_status(ctl[k].status);
    if (sk != GPCG_OK && first_bad == GPCG_OK) first_bad = sk;
  }
  if (first_bad != GPCG_OK)
    return fail(first_bad, "solve ended with status %d", (int)first_bad);
  return GPCG_OK;
}

extern "C" gpcg_status gpcg_solve(gpcg_problem* p, const gpcg_options* opt) {
  if (!p) return fail(GPCG_ERR_ARG, "problem is NULL");
  gpcg_status st = check_options(opt);
  if (st != GPCG_OK) return st;
  gpcg_problem* one[1] = {p};
  return solve_set(one, 1, opt, p->sc);
}

extern "C" gpcg_status gpcg_solve_batch(gpcg_problem* const* probs, int count,
                                        const gpcg_options* opt) {
  if (!probs || count < 1) return fail(GPCG_ERR_ARG, "empty batch");
  for (int k = 0; k < count; ++k)
    if (!probs[k]) return fail(GPCG_ERR_ARG, "problem %d is NULL", k);
  gpcg_status st = check_options(opt);
  if (st != GPCG_OK) return st;
  Scratch sc;
  return solve_set(probs, count, opt, sc);
}

static void fill_stats(const gpcg_problem* p, gpcg_stats* s) {
  const Ctl& C = p->last;
  memset(s, 0, sizeof(*s));
  s->q = 0.5 * C.xgb + p->c;
  s->pg_norm = std::sqrt(C.pg2);
  s->pg_norm0 = C.pg0;
  s->tau = C.tau;
  s->n_active = (int64_t)C.nA;
  s->n_binding = (int64_t)C.nB;
  s->n_free = p->n - (int64_t)C.nA;
  s->outer_iters = C.outer_iters;
  s->gp_iters = C.gp_iters;
  s->cg_iters = C.cg_iters;
  s->ls_trials = C.ls_trials;
  s->refine_cg_iters = C.refine_cg_iters;
  s->passes = C.passes;
  s->status = to_status(C.status);
  s->err_bound = p->lambda_min > 0.0 ? s->pg_norm / p->lambda_min : -1.0;
  s->alg_bytes = C.alg_bytes;
  s->launches = p->launches;
  const DevInst& I = p->inst;
  s->staged = (I.tma_mask ? 1 : 0) | (I.tma64 ? 2 : 0) | (I.tma32 ? 4 : 0) | (I.tma_gp ? 8 : 0);
  s->fp64_gp_iters = C.fp64_gp;
  s->mixed_n_active = (int64_t)C.mixed_nA;
  s->path = p->last_path;
  s->reserved = 0;
}

extern "C" gpcg_status gpcg_result(const gpcg_problem* p, double* x_out, gpcg_stats* stats) {
  if (!p) return fail(GPCG_ERR_ARG, "problem is NULL");
  if (!p->have) return fail(GPCG_ERR_PENDING, "no solve has run on this problem");
  if (x_out) {
    const double* x = p->inst.x[p->last.cur];
    CK(cudaMemcpy2D(x_out, sizeof(double) * p->nx, x, sizeof(double) * p->px,
                    sizeof(double) * p->nx, (size_t)p->ny * p->nz, cudaMemcpyDefault));
  }
  if (stats) fill_stats(p, stats);
  return GPCG_OK;
}

// ------------------------------------------- masked product entry points --

static bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The pass kernel's feature set a pass needs.
static int pass_feature(int pass) {
  if (pass == P_CG_Z) return FEAT_TILE;
  if (pass >= P_RX_COUNT && pass <= P_RW) return FEAT_EXT;
  return 0;
}

static gpcg_status one_pass(gpcg_problem* p, Ctl C, cudaStream_t s, Ctl* out) {
  Scratch& sc = p->sc;
  gpcg_status st = sc.ensure(1, p->n_groups);
  if (st != GPCG_OK) return st;
  std::vector<int2> table((size_t)p->n_groups);
  for (int j = 0; j < p->n_groups; ++j) table[(size_t)j] = make_int2(0, j);
  DevInst I = p->inst;
  I.opt = Opts{};
  CK(cudaMemcpyAsync(sc.d_insts, &I, sizeof(DevInst), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(sc.d_ctl, &C, sizeof(Ctl), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(sc.d_tiles, table.data(), sizeof(int2) * table.size(),
                     cudaMemcpyHostToDevice, s));
  sc.h_pin[0] = 1;
  sc.h_pin[1] = 0;
  CK(cudaMemcpyAsync(sc.d_live, &sc.h_pin[0], sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(sc.d_npass, &sc.h_pin[1], sizeof(unsigned), cudaMemcpyHostToDevice, s));
  EngineArgs E{sc.d_insts, sc.d_ctl,  sc.d_tiles,    p->n_groups, sc.d_queue, (unsigned*)(sc.d_queue + 1),
               sc.d_live,   sc.d_npass, sc.d_queue + 2, 0xffffffffu, 0ull};
  CK(launch_pass(E, pass_grid(p->n_groups), s, pass_feature(C.pass)));
  if (out) {
    CK(cudaMemcpyAsync(out, sc.d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return GPCG_OK;
}

static Ctl spmv_ctl(bool f32, int cur, int pcur) {
  Ctl C = fresh_ctl();
  C.pass = P_CG_B;
  C.first_cg = 0;
  C.beta = 0.0;
  C.cur = cur;
  C.pcur = pcur;
  C.cg32 = f32 ? 1 : 0;
  C.hold = 1;
  return C;
}

// The standalone masked product runs its own kernel on 2-D instances whose
// maps of the precision are valid (the generic engine pass otherwise).
static bool lean_spmv(const gpcg_problem* p, bool f32) {
  return p->dim == 2 && p->inst.tma_mask && (f32 ? p->inst.tma32 : p->inst.tma64) != 0;
}

static gpcg_status ms_scratch(gpcg_problem* p, cudaStream_t s) {
  if (p->ms_buf) return GPCG_OK;
  const size_t n = (size_t)ms_max_ctas() + 8;
  CK(cudaMalloc(&p->ms_buf, n * sizeof(double)));
  CK(cudaMemsetAsync(p->ms_buf, 0, n * sizeof(double), s));
  return GPCG_OK;
}

// One launch of the standalone kernel on the problem's p[0] (operand) and
// Ap[1] (result) with free-set words `mask`.
static gpcg_status ms_launch(gpcg_problem* p, bool f32, int mask, cudaStream_t s,
                             bool pdl = false) {
  const size_t c = (size_t)ms_max_ctas();
  double* part = p->ms_buf;
  DevInst& I = p->inst;
  void* y = f32 ? (void*)I.Ap32[1] : (void*)I.Ap64[1];
  CK(launch_mspmv(I, f32, mask, y, part, (unsigned*)(part + c + 1), part + c, (int*)(part + c + 2),
                  s, pdl));
  return GPCG_OK;
}

static gpcg_status ms_check(gpcg_problem* p, cudaStream_t s, double* result) {
  const size_t c = (size_t)ms_max_ctas();
  double r = 0.0;
  int err = 0;
  CK(cudaMemcpyAsync(&r, p->ms_buf + c, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&err, (int*)(p->ms_buf + c + 2), sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (err) {
    // the CTAs that gave up never counted themselves: reset flag and counter
    cudaMemsetAsync(p->ms_buf + c + 1, 0, 2 * sizeof(double), s);
    cudaStreamSynchronize(s);
    return fail(GPCG_ERR_TIMEOUT, "a bounded wait for a TMA copy gave up");
  }
  if (result) *result = r;
  return GPCG_OK;
}

extern "C" gpcg_status gpcg_masked_spmv(gpcg_problem* p, const uint8_t* free_mask,
                                        const double* pv, double* y, double* pAp, int precision,
                                        void* cuda_stream) {
  if (!p || !free_mask || !pv || !y) return fail(GPCG_ERR_ARG, "NULL argument");
  {
    const gpcg_status ps = settle_now(p);
    if (ps != GPCG_OK) return ps;
  }
  if (precision != GPCG_FP64 && precision != GPCG_MIXED)
    return fail(GPCG_ERR_ARG, "unknown precision");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const bool f32 = precision == GPCG_MIXED;
  gpcg_status st;
  if (f32 && (st = ensure_mixed(p, s, true)) != GPCG_OK) return st;
  uint8_t* dm = nullptr;
  double* dp = nullptr;
  double* dy = nullptr;
  const bool m_dev = is_device_ptr(free_mask), p_dev = is_device_ptr(pv), y_dev = is_device_ptr(y);
  std::vector<void*> temps;
  auto cleanup = [&]() {
    for (void* t : temps) cudaFree(t);
  };
  st = GPCG_OK;
  do {
    if (m_dev) {
      dm = const_cast<uint8_t*>(free_mask);
    } else {
      if (cudaMalloc(&dm, p->n) != cudaSuccess) { st = fail(GPCG_ERR_OOM, "temp alloc"); break; }
      temps.push_back(dm);
      if (cudaMemcpyAsync(dm, free_mask, p->n, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        st = fail(GPCG_ERR_CUDA, "copy mask");
        break;
      }
    }
    if (p_dev) {
      dp = const_cast<double*>(pv);
    } else {
      if (cudaMalloc(&dp, sizeof(double) * p->n) != cudaSuccess) { st = fail(GPCG_ERR_OOM, "temp alloc"); break; }
      temps.push_back(dp);
      if (cudaMemcpyAsync(dp, pv, sizeof(double) * p->n, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        st = fail(GPCG_ERR_CUDA, "copy p");
        break;
      }
    }
    if (y_dev) {
      dy = y;
    } else {
      if (cudaMalloc(&dy, sizeof(double) * p->n) != cudaSuccess) { st = fail(GPCG_ERR_OOM, "temp alloc"); break; }
      temps.push_back(dy);
    }
    DevInst& I = p->inst;
    if (lean_spmv(p, f32)) {
      void* pm = f32 ? (void*)I.p32[0] : (void*)I.p64[0];
      double r = 0.0;
      if ((st = ms_scratch(p, s)) != GPCG_OK) break;
      if (launch_mspmv_setup(I, dm, dp, I.mask[0], pm, f32, s) != cudaSuccess) {
        st = fail(GPCG_ERR_CUDA, "spmv set-up launch");
        break;
      }
      if ((st = ms_launch(p, f32, 0, s)) != GPCG_OK) break;
      const void* yb = f32 ? (const void*)I.Ap32[1] : (const void*)I.Ap64[1];
      if (launch_unpad(I, yb, f32, dy, s) != cudaSuccess) {
        st = fail(GPCG_ERR_CUDA, "unpad launch");
        break;
      }
      if (!y_dev &&
          cudaMemcpyAsync(y, dy, sizeof(double) * p->n, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
        st = fail(GPCG_ERR_CUDA, "copy y");
        break;
      }
      if ((st = ms_check(p, s, &r)) != GPCG_OK) break;
      if (pAp) *pAp = r;
      p->have = false;  // the solve's vectors were overwritten
      break;
    }
    // the standalone pass is a CG_B step at pcur = 0 with beta = 0: it reads
    // r[1] (p = -r) and writes p[1], Ap[1]
    void* r = f32 ? (void*)I.r32[1] : (void*)I.r64[1];
    void* p0 = f32 ? (void*)I.p32[0] : (void*)I.p64[0];
    if (launch_spmv_setup(I, dm, dp, I.mask[0], r, p0, f32, s) != cudaSuccess) {
      st = fail(GPCG_ERR_CUDA, "spmv set-up launch");
      break;
    }
    Ctl out;
    if ((st = one_pass(p, spmv_ctl(f32, 0, 0), s, &out)) != GPCG_OK) break;
    const void* ap = f32 ? (const void*)I.Ap32[1] : (const void*)I.Ap64[1];
    if (launch_unpad(I, ap, f32, dy, s) != cudaSuccess) {
      st = fail(GPCG_ERR_CUDA, "unpad launch");
      break;
    }
    if (!y_dev &&
        cudaMemcpyAsync(y, dy, sizeof(double) * p->n, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
      st = fail(GPCG_ERR_CUDA, "copy y");
      break;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      st = fail(GPCG_ERR_CUDA, "synchronize: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    if (pAp) *pAp = out.red[0];
    p->have = false;  // the solve's vectors were overwritten
  } while (0);
  cleanup();
  return st;
}

extern "C" gpcg_status gpcg_reduced_system(gpcg_problem* p, const uint8_t* free_mask,
                                           int precision, int64_t* m, int32_t* fidx,
                                           double* diag, int32_t* nb, double* val,
                                           void* cuda_stream) {
  if (!p || !free_mask || !m || !fidx || !diag || !nb || !val)
    return fail(GPCG_ERR_ARG, "NULL argument");
  if (precision != GPCG_FP64 && precision != GPCG_MIXED)
    return fail(GPCG_ERR_ARG, "unknown precision");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const bool f32 = precision == GPCG_MIXED;
  gpcg_status st;
  if ((st = settle_now(p)) != GPCG_OK) return st;
  if (f32 && (st = ensure_mixed(p, s, true)) != GPCG_OK) return st;
  if ((st = ensure_extract(p, f32, s, true)) != GPCG_OK) return st;
  DevInst& I = p->inst;
  uint8_t* dm = nullptr;
  CK(cudaMalloc(&dm, (size_t)p->n));
  st = GPCG_OK;
  do {
    if (cudaMemcpyAsync(dm, free_mask, (size_t)p->n, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      st = fail(GPCG_ERR_CUDA, "copy mask");
      break;
    }
    // free-set words into mask[0] (the set-up also fills two CG scratch
    // vectors; its value operand is unused here)
    if (launch_spmv_setup(I, dm, I.diag, I.mask[0], I.r64[1], I.p64[1], false, s) !=
        cudaSuccess) {
      st = fail(GPCG_ERR_CUDA, "set-up launch");
      break;
    }
    Ctl C = fresh_ctl();
    C.cur = 0;
    C.pcur = 0;
    C.cg32 = f32 ? 1 : 0;
    C.gp32 = 0;
    C.hold = 1;
    Ctl out;
    C.pass = P_RX_COUNT;
    if ((st = one_pass(p, C, s, &out)) != GPCG_OK) break;
    const long long mm = (long long)out.red[4];
    C.m = (int)mm;
    C.pass = P_RX_MAP;
    if ((st = one_pass(p, C, s, &out)) != GPCG_OK) break;
    C.pass = P_RX_BUILD;
    if ((st = one_pass(p, C, s, &out)) != GPCG_OK) break;
    *m = mm;
    const int nn = 2 * p->dim;
    std::vector<int32_t> fx((size_t)mm);
    if (mm > 0 &&
        cudaMemcpyAsync(fx.data(), I.fidx, sizeof(int) * mm, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess) {
      st = fail(GPCG_ERR_CUDA, "copy fidx");
      break;
    }
    for (int j = 0; j < nn && mm > 0; ++j)
      if (cudaMemcpyAsync(nb + (size_t)j * mm, I.rnb + (size_t)j * p->n, sizeof(int) * mm,
                          cudaMemcpyDeviceToHost, s) != cudaSuccess) {
        st = fail(GPCG_ERR_CUDA, "copy neighbours");
        break;
      }
    if (st != GPCG_OK) break;
    const size_t es = f32 ? sizeof(float) : sizeof(double);
    std::vector<char> dv((size_t)mm * es), vv((size_t)mm * nn * es);
    const char* rd = f32 ? (const char*)I.rd32 : (const char*)I.rd64;
    const char* rv = f32 ? (const char*)I.rv32 : (const char*)I.rv64;
    if (mm > 0 && cudaMemcpyAsync(dv.data(), rd, es * mm, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
      st = fail(GPCG_ERR_CUDA, "copy diagonal");
      break;
    }
    for (int j = 0; j < nn && mm > 0; ++j)
      if (cudaMemcpyAsync(vv.data() + (size_t)j * mm * es, rv + (size_t)j * p->n * es, es * mm,
                          cudaMemcpyDeviceToHost, s) != cudaSuccess) {
        st = fail(GPCG_ERR_CUDA, "copy couplings");
        break;
      }
    if (st != GPCG_OK) break;
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      st = fail(GPCG_ERR_CUDA, "synchronize: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    // padded point index -> row-major index of the unpadded grid
    for (long long k = 0; k < mm; ++k) {
      const long long i = fx[(size_t)k];
      const long long ix = i % p->px, row = i / p->px;
      fidx[k] = (int32_t)(ix + (long long)p->nx * row);
    }
    for (size_t k = 0; k < (size_t)mm; ++k)
      diag[k] = f32 ? (double)((const float*)dv.data())[k] : ((const double*)dv.data())[k];
    for (size_t k = 0; k < (size_t)mm * nn; ++k)
      val[k] = f32 ? (double)((const float*)vv.data())[k] : ((const double*)vv.data())[k];
    p->have = false;  // the solve's vectors were overwritten
  } while (0);
  cudaFree(dm);
  return st;
}

extern "C" gpcg_status gpcg_tile_precondition(gpcg_problem* p, const uint8_t* free_mask,
                                              const double* r, double* z, double* rz,
                                              int precision, void* cuda_stream) {
  if (!p || !free_mask || !r || !z) return fail(GPCG_ERR_ARG, "NULL argument");
  {
    const gpcg_status ps = settle_now(p);
    if (ps != GPCG_OK) return ps;
  }
  if (precision != GPCG_FP64 && precision != GPCG_MIXED)
    return fail(GPCG_ERR_ARG, "unknown precision");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const bool f32 = precision == GPCG_MIXED;
  gpcg_status st;
  if (f32 && (st = ensure_mixed(p, s, true)) != GPCG_OK) return st;
  if ((st = ensure_tile(p, f32, s, true)) != GPCG_OK) return st;
  std::vector<void*> temps;
  auto dev_copy = [&](const void* src, size_t bytes, void** out) -> gpcg_status {
    if (is_device_ptr(src)) {
      *out = const_cast<void*>(src);
      return GPCG_OK;
    }
    CK(cudaMalloc(out, bytes));
    temps.push_back(*out);
    CK(cudaMemcpyAsync(*out, src, bytes, cudaMemcpyHostToDevice, s));
    return GPCG_OK;
  };
  do {
    void *dm = nullptr, *dr = nullptr, *dz = z;
    if ((st = dev_copy(free_mask, (size_t)p->n, &dm)) != GPCG_OK) break;
    if ((st = dev_copy(r, sizeof(double) * (size_t)p->n, &dr)) != GPCG_OK) break;
    const bool z_dev = is_device_ptr(z);
    if (!z_dev) {
      if (cudaMalloc(&dz, sizeof(double) * (size_t)p->n) != cudaSuccess) {
        st = fail(GPCG_ERR_OOM, "temp alloc");
        break;
      }
      temps.push_back(dz);
    }
    DevInst& I = p->inst;
    // free-set words into mask[0] (the set-up also fills two CG scratch
    // vectors the pass overwrites), r into the FP64 gradient g[0]
    if (launch_spmv_setup(I, (const uint8_t*)dm, (const double*)dr, I.mask[0], I.r64[1],
                          I.p64[1], false, s) != cudaSuccess) {
      st = fail(GPCG_ERR_CUDA, "set-up launch");
      break;
    }
    if ((st = copy_in(p, I.g[0], (const double*)dr, s)) != GPCG_OK) break;
    Ctl C = fresh_ctl();
    C.pass = P_CG_Z;
    C.cur = 0;
    C.pcur = 0;
    C.cg32 = f32 ? 1 : 0;
    C.gp32 = 0;
    C.hold = 1;
    Ctl out;
    if ((st = one_pass(p, C, s, &out)) != GPCG_OK) break;
    const void* zb = f32 ? (const void*)I.z32[0] : (const void*)I.z64[0];
    if (launch_unpad(I, zb, f32, (double*)dz, s) != cudaSuccess) {
      st = fail(GPCG_ERR_CUDA, "unpad launch");
      break;
    }
    if (!z_dev &&
        cudaMemcpyAsync(z, dz, sizeof(double) * (size_t)p->n, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess) {
      st = fail(GPCG_ERR_CUDA, "copy z");
      break;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      st = fail(GPCG_ERR_CUDA, "synchronize: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    if (rz) *rz = out.red[0];
    p->have = false;  // the solve's vectors were overwritten
  } while (0);
  for (void* t : temps) cudaFree(t);
  return st;
}

// The operand of the timed products: the free set and p of the latest solve
// (words mask[*cur]), or all points free and p = 1 before any solve.
static gpcg_status ms_prepare(gpcg_problem* p, bool f32, cudaStream_t s, int* cur) {
  gpcg_status st;
  if (f32 && (st = ensure_mixed(p, s, true)) != GPCG_OK) return st;
  *cur = p->have ? p->last.cur : 0;
  if (!p->have) {
    uint8_t* dm = nullptr;
    double* dp = nullptr;
    CK(cudaMalloc(&dm, p->n));
    CK(cudaMalloc(&dp, sizeof(double) * p->n));
    CK(cudaMemsetAsync(dm, 1, p->n, s));
    std::vector<double> ones((size_t)p->n, 1.0);
    CK(cudaMemcpyAsync(dp, ones.data(), sizeof(double) * p->n, cudaMemcpyHostToDevice, s));
    DevInst& I = p->inst;
    if (lean_spmv(p, f32))
      CK(launch_mspmv_setup(I, dm, dp, I.mask[0], f32 ? (void*)I.p32[0] : (void*)I.p64[0], f32,
                            s));
    else
      CK(launch_spmv_setup(I, dm, dp, I.mask[0], f32 ? (void*)I.r32[1] : (void*)I.r64[1],
                           f32 ? (void*)I.p32[0] : (void*)I.p64[0], f32, s));
    CK(cudaStreamSynchronize(s));
    cudaFree(dm);
    cudaFree(dp);
    *cur = 0;
  }
  return GPCG_OK;
}

// Algorithmic bytes of one masked product: the bands and p read once, y
// written once, the mask bits.
static double ms_bytes(const gpcg_problem* p, bool f32) {
  const double sv = f32 ? 4.0 : 8.0;
  return (double)p->n * (sv * p->kc + 2.0 * sv + 0.125);
}

extern "C" gpcg_status gpcg_time_masked_spmv_stream(gpcg_problem** probs, int count,
                                                    int precision, int reps, void* cuda_stream,
                                                    double* ms_per_launch,
                                                    double* bytes_per_launch) {
  if (!probs || count < 2 || count > 64 || reps < 1) return fail(GPCG_ERR_ARG, "bad argument");
  if (precision != GPCG_FP64 && precision != GPCG_MIXED)
    return fail(GPCG_ERR_ARG, "unknown precision");
  const bool f32 = precision == GPCG_MIXED;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  for (int k = 0; k < count; ++k) {
    if (!probs[k]) return fail(GPCG_ERR_ARG, "NULL problem %d", k);
    for (int j = 0; j < k; ++j)
      if (probs[j] == probs[k]) return fail(GPCG_ERR_ARG, "problem %d appears twice", k);
  }
  std::vector<int> cur((size_t)count, 0);
  double bytes = 0.0;
  gpcg_status st;
  for (int k = 0; k < count; ++k) {
    gpcg_problem* p = probs[k];
    if ((st = settle_now(p)) != GPCG_OK) return st;
    if ((st = ms_prepare(p, f32, s, &cur[(size_t)k])) != GPCG_OK) return st;
    if (!lean_spmv(p, f32))
      return fail(GPCG_ERR_ARG, "problem %d: not a 2-D problem on the staged path", k);
    if ((st = ms_scratch(p, s)) != GPCG_OK) return st;
    if ((st = ms_launch(p, f32, cur[(size_t)k], s)) != GPCG_OK) return st;  // untimed
    bytes += ms_bytes(p, f32);
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, s));
  // consecutive launches are distinct problems, so each may start while the
  // previous one drains (programmatic dependent launches)
  for (int r = 0; r < reps && st == GPCG_OK; ++r)
    for (int k = 0; k < count && st == GPCG_OK; ++k)
      st = ms_launch(probs[k], f32, cur[(size_t)k], s, true);
  CK(cudaEventRecord(e1, s));
  CK(cudaStreamSynchronize(s));
  float ms = 0.f;
  const cudaError_t et = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != GPCG_OK) return st;
  if (et != cudaSuccess) return fail(GPCG_ERR_CUDA, "event timing: %s", cudaGetErrorString(et));
  for (int k = 0; k < count; ++k)
    if ((st = ms_check(probs[k], s, nullptr)) != GPCG_OK) return st;
  if (ms_per_launch) *ms_per_launch = (double)ms / ((double)reps * count);
  if (bytes_per_launch) *bytes_per_launch = bytes / count;
  return GPCG_OK;
}

extern "C" gpcg_status gpcg_time_masked_spmv(gpcg_problem* p, int precision, int reps,
                                             int flush_l2, void* cuda_stream,
                                             double* ms_per_launch, double* bytes_per_launch) {
  if (!p || reps < 1) return fail(GPCG_ERR_ARG, "bad argument");
  {
    const gpcg_status ps = settle_now(p);
    if (ps != GPCG_OK) return ps;
  }
  if (precision != GPCG_FP64 && precision != GPCG_MIXED)
    return fail(GPCG_ERR_ARG, "unknown precision");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const bool f32 = precision == GPCG_MIXED;
  gpcg_status st;
  int cur = 0;
  if ((st = ms_prepare(p, f32, s, &cur)) != GPCG_OK) return st;
  if (lean_spmv(p, f32)) {
    DevInst& I = p->inst;
    const int mask = cur;
    (void)I;
    if ((st = ms_scratch(p, s)) != GPCG_OK) return st;
    if ((st = ms_launch(p, f32, mask, s)) != GPCG_OK) return st;  // untimed
    const size_t flush_bytes = (size_t)256 << 20;
    void* flush = nullptr;
    if (flush_l2) CK(cudaMalloc(&flush, flush_bytes));
    std::vector<cudaEvent_t> ev(2 * (size_t)reps);
    for (auto& e : ev) CK(cudaEventCreate(&e));
    for (int k = 0; k < reps; ++k) {
      if (flush) CK(cudaMemsetAsync(flush, k & 0xff, flush_bytes, s));
      CK(cudaEventRecord(ev[2 * k], s));
      if ((st = ms_launch(p, f32, mask, s)) != GPCG_OK) return st;
      CK(cudaEventRecord(ev[2 * k + 1], s));
    }
    CK(cudaStreamSynchronize(s));
    double total = 0.0;
    for (int k = 0; k < reps; ++k) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]));
      total += ms;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (flush) cudaFree(flush);
    if ((st = ms_check(p, s, nullptr)) != GPCG_OK) return st;
    if (ms_per_launch) *ms_per_launch = total / reps;
    if (bytes_per_launch) *bytes_per_launch = ms_bytes(p, f32);
    return GPCG_OK;
  }
  // one untimed launch sets up the tables, then `reps` timed launches
  if ((st = one_pass(p, spmv_ctl(f32, cur, 0), s, nullptr)) != GPCG_OK) return st;
  Scratch& sc = p->sc;
  EngineArgs E{sc.d_insts, sc.d_ctl,  sc.d_tiles,    p->n_groups, sc.d_queue, (unsigned*)(sc.d_queue + 1),
               sc.d_live,   sc.d_npass, sc.d_queue + 2, 0xffffffffu, 0ull};
  const int grid = pass_grid(p->n_groups);
  const size_t flush_bytes = (size_t)256 << 20;
  void* flush = nullptr;
  if (flush_l2) CK(cudaMalloc(&flush, flush_bytes));
  std::vector<cudaEvent_t> ev(2 * (size_t)reps);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  for (int k = 0; k < reps; ++k) {
    if (flush) CK(cudaMemsetAsync(flush, k & 0xff, flush_bytes, s));
    CK(cudaEventRecord(ev[2 * k], s));
    CK(launch_pass(E, grid, s, 0));
    CK(cudaEventRecord(ev[2 * k + 1], s));
  }
  CK(cudaStreamSynchronize(s));
  double total = 0.0;
  for (int k = 0; k < reps; ++k) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]));
    total += ms;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (flush) cudaFree(flush);
  if (ms_per_launch) *ms_per_launch = total / reps;
  const double sv = f32 ? 4.0 : 8.0;
  if (bytes_per_launch) *bytes_per_launch = (double)p->n * (sv * p->kc + 4.0 * sv + 0.125);
  return GPCG_OK;
}

// -------------------------------------------------------------- server --
//
// The host thread that calls gpcg_server_step moves requests in and out of
// the engine's slots, launches the passes of the running slots and waits for
// them.  Worker threads, each on its own stream, do the rest while the passes
// run: they set up the uploads of admitted requests and read back the results
// of finished ones.  Device memory comes from a stream-ordered pool, so
// neither allocation nor release waits for the running passes.  An upload
// joins a free slot at the first step after it has completed (its event); a
// finished request leaves its slot at the next step, before the launch.

namespace {
// R_QUEUED: waiting for memory; R_STAGING: a worker sets up its upload;
// R_UPLOADING: the set-up is enqueued, waiting for its event; R_RUNNING: in an
// engine slot; R_RETIRING: finished, a worker reads x back; R_DONE and
// R_CANCELLED are final.
enum ReqState { R_QUEUED, R_STAGING, R_UPLOADING, R_RUNNING, R_RETIRING, R_DONE, R_CANCELLED };

struct Req {
  int64_t ticket = 0;
  gpcg_stencil A{};
  const double *b = nullptr, *l = nullptr, *u = nullptr;
  double c = 0.0;
  double* x_out = nullptr;
  int state = R_QUEUED;
  bool cancel = false;        // cancelled while a worker held it
  gpcg_problem* prob = nullptr;
  size_t bytes = 0;
  bool held = false;          // bytes counted against the budget
  bool fresh = false;         // took its slot in this step (its input checks are pending)
  int slot = -1;
  int flag = -1;              // its word among the server's pinned check words
  cudaEvent_t ev = nullptr;   // end of its upload on a worker's stream
  DevInst inst{};
  double t_submit = 0.0, t_done = 0.0;
  gpcg_stats st{};
};

struct Job {
  Req* r;
  bool upload;  // else: read back
};

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

constexpr int kServerWorkers = 4;
}  // namespace

struct gpcg_server {
  size_t budget = 0, used = 0;
  int max_live = 0;
  int dev = 0;
  gpcg_options opt{};
  cudaStream_t stream = nullptr;  // the engine's passes
  cudaMemPool_t pool = nullptr;
  cudaEvent_t ev_start = nullptr;  // start and end of the running step's passes
  cudaEvent_t ev_step = nullptr;
  double timing[8] = {};           // gpcg_server_timing
  int* h_flags = nullptr;          // pinned: the input-check word of each upload in flight
  Ctl* h_ctl = nullptr;            // pinned: the slots' control blocks after a step
  std::vector<int> free_flags;
  std::mutex mu;
  std::condition_variable cv;       // a job is queued, or stop
  std::condition_variable idle_cv;  // a step's passes are done
  std::condition_variable job_cv;   // a worker finished a job
  bool stop = false, stepping = false;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> wstreams;  // per worker: uploads, then read-backs
  std::vector<Stager> stagers;         // per worker
  std::deque<Job> jobs;
  std::deque<Req*> queue;
  std::vector<Req*> uploading;
  std::vector<Req*> slots;  // request per slot (nullptr = free)
  std::map<int64_t, Req*> all;
  int64_t next_ticket = 1;
  int finished = 0, n_staging = 0, n_retiring = 0;
  Scratch sc;
  bool dirty = true;
  long long tiles = 0;
  ~gpcg_server() {
    {
      std::lock_guard<std::mutex> g(mu);
      stop = true;
    }
    cv.notify_all();
    for (std::thread& t : workers) t.join();
    if (stream) cudaStreamSynchronize(stream);
    for (cudaStream_t w : wstreams) cudaStreamSynchronize(w);
    for (auto& kv : all) {
      delete kv.second->prob;  // pool frees, ordered on the stream of its upload
      if (kv.second->ev) cudaEventDestroy(kv.second->ev);
      delete kv.second;
    }
    for (cudaStream_t w : wstreams) cudaStreamSynchronize(w);
    for (Stager& g : stagers) g.release();
    sc.release();
    if (pool) cudaMemPoolDestroy(pool);
    if (h_flags) cudaFreeHost(h_flags);
    if (h_ctl) cudaFreeHost(h_ctl);
    if (ev_step) cudaEventDestroy(ev_step);
    if (ev_start) cudaEventDestroy(ev_start);
    if (stream) cudaStreamDestroy(stream);
    for (cudaStream_t w : wstreams) cudaStreamDestroy(w);
  }
};

static size_t footprint(const gpcg_stencil* A, bool mixed, bool tile, bool extract) {
  gpcg_problem tmp;
  geometry(A->dim, A->nx, A->ny, A->nz, &tmp);
  size_t b = arena64_bytes(&tmp);
  if (mixed) b += arena32_bytes(&tmp);
  if (tile) b += arena_tile_bytes(&tmp, false) + (mixed ? arena_tile_bytes(&tmp, true) : 0);
  if (extract)
    b += arena_rx_index_bytes(&tmp) + arena_rx_value_bytes(&tmp, false) +
         (mixed ? arena_rx_value_bytes(&tmp, true) : 0);
  return b + 4096;
}

// A request reaches a final state (server lock held): its device memory goes
// back to the pool (ordered on the stream of its upload) and its budget share
// and check word are released.
static void finish(gpcg_server* s, Req* r, int state) {
  delete r->prob;
  r->prob = nullptr;
  if (r->held) s->used -= r->bytes;
  r->held = false;
  if (r->flag >= 0) s->free_flags.push_back(r->flag);
  r->flag = -1;
  if (r->ev) cudaEventDestroy(r->ev);
  r->ev = nullptr;
  r->state = state;
  r->t_done = now_s();
  s->finished++;
}

// Enqueue a request's upload on stream ws (no lock held): its arenas from
// the pool, the copies of its arrays and of the tensor maps its options need,
// then the event that marks the end.  Only copy engines work on ws: the
// device-side set-up (device_init) runs on the engine's stream when the
// request takes a slot, since a step's passes hold every SM until it ends.
static gpcg_status start_upload(gpcg_server* s, Req* r, cudaStream_t ws, Stager* sg) {
  gpcg_status st = new_problem(&r->A, r->c, s->pool, ws, &r->prob, false);
  if (st != GPCG_OK) return st;
  if ((st = upload_copies(r->prob, &r->A, r->b, r->l, r->u, ws, sg)) != GPCG_OK) return st;
  make_fp64_maps(r->prob, ws);
  if ((st = prepare_instance(r->prob, &s->opt, ws, &r->inst, false)) != GPCG_OK) return st;
  // a server's launches are crowded: coarse work items
  r->inst.span = item_span(r->prob, 1LL << 40, s->opt.cg_system == GPCG_CG_EXTRACTED);
  CK(cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming));
  CK(cudaEventRecord(r->ev, ws));
  return GPCG_OK;
}

// Copy a finished request's x to its caller's buffer and fill its statistics
// (no lock held; its passes are complete).
static gpcg_status read_back(Req* r, cudaStream_t ws, Stager* sg) {
  gpcg_problem* p = r->prob;
  const double* x = p->inst.x[p->last.cur];
  if (sizeof(double) * (size_t)p->px <= Stager::kBytes && pageable(r->x_out)) {
    gpcg_status st = staged_out(*sg, r->x_out, x, (size_t)p->nx, (size_t)p->px,
                                (size_t)p->ny * p->nz, ws);
    if (st != GPCG_OK) return st;
  } else {
    CK(cudaMemcpy2DAsync(r->x_out, sizeof(double) * p->nx, x, sizeof(double) * p->px,
                         sizeof(double) * p->nx, (size_t)p->ny * p->nz, cudaMemcpyDefault, ws));
    CK(cudaStreamSynchronize(ws));
  }
  fill_stats(p, &r->st);
  return GPCG_OK;
}

static void server_worker(gpcg_server* s, int w) {
  cudaSetDevice(s->dev);
  // a read-back is ordered after no upload of the same worker
  cudaStream_t up = s->wstreams[2 * (size_t)w], down = s->wstreams[2 * (size_t)w + 1];
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv.wait(lk, [&] { return s->stop || !s->jobs.empty(); });
    if (s->stop) return;
    const Job j = s->jobs.front();
    s->jobs.pop_front();
    Req* r = j.r;
    lk.unlock();
    const double t0 = now_s();
    Stager* sg = &s->stagers[(size_t)w];
    const gpcg_status st = j.upload ? start_upload(s, r, up, sg) : read_back(r, down, sg);
    lk.lock();
    if (st == GPCG_OK && j.upload && r->cancel) {
      // cancelled meanwhile: its copies finish before the request ends
      lk.unlock();
      cudaEventSynchronize(r->ev);
      lk.lock();
    }
    s->timing[j.upload ? 3 : 2] += now_s() - t0;
    if (j.upload) {
      s->n_staging--;
      if (r->cancel) {
        finish(s, r, R_CANCELLED);
      } else if (st != GPCG_OK) {
        r->st.status = st;
        finish(s, r, R_DONE);
      } else {
        r->state = R_UPLOADING;
        s->uploading.push_back(r);
      }
    } else {
      s->n_retiring--;
      if (st != GPCG_OK) r->st.status = st;
      finish(s, r, r->cancel ? R_CANCELLED : R_DONE);
    }
    s->job_cv.notify_all();
  }
}

extern "C" gpcg_status gpcg_server_create(size_t hbm_budget, int max_live, const gpcg_options* opt,
                                          gpcg_server** out) {
  if (!out) return fail(GPCG_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (hbm_budget == 0 || max_live < 1) return fail(GPCG_ERR_ARG, "bad budget or slot count");
  gpcg_status st = check_options(opt);
  if (st != GPCG_OK) return st;
  gpcg_server* s = new gpcg_server();
  s->budget = hbm_budget;
  s->max_live = max_live;
  s->opt = *opt;
  s->opt.x0 = nullptr;
  s->slots.assign(max_live, nullptr);
  for (int k = max_live - 1; k >= 0; --k) s->free_flags.push_back(k);
  cudaMemPoolProps props;
  memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  cudaError_t e = cudaGetDevice(&s->dev);
  props.location.id = s->dev;
  // the passes run at the lowest stream priority and the workers' streams at
  // the highest; the workers' streams carry copies only (a request's
  // device-side set-up runs on the passes' stream), which the copy engines
  // move while the passes hold the SMs
  int lo = 0, hi = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->stream, cudaStreamNonBlocking, lo);
  for (int w = 0; w < 2 * kServerWorkers && e == cudaSuccess; ++w) {
    cudaStream_t ws = nullptr;
    e = cudaStreamCreateWithPriority(&ws, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) s->wstreams.push_back(ws);
  }
  if (e == cudaSuccess) e = cudaMemPoolCreate(&s->pool, &props);
  if (e == cudaSuccess) {
    // keep released memory in the pool (the budget bounds what it holds)
    cuuint64_t keep = ~0ull;
    e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  if (e == cudaSuccess) e = cudaEventCreate(&s->ev_step);
  if (e == cudaSuccess) e = cudaEventCreate(&s->ev_start);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_flags, sizeof(int) * max_live);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_ctl, sizeof(Ctl) * max_live);
  s->stagers.resize(kServerWorkers);
  for (int w = 0; w < kServerWorkers && e == cudaSuccess; ++w) e = s->stagers[(size_t)w].init();
  if (e != cudaSuccess) {
    delete s;
    return fail(GPCG_ERR_CUDA, "server set-up: %s", cudaGetErrorString(e));
  }
  // the work-item table is sized for max_live instances of the largest
  // group count, so admissions never reallocate it
  if ((st = s->sc.ensure(max_live, (long long)max_live * kMaxGroups)) != GPCG_OK) {
    delete s;
    return st;
  }
  for (int w = 0; w < kServerWorkers; ++w) s->workers.emplace_back(server_worker, s, w);
  *out = s;
  return GPCG_OK;
}

extern "C" gpcg_status gpcg_server_submit(gpcg_server* s, const gpcg_stencil* A, const double* b,
                                          const double* l, const double* u, double c,
                                          double* x_out, int64_t* ticket) {
  if (!s || !A || !b || !x_out || !ticket) return fail(GPCG_ERR_ARG, "NULL argument");
  gpcg_status st = check_problem(A, b, c);
  if (st != GPCG_OK) return st;
  if (s->opt.precond == GPCG_PRECOND_TILE && A->dim != 2)
    return fail(GPCG_ERR_ARG, "the tile preconditioner is for 2-D problems only");
  const size_t bytes =
      footprint(A, s->opt.precision == GPCG_MIXED, s->opt.precond == GPCG_PRECOND_TILE,
                s->opt.cg_system == GPCG_CG_EXTRACTED);
  if (bytes > s->budget) return fail(GPCG_ERR_BUDGET, "request needs %zu bytes, budget %zu",
                                     bytes, s->budget);
  Req* r = new Req();
  r->A = *A;
  r->b = b;
  r->l = l;
  r->u = u;
  r->c = c;
  r->x_out = x_out;
  r->bytes = bytes;
  r->t_submit = now_s();
  std::lock_guard<std::mutex> g(s->mu);
  r->ticket = s->next_ticket++;
  s->queue.push_back(r);
  s->all[r->ticket] = r;
  *ticket = r->ticket;
  return GPCG_OK;
}

static gpcg_status server_upload_table(gpcg_server* s) {
  std::vector<int2> table;
  for (int k = 0; k < s->max_live; ++k) {
    Req* r = s->slots[k];
    if (!r) continue;
    for (int j = 0; j < r->prob->n_groups; j += std::max(1, r->inst.span))
      table.push_back(make_int2(k, j));
  }
  s->tiles = (long long)table.size();
  s->dirty = false;
  if (s->tiles == 0) return GPCG_OK;
  gpcg_status st = s->sc.ensure(s->max_live, s->tiles);
  if (st != GPCG_OK) return st;
  CK(cudaMemcpyAsync(s->sc.d_tiles, table.data(), sizeof(int2) * table.size(),
                     cudaMemcpyHostToDevice, s->stream));
  return GPCG_OK;
}

extern "C" gpcg_status gpcg_server_step(gpcg_server* s, int passes) {
  if (!s || passes < 1) return fail(GPCG_ERR_ARG, "bad argument");
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->stepping) return fail(GPCG_ERR_ARG, "another thread is stepping this server");
  cudaStream_t st_ = s->stream;
  double t0 = now_s(), t1;
  // (1) requests that finished leave their slots; completed uploads take
  // free ones
  for (int k = 0; k < s->max_live; ++k) {
    Req* r = s->slots[k];
    if (r && r->state != R_RUNNING) {
      r->slot = -1;
      s->slots[k] = nullptr;
      s->dirty = true;
    }
  }
  for (size_t i = 0; i < s->uploading.size();) {
    Req* r = s->uploading[i];
    const cudaError_t q = cudaEventQuery(r->ev);
    if (q == cudaErrorNotReady) {
      ++i;
      continue;
    }
    if (q != cudaSuccess) return fail(GPCG_ERR_CUDA, "upload: %s", cudaGetErrorString(q));
    int slot = -1;
    for (int k = 0; k < s->max_live && slot < 0; ++k)
      if (!s->slots[k]) slot = k;
    if (slot < 0) break;
    s->uploading.erase(s->uploading.begin() + (long)i);
    gpcg_status st = device_init(r->prob, r->l == nullptr, r->u == nullptr, st_);
    if (st != GPCG_OK) return st;
    CK(cudaMemcpyAsync(&s->h_flags[r->flag], r->prob->d_flags, sizeof(int),
                       cudaMemcpyDeviceToHost, st_));
    r->fresh = true;
    Ctl C = fresh_ctl();
    C.gp32 = s->opt.precision == GPCG_MIXED ? 1 : 0;
    CK(cudaMemcpyAsync(s->sc.d_insts + slot, &r->inst, sizeof(DevInst), cudaMemcpyHostToDevice,
                       st_));
    CK(cudaMemcpyAsync(s->sc.d_ctl + slot, &C, sizeof(Ctl), cudaMemcpyHostToDevice, st_));
    r->slot = slot;
    r->state = R_RUNNING;
    s->slots[slot] = r;
    s->dirty = true;
  }
  t1 = now_s();
  s->timing[0] += t1 - t0;
  t0 = t1;
  // (2) launch the passes of the running slots
  int live = 0;
  for (Req* r : s->slots)
    if (r) live++;
  bool launched = false;
  if (live > 0) {
    gpcg_status st = s->dirty ? server_upload_table(s) : GPCG_OK;
    if (st != GPCG_OK) return st;
    s->sc.h_pin[0] = live;
    CK(cudaMemcpyAsync(s->sc.d_live, &s->sc.h_pin[0], sizeof(int), cudaMemcpyHostToDevice, st_));
    // a server may admit 3-D requests at any time: its kernel has the fused
    // 3-D step whenever its options allow it
    st = get_graph(s->sc, s->tiles, 1, passes, 0xffffffffu, feature_set(&s->opt, true));
    if (st != GPCG_OK) return st;
    CK(cudaEventRecord(s->ev_start, st_));
    CK(cudaGraphLaunch(s->sc.gexec, st_));
    CK(cudaMemcpyAsync(s->h_ctl, s->sc.d_ctl, sizeof(Ctl) * s->max_live, cudaMemcpyDeviceToHost,
                       st_));
    CK(cudaEventRecord(s->ev_step, st_));
    launched = true;
  }
  // (3) admit queued requests that fit the budget: their uploads go to the
  // workers
  while (!s->queue.empty()) {
    Req* r = s->queue.front();
    if (r->state == R_CANCELLED) {
      s->queue.pop_front();
      continue;
    }
    if (s->free_flags.empty() || s->used + r->bytes > s->budget) break;
    s->queue.pop_front();
    s->used += r->bytes;
    r->held = true;
    r->flag = s->free_flags.back();
    s->free_flags.pop_back();
    r->state = R_STAGING;
    s->n_staging++;
    s->jobs.push_back(Job{r, true});
    s->cv.notify_one();
  }
  t1 = now_s();
  s->timing[1] += t1 - t0;
  t0 = t1;
  if (!launched) {
    s->timing[6] += 1.0;
    return GPCG_OK;
  }
  // (4) wait for the passes (lock released: the workers post their results
  // meanwhile); finished requests go to the workers for read-back
  s->stepping = true;
  lk.unlock();
  const cudaError_t we = cudaEventSynchronize(s->ev_step);
  lk.lock();
  s->stepping = false;
  s->idle_cv.notify_all();
  if (we != cudaSuccess) return fail(GPCG_ERR_CUDA, "server step: %s", cudaGetErrorString(we));
  for (int k = 0; k < s->max_live; ++k) {
    Req* r = s->slots[k];
    if (!r || r->state != R_RUNNING) continue;
    if (r->fresh) {
      // the input checks of a request that joined in this step: one that
      // fails them ends with that status (its passes ran on its data
      // harmlessly, every loop of the engine being bounded)
      r->fresh = false;
      const gpcg_status fs = flags_status(s->h_flags[r->flag]);
      if (fs != GPCG_OK) {
        r->st.status = fs;
        finish(s, r, R_DONE);
        continue;
      }
    }
    if (!s->h_ctl[k].done) continue;
    r->prob->last = s->h_ctl[k];
    r->prob->have = true;
    r->prob->lambda_min = s->opt.lambda_min;
    r->state = R_RETIRING;
    s->n_retiring++;
    s->jobs.push_back(Job{r, false});
    s->cv.notify_one();
  }
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, s->ev_start, s->ev_step) == cudaSuccess) s->timing[5] += 1e-3 * ms;
  s->timing[4] += now_s() - t0;
  s->timing[6] += 1.0;
  s->timing[7] += 1.0;
  return GPCG_OK;
}

extern "C" gpcg_status gpcg_server_timing(gpcg_server* s, double* out) {
  if (!s || !out) return fail(GPCG_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> g(s->mu);
  for (int k = 0; k < 8; ++k) out[k] = s->timing[k];
  return GPCG_OK;
}

extern "C" int gpcg_server_done(gpcg_server* s, int64_t ticket) {
  if (!s) return 0;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->all.find(ticket);
  return it != s->all.end() && it->second->state == R_DONE;
}

extern "C" gpcg_status gpcg_server_stats(gpcg_server* s, int64_t ticket, gpcg_stats* st,
                                         double* latency_s) {
  if (!s) return fail(GPCG_ERR_ARG, "server is NULL");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(GPCG_ERR_ARG, "unknown ticket");
  Req* r = it->second;
  if (r->state == R_CANCELLED) return fail(GPCG_ERR_CANCELLED, "ticket cancelled");
  if (r->state != R_DONE) return fail(GPCG_ERR_PENDING, "ticket still running");
  if (st) *st = r->st;
  if (latency_s) *latency_s = r->t_done - r->t_submit;
  return GPCG_OK;
}

extern "C" gpcg_status gpcg_server_cancel(gpcg_server* s, int64_t ticket) {
  if (!s) return fail(GPCG_ERR_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  // a slot's control block is rewritten only between steps
  s->idle_cv.wait(lk, [&] { return !s->stepping; });
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(GPCG_ERR_ARG, "unknown ticket");
  Req* r = it->second;
  if (r->state == R_DONE || r->state == R_CANCELLED || r->cancel)
    return fail(GPCG_ERR_ARG, "ticket already finished");
  if (r->state == R_STAGING || r->state == R_RETIRING) {
    // a job not yet taken is dropped here; one a worker holds ends cancelled
    for (size_t i = 0; i < s->jobs.size(); ++i)
      if (s->jobs[i].r == r) {
        s->jobs.erase(s->jobs.begin() + (long)i);
        if (r->state == R_STAGING) s->n_staging--;
        else s->n_retiring--;
        if (r->slot >= 0) {
          s->slots[r->slot] = nullptr;
          r->slot = -1;
          s->dirty = true;
        }
        finish(s, r, R_CANCELLED);
        return GPCG_OK;
      }
    // a worker holds it: wait until it lets go (no copy of the request's
    // arrays is in flight when cancel returns)
    r->cancel = true;
    s->job_cv.wait(lk, [&] { return r->state == R_CANCELLED || r->state == R_UPLOADING ||
                                    r->state == R_DONE; });
    if (r->state != R_UPLOADING) return GPCG_OK;
  }
  if (r->state == R_UPLOADING) {
    CK(cudaEventSynchronize(r->ev));
    for (size_t i = 0; i < s->uploading.size(); ++i)
      if (s->uploading[i] == r) {
        s->uploading.erase(s->uploading.begin() + (long)i);
        break;
      }
  } else if (r->state == R_RUNNING) {
    Ctl C = fresh_ctl();
    C.pass = P_NONE;
    C.done = 1;
    C.status = S_OK;
    CK(cudaMemcpyAsync(s->sc.d_ctl + r->slot, &C, sizeof(Ctl), cudaMemcpyHostToDevice,
                       s->stream));
    CK(cudaStreamSynchronize(s->stream));
  }
  if (r->slot >= 0) {
    s->slots[r->slot] = nullptr;
    r->slot = -1;
    s->dirty = true;
  }
  finish(s, r, R_CANCELLED);
  return GPCG_OK;
}

extern "C" void gpcg_server_counts(gpcg_server* s, int* queued, int* running, int* finished) {
  if (!s) return;
  std::lock_guard<std::mutex> g(s->mu);
  int q = s->n_staging + (int)s->uploading.size(), run = s->n_retiring;
  for (Req* r : s->queue)
    if (r->state == R_QUEUED) q++;
  for (Req* r : s->slots)
    if (r && r->state == R_RUNNING) run++;
  if (queued) *queued = q;
  if (running) *running = run;
  if (finished) *finished = s->finished;
}

extern "C" void gpcg_server_destroy(gpcg_server* s) {
  if (!s) return;
  delete s;
}

extern "C" const char* gpcg_last_error(void) { return g_err; }

namespace gpcg {
// Lets the other translation units of the library report through
// gpcg_last_error().
void set_last_error(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }
}  // namespace gpcg

extern "C" const char* gpcg_version(void) { return "gpcg-gb300 0.1 (sm_103a)"; }
