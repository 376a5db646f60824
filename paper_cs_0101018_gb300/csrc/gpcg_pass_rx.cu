// gpcg_pass_rx.cu -- the pass kernel instantiated with the explicit reduced system's passes (P_RX_COUNT, P_RX_MAP, P_RX_BUILD,
// P_RCG, P_RW).
// A translation unit of its own so that it compiles in parallel with the
// default instantiation in gpcg_kernels.cu.
#include "pass_engine.cuh"

namespace gpcg {

namespace {  // the header's namespace
template __global__ void pass_kernel<true, FEAT_EXT>(EngineArgs);
template __global__ void pass_kernel<false, FEAT_EXT>(EngineArgs);
}  // namespace

const void* pass_kernel_ptr_rx(bool cond) {
  return cond ? (const void*)pass_kernel<true, FEAT_EXT> : (const void*)pass_kernel<false, FEAT_EXT>;
}

}  // namespace gpcg
