// gpcg_coop.cu -- the cooperative pass kernel (every pass of one solve in one
// launch, the blocks meeting at a grid barrier between passes) for the
// default passes and for 3-D grids.  A translation unit of its own: the
// cooperative kernel reads engine data through the coherent path only
// (GPCG_COOP), so its device code is compiled apart from the other kernels'.
#define GPCG_COOP 1
#include "pass_engine.cuh"

namespace gpcg {

namespace {  // the header's namespace
template __global__ void pass_kernel_coop<0>(EngineArgs);
template __global__ void pass_kernel_coop<FEAT_3D>(EngineArgs);
}  // namespace

const void* pass_kernel_coop_ptr_a(int feat) {
  return feat == FEAT_3D ? (const void*)pass_kernel_coop<FEAT_3D> : (const void*)pass_kernel_coop<0>;
}

}  // namespace gpcg
