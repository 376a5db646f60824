// gpcg_coop_f64.cu -- the cooperative pass kernel (see gpcg_coop.cu) for FP64
// solves and for the tile preconditioner.
#define GPCG_COOP 1
#include "pass_engine.cuh"

namespace gpcg {

namespace {  // the header's namespace
template __global__ void pass_kernel_coop<FEAT_F64>(EngineArgs);
template __global__ void pass_kernel_coop<FEAT_TILE>(EngineArgs);
}  // namespace

const void* pass_kernel_coop_ptr_b(int feat) {
  return feat == FEAT_TILE ? (const void*)pass_kernel_coop<FEAT_TILE>
                           : (const void*)pass_kernel_coop<FEAT_F64>;
}

}  // namespace gpcg
