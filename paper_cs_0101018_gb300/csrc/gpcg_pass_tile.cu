// gpcg_pass_tile.cu -- the pass kernel instantiated with the tile preconditioner's passes (P_CG_Z and the tile variant of P_CG_F).
// A translation unit of its own so that it compiles in parallel with the
// default instantiation in gpcg_kernels.cu.
#include "pass_engine.cuh"

namespace gpcg {

namespace {  // the header's namespace
template __global__ void pass_kernel<true, FEAT_TILE>(EngineArgs);
template __global__ void pass_kernel<false, FEAT_TILE>(EngineArgs);
}  // namespace

const void* pass_kernel_ptr_tile(bool cond) {
  return cond ? (const void*)pass_kernel<true, FEAT_TILE> : (const void*)pass_kernel<false, FEAT_TILE>;
}

}  // namespace gpcg
