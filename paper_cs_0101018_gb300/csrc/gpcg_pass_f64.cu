// gpcg_pass_f64.cu -- the pass kernel instantiated for FP64 solves: the
// default passes and the staged FP64 alpha0 pass.  A translation unit of its
// own so that it compiles in parallel with the default instantiation.
#include "pass_engine.cuh"

namespace gpcg {

namespace {  // the header's namespace
template __global__ void pass_kernel<true, FEAT_F64>(EngineArgs);
template __global__ void pass_kernel<false, FEAT_F64>(EngineArgs);
}  // namespace

const void* pass_kernel_ptr_f64(bool cond) {
  return cond ? (const void*)pass_kernel<true, FEAT_F64> : (const void*)pass_kernel<false, FEAT_F64>;
}

}  // namespace gpcg
