// gpcg_pass_3d.cu -- the pass kernel instantiated with the fused FP32 CG
// step of 3-D grids (P_CG_F on 3-D instances), for mixed-precision solves
// that have 3-D instances.  A translation unit of its own: the step's code
// would otherwise enlarge the default kernel that 2-D solves run.
#include "pass_engine.cuh"

namespace gpcg {

namespace {  // the header's namespace
template __global__ void pass_kernel<true, FEAT_3D>(EngineArgs);
template __global__ void pass_kernel<false, FEAT_3D>(EngineArgs);
}  // namespace

const void* pass_kernel_ptr_3d(bool cond) {
  return cond ? (const void*)pass_kernel<true, FEAT_3D> : (const void*)pass_kernel<false, FEAT_3D>;
}

}  // namespace gpcg
