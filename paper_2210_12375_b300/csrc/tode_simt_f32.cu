// FP32-state instantiation of the SIMT solver (time stays FP64).  Built with
// -fmad=false: every multiply-add it performs is an explicit fused operation
// (madd), so the plain and fused kernels round identically.
#include "tode_simt_adjoint.cuh"
#include "tode_simt_joint.cuh"

namespace tode {
tode_err simt_solve_f32(const SolveReq& r) {
  return r.o->joint ? simt_joint<float>(r) : simt_solve<float>(r);
}
tode_err simt_adjoint_f32(const AdjReq& r) { return simt_adjoint<float>(r); }
tode_err simt_t_bounds_f32(const AdjReq& r, const void* yp, double* gt0, double* gt1) {
  return simt_t_bounds<float>(r, yp, gt0, gt1);
}
}  // namespace tode
