// FP32-state instantiation of the SIMT solver (time stays FP64).  Built with
// -fmad=false: every multiply-add it performs is an explicit fused operation
// (madd), so the plain and fused kernels round identically.
#include "tode_simt_adjoint.cuh"
#include "tode_simt_joint.cuh"

namespace tode {
// dopri5 here; the tsit5 instantiations live in their own unit
tode_err simt_solve_f32(const SolveReq& r) {
  if (r.o->method == TODE_TSIT5) return simt_solve_ts5_f32(r);
  return r.o->joint ? simt_joint<float>(r) : simt_solve<DP5, float>(r);
}
tode_err simt_adjoint_f32(const AdjReq& r) {
  if (r.o->method == TODE_TSIT5) return simt_adjoint_ts5_f32(r);
  return simt_adjoint<DP5, float>(r);
}
tode_err simt_t_bounds_f32(const AdjReq& r, const void* yp, double* gt0, double* gt1) {
  if (r.o->method == TODE_TSIT5) return simt_t_bounds_ts5_f32(r, yp, gt0, gt1);
  return simt_t_bounds<DP5, float>(r, yp, gt0, gt1);
}
}  // namespace tode
