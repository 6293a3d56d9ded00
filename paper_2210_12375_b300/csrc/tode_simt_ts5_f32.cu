// FP32-state instantiation of the SIMT solver with the Tsitouras 5(4) pair
// (tsit5, App. A): the same kernels as the dopri5 unit with the other
// tableau, in a unit of their own so that the two compile side by side.
// Built with -fmad=false like the dopri5 unit (explicit fused operations
// only), so the FP64 path's step sequences are reproducible bit for bit.
#include "tode_simt_adjoint.cuh"
#include "tode_simt_joint.cuh"

namespace tode {
tode_err simt_solve_ts5_f32(const SolveReq& r) {
  return r.o->joint ? simt_joint<float, TS5>(r) : simt_solve<TS5, float>(r);
}
tode_err simt_adjoint_ts5_f32(const AdjReq& r) { return simt_adjoint<TS5, float>(r); }
tode_err simt_t_bounds_ts5_f32(const AdjReq& r, const void* yp, double* gt0, double* gt1) {
  return simt_t_bounds<TS5, float>(r, yp, gt0, gt1);
}
}  // namespace tode
