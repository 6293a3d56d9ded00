// FP64 instantiation of the SIMT solver.  Built with -fmad=false so that no
// multiply-add is contracted and every sum is taken left to right: the FP64
// path's accept/reject decisions are reproducible on any IEEE-754 machine.
#include "tode_simt_adjoint.cuh"
#include "tode_simt_joint.cuh"

namespace tode {
// dopri5 here; the tsit5 instantiations live in their own unit
tode_err simt_solve_f64(const SolveReq& r) {
  if (r.o->method == TODE_TSIT5) return simt_solve_ts5_f64(r);
  return r.o->joint ? simt_joint<double>(r) : simt_solve<DP5, double>(r);
}
tode_err simt_adjoint_f64(const AdjReq& r) {
  if (r.o->method == TODE_TSIT5) return simt_adjoint_ts5_f64(r);
  return simt_adjoint<DP5, double>(r);
}
tode_err simt_t_bounds_f64(const AdjReq& r, const void* yp, double* gt0, double* gt1) {
  if (r.o->method == TODE_TSIT5) return simt_t_bounds_ts5_f64(r, yp, gt0, gt1);
  return simt_t_bounds<DP5, double>(r, yp, gt0, gt1);
}
}  // namespace tode
