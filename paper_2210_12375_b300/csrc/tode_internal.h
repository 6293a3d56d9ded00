// tode_internal.h -- host-side requests passed from the C-ABI layer
// (tode_api.cu) to the per-precision launchers (tode_simt_f64.cu,
// tode_simt_f32.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/tode.h"

namespace tode {

struct SolveReq {
  const tode_field_desc* f;
  const tode_options* o;
  int B, D, K;
  const void* y0;
  const double* t0;
  const double* t1;
  const double* te;
  void* ye;
  void* yp;   // may be NULL: dy/dt at the evaluation points
  void* yf;
  int32_t *n_acc, *n_rej, *n_fe, *status;
  const tode_tape* tape;    // may be NULL
  const tode_trace* trace;  // may be NULL
  char* ws;                 // carved by the launcher
  size_t ws_bytes;
  cudaStream_t stream;
  int num_sms;
  // MLP field, re-solve of one checkpointed segment (tode_mlp_resolve)
  bool resolve;
  int rs_seg;
  const tode_tape* ck;
  int32_t* rs_n;
  double* rs_t0;
  double* rs_t1;
};

struct AdjReq {
  const tode_field_desc* f;
  const tode_options* o;
  int B, D, K;
  const double* t0;
  const double* t1;
  const double* te;
  const int32_t* n_acc;
  const int32_t* status;
  const tode_tape* tape;
  const void* gye;
  const void* gyf;
  void* gy0;
  void* gparam;
  float* const* gW;
  float* const* gb;
  int32_t* overflow;
  char* scratch;
  size_t scratch_bytes;
  cudaStream_t stream;
  int num_sms;
};

#define TODE_CUDA_TRY(x)        \
  do {                          \
    if ((x) != cudaSuccess) {   \
      (void)cudaGetLastError(); \
      return TODE_ECUDA;        \
    }                           \
  } while (0)

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Work order (k_counting_order and its multi-CTA form): 256 bins; a batch
// above ORDER_SMALL_B instances is counted by up to 1024 CTAs, whose per-CTA
// bin counts (then their queue offsets) live in scratch.
constexpr int ORDER_BINS = 256;
constexpr int ORDER_THREADS = 1024;
constexpr int ORDER_SMALL_B = 2048;
inline int order_ctas(int B) {
  const int g = (B + ORDER_THREADS - 1) / ORDER_THREADS;
  return g > 1024 ? 1024 : g;
}
inline size_t order_part_bytes(int B) {
  return B <= ORDER_SMALL_B ? 0 : align256((size_t)order_ctas(B) * ORDER_BINS * 4);
}


// Joint solve: a control block, three partial sums per CTA (at most one CTA
// per instance) and a double buffer of the per-instance state y, y_lo, k1.
constexpr size_t JOINT_CTL_BYTES = 512;
inline size_t joint_ws_offset(int B) {
  return align256(256) + align256((size_t)B * 4) + order_part_bytes(B);
}
inline size_t joint_part_bytes(int B) { return align256((size_t)(B + 1) * 3 * 8); }
inline size_t joint_state_bytes(int B, int D, size_t ts) {
  return 6 * align256((size_t)B * D * ts);
}

// Workspace bytes of the SIMT solver for state dtype size `ts`.
inline size_t simt_workspace_bytes(int B, int D, size_t ts, int form, int joint) {
  size_t s = 0;
  s += align256(256);             // any-active flag + work counter
  s += align256((size_t)B * 4);    // work order
  s += order_part_bytes(B);        // and the sort's per-CTA counts
  if (joint) return s + JOINT_CTL_BYTES + joint_part_bytes(B) + joint_state_bytes(B, D, ts);
  if (form == TODE_PLAIN) {
    s += 3 * align256((size_t)B * D * ts);  // y, y_lo, k1
    s += align256((size_t)B * 8);           // t
    s += 3 * align256((size_t)B * ts);      // h, err_prev, err_prev2
    s += 2 * align256((size_t)B * 4);       // cursor, flags
  }
  return s;
}

// Scratch bytes of the SIMT adjoint: the work counter, the work order (one
// int32 per instance) and one segment of `stride` step-start states per
// instance (y, k1, t, h).
inline size_t simt_adjoint_scratch_bytes(int B, int D, size_t ts, int stride) {
  return align256(256) + align256((size_t)B * 4) + order_part_bytes(B) +
         2 * align256((size_t)stride * B * D * ts) +
         align256((size_t)stride * B * 8) + align256((size_t)stride * B * ts);
}

tode_err simt_solve_f64(const SolveReq& r);  // both: independent or joint (o->joint)
tode_err simt_solve_f32(const SolveReq& r);
tode_err simt_adjoint_f64(const AdjReq& r);
tode_err simt_adjoint_f32(const AdjReq& r);
tode_err simt_t_bounds_f64(const AdjReq& r, const void* yp, double* gt0, double* gt1);
tode_err simt_t_bounds_f32(const AdjReq& r, const void* yp, double* gt0, double* gt1);
// the same for the tsit5 pair (tode_simt_ts5_f64.cu, tode_simt_ts5_f32.cu);
// the functions above hand over to these when o->method is TODE_TSIT5
// the joint continuous adjoint of the MLP field (tode_mlp.cu)
struct JadjReq {
  const tode_field_desc* f;
  const tode_options* o;
  int B, K;
  double t0, t1;
  const double* te;  // host [K]
  const float* y1;
  const float* gye;
  const float* gyf;
  float* gy0;
  float* y0;
  float* const* gW;
  float* const* gb;
  int32_t* stats;  // host [4]
  char* ws;
  cudaStream_t stream;
};
size_t mlp_jadj_workspace_bytes(const tode_field_desc* f);
tode_err mlp_joint_adjoint(const JadjReq& r);
tode_err simt_solve_ts5_f64(const SolveReq& r);
tode_err simt_solve_ts5_f32(const SolveReq& r);
tode_err simt_adjoint_ts5_f64(const AdjReq& r);
tode_err simt_adjoint_ts5_f32(const AdjReq& r);
tode_err simt_t_bounds_ts5_f64(const AdjReq& r, const void* yp, double* gt0, double* gt1);
tode_err simt_t_bounds_ts5_f32(const AdjReq& r, const void* yp, double* gt0, double* gt1);

bool simt_supported(int kind, int D);

// the MLP field's most weight layers
constexpr int MLP_MAX_LAYERS = 4;
bool mlp_supported(const tode_field_desc* f);
size_t mlp_workspace_bytes(const tode_field_desc* f, const tode_options* o);
tode_err mlp_solve(const SolveReq& r, bool split);
size_t mlp_adjoint_scratch_bytes(const tode_field_desc* f, const tode_options* o, int slots,
                                 int num_sms);
tode_err mlp_adjoint(const AdjReq& r);
tode_err mlp_t_bounds(const AdjReq& r, const void* yp, double* gt0, double* gt1);

}  // namespace tode
