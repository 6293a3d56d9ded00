// tode_api.cu -- the C ABI (include/tode.h): argument validation, workspace
// sizing and dispatch to the per-precision launchers.  No entry point
// allocates device memory.
#include <cmath>
#include <cstring>

#include "tode_internal.h"

namespace tode {

bool simt_supported(int kind, int D) {
  if (kind == TODE_VDP) return D == 2;
  if (kind == TODE_LINEAR) return D == 1 || D == 2 || D == 4 || D == 8 || D == 16 || D == 32;
  return false;
}

static bool opts_ok(const tode_options* o) {
  if (!o) return false;
  if (!(o->rtol >= 0.0) || !(o->atol >= 0.0) || !std::isfinite(o->rtol) ||
      !std::isfinite(o->atol))
    return false;
  if (!o->rtol_b && !o->atol_b && !(o->rtol + o->atol > 0.0)) return false;
  if (!(o->safety > 0.0) || !(o->fac_min > 0.0) || !(o->fac_min <= 1.0) || !(o->fac_max >= 1.0))
    return false;
  if (!(o->beta1 > 0.0) || !std::isfinite(o->beta1) || !std::isfinite(o->beta2) ||
      !std::isfinite(o->beta3))
    return false;
  if (!(o->h0 >= 0.0) || !std::isfinite(o->h0)) return false;
  if (o->max_steps < 1) return false;
  if (o->form != TODE_PLAIN && o->form != TODE_FUSED) return false;
  if (o->block < 0 || o->group < 0 || o->ctas_per_sm < 0 || o->poll_every < 0) return false;
  if (o->order != 0 && o->order != 1) return false;
  if (o->joint != 0 && o->joint != 1) return false;
  if (o->method != TODE_DOPRI5 && o->method != TODE_TSIT5) return false;
  return true;
}

static size_t state_size(const tode_options* o) { return o->prec == TODE_F64 ? 8 : 4; }

static tode_err field_ok(const tode_field_desc* f, const tode_options* o) {
  if (!f || !o) return TODE_EINVAL;
  if (f->B < 0 || f->D < 1) return TODE_EINVAL;
  if (f->kind == TODE_VDP || f->kind == TODE_LINEAR) {
    if (o->prec != TODE_F64 && o->prec != TODE_F32) return TODE_EUNSUPPORTED;
    if (!simt_supported(f->kind, f->D)) return TODE_EUNSUPPORTED;
    if (f->B > 0 && f->kind == TODE_VDP && !f->mu) return TODE_EINVAL;
    if (f->B > 0 && f->kind == TODE_LINEAR && !f->A) return TODE_EINVAL;
    return TODE_OK;
  }
  if (f->kind == TODE_MLP) {
    if (o->prec != TODE_BF16W && o->prec != TODE_BF16W_SPLIT) return TODE_EUNSUPPORTED;
    // tsit5 on the split form only (the adjoints and the reported form)
    if (o->method == TODE_TSIT5 && o->prec != TODE_BF16W_SPLIT) return TODE_EUNSUPPORTED;
    if (!f->widths || !f->W || !f->b) return TODE_EINVAL;
    if (!mlp_supported(f)) return TODE_EUNSUPPORTED;
    if (f->B > 0)
      for (int l = 0; l < f->n_layers; ++l)
        if (!f->W[l]) return TODE_EINVAL;
    return TODE_OK;
  }
  return TODE_EINVAL;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

static bool tape_ok(const tode_tape* tp, const tode_options* o, const tode_field_desc* f) {
  const void* arrays[] = {tp->y,     tp->y_lo,  tp->k1,      tp->t,        tp->h,
                          tp->err_prev, tp->flags, tp->h_acc, tp->y_stage, tp->err_prev2};
  for (const void* p : arrays)
    if (!aligned16(p)) return false;  // NULL passes
  if (tp->slots < 1 || tp->stride < 1 || !tp->y || !tp->t) return false;
  if (f->kind == TODE_MLP) {
    if (tp->stride == 1) return tp->h_acc && tp->y_stage;
    // checkpoints of a budgeted solve: the whole solver state at each one
    return tp->k1 && tp->y_lo && tp->h && tp->err_prev && tp->flags &&
           (o->beta3 == 0.0 || tp->err_prev2);
  }
  // stride 1 with the accepted step sizes: reversed straight from the slots,
  // which need the FSAL stage only when the stage inputs are not recorded
  if (tp->stride == 1 && tp->h_acc) return tp->k1 || tp->y_stage;
  // otherwise segments are re-run from their slots: the whole solver state
  return tp->k1 && tp->h && tp->err_prev && tp->flags && (o->prec == TODE_F64 || tp->y_lo) &&
         (o->beta3 == 0.0 || tp->err_prev2);
}

static int sm_count_or_zero() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return sms;
}

static tode_err device_sms(int* sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return TODE_ECUDA;
  }
  if (cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return TODE_ECUDA;
  }
  return TODE_OK;
}

static bool aligned256(const void* p) { return ((uintptr_t)p & 255u) == 0; }

}  // namespace tode

using namespace tode;

extern "C" {

int tode_version(void) { return TODE_VERSION; }

const char* tode_strerror(tode_err e) {
  switch (e) {
    case TODE_OK: return "ok";
    case TODE_EINVAL: return "invalid argument";
    case TODE_EWORKSPACE: return "workspace, tape or scratch too small or misaligned";
    case TODE_ECUDA: return "CUDA runtime error";
    case TODE_EUNSUPPORTED: return "unsupported field / dimension / precision combination";
    case TODE_ETIMEOUT: return "bounded wait gave up";
  }
  return "unknown error";
}

void tode_default_options(tode_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->rtol = 1e-6;
  o->atol = 1e-6;
  o->safety = 0.9;
  o->fac_min = 0.2;
  o->fac_max = 10.0;
  o->beta1 = 0.2;
  o->beta2 = 0.0;
  o->h0 = 0.0;
  o->max_steps = 100000;
  o->prec = TODE_F32;
  o->form = TODE_FUSED;
}

// Joint solving (Sec. 4.1) covers the Van der Pol and linear fields with
// scalar tolerances (one problem has one norm).
static tode_err joint_ok(const tode_field_desc* f, const tode_options* o) {
  if (!o->joint) return TODE_OK;
  if (f->kind == TODE_MLP) return TODE_EUNSUPPORTED;
  if (o->rtol_b || o->atol_b) return TODE_EINVAL;
  return TODE_OK;
}

size_t tode_workspace_size(const tode_field_desc* f, const tode_options* o, int K) {
  if (K < 0 || !opts_ok(o) || field_ok(f, o) != TODE_OK || joint_ok(f, o) != TODE_OK) return 0;
  if (f->kind == TODE_MLP) return mlp_workspace_bytes(f, o);
  return simt_workspace_bytes(f->B, f->D, state_size(o), o->form, o->joint);
}

tode_err tode_solve(const tode_field_desc* f, const tode_options* o, const void* y0,
                    const double* t0, const double* t1, const double* t_eval, int K,
                    void* y_eval, void* yp_eval, void* y_final, int32_t* n_acc, int32_t* n_rej,
                    int32_t* n_feval, int32_t* status, const tode_tape* tape,
                    const tode_trace* trace, void* workspace, size_t ws_bytes, void* stream) {
  if (!opts_ok(o) || K < 0) return TODE_EINVAL;
  tode_err e = field_ok(f, o);
  if (e != TODE_OK) return e;
  e = joint_ok(f, o);
  if (e != TODE_OK) return e;
  if (f->B == 0) return TODE_OK;
  if (!y0 || !t0 || !t1 || !y_final || !n_acc || !n_rej || !n_feval || !status)
    return TODE_EINVAL;
  if (K > 0 && (!t_eval || !y_eval)) return TODE_EINVAL;
  // the derivative at the points: every field, solved independently
  if (K > 0 && yp_eval && o->joint) return TODE_EUNSUPPORTED;
  if (tape && !tape_ok(tape, o, f)) return TODE_EINVAL;
  // a joint mesh is reversed from the tape, never re-run per instance
  if (tape && o->joint && !(tape->stride == 1 && tape->h_acc)) return TODE_EINVAL;
  if (trace) {
    if (trace->cap < 0) return TODE_EINVAL;
    if (trace->cap > 0 &&
        (!trace->t || !trace->h || !trace->err || !trace->accepted || !trace->len))
      return TODE_EINVAL;
  }
  const size_t need = tode_workspace_size(f, o, K);
  if (!workspace || !aligned256(workspace) || ws_bytes < need) return TODE_EWORKSPACE;
  SolveReq r{};
  r.f = f;
  r.o = o;
  r.B = f->B;
  r.D = f->D;
  r.K = K;
  r.y0 = y0;
  r.t0 = t0;
  r.t1 = t1;
  r.te = t_eval;
  r.ye = y_eval;
  r.yp = K > 0 ? yp_eval : nullptr;
  r.yf = y_final;
  r.n_acc = n_acc;
  r.n_rej = n_rej;
  r.n_fe = n_feval;
  r.status = status;
  r.tape = tape;
  r.trace = trace;
  r.ws = (char*)workspace;
  r.ws_bytes = ws_bytes;
  r.stream = (cudaStream_t)stream;
  e = device_sms(&r.num_sms);
  if (e != TODE_OK) return e;
  if (f->kind == TODE_MLP) return mlp_solve(r, o->prec == TODE_BF16W_SPLIT);
  return o->prec == TODE_F64 ? simt_solve_f64(r) : simt_solve_f32(r);
}

tode_err tode_mlp_resolve(const tode_field_desc* f, const tode_options* o, const double* t0,
                          const double* t1, const int32_t* n_acc, const tode_tape* ckpt, int seg,
                          const tode_tape* seg_tape, int32_t* seg_n, double* seg_t0,
                          double* seg_t1, void* workspace, size_t ws_bytes, void* stream) {
  if (!opts_ok(o) || seg < 0) return TODE_EINVAL;
  tode_err e = field_ok(f, o);
  if (e != TODE_OK) return e;
  if (f->kind != TODE_MLP || o->prec != TODE_BF16W_SPLIT || o->joint || o->form != TODE_FUSED)
    return TODE_EUNSUPPORTED;
  if (f->B == 0) return TODE_OK;
  if (!t0 || !t1 || !n_acc || !ckpt || !seg_tape || !seg_n || !seg_t0 || !seg_t1)
    return TODE_EINVAL;
  if (!tape_ok(ckpt, o, f) || ckpt->stride < 2) return TODE_EINVAL;
  if (!tape_ok(seg_tape, o, f) || seg_tape->stride != 1 || seg_tape->slots < ckpt->stride)
    return TODE_EINVAL;
  const size_t need = tode_workspace_size(f, o, 0);
  if (!workspace || !aligned256(workspace) || ws_bytes < need) return TODE_EWORKSPACE;
  SolveReq r{};
  r.f = f;
  r.o = o;
  r.B = f->B;
  r.D = f->D;
  r.K = 0;
  r.t0 = t0;
  r.t1 = t1;
  r.n_acc = const_cast<int32_t*>(n_acc);
  r.tape = seg_tape;
  r.ws = (char*)workspace;
  r.ws_bytes = ws_bytes;
  r.stream = (cudaStream_t)stream;
  r.resolve = true;
  r.rs_seg = seg;
  r.ck = ckpt;
  r.rs_n = seg_n;
  r.rs_t0 = seg_t0;
  r.rs_t1 = seg_t1;
  e = device_sms(&r.num_sms);
  if (e != TODE_OK) return e;
  return mlp_solve(r, true);
}

size_t tode_adjoint_scratch_size(const tode_field_desc* f, const tode_options* o,
                                 const tode_tape* tape) {
  if (!opts_ok(o) || field_ok(f, o) != TODE_OK || !tape || tape->stride < 1) return 0;
  if (f->kind == TODE_MLP) {
    // sized for one CTA per SM of the current device (at least one SM)
    const int sms = sm_count_or_zero();
    return (tape->stride == 1 && o->prec == TODE_BF16W_SPLIT)
               ? mlp_adjoint_scratch_bytes(f, o, tape->slots, sms > 0 ? sms : 1)
               : 0;
  }
  return simt_adjoint_scratch_bytes(f->B, f->D, state_size(o), tape->stride);
}

tode_err tode_adjoint(const tode_field_desc* f, const tode_options* o, const double* t0,
                      const double* t1, const double* t_eval, int K, const int32_t* n_acc,
                      const int32_t* status, const tode_tape* tape, const void* gy_eval,
                      const void* gy_final, void* gy0, void* gparam, float* const* gW,
                      float* const* gb, int32_t* overflow, void* scratch, size_t scratch_bytes,
                      void* stream) {
  if (!opts_ok(o) || K < 0) return TODE_EINVAL;
  tode_err e = field_ok(f, o);
  if (e != TODE_OK) return e;
  if (f->kind == TODE_MLP && o->prec != TODE_BF16W_SPLIT) return TODE_EUNSUPPORTED;
  if (f->B == 0) return TODE_OK;
  if (!t0 || !t1 || !n_acc || !status || !tape || !gy0 || !overflow) return TODE_EINVAL;
  if (K > 0 && !t_eval) return TODE_EINVAL;
  if (!tape_ok(tape, o, f)) return TODE_EINVAL;
  const size_t need = tode_adjoint_scratch_size(f, o, tape);
  if (!scratch || !aligned256(scratch) || scratch_bytes < need) return TODE_EWORKSPACE;
  AdjReq r{};
  r.f = f;
  r.o = o;
  r.B = f->B;
  r.D = f->D;
  r.K = K;
  r.t0 = t0;
  r.t1 = t1;
  r.te = t_eval;
  r.n_acc = n_acc;
  r.status = status;
  r.tape = tape;
  r.gye = gy_eval;
  r.gyf = gy_final;
  r.gy0 = gy0;
  r.gparam = gparam;
  r.gW = gW;
  r.gb = gb;
  r.overflow = overflow;
  r.scratch = (char*)scratch;
  r.scratch_bytes = scratch_bytes;
  r.stream = (cudaStream_t)stream;
  e = device_sms(&r.num_sms);
  if (e != TODE_OK) return e;
  if (f->kind == TODE_MLP) return mlp_adjoint(r);
  return o->prec == TODE_F64 ? simt_adjoint_f64(r) : simt_adjoint_f32(r);
}

static bool jadj_ok(const tode_field_desc* f, const tode_options* o) {
  return f->kind == TODE_MLP && o->prec == TODE_BF16W_SPLIT && !o->rtol_b && !o->atol_b &&
         !o->joint;
}

size_t tode_joint_adjoint_workspace_size(const tode_field_desc* f, const tode_options* o) {
  if (!opts_ok(o) || field_ok(f, o) != TODE_OK || !jadj_ok(f, o)) return 0;
  return mlp_jadj_workspace_bytes(f);
}

tode_err tode_joint_adjoint(const tode_field_desc* f, const tode_options* o, double t0, double t1,
                            const double* t_eval, int K, const void* y1, const void* gy_eval,
                            const void* gy_final, void* gy0, float* const* gW, float* const* gb,
                            void* y0, int32_t* stats, void* workspace, size_t ws_bytes,
                            void* stream) {
  if (!opts_ok(o) || K < 0 || !stats) return TODE_EINVAL;
  tode_err e = field_ok(f, o);
  if (e != TODE_OK) return e;
  if (f->kind != TODE_MLP || o->prec != TODE_BF16W_SPLIT || o->joint) return TODE_EUNSUPPORTED;
  if (o->rtol_b || o->atol_b) return TODE_EINVAL;
  if (!std::isfinite(t0) || !std::isfinite(t1) || !(t0 < t1)) return TODE_EINVAL;
  if (K > 0 && !t_eval) return TODE_EINVAL;
  for (int q = 0; q < K; ++q)
    if (!(t_eval[q] >= t0 && t_eval[q] <= t1) || (q > 0 && t_eval[q] < t_eval[q - 1]))
      return TODE_EINVAL;
  stats[0] = stats[1] = stats[2] = 0;
  stats[3] = TODE_S_SUCCESS;
  if (f->B == 0) return TODE_OK;
  if (!y1 || !gy0 || !gW || !gW[0] || !gW[1] || !gW[2]) return TODE_EINVAL;
  const size_t need = mlp_jadj_workspace_bytes(f);
  if (need == 0) return TODE_EUNSUPPORTED;
  if (!workspace || !aligned256(workspace) || ws_bytes < need) return TODE_EWORKSPACE;
  JadjReq r{};
  r.f = f;
  r.o = o;
  r.B = f->B;
  r.K = K;
  r.t0 = t0;
  r.t1 = t1;
  r.te = t_eval;
  r.y1 = (const float*)y1;
  r.gye = (const float*)gy_eval;
  r.gyf = (const float*)gy_final;
  r.gy0 = (float*)gy0;
  r.y0 = (float*)y0;
  r.gW = gW;
  r.gb = gb;
  r.stats = stats;
  r.ws = (char*)workspace;
  r.stream = (cudaStream_t)stream;
  return mlp_joint_adjoint(r);
}

tode_err tode_t_bounds_grad(const tode_field_desc* f, const tode_options* o, const double* t0,
                            const double* t1, const double* t_eval, int K, const int32_t* n_acc,
                            const int32_t* status, const tode_tape* tape, const void* gy_eval,
                            const void* gy_final, const void* yp_eval, double* g_t0,
                            double* g_t1, void* stream) {
  if (!opts_ok(o) || K < 0) return TODE_EINVAL;
  tode_err e = field_ok(f, o);
  if (e != TODE_OK) return e;
  if (o->joint) return TODE_EUNSUPPORTED;
  if (f->kind == TODE_MLP && o->prec != TODE_BF16W_SPLIT) return TODE_EUNSUPPORTED;
  if (f->B == 0) return TODE_OK;
  if (!t0 || !t1 || !n_acc || !status || !tape || !g_t1) return TODE_EINVAL;
  if (K > 0 && !t_eval) return TODE_EINVAL;
  if (g_t0 && K > 0 && gy_eval && !yp_eval) return TODE_EINVAL;
  if (!tape_ok(tape, o, f) || tape->stride != 1 || !tape->h_acc) return TODE_EINVAL;
  AdjReq r{};
  r.f = f;
  r.o = o;
  r.B = f->B;
  r.D = f->D;
  r.K = K;
  r.t0 = t0;
  r.t1 = t1;
  r.te = t_eval;
  r.n_acc = n_acc;
  r.status = status;
  r.tape = tape;
  r.gye = gy_eval;
  r.gyf = gy_final;
  r.stream = (cudaStream_t)stream;
  e = device_sms(&r.num_sms);
  if (e != TODE_OK) return e;
  if (f->kind == TODE_MLP) return mlp_t_bounds(r, yp_eval, g_t0, g_t1);
  return o->prec == TODE_F64 ? simt_t_bounds_f64(r, yp_eval, g_t0, g_t1)
                             : simt_t_bounds_f32(r, yp_eval, g_t0, g_t1);
}

}  // extern "C"

namespace tode {
// g[i][q] = sum_j gy[i][q][j] yp[i][q][j], one warp per row, FP64 sums in a
// fixed order (lane-strided partial sums, then a butterfly).
template <typename T>
__global__ void k_t_eval_grad(long long rows, int D, const T* gy, const T* yp, double* g) {
  const long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;  // whole warps leave together
  double s = 0.0;
  for (int j = lane; j < D; j += 32) s += (double)gy[row * D + j] * (double)yp[row * D + j];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) g[row] = s;
}
}  // namespace tode

extern "C" {
tode_err tode_t_eval_grad(int B, int K, int D, tode_prec prec, const void* gy_eval,
                          const void* yp_eval, double* g_t_eval, void* stream) {
  if (B < 0 || K < 0 || D < 1) return TODE_EINVAL;
  if (prec != TODE_F64 && prec != TODE_F32) return TODE_EUNSUPPORTED;
  const long long rows = (long long)B * K;
  if (rows == 0) return TODE_OK;
  if (!gy_eval || !yp_eval || !g_t_eval) return TODE_EINVAL;
  const int block = 256;
  const long long grid = (rows * 32 + block - 1) / block;
  if (grid > 0x7fffffffLL) return TODE_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  if (prec == TODE_F64)
    tode::k_t_eval_grad<double><<<(unsigned)grid, block, 0, st>>>(
        rows, D, (const double*)gy_eval, (const double*)yp_eval, g_t_eval);
  else
    tode::k_t_eval_grad<float><<<(unsigned)grid, block, 0, st>>>(
        rows, D, (const float*)gy_eval, (const float*)yp_eval, g_t_eval);
  TODE_CUDA_TRY(cudaGetLastError());
  return TODE_OK;
}
}  // extern "C"
