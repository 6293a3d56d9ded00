// tode_simt.cuh -- forward kernels for the SIMT fields (Van der Pol, linear):
// the plain form (one launch per step over the masked batch) and the fused
// persistent form with work stealing.  Both call the same inst_init /
// inst_attempt / inst_finalize routines, so their results are bit-identical.
#pragma once
#include "tode_core.cuh"
#include "tode_fields.cuh"
#include "tode_internal.h"

namespace tode {

template <typename T> struct SolveArgs {
  int B, D, K;
  const T* y0;
  const double* t0;
  const double* t1;
  const double* te;
  const double* rtol_b;
  const double* atol_b;
  double rtol, atol;
  T* ye;
  T* yp;  // NULL unless requested
  T* yf;
  int32_t *n_acc, *n_rej, *n_fe, *status;
  SolveOpts o;
  TapeDev<T> tape;
  TraceDev trace;
  const T* fparam;  // mu [B] or A [B][D][D]
  // plain-form state, lane-interleaved: y[(r*B + i)*G + g]
  T* wy;
  T* wylo;
  T* wk;
  double* wt;
  T* wh;
  T* wep;
  T* wep2;
  int32_t* wcur;
  int32_t* wfl;
  int32_t* active;
  int32_t* counter;  // fused form: next queue position to hand out
  const int32_t* order;  // work queue: instance at each position (NULL: index order)
  int* order_part;       // the large-batch sort's per-CTA counts
};

// Instance at queue position j (B past the end of the queue).
template <typename T> __device__ __forceinline__ int queued(const SolveArgs<T>& a, int j) {
  return j >= a.B ? a.B : (a.order ? a.order[j] : j);
}

template <typename T>
__device__ __forceinline__ InstOut<T> inst_out(const SolveArgs<T>& a, int i) {
  InstOut<T> o;
  o.K = a.K;
  o.te = a.te + (size_t)i * a.K;
  o.ye = a.ye + (size_t)i * a.K * a.D;
  o.yp = a.yp ? a.yp + (size_t)i * a.K * a.D : nullptr;
  return o;
}

// The field's direction factor for instance i (-1: backward in time).
template <typename T> __device__ __forceinline__ T dir_of(const SolveArgs<T>& a, int i) {
  return reversed_at(a.t0, a.t1, i) ? T(-1) : T(1);
}

template <typename T> __device__ __forceinline__ double rtol_of(const SolveArgs<T>& a, int i) {
  return a.rtol_b ? a.rtol_b[i] : a.rtol;
}
template <typename T> __device__ __forceinline__ double atol_of(const SolveArgs<T>& a, int i) {
  return a.atol_b ? a.atol_b[i] : a.atol;
}

// Plain-form state between launches, kept at the queue position j (so a
// warp's accesses stay contiguous); the outputs are at the instance i.
template <typename T, int R, int G>
__device__ __forceinline__ void plain_store(const SolveArgs<T>& a, int j, int i,
                                            const Inst<T, R>& s) {
  const int g = Grp<G>::rank();
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const size_t q = ((size_t)r * a.B + j) * G + g;
    a.wy[q] = s.y[r];
    if constexpr (Comp<T>::on) a.wylo[q] = s.ylo[r];
    a.wk[q] = s.k1[r];
  }
  if (g == 0) {
    a.wt[j] = s.t;
    a.wh[j] = s.h;
    a.wep[j] = s.err_prev;
    a.wep2[j] = s.err_prev2;
    a.wcur[j] = s.cursor;
    a.wfl[j] = s.flags;
    a.n_acc[i] = s.n_acc;
    a.n_rej[i] = s.n_rej;
    a.status[i] = s.status;
  }
}

template <typename T, int R, int G>
__device__ __forceinline__ void plain_load(const SolveArgs<T>& a, int j, int i,
                                           Inst<T, R>& s) {
  const int g = Grp<G>::rank();
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const size_t q = ((size_t)r * a.B + j) * G + g;
    s.y[r] = a.wy[q];
    s.ylo[r] = Comp<T>::on ? a.wylo[q] : T(0);
    s.k1[r] = a.wk[q];
  }
  s.t = a.wt[j];
  s.flags = a.wfl[j];
  const unsigned long long m = rev_mask(s.flags);
  s.t0 = flip(a.t0[i], m);
  s.t1 = flip(a.t1[i], m);
  s.h = a.wh[j];
  s.err_prev = a.wep[j];
  s.err_prev2 = a.wep2[j];
  s.cursor = a.wcur[j];
  const InstOut<T> out = inst_out(a, i);
  s.tq = te_at(out, s.cursor, m);
  s.tq2 = te_at(out, s.cursor + 1, m);
  s.n_acc = a.n_acc[i];
  s.n_rej = a.n_rej[i];
  s.status = a.status[i];
  s.rtol = T(rtol_of(a, i));
  s.atol = T(atol_of(a, i));
  if constexpr (Comp<T>::on) {  // functions of (t, t0, t1), as in the fused form
    s.rem = __double2float_rd(s.t1 - s.t);
    s.hmin = T(1e-14 * tmax(fabs(s.t0), fabs(s.t1)));
  }
}

// ---------------------------------------------------------------- plain form
template <class Field, typename T, int R, int G>
__global__ void k_plain_init(SolveArgs<T> a) {
  const int j = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) / G);
  if (j >= a.B) return;
  const int i = queued(a, j);
  Field F;
  F.load(a.fparam, i, dir_of(a, i));
  Inst<T, R> s;
  const bool run =
      inst_init<Field, T, R, G>(F, s, a.o, i, a.D, a.y0, a.t0, a.t1, rtol_of(a, i),
                                atol_of(a, i), inst_out(a, i));
  if (run) tape_store<T, R, G>(a.tape, i, s);
  plain_store<T, R, G>(a, j, i, s);
  if (!run)
    inst_finalize<T, R, G>(s, a.o, i, a.D, inst_out(a, i), a.yf, a.n_acc, a.n_rej, a.n_fe,
                           a.status, a.trace);
}

template <class Tab, class Field, typename T, int R, int G, bool YP>
__global__ void k_plain_step(SolveArgs<T> a) {
  const int j = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) / G);
  if (j >= a.B) return;
  const int i = queued(a, j);
  if (a.status[i] != ST_RUNNING) return;  // masked: finished instances do no work
  Field F;
  F.load(a.fparam, i, dir_of(a, i));
  Inst<T, R> s;
  plain_load<T, R, G>(a, j, i, s);
  const int acc_before = s.n_acc;
  T ys[6][R];
  const bool run =
      inst_attempt<Tab, Field, T, R, G, YP>(F, s, a.o, i, a.D, inst_out(a, i), a.trace, ys);
  if (s.n_acc != acc_before) {
    tape_store_hacc<T, R, G>(a.tape, i, s, ys);
    if (run) tape_store<T, R, G>(a.tape, i, s);
  }
  plain_store<T, R, G>(a, j, i, s);
  if (!run) {
    inst_finalize<T, R, G>(s, a.o, i, a.D, inst_out(a, i), a.yf, a.n_acc, a.n_rej, a.n_fe,
                           a.status, a.trace);
  } else if (Grp<G>::rank() == 0) {
    *a.active = 1;
  }
}

// ---------------------------------------------------------------- fused form
// Persistent kernel: each group integrates one instance at a time to its end
// and then steals the next; one loop iteration is one attempt, so a group
// whose instance finished refills at once instead of waiting for its warp.
template <class Tab, class Field, typename T, int R, int G, bool YP>
__global__ void __launch_bounds__(256) k_fused(SolveArgs<T> a) {
  const int groups_total = (int)((gridDim.x * (size_t)blockDim.x) / G);
  int i = queued(a, (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) / G));
  Field F;
  Inst<T, R> s;
  bool have = false;
  while (true) {
    if (!have) {
      if (i >= a.B) break;
      F.load(a.fparam, i, dir_of(a, i));
      have = inst_init<Field, T, R, G>(F, s, a.o, i, a.D, a.y0, a.t0, a.t1, rtol_of(a, i),
                                       atol_of(a, i), inst_out(a, i));
      if (!have) {
        inst_finalize<T, R, G>(s, a.o, i, a.D, inst_out(a, i), a.yf, a.n_acc, a.n_rej,
                               a.n_fe, a.status, a.trace);
        i = queued(a, grab_instance<G>(a.counter, groups_total));
        continue;
      }
      tape_store<T, R, G>(a.tape, i, s);
    }
    const int acc_before = s.n_acc;
    T ys[6][R];
    const bool run =
        inst_attempt<Tab, Field, T, R, G, YP>(F, s, a.o, i, a.D, inst_out(a, i), a.trace, ys);
    if (s.n_acc != acc_before) tape_store_hacc<T, R, G>(a.tape, i, s, ys);
    if (run) {
      if (s.n_acc != acc_before) tape_store<T, R, G>(a.tape, i, s);
    } else {
      inst_finalize<T, R, G>(s, a.o, i, a.D, inst_out(a, i), a.yf, a.n_acc, a.n_rej, a.n_fe,
                           a.status, a.trace);
      have = false;
      i = queued(a, grab_instance<G>(a.counter, groups_total));
    }
  }
}

// ---------------------------------------------------------------- host side
template <typename T> TapeDev<T> make_tape(const tode_tape* tp, int B, int D) {
  TapeDev<T> d{};
  d.B = B;
  d.D = D;
  if (!tp) {
    d.slots = 0;
    d.stride = 1;
    return d;
  }
  d.slots = tp->slots;
  d.stride = tp->stride;
  d.y = (T*)tp->y;
  d.ylo = (T*)tp->y_lo;
  d.k1 = (T*)tp->k1;
  d.t = tp->t;
  d.h = (T*)tp->h;
  d.err_prev = (T*)tp->err_prev;
  d.err_prev2 = (T*)tp->err_prev2;
  d.flags = tp->flags;
  d.h_acc = (T*)tp->h_acc;
  d.ystage = (T*)tp->y_stage;
  return d;
}

inline SolveOpts make_opts(const tode_options* o) {
  SolveOpts s;
  s.safety = o->safety;
  s.fac_min = o->fac_min;
  s.fac_max = o->fac_max;
  s.beta1 = o->beta1;
  s.beta2 = o->beta2;
  s.beta3 = o->beta3;
  s.h0 = o->h0;
  s.max_steps = o->max_steps;
  opts_round_f32(s);
  return s;
}

template <typename T> SolveArgs<T> make_solve_args(const SolveReq& r) {
  SolveArgs<T> a{};
  a.B = r.B;
  a.D = r.D;
  a.K = r.K;
  a.y0 = (const T*)r.y0;
  a.t0 = r.t0;
  a.t1 = r.t1;
  a.te = r.te;
  a.rtol_b = r.o->rtol_b;
  a.atol_b = r.o->atol_b;
  a.rtol = r.o->rtol;
  a.atol = r.o->atol;
  a.ye = (T*)r.ye;
  a.yp = (T*)r.yp;
  a.yf = (T*)r.yf;
  a.n_acc = r.n_acc;
  a.n_rej = r.n_rej;
  a.n_fe = r.n_fe;
  a.status = r.status;
  a.o = make_opts(r.o);
  a.tape = make_tape<T>(r.tape, r.B, r.D);
  if (r.trace) {
    a.trace.cap = r.trace->cap;
    a.trace.t = r.trace->t;
    a.trace.h = r.trace->h;
    a.trace.err = r.trace->err;
    a.trace.acc = r.trace->accepted;
    a.trace.len = r.trace->len;
  } else {
    a.trace.cap = 0;
  }
  a.fparam = (const T*)(r.f->kind == TODE_VDP ? r.f->mu : r.f->A);
  // workspace carve (must match simt_workspace_bytes)
  char* p = r.ws;
  a.active = (int32_t*)p;
  a.counter = (int32_t*)(p + 128);
  p += align256(256);
  a.order = r.o->order == 1 ? (const int32_t*)p : nullptr;
  p += align256((size_t)r.B * 4);
  a.order_part = (int*)p;
  p += order_part_bytes(r.B);
  if (r.o->form == TODE_PLAIN) {
    const size_t ts = sizeof(T);
    a.wy = (T*)p;
    p += align256((size_t)r.B * r.D * ts);
    a.wylo = (T*)p;
    p += align256((size_t)r.B * r.D * ts);
    a.wk = (T*)p;
    p += align256((size_t)r.B * r.D * ts);
    a.wt = (double*)p;
    p += align256((size_t)r.B * 8);
    a.wh = (T*)p;
    p += align256((size_t)r.B * ts);
    a.wep = (T*)p;
    p += align256((size_t)r.B * ts);
    a.wep2 = (T*)p;
    p += align256((size_t)r.B * ts);
    a.wcur = (int32_t*)p;
    p += align256((size_t)r.B * 4);
    a.wfl = (int32_t*)p;
    p += align256((size_t)r.B * 4);
  }
  return a;
}

// Default threads per CTA: 128, or fewer (down to one warp) when the batch
// has fewer than 128 threads per SM, so that a small batch still spreads
// over every SM instead of filling a few.
inline int default_block(long long threads, int num_sms) {
  const long long per_sm = (threads + num_sms - 1) / (num_sms > 0 ? num_sms : 1);
  int b = 32;
  while (b < 128 && b < per_sm) b *= 2;
  return b;
}

template <class Tab, class Field, typename T, int R, int G, bool YP>
tode_err launch_solve_yp(const SolveReq& r) {
  SolveArgs<T> a = make_solve_args<T>(r);
  const cudaStream_t st = r.stream;
  const long long threads = (long long)r.B * G;
  const int block = r.o->block > 0 ? r.o->block : default_block(threads, r.num_sms);
  if (block % 32 != 0 || block > 256) return TODE_EINVAL;
  if (a.order) {
    TODE_CUDA_TRY(launch_order(r.B, IntervalBin{r.t0, r.t1}, const_cast<int32_t*>(a.order),
                               a.order_part, st));
  }
  if (r.o->form == TODE_PLAIN) {
    const int grid = (int)((threads + block - 1) / block);
    if (grid == 0) return TODE_OK;
    k_plain_init<Field, T, R, G><<<grid, block, 0, st>>>(a);
    TODE_CUDA_TRY(cudaGetLastError());
    const int poll = r.o->poll_every > 0 ? r.o->poll_every : 16;
    long long launched = 0;
    const long long limit = (long long)r.o->max_steps + 2LL * poll + 2;
    while (true) {
      for (int c = 0; c < poll - 1; ++c)
        k_plain_step<Tab, Field, T, R, G, YP><<<grid, block, 0, st>>>(a);
      TODE_CUDA_TRY(cudaMemsetAsync(a.active, 0, sizeof(int32_t), st));
      k_plain_step<Tab, Field, T, R, G, YP><<<grid, block, 0, st>>>(a);
      TODE_CUDA_TRY(cudaGetLastError());
      launched += poll;
      int32_t any = 0;
      TODE_CUDA_TRY(cudaMemcpyAsync(&any, a.active, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      TODE_CUDA_TRY(cudaStreamSynchronize(st));
      if (!any) break;
      // every launch advances each running instance by one attempt, so
      // max_steps bounds the loop; this guard is never expected to fire
      if (launched > limit) return TODE_ETIMEOUT;
    }
    return TODE_OK;
  }
  // fused persistent form
  int per_sm = r.o->ctas_per_sm;
  if (per_sm <= 0) {
    TODE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, k_fused<Tab, Field, T, R, G, YP>, block, 0));
    if (per_sm < 1) per_sm = 1;
  }
  long long grid = (long long)r.num_sms * per_sm;
  const long long need = (threads + block - 1) / block;
  if (grid > need) grid = need;
  if (grid == 0) return TODE_OK;
  TODE_CUDA_TRY(cudaMemsetAsync(a.counter, 0, sizeof(int32_t), st));
  k_fused<Tab, Field, T, R, G, YP><<<(int)grid, block, 0, st>>>(a);
  TODE_CUDA_TRY(cudaGetLastError());
  return TODE_OK;
}

template <class Tab, class Field, typename T, int R, int G>
tode_err launch_solve(const SolveReq& r) {
  return r.yp ? launch_solve_yp<Tab, Field, T, R, G, true>(r)
              : launch_solve_yp<Tab, Field, T, R, G, false>(r);
}

// Lanes per instance of the linear field (0 = unsupported combination).
// D <= 8: one row per lane.  D = 16: 4, 8 or 16 lanes, default 8 (fastest of
// the three on B300 for the D = 16, B = 8192 workload: 0.123 ms vs 0.131 ms
// for 16 and 0.135 ms for 4).  D = 32: 16 lanes of two rows.
inline int linear_group(int D, int requested) {
  switch (D) {
    case 1: case 2: case 4: case 8: return (requested == 0 || requested == D) ? D : 0;
    case 16: return requested == 0 ? 8 : (requested == 4 || requested == 8 || requested == 16)
                                             ? requested : 0;
    case 32: return (requested == 0 || requested == 16) ? 16 : 0;
    default: return 0;
  }
}

// Field / group dispatch for one state dtype and pair.
template <class Tab, typename T> tode_err simt_solve(const SolveReq& r) {
  if (r.f->kind == TODE_VDP) return launch_solve<Tab, VdpField<T>, T, 2, 1>(r);
  switch (linear_group(r.D, r.o->group)) {
    case 1: return launch_solve<Tab, LinearField<T, 1, 1>, T, 1, 1>(r);
    case 2: return launch_solve<Tab, LinearField<T, 1, 2>, T, 1, 2>(r);
    case 4: return r.D == 4 ? launch_solve<Tab, LinearField<T, 1, 4>, T, 1, 4>(r)
                            : launch_solve<Tab, LinearField<T, 4, 4>, T, 4, 4>(r);
    case 8: return r.D == 8 ? launch_solve<Tab, LinearField<T, 1, 8>, T, 1, 8>(r)
                            : launch_solve<Tab, LinearField<T, 2, 8>, T, 2, 8>(r);
    case 16: return r.D == 16 ? launch_solve<Tab, LinearField<T, 1, 16>, T, 1, 16>(r)
                              : launch_solve<Tab, LinearField<T, 2, 16>, T, 2, 16>(r);
    default: return TODE_EUNSUPPORTED;
  }
}

}  // namespace tode
