// tode_simt_joint.cuh -- joint ("stacked") solving for the SIMT fields
// (Sec. 4.1): the batch is treated as one problem of size B*D with one time
// axis, one step size, one error norm over all B*D components and one
// accept/reject decision.  These are the semantics the paper's batching
// experiment (Fig. 1) compares independent solving against; every instance
// still evaluates its own field.
//
// One launch per attempt.  Launch n commits the decision taken on attempt
// n-1 (its trace entry and the decision-dependent tape fields), then, while
// the problem runs, computes attempt n for every instance with each CTA's
// partial sum of squared scaled errors.  The CTA that finishes last (a
// ticket counter: no CTA ever waits for another) sums the partials in CTA
// order, takes the decision, runs the controller and writes the control
// block that launch n+1 reads.
//
// Every instance shares the decision, so an attempt writes its results as if
// it were accepted: the candidate state goes to the other half of a double
// buffer (an acceptance only flips the buffer index), the dense output of
// the points in (t, t + h] and the tape slots straight to their places.  A
// rejected attempt's points are written again by the accepted step that
// later covers them, and a failed solve turns every point past its last
// accepted step into NaN, so nothing but the state is ever staged.  Two
// launches before the first attempt validate the batch and pick the first
// step (the HNW Sec. II.4 heuristic with its norms over the whole batch).
#pragma once
#include "tode_simt.cuh"

namespace tode {

enum : int { JP_H0 = 1, JP_RUN = 2, JP_DONE = 3 };  // phase of the joint solve
enum : int { JD_NONE = 0, JD_ACC = 1, JD_REJ = 2 };  // decision the next launch commits

// Control block of the joint solve (device memory; written only by the CTA
// that finishes last in a launch, after every other CTA has read it).
template <typename T> struct JointCtl {
  double t, t0, t1;
  double dec_t;              // start of the decided attempt
  T h;                       // step proposed for the next attempt
  T h_use;                   // the next attempt's step, clipped at t1
  T err_prev, err_prev2, rem, hmin;
  T d1, h0;                  // starting-step heuristic between its two launches
  T dec_h, dec_err;
  int use_last, flags, n_acc, n_rej, status, phase, cursor;
  int cur;                   // half of the state double buffer that holds the state
  int dec, dec_att;
  unsigned int ticket;       // CTAs finished in the current launch
};
static_assert(sizeof(JointCtl<double>) <= JOINT_CTL_BYTES, "control block");

template <typename T> struct JointArgs {
  SolveArgs<T> a;  // problem, outputs, options
  JointCtl<T>* ctl;
  double* part;    // [grid][3] per-CTA partial sums
  T* y[2];         // state double buffer: y, its compensation term, k1 (FSAL)
  T* ylo[2];
  T* k1[2];
};

// Per-instance arrays are lane-interleaved like the plain form's state:
// component r of instance i on lane g at ((r*B + i)*G + g).
template <typename T, int R, int G>
__device__ __forceinline__ void jld(const T* p, int B, int i, T (&v)[R]) {
  const int g = Grp<G>::rank();
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = p[((size_t)r * B + i) * G + g];
}
template <typename T, int R, int G>
__device__ __forceinline__ void jst(T* p, int B, int i, const T (&v)[R]) {
  const int g = Grp<G>::rank();
#pragma unroll
  for (int r = 0; r < R; ++r) p[((size_t)r * B + i) * G + g] = v[r];
}

// Sum of one value per thread over the CTA in a fixed order (a butterfly in
// each warp, then the warps in order), in the state type: an FP32 batch
// reduces on the FP32 pipe (B300's FP64 pipe is narrow), an FP64 batch in
// FP64.  The result is valid in thread 0.
template <typename T> __device__ __forceinline__ T cta_sum(T v, double* red_d) {
  T* red = reinterpret_cast<T*>(red_d);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = T(0);
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  __syncthreads();
  return s;
}

// Thread 0 has written this CTA's partials; takes a ticket and returns, in
// every thread, whether this CTA is the last of the launch to finish.
__device__ __forceinline__ bool joint_last_cta(unsigned int* ticket, int* flag) {
  if (threadIdx.x == 0) {
    __threadfence();
    *flag = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  const bool last = *flag != 0;
  if (last) __threadfence();
  return last;
}

// The last CTA's sum of partial k over all CTAs, in CTA order per thread
// and then a fixed tree, in FP64; valid in thread 0.
__device__ __forceinline__ double joint_total(const double* part, int k, double* red) {
  double s = 0.0;
  const int n = (int)gridDim.x, stride = (int)blockDim.x;
  for (int b0 = threadIdx.x; b0 < n; b0 += 4 * stride) {
    double v[4];  // four loads in flight, added in order
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int b = b0 + u * stride;
      v[u] = b < n ? __ldcg(part + 3 * b + k) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) s += v[u];
  }
  return cta_sum<double>(s, red);
}

// The next attempt's step: the proposal, clipped so that the step ends at t1.
template <typename T> __device__ __forceinline__ void joint_clip(JointCtl<T>& c) {
  T h = c.h;
  int last = 0;
  if constexpr (Comp<T>::on) {
    if (h >= c.rem) {
      h = c.rem;
      last = 1;
    }
  } else if (c.t + (double)h >= c.t1) {
    h = T(c.t1 - c.t);
    last = 1;
  }
  c.h_use = h;
  c.use_last = last;
}

// ---------------------------------------------------------------- launch 1: init
// Validates every instance (its own time arguments, and the same t0, t1 and
// evaluation points as instance 0: one problem has one time axis), writes
// the points at t0, evaluates k1 = f(t0, y0) and sums the squared scaled y0
// and k1 for the starting-step heuristic.
template <class Field, typename T, int R, int G>
__global__ void __launch_bounds__(256) k_joint_init(JointArgs<T> ja) {
  const SolveArgs<T>& a = ja.a;
  __shared__ double red[32];
  __shared__ int last_s;
  const int g = Grp<G>::rank();
  T s0 = T(0), s1 = T(0);
  bool bad = false;
  // grid-stride over the instances (lane groups stay within one warp);
  // each thread accumulates its instances in index order
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j / G < a.B;
       j += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(j / G);
    Field F;
    F.load(a.fparam, i, dir_of(a, i));
    Inst<T, R> s;
    SolveOpts o1 = a.o;
    o1.h0 = 1.0;  // the first step is the batch's: no per-instance heuristic here
    const InstOut<T> out = inst_out(a, i);
    const bool run = inst_init<Field, T, R, G>(F, s, o1, i, a.D, a.y0, a.t0, a.t1, a.rtol, a.atol,
                                               out);
    bool same = tkey(a.t0[i]) == tkey(a.t0[0]) && tkey(a.t1[i]) == tkey(a.t1[0]);
    for (int q = g; q < a.K; q += G) same = same && tkey(out.te[q]) == tkey(a.te[q]);
    if constexpr (G > 1) same = __all_sync(Grp<G>::mask(), same) != 0;
    jst<T, R, G>(ja.y[0], a.B, i, s.y);
    if constexpr (Comp<T>::on) jst<T, R, G>(ja.ylo[0], a.B, i, s.ylo);
    jst<T, R, G>(ja.k1[0], a.B, i, s.k1);
    T q0[R], q1[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const T sc = madd(s.rtol, T(fabs(s.y[r])), s.atol);
      const T u = s.y[r] / sc, v = s.k1[r] / sc;
      q0[r] = u * u;
      q1[r] = v * v;
    }
    const T S0 = group_sum<T, R, G>(q0), S1 = group_sum<T, R, G>(q1);
    if (g == 0) {
      bad = bad || s.status == ST_INVALID || !same;
      if (run) {
        s0 += S0;
        s1 += S1;
      }
    }
  }
  const int nbad = __syncthreads_count(bad);
  s0 = cta_sum<T>(s0, red);
  s1 = cta_sum<T>(s1, red);
  if (threadIdx.x == 0) {
    ja.part[3 * blockIdx.x + 0] = (double)s0;
    ja.part[3 * blockIdx.x + 1] = (double)s1;
    ja.part[3 * blockIdx.x + 2] = (double)nbad;
  }
  if (!joint_last_cta(&ja.ctl->ticket, &last_s)) return;
  const double S0 = joint_total(ja.part, 0, red);
  const double S1 = joint_total(ja.part, 1, red);
  const double NB = joint_total(ja.part, 2, red);
  if (threadIdx.x != 0) return;
  JointCtl<T> c{};
  const bool rev = reversed_at(a.t0, a.t1, 0);  // every instance's direction
  const unsigned long long m = rev ? SIGN_BIT : 0ULL;
  c.flags = rev ? FL_REVERSE : 0;
  c.t0 = flip(a.t0[0], m);
  c.t1 = flip(a.t1[0], m);
  c.t = c.t0;
  c.err_prev = T(1);
  c.err_prev2 = T(1);
  c.phase = JP_RUN;
  c.dec = JD_NONE;
  while (c.cursor < a.K && tkey(flip(a.te[c.cursor], m)) == tkey(c.t0)) c.cursor++;
  if (NB > 0.0) {
    c.status = ST_INVALID;
  } else if (tkey(c.t1) == tkey(c.t0)) {
    c.status = ST_SUCCESS;
  } else {
    c.status = ST_RUNNING;
    if constexpr (Comp<T>::on) {
      c.rem = __double2float_rd(c.t1 - c.t0);
      c.hmin = T(1e-14 * tmax(fabs(c.t0), fabs(c.t1)));
    }
    if (a.o.h0 > 0.0) {
      c.h = T(a.o.h0);
      joint_clip(c);
    } else {
      // HNW Sec. II.4 with the RMS norms taken over all B*D components
      const double n = (double)a.B * a.D;
      const T d0 = T(sqrt(S0 / n)), d1 = T(sqrt(S1 / n));
      c.h0 = (d0 < T(1e-5) || d1 < T(1e-5)) ? T(1e-6) : T(0.01) * (d0 / d1);
      c.d1 = d1;
      c.phase = JP_H0;
    }
  }
  *ja.ctl = c;
}

// ---------------------------------------------------------------- launch 2: first step
// The heuristic's second evaluation f(t0 + h0, y0 + h0 k1); a no-op when the
// first step was given.
template <class Field, typename T, int R, int G>
__global__ void __launch_bounds__(256) k_joint_h0(JointArgs<T> ja) {
  const SolveArgs<T>& a = ja.a;
  const JointCtl<T> c = *ja.ctl;
  if (c.phase != JP_H0) return;
  __shared__ double red[32];
  __shared__ int last_s;
  T s2 = T(0);
  // grid-stride over the instances (lane groups stay within one warp);
  // each thread accumulates its instances in index order
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j / G < a.B;
       j += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(j / G);
    Field F;
    F.load(a.fparam, i, dir_of(a, i));
    const T rtol = T(a.rtol), atol = T(a.atol);
    T y[R], k1[R], w[R], f1[R], q[R];
    jld<T, R, G>(ja.y[0], a.B, i, y);
    jld<T, R, G>(ja.k1[0], a.B, i, k1);
#pragma unroll
    for (int r = 0; r < R; ++r) w[r] = madd(c.h0, k1[r], y[r]);
    F.eval(c.t0 + (double)c.h0, w, f1);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const T sc = madd(rtol, T(fabs(y[r])), atol);
      const T u = (f1[r] - k1[r]) / sc;
      q[r] = u * u;
    }
    const T S2 = group_sum<T, R, G>(q);
    if (Grp<G>::rank() == 0) s2 += S2;
  }
  s2 = cta_sum<T>(s2, red);
  if (threadIdx.x == 0) ja.part[3 * blockIdx.x] = (double)s2;
  if (!joint_last_cta(&ja.ctl->ticket, &last_s)) return;
  const double S2 = joint_total(ja.part, 0, red);
  if (threadIdx.x != 0) return;
  JointCtl<T> n = c;
  const T h0 = c.h0;
  const T d2 = T(sqrt(S2 / ((double)a.B * a.D))) / h0;
  const T m = (c.d1 > d2) ? c.d1 : d2;
  const T h1 = (m <= T(1e-15)) ? tmax(T(1e-6), h0 * T(1e-3)) : ctl_pow(T(0.01) / m, T(1.0 / 5.0));
  T h = tmin(T(100) * h0, h1);
  h = tmin(h, T(c.t1 - c.t0));
  if (!(h > T(0) && finite_(h))) h = T(c.t1 - c.t0);
  n.h = h;
  n.phase = JP_RUN;
  n.ticket = 0;
  joint_clip(n);
  *ja.ctl = n;
}

// ---------------------------------------------------------------- launch 3..: attempts
// The state slot that an accepted attempt opens, written before the
// decision: y, y_lo, k1 and t (h, err_prev and flags follow the decision).
// Joint tapes have stride 1.
template <typename T, int R, int G>
__device__ __forceinline__ void joint_tape_state(const TapeDev<T>& tp, int i, int j, double t,
                                                 const T (&y)[R], const T (&ylo)[R],
                                                 const T (&k1)[R]) {
  if (tp.slots == 0 || j >= tp.slots) return;
  const size_t o = (size_t)i * tp.slots + j;
  const int g = Grp<G>::rank();
  st_row<T, R>(tp.y + o * tp.D + g * R, y);
  if (tp.k1) st_row<T, R>(tp.k1 + o * tp.D + g * R, k1);
  if constexpr (Comp<T>::on) {
    if (tp.ylo) st_row<T, R>(tp.ylo + o * tp.D + g * R, ylo);
  }
  if (g == 0) tp.t[o] = t;
}

template <class Field, typename T, int R, int G, class Tab = DP5>
__global__ void __launch_bounds__(256) k_joint_step(JointArgs<T> ja) {
  const SolveArgs<T>& a = ja.a;
  const JointCtl<T> c = *ja.ctl;
  if (c.phase != JP_RUN) return;
  __shared__ double red[32];
  __shared__ int last_s;
  const int g = Grp<G>::rank();
  T sq = T(0);
  bool nonfin = false;
  // grid-stride over the instances (lane groups stay within one warp);
  // each thread accumulates its instances in index order.  The next
  // instance's state and field are loaded one iteration ahead, so that
  // their latency overlaps the current instance's attempt.
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  T ny[R], nylo[R], nk1[R];
  Field nF;
  const T dir = (c.flags & FL_REVERSE) ? T(-1) : T(1);  // the batch's direction
  auto fetch = [&](int i) {
    jld<T, R, G>(ja.y[c.cur], a.B, i, ny);
    if constexpr (Comp<T>::on) jld<T, R, G>(ja.ylo[c.cur], a.B, i, nylo);
    jld<T, R, G>(ja.k1[c.cur], a.B, i, nk1);
    nF.load(a.fparam, i, dir);
  };
  if (j / G < a.B) fetch((int)(j / G));
  for (; j / G < a.B; j += stride) {
    const int i = (int)(j / G);
    Inst<T, R> s;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      s.y[r] = ny[r];
      s.ylo[r] = Comp<T>::on ? nylo[r] : T(0);
      s.k1[r] = nk1[r];
    }
    const Field F = nF;
    if ((j + stride) / G < a.B) fetch((int)((j + stride) / G));
    const InstOut<T> out = inst_out(a, i);
    // ---- commit the decided attempt: its trace entry, and the controller
    // state of the tape slot it opened
    if (c.dec != JD_NONE && a.trace.cap > 0 && c.dec_att < a.trace.cap && g == 0) {
      const size_t q = (size_t)i * a.trace.cap + c.dec_att;
      a.trace.t[q] = flip(c.dec_t, rev_mask(c.flags));  // the caller's time and signed step
      a.trace.h[q] = flip((double)c.dec_h, rev_mask(c.flags));
      a.trace.err[q] = (double)c.dec_err;
      a.trace.acc[q] = c.dec == JD_ACC ? 1 : 0;
    }
    if (c.dec == JD_ACC && c.status == ST_RUNNING && g == 0 && c.n_acc < a.tape.slots) {
      const size_t o = (size_t)i * a.tape.slots + c.n_acc;
      if (a.tape.h) a.tape.h[o] = c.h;
      if (a.tape.err_prev) a.tape.err_prev[o] = c.err_prev;
      if (a.tape.err_prev2) a.tape.err_prev2[o] = c.err_prev2;
      if (a.tape.flags) a.tape.flags[o] = c.flags;
    }
    s.t0 = c.t0;
    s.t1 = c.t1;
    s.t = c.t;
    s.h = c.h;
    s.err_prev = c.err_prev;
    s.err_prev2 = c.err_prev2;
    s.flags = c.flags;
    s.rtol = T(a.rtol);
    s.atol = T(a.atol);
    s.n_acc = c.n_acc;
    s.n_rej = c.n_rej;
    s.status = c.status;
    s.cursor = c.cursor;
    if (c.dec == JD_NONE && c.status == ST_RUNNING) tape_store<T, R, G>(a.tape, i, s);  // slot 0
    if (c.status != ST_RUNNING) {
      if (c.status == ST_INVALID) {  // the batch is not one problem: no output is defined
        T nanv[R];
#pragma unroll
        for (int r = 0; r < R; ++r) nanv[r] = nan_(T(0));
        for (int q = 0; q < a.K; ++q) store_point<T, R, G>(out.ye + (size_t)q * a.D, nanv);
      }
      inst_finalize<T, R, G>(s, a.o, i, a.D, out, a.yf, a.n_acc, a.n_rej, a.n_fe, a.status,
                             a.trace);
    } else {
      // ---- attempt n with the batch's step
      const T h = c.h_use;
      const double hd = (double)h;
      T ys[6][R], y1[R], inc[R], ev[R], sc[R], q2[R];
      Stages<T, R> K;  // the pair Tab (dopri5 or tsit5)
#pragma unroll
      for (int r = 0; r < R; ++r) K.k[0][r] = s.k1[r];
      attempt_stages<Tab, Field, T, R>(F, c.t, h, s.y, K, ys, y1, inc);
      const T (&k7)[R] = K.k[6];
      bool fin = error_terms<Tab, T, R>(h, s.y, y1, K, s.rtol, s.atol, ev, sc);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const T u = ev[r] / sc[r];
        q2[r] = u * u;
      }
      const T S = group_sum<T, R, G>(q2);
      if constexpr (G > 1) fin = __all_sync(Grp<G>::mask(), fin) != 0;
      if (g == 0) {
        sq += S;
        nonfin = nonfin || !fin;
      }
      T yn[R], ylon[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if constexpr (Comp<T>::on) {  // compensated y + (inc + y_lo), as in the independent form
          const T u = inc[r] + s.ylo[r];
          yn[r] = s.y[r] + u;
          ylon[r] = (s.y[r] - yn[r]) + u;
        } else {
          yn[r] = y1[r];
          ylon[r] = T(0);
        }
      }
      const int nb = c.cur ^ 1;
      jst<T, R, G>(ja.y[nb], a.B, i, yn);
      if constexpr (Comp<T>::on) jst<T, R, G>(ja.ylo[nb], a.B, i, ylon);
      jst<T, R, G>(ja.k1[nb], a.B, i, k7);  // FSAL
      // ---- the results of an acceptance, written before the decision
      double t_next = c.use_last ? c.t1 : c.t + hd;
      if constexpr (Comp<T>::on) {
        if (!c.use_last && tkey(t_next) >= tkey(c.t1)) t_next = c.t1;  // landed on t1
      }
      const long long kn = tkey(t_next);
      for (int q = c.cursor; q < a.K; ++q) {  // the points in (t, t_next]
        // the batch's evaluation times (equal in every row)
        const double tq = flip(a.te[q], rev_mask(c.flags));
        const long long kq = tkey(tq);
        if (kq > kn) break;
        T* dst = out.ye + (size_t)q * a.D;
        if (kq == kn) {
          store_point<T, R, G>(dst, yn);
        } else {
          T theta;
          if constexpr (Comp<T>::on) theta = T(tq - c.t) / h;
          else theta = T((tq - c.t) / hd);
          T v[R];
          dense_point<Tab, T, R>(theta, h, s.y, s.ylo, K, v);
          store_point<T, R, G>(dst, v);
        }
      }
      if (a.tape.slots > 0) {
        s.n_acc = c.n_acc + 1;
        s.h_last = h;
        tape_store_hacc<T, R, G>(a.tape, i, s, ys);
        joint_tape_state<T, R, G>(a.tape, i, c.n_acc + 1, t_next, yn, ylon, k7);
      }
    }
  }
  const int nnf = __syncthreads_count(nonfin);
  sq = cta_sum<T>(sq, red);
  if (threadIdx.x == 0) {
    ja.part[3 * blockIdx.x + 0] = (double)sq;
    ja.part[3 * blockIdx.x + 1] = (double)nnf;
  }
  if (!joint_last_cta(&ja.ctl->ticket, &last_s)) return;
  const double S = joint_total(ja.part, 0, red);
  const double NF = joint_total(ja.part, 1, red);
  if (threadIdx.x != 0) return;
  // ---- the batch's decision (a5..a9 on the concatenated problem)
  JointCtl<T> n = c;
  n.ticket = 0;
  n.dec = JD_NONE;
  if (c.status != ST_RUNNING) {
    n.phase = JP_DONE;
    *ja.ctl = n;
    return;
  }
  const T err = T(sqrt(S / ((double)a.B * a.D)));
  const bool finite = NF == 0.0 && finite_(err);
  const bool accept = finite && err <= T(1);
  const T h = c.h_use;
  const double hd = (double)h;
  bool last = c.use_last != 0;
  n.dec_t = c.t;
  n.dec_h = h;
  n.dec_err = err;
  n.dec_att = c.n_acc + c.n_rej;
  T h_next;
  if (accept) {
    double t_next = last ? c.t1 : c.t + hd;
    if constexpr (Comp<T>::on) {
      if (!last && tkey(t_next) >= tkey(c.t1)) {  // landed on t1 by rounding
        last = true;
        t_next = c.t1;
      }
    }
    const long long kn = tkey(t_next);
    while (n.cursor < a.K && tkey(flip(a.te[n.cursor], rev_mask(c.flags))) <= kn) n.cursor++;
    T fac;
    if (err == T(0)) {
      fac = opt_v<T>(a.o.fac_max, a.o.fac_max_f);
    } else {
      fac = opt_v<T>(a.o.safety, a.o.safety_f) * ctl_pow(err, -opt_v<T>(a.o.beta1, a.o.beta1_f));
      if (a.o.beta2 != 0.0) fac = fac * ctl_pow(c.err_prev, opt_v<T>(a.o.beta2, a.o.beta2_f));
      if (a.o.beta3 != 0.0)
        fac = fac * ctl_pow(c.err_prev2, -opt_v<T>(a.o.beta3, a.o.beta3_f));
    }
    fac = tmin(tmax(fac, opt_v<T>(a.o.fac_min, a.o.fac_min_f)),
               opt_v<T>(a.o.fac_max, a.o.fac_max_f));
    if (c.flags & FL_PREV_REJ) fac = tmin(fac, T(1));
    h_next = h * fac;
    n.err_prev2 = c.err_prev;
    n.err_prev = tmax(err, T(1e-4));
    n.flags = c.flags & ~FL_PREV_REJ;
    n.n_acc = c.n_acc + 1;
    n.t = t_next;
    n.cur = c.cur ^ 1;
    if constexpr (Comp<T>::on) {
      if (!last) n.rem = __double2float_rd(c.t1 - t_next);
    }
    if (last) n.status = ST_SUCCESS;
    n.dec = JD_ACC;
  } else {
    const T fmin = opt_v<T>(a.o.fac_min, a.o.fac_min_f);
    const T fac =
        finite ? tmin(tmax(opt_v<T>(a.o.safety, a.o.safety_f) *
                               ctl_pow(err, -opt_v<T>(a.o.beta1, a.o.beta1_f)),
                           fmin),
                      T(1))
               : fmin;
    h_next = h * fac;
    n.flags = c.flags | FL_PREV_REJ;
    n.n_rej = c.n_rej + 1;
    n.dec = JD_REJ;
  }
  n.h = h_next;
  if (n.status == ST_RUNNING) {
    bool under;
    if constexpr (Comp<T>::on) {
      under = !(h_next >= c.hmin) || !(h_next > T(0));
    } else {
      const double scale = tmax(fabs(n.t), fabs(c.t1));
      const double hn = (double)h_next;
      under = n.t + hn == n.t || hn < 1e-14 * scale || !(h_next > T(0));
    }
    if (under)
      n.status = finite ? ST_DT_UNDERFLOW : ST_NONFINITE;
    else if (n.n_acc + n.n_rej >= a.o.max_steps)
      n.status = ST_MAX_STEPS;
  }
  if (n.status == ST_RUNNING) joint_clip(n);
  *ja.ctl = n;
}

// ---------------------------------------------------------------- host side
// Workspace of the joint solve (must match simt_workspace_bytes).
template <typename T> JointArgs<T> make_joint_args(const SolveReq& r) {
  JointArgs<T> j{};
  j.a = make_solve_args<T>(r);
  j.a.order = nullptr;  // one problem: every instance takes every attempt
  char* p = r.ws + joint_ws_offset(r.B);
  const size_t bd = align256((size_t)r.B * r.D * sizeof(T));
  j.ctl = (JointCtl<T>*)p;
  p += JOINT_CTL_BYTES;
  j.part = (double*)p;
  p += joint_part_bytes(r.B);
  T** arrays[6] = {&j.y[0], &j.y[1], &j.ylo[0], &j.ylo[1], &j.k1[0], &j.k1[1]};
  for (T** q : arrays) {
    *q = (T*)p;
    p += bd;
  }
  return j;
}

template <class Field, typename T, int R, int G, class Tab>
tode_err launch_joint(const SolveReq& r) {
  if (r.B == 0) return TODE_OK;
  JointArgs<T> ja = make_joint_args<T>(r);
  const cudaStream_t st = r.stream;
  const long long threads = (long long)r.B * G;
  const int block = r.o->block > 0 ? r.o->block : default_block(threads, r.num_sms);
  if (block % 32 != 0 || block > 256) return TODE_EINVAL;
  // as many CTAs as are resident at once (one partial sum each, so the CTA
  // that finishes last has few to add), at most one per lane group
  int per_sm = r.o->ctas_per_sm;
  if (per_sm <= 0) {
    TODE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, k_joint_step<Field, T, R, G, Tab>, block, 0));
    if (per_sm < 1) per_sm = 1;
  }
  long long grid_ll = (threads + block - 1) / block;
  if (grid_ll > (long long)r.num_sms * per_sm) grid_ll = (long long)r.num_sms * per_sm;
  const int grid = (int)grid_ll;
  TODE_CUDA_TRY(cudaMemsetAsync(ja.ctl, 0, sizeof(JointCtl<T>), st));
  k_joint_init<Field, T, R, G><<<grid, block, 0, st>>>(ja);
  k_joint_h0<Field, T, R, G><<<grid, block, 0, st>>>(ja);
  TODE_CUDA_TRY(cudaGetLastError());
  const int poll = r.o->poll_every > 0 ? r.o->poll_every : 16;
  // one launch per attempt plus the one that finalizes
  const long long limit = (long long)r.o->max_steps + 2LL * poll + 2;
  long long launched = 0;
  while (true) {
    for (int k = 0; k < poll; ++k) k_joint_step<Field, T, R, G, Tab><<<grid, block, 0, st>>>(ja);
    TODE_CUDA_TRY(cudaGetLastError());
    launched += poll;
    int phase = 0;
    TODE_CUDA_TRY(cudaMemcpyAsync(&phase, &ja.ctl->phase, sizeof(int), cudaMemcpyDeviceToHost,
                                  st));
    TODE_CUDA_TRY(cudaStreamSynchronize(st));
    if (phase == JP_DONE) break;
    if (launched > limit) return TODE_ETIMEOUT;  // never expected: max_steps bounds the loop
  }
  return TODE_OK;
}

// Field / group dispatch of the joint solve (the same lane groups as the
// independent solver).
template <typename T, class Tab = DP5> tode_err simt_joint(const SolveReq& r) {
  if (r.f->kind == TODE_VDP) return launch_joint<VdpField<T>, T, 2, 1, Tab>(r);
  switch (linear_group(r.D, r.o->group)) {
    case 1: return launch_joint<LinearField<T, 1, 1>, T, 1, 1, Tab>(r);
    case 2: return launch_joint<LinearField<T, 1, 2>, T, 1, 2, Tab>(r);
    case 4: return r.D == 4 ? launch_joint<LinearField<T, 1, 4>, T, 1, 4, Tab>(r)
                            : launch_joint<LinearField<T, 4, 4>, T, 4, 4, Tab>(r);
    case 8: return r.D == 8 ? launch_joint<LinearField<T, 1, 8>, T, 1, 8, Tab>(r)
                            : launch_joint<LinearField<T, 2, 8>, T, 2, 8, Tab>(r);
    case 16: return r.D == 16 ? launch_joint<LinearField<T, 1, 16>, T, 1, 16, Tab>(r)
                              : launch_joint<LinearField<T, 2, 16>, T, 2, 16, Tab>(r);
    default: return TODE_EUNSUPPORTED;
  }
}

}  // namespace tode
