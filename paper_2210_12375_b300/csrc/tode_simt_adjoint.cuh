// tode_simt_adjoint.cuh -- discrete adjoint of the fixed-mesh map of the pair (dopri5 or tsit5) for
// the SIMT fields (torchode App. A: gradients by backpropagation through the
// solver, i.e. discretize-then-optimize).
//
// Per instance, in reverse over its accepted steps n with (t_n, h_n) frozen:
//   kbar_i = h b_i ybar_{n+1} + sum_{tau in (t_n, t_n+1]} h b_i(theta_tau) ybar_tau
//   for i = 7..1:  g_i = J_f(Y_i)^T kbar_i,  dtheta += (df/dtheta)^T kbar_i,
//                  kbar_j += h a_ij g_i  (j < i)
//   ybar_n = ybar_{n+1} + sum_tau ybar_tau + sum_i g_i.
// Step-start states come from the checkpoint tape: slot j holds the solver
// state (including its FSAL stage) at the start of accepted step j*stride.
// With one slot per accepted step and the accepted step sizes recorded, each
// step is reversed straight from its slot.  Otherwise the segment up to the
// next slot is re-run with the forward routine (a bit-identical mesh), its
// step-start states parked in scratch, then reversed.  Either way the first
// stage derivative is the forward's own FSAL value k1.
#pragma once
#include "tode_simt.cuh"

namespace tode {

// ---------------------------------------------------------------- adjoint fields
template <typename T> struct VdpAdj {
  static constexpr int R = 2, G = 1;
  VdpField<T> f;
  T gmu;
  __device__ __forceinline__ void load(const T* p, int i, T dir) {
    f.load(p, i, dir);
    gmu = T(0);
  }
  __device__ __forceinline__ void eval(double t, const T (&y)[2], T (&o)[2]) const {
    f.eval(t, y, o);
  }
  // gy = J^T v with J = [[0, 1], [-2 mu y1 y2 - 1, mu (1 - y1^2)]] the
  // Jacobian of f; the field evaluated is dir f, so v enters as dir v
  __device__ __forceinline__ void vjp(const T (&y)[2], const T (&vin)[2], T (&gy)[2]) {
    const T v[2] = {f.dir * vin[0], f.dir * vin[1]};
    const T mu = f.mu;
    const T one_m = madd(-y[0], y[0], T(1));  // 1 - y1^2
    gy[0] = v[1] * madd(T(-2) * mu * y[0], y[1], T(-1));
    gy[1] = madd(v[1], mu * one_m, v[0]);
    gmu = madd(v[1], one_m * y[1], gmu);
  }
  __device__ __forceinline__ void store_param(T* gp, int i, bool bad) const {
    gp[i] = bad ? nan_(T(0)) : gmu;
  }
};

template <typename T, int R_, int G_> struct LinearAdj {
  static constexpr int R = R_, G = G_, D = R_ * G_;
  // One column per lane (R = 1) stays in registers; wider lanes read their
  // columns through the L1 cache to keep the register count at two CTAs/SM.
  static constexpr bool REG_COLS = (R == 1);
  LinearField<T, R, G> f;   // holds dir A_i (the field evaluated)
  const T* acol;       // column g*R of A_i: A[j][g*R + r] = acol[j*D + r]
  T acr[REG_COLS ? D : 1];  // R = 1: the column itself
  T gA[R][D];          // columns g*R+r of dL/dA_i: gA[r][j] = dL/dA[j][g*R + r]
  T dir;
  __device__ __forceinline__ void load(const T* p, int i, T d) {
    f.load(p, i, d);
    dir = d;
    acol = p + (size_t)i * D * D + Grp<G>::rank() * R;
    if constexpr (REG_COLS) {
#pragma unroll
      for (int j = 0; j < D; ++j) acr[j] = acol[j * D];
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int j = 0; j < D; ++j) gA[r][j] = T(0);
  }
  __device__ __forceinline__ T a_col(int j, int r) const {
    if constexpr (REG_COLS) return acr[j];
    else return __ldg(acol + j * D + r);
  }
  __device__ __forceinline__ void eval(double t, const T (&y)[R], T (&o)[R]) const {
    f.eval(t, y, o);
  }
  // gy = A^T v,  dL/dA += v Y^T (v taken as dir v: the field is dir A y).
  // The lane owns columns of dL/dA, so both products need the gathered v
  // and only the lane's own components of Y.
  __device__ __forceinline__ void vjp(const T (&y)[R], const T (&vin)[R], T (&gy)[R]) {
    T v[R], vall[D];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = dir * vin[r];
    f.gather(v, vall);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if constexpr (sizeof(T) == 8 || D < 8) {
        T s = T(0);  // FP64: left-to-right (the oracle's order)
#pragma unroll
        for (int j = 0; j < D; ++j) s = madd(a_col(j, r), vall[j], s);
        gy[r] = s;
      } else {
        // partial sums over j = 0, 1, 2, 3 (mod 4) as two FP32x2 pairs of
        // adjacent rows (same bits as scalar fused multiply-adds)
        float2 p01 = make_float2(0.0f, 0.0f), p23 = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int j = 0; j < D; j += 4) {
          p01 = __ffma2_rn(make_float2(a_col(j, r), a_col(j + 1, r)),
                           make_float2(vall[j], vall[j + 1]), p01);
          p23 = __ffma2_rn(make_float2(a_col(j + 2, r), a_col(j + 3, r)),
                           make_float2(vall[j + 2], vall[j + 3]), p23);
        }
        gy[r] = (p01.x + p01.y) + (p23.x + p23.y);
      }
      if constexpr (sizeof(T) == 4 && D % 2 == 0) {
        const float2 yy = make_float2(y[r], y[r]);
#pragma unroll
        for (int j = 0; j < D; j += 2) {
          const float2 g2 = __ffma2_rn(make_float2(vall[j], vall[j + 1]), yy,
                                       make_float2(gA[r][j], gA[r][j + 1]));
          gA[r][j] = g2.x;
          gA[r][j + 1] = g2.y;
        }
      } else {
#pragma unroll
        for (int j = 0; j < D; ++j) gA[r][j] = madd(vall[j], y[r], gA[r][j]);
      }
    }
  }
  __device__ __forceinline__ void store_param(T* gp, int i, bool bad) const {
    const int g = Grp<G>::rank();
    T* dst = gp + (size_t)i * D * D + (size_t)g * R;
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
      for (int r = 0; r < R; ++r) dst[(size_t)j * D + r] = bad ? nan_(T(0)) : gA[r][j];
  }
};

template <typename T> struct AdjArgs {
  int B, D, K;
  const double* t0;
  const double* t1;
  const double* te;
  const double* rtol_b;
  const double* atol_b;
  double rtol, atol;
  const int32_t* n_acc;
  const int32_t* status;
  TapeDev<T> tape;
  SolveOpts o;
  const T* gye;
  const T* gyf;
  T* gy0;
  T* gparam;
  const T* fparam;
  int32_t* overflow;
  int32_t* counter;
  const int32_t* order;  // instances by decreasing step count (work queue order)
  T* sy;        // [stride][B][D]
  T* sk1;       // [stride][B][D]
  double* st;   // [stride][B]
  T* sh;        // [stride][B]
};

// Cursor over an instance's evaluation points, from the last backwards: the
// time of point q and of point q - 1 (-inf before the first) and the
// cotangent of point q, held in registers so that a step with no point of
// its own loads nothing, and a consumed point's successor is fetched while
// the step is reversed.
template <typename T, int R> struct AdjCursor {
  int q;
  double tq, tq2;   // in the direction of integration (-t backward in time)
  unsigned long long m;  // the instance's rev_mask
  T gq[R];
};

template <typename T>
__device__ __forceinline__ double adj_te(const AdjArgs<T>& a, int i, int q,
                                         unsigned long long m) {
  return q >= 0 ? flip(a.te[(size_t)i * a.K + q], m)
                : __longlong_as_double((long long)0xfff0000000000000ULL);
}

template <typename T, int R, int G>
__device__ __forceinline__ void adj_gq(const AdjArgs<T>& a, int i, int D, int q, T (&gq)[R]) {
  const int g = Grp<G>::rank();
#pragma unroll
  for (int r = 0; r < R; ++r)
    gq[r] = (a.gye && q >= 0) ? a.gye[((size_t)i * a.K + q) * D + g * R + r] : T(0);
}

template <typename T, int R, int G>
__device__ __forceinline__ void adj_cursor_start(AdjCursor<T, R>& c, const AdjArgs<T>& a, int i,
                                                 int D) {
  c.q = a.K - 1;
  c.m = reversed_at(a.t0, a.t1, i) ? SIGN_BIT : 0ULL;
  c.tq = adj_te(a, i, c.q, c.m);
  c.tq2 = adj_te(a, i, c.q - 1, c.m);
  adj_gq<T, R, G>(a, i, D, c.q, c.gq);
}

template <typename T, int R, int G>
__device__ __forceinline__ void adj_cursor_next(AdjCursor<T, R>& c, const AdjArgs<T>& a, int i,
                                                int D) {
  c.q--;
  c.tq = c.tq2;
  c.tq2 = adj_te(a, i, c.q - 1, c.m);
  adj_gq<T, R, G>(a, i, D, c.q, c.gq);
}

// One accepted step as the reverse sweep needs it: its start state y, the
// FSAL stage k1 (when the stage inputs are recomputed) or the recorded stage
// inputs Y_2..Y_7 (this lane's components), its start time and its size.
template <typename T, int R> struct AdjSlot {
  T y[R];
  T k1[R];
  T ys[6][R];
  double t;
  T h;
};

// Loads slot n of instance i from a stride-1 tape (YS: with stage inputs).
template <bool YS, typename T, int R, int G>
__device__ __forceinline__ void adj_load_slot(const AdjArgs<T>& a, int i, int D, int n,
                                              AdjSlot<T, R>& sl) {
  const int g = Grp<G>::rank();
  const size_t o = (size_t)i * a.tape.slots + n;
  ld_row<T, R>(a.tape.y + o * D + g * R, sl.y);
  if constexpr (YS) {
    const T* ys = a.tape.ystage + o * 6 * D + g * R;
#pragma unroll
    for (int q = 0; q < 6; ++q) ld_row<T, R>(ys + q * D, sl.ys[q]);
  } else {
    ld_row<T, R>(a.tape.k1 + o * D + g * R, sl.k1);
  }
  sl.t = a.tape.t[o];
  sl.h = a.tape.h_acc[o];
}

// Reverse one accepted step.  sl: the step (YS: with its recorded stage
// inputs), yb: running cotangent, c: cursor over the instance's evaluation
// points, from the last backwards.
template <class Tab, bool YS, class AF, typename T, int R, int G>
__device__ __forceinline__ void reverse_step(AF& F, const AdjArgs<T>& a, int i, int D,
                                             const AdjSlot<T, R>& sl, double t_next, T (&yb)[R],
                                             AdjCursor<T, R>& c) {
  const double t = sl.t;
  const T h = sl.h;
  const T (&y)[R] = sl.y;
  T Y[7][R];
#pragma unroll
  for (int r = 0; r < R; ++r) Y[0][r] = y[r];
  if constexpr (YS) {
    // the forward recorded this step's stage inputs Y_2..Y_7
#pragma unroll
    for (int q6 = 0; q6 < 6; ++q6)
#pragma unroll
      for (int r = 0; r < R; ++r) Y[q6 + 1][r] = sl.ys[q6][r];
  } else {
    // recompute them with the forward's own stage code (bit for bit), less
    // the evaluation at y_{n+1}
    Stages<T, R> K;
    T ysr[6][R], y1[R], inc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) K.k[0][r] = sl.k1[r];
    attempt_stages<Tab, AF, T, R, false>(F, t, h, y, K, ysr, y1, inc);
#pragma unroll
    for (int q6 = 0; q6 < 6; ++q6)
#pragma unroll
      for (int r = 0; r < R; ++r) Y[q6 + 1][r] = ysr[q6][r];
  }

  // cotangents of the stage derivatives
  T bw[7];
#pragma unroll
  for (int s = 0; s < 7; ++s) bw[s] = T(Tab::b(s + 1));
  T kb[7][R];
#pragma unroll
  for (int s = 0; s < 7; ++s)
#pragma unroll
    for (int r = 0; r < R; ++r) kb[s][r] = h * bw[s] * yb[r];
  bool dense7 = false;
  const long long kt = tkey(t), kn = tkey(t_next);
  while (true) {  // the points in (t, t_next]
    const double tq = c.tq;
    const long long kq = tkey(tq);
    if (!(kq > kt)) break;
    if (a.gye) {
      const T (&gq)[R] = c.gq;
      T w[7];
      if (kq == kn) {
#pragma unroll
        for (int s = 0; s < 7; ++s) w[s] = bw[s];
      } else {
        T th;
        if constexpr (Comp<T>::on) th = T(tq - t) / h;
        else th = T((tq - t) / (double)h);
        dense_weights<Tab, T>(th, w);
        dense7 = true;
      }
#pragma unroll
      for (int s = 0; s < 7; ++s)
#pragma unroll
        for (int r = 0; r < R; ++r) kb[s][r] = madd(h * w[s], gq[r], kb[s][r]);
#pragma unroll
      for (int r = 0; r < R; ++r) yb[r] = yb[r] + gq[r];
    }
    adj_cursor_next<T, R, G>(c, a, i, D);
  }
  // reverse stage sweep (b_7 = 0: kbar_7 = 0 without interior dense points)
#pragma unroll
  for (int s = 6; s >= 0; --s) {
    if (s == 6 && !dense7) continue;
    T gs[R];
    F.vjp(Y[s], kb[s], gs);
#pragma unroll
    for (int l = 0; l < s; ++l)
      if (Tab::a(s + 1, l + 1) != 0.0)
#pragma unroll
        for (int r = 0; r < R; ++r)
          kb[l][r] = madd(h * T(Tab::a(s + 1, l + 1)), gs[r], kb[l][r]);
#pragma unroll
    for (int r = 0; r < R; ++r) yb[r] = yb[r] + gs[r];
  }
}

// ---------------------------------------------------------------- work order
// The reverse sweeps are handed out longest first (by the forward's accepted
// step counts, StepsBin), so that the long instances do not start last and
// stretch the tail of the persistent grid.

// Instance at queue position j (B past the end of the queue).
template <typename T> __device__ __forceinline__ int queued(const AdjArgs<T>& a, int j) {
  return j < a.B ? a.order[j] : a.B;
}

// Cotangents of evaluation points sitting at t0 (they are y0 itself), then
// the instance's results: dL/dy0 and the field's parameter gradient.
template <class AF, typename T>
__device__ __forceinline__ void adjoint_finish(AF& F, const AdjArgs<T>& a, int i, int q, bool bad,
                                               T (&yb)[AF::R]) {
  constexpr int R = AF::R, G = AF::G;
  const int D = a.D;
  const int g = Grp<G>::rank();
  if (!bad && a.gye) {
    const long long k0 = tkey(a.t0[i]);
    for (; q >= 0; --q) {
      if (tkey(a.te[(size_t)i * a.K + q]) == k0) {
#pragma unroll
        for (int r = 0; r < R; ++r)
          yb[r] = yb[r] + a.gye[((size_t)i * a.K + q) * D + g * R + r];
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) a.gy0[(size_t)i * D + g * R + r] = bad ? nan_(T(0)) : yb[r];
  if (a.gparam) F.store_param(a.gparam, i, bad);
}

// Direct form (stride-1 tape with the accepted step sizes): one loop
// iteration reverses one step straight from its slot, and a group whose
// instance is done finishes it and steals the next at once, so the groups of
// a warp stay on the common step body whatever their step counts.
template <class Tab, class AF, typename T, bool YS>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_adjoint_steps(AdjArgs<T> a) {
  constexpr int R = AF::R, G = AF::G;
  const int D = a.D;
  const int groups_total = (int)((gridDim.x * (size_t)blockDim.x) / G);
  int i = queued(a, (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) / G));
  const int g = Grp<G>::rank();
  AF F;
  T yb[R];
  int n = -1;          // next step to reverse; < 0: the instance is done
  AdjCursor<T, R> c;   // evaluation-point cursor, from the last backwards
  c.q = -1;
  bool bad = false;
  bool have = false;
  double t_after = 0.0;  // end of step n: t1, or the start of step n+1 (its slot's t)
  AdjSlot<T, R> cur, nxt;  // step n, and step n - 1 in flight
  while (true) {
    if (n < 0) {
      if (have) {
        adjoint_finish<AF, T>(F, a, i, c.q, bad, yb);
        have = false;
        i = queued(a, grab_instance<G>(a.counter, groups_total));
      }
      if (i >= a.B) break;
      F.load(a.fparam, i, reversed_at(a.t0, a.t1, i) ? T(-1) : T(1));
      const int N = a.n_acc[i];
      bad = a.status[i] != ST_SUCCESS;
      if (!bad && N > a.tape.slots) {
        bad = true;
        if (g == 0) *a.overflow = 1;
      }
#pragma unroll
      for (int r = 0; r < R; ++r) yb[r] = a.gyf ? a.gyf[(size_t)i * D + g * R + r] : T(0);
      adj_cursor_start<T, R, G>(c, a, i, D);
      t_after = flip(a.t1[i], c.m);
      n = bad ? -1 : N - 1;
      have = true;
      if (n < 0) continue;
      adj_load_slot<YS, T, R, G>(a, i, D, n, cur);
    }
    // the next step's slot is fetched while this one is reversed
    if (n > 0) adj_load_slot<YS, T, R, G>(a, i, D, n - 1, nxt);
    const double t_next = t_after;  // the forward's t + h, bit for bit
    t_after = cur.t;
    reverse_step<Tab, YS, AF, T, R, G>(F, a, i, D, cur, t_next, yb, c);
    cur = nxt;
    --n;
  }
}

// Re-running form (strided tape, or no recorded step sizes): each segment
// between slots is re-run with the forward routine from its slot, its
// step-start states parked in scratch, then reversed.
template <class Tab, class AF, typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_adjoint(AdjArgs<T> a) {
  constexpr int R = AF::R, G = AF::G;
  const int D = a.D;
  const int groups_total = (int)((gridDim.x * (size_t)blockDim.x) / G);
  int i = queued(a, (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) / G));
  const int g = Grp<G>::rank();
  SolveOpts ro = a.o;
  ro.max_steps = 0x7fffffff;  // the re-run never stops on a step count
  TraceDev no_trace{};
  no_trace.cap = 0;
  InstOut<T> no_out{};
  no_out.K = 0;
  while (i < a.B) {
    AF F;
    F.load(a.fparam, i, reversed_at(a.t0, a.t1, i) ? T(-1) : T(1));
    const int N = a.n_acc[i];
    const int m = a.tape.stride;
    const int nseg = (N + m - 1) / m;
    bool bad = a.status[i] != ST_SUCCESS;
    if (!bad && nseg > a.tape.slots) {
      bad = true;
      if (g == 0) *a.overflow = 1;
    }
    T yb[R];
#pragma unroll
    for (int r = 0; r < R; ++r) yb[r] = a.gyf ? a.gyf[(size_t)i * D + g * R + r] : T(0);
    AdjCursor<T, R> c;
    adj_cursor_start<T, R, G>(c, a, i, D);
    const double t1 = flip(a.t1[i], c.m);  // in the direction of integration
    for (int j = nseg - 1; j >= 0 && !bad; --j) {
      const int n0 = j * m;
      const int n1 = (n0 + m < N) ? n0 + m : N;
      // restore the slot and re-run the forward over the segment
      Inst<T, R> s;
      const size_t o = (size_t)i * a.tape.slots + j;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        s.y[r] = a.tape.y[o * D + g * R + r];
        s.ylo[r] = Comp<T>::on ? a.tape.ylo[o * D + g * R + r] : T(0);
        s.k1[r] = a.tape.k1[o * D + g * R + r];
      }
      s.t = a.tape.t[o];
      s.h = a.tape.h[o];
      s.err_prev = a.tape.err_prev[o];
      s.err_prev2 = a.tape.err_prev2 ? a.tape.err_prev2[o] : T(1);  // present when beta3 != 0
      s.flags = a.tape.flags[o];
      s.t0 = flip(a.t0[i], c.m);
      s.t1 = t1;
      s.rtol = T(a.rtol_b ? a.rtol_b[i] : a.rtol);
      s.atol = T(a.atol_b ? a.atol_b[i] : a.atol);
      s.n_acc = n0;
      s.n_rej = 0;
      s.cursor = 0;
      s.tq = s.tq2 = te_at(no_out, 0, 0ULL);  // no evaluation points in a re-run
      s.status = ST_RUNNING;
      if constexpr (Comp<T>::on) {  // functions of (t, t0, t1), as in the forward
        s.rem = __double2float_rd(s.t1 - s.t);
        s.hmin = T(1e-14 * tmax(fabs(s.t0), fabs(s.t1)));
      }
      while (s.n_acc < n1 && s.status == ST_RUNNING) {
        const int before = s.n_acc;
        const double tb = s.t;
        T ys[R], ks[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          ys[r] = s.y[r];
          ks[r] = s.k1[r];
        }
        T ysd[6][R];
        inst_attempt<Tab, AF, T, R, G>(F, s, ro, i, D, no_out, no_trace, ysd);
        const T hb = s.h_last;
        if (s.n_acc != before) {
          const size_t p = (size_t)(before - n0) * a.B + i;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            a.sy[p * D + g * R + r] = ys[r];
            a.sk1[p * D + g * R + r] = ks[r];
          }
          if (g == 0) {
            a.st[p] = tb;
            a.sh[p] = hb;
          }
        }
      }
      if (s.n_acc < n1) {  // the re-run left the forward's mesh: cannot happen
        bad = true;
        break;
      }
      if constexpr (G > 1) __syncwarp(Grp<G>::mask());
      for (int n = n1 - 1; n >= n0; --n) {
        const size_t p = (size_t)(n - n0) * a.B + i;
        AdjSlot<T, R> sl;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          sl.y[r] = a.sy[p * D + g * R + r];
          sl.k1[r] = a.sk1[p * D + g * R + r];
        }
        sl.t = a.st[p];
        sl.h = a.sh[p];
        const double t_next = (n == N - 1) ? t1 : sl.t + (double)sl.h;
        reverse_step<Tab, false, AF, T, R, G>(F, a, i, D, sl, t_next, yb, c);
      }
      if constexpr (G > 1) __syncwarp(Grp<G>::mask());
    }
    adjoint_finish<AF, T>(F, a, i, c.q, bad, yb);
    i = queued(a, grab_instance<G>(a.counter, groups_total));
  }
}

template <class Tab, class AF, typename T> tode_err launch_adjoint(const AdjReq& r) {
  const bool direct = r.tape->stride == 1 && r.tape->h_acc != nullptr;
  AdjArgs<T> a{};
  a.B = r.B;
  a.D = r.D;
  a.K = r.K;
  a.t0 = r.t0;
  a.t1 = r.t1;
  a.te = r.te;
  a.rtol_b = r.o->rtol_b;
  a.atol_b = r.o->atol_b;
  a.rtol = r.o->rtol;
  a.atol = r.o->atol;
  a.n_acc = r.n_acc;
  a.status = r.status;
  a.tape = make_tape<T>(r.tape, r.B, r.D);
  a.o = make_opts(r.o);
  a.gye = (const T*)r.gye;
  a.gyf = (const T*)r.gyf;
  a.gy0 = (T*)r.gy0;
  a.gparam = (T*)r.gparam;
  a.fparam = (const T*)(r.f->kind == TODE_VDP ? r.f->mu : r.f->A);
  a.overflow = r.overflow;
  char* p = r.scratch;
  a.counter = (int32_t*)p;
  p += align256(256);
  int32_t* order = (int32_t*)p;
  a.order = order;
  p += align256((size_t)r.B * 4);
  int* order_part = (int*)p;
  p += order_part_bytes(r.B);
  const int m = r.tape->stride;
  a.sy = (T*)p;
  p += align256((size_t)m * r.B * r.D * sizeof(T));
  a.sk1 = (T*)p;
  p += align256((size_t)m * r.B * r.D * sizeof(T));
  a.st = (double*)p;
  p += align256((size_t)m * r.B * 8);
  a.sh = (T*)p;
  const long long threads = (long long)r.B * AF::G;
  const int block = r.o->block > 0 ? r.o->block : default_block(threads, r.num_sms);
  if (block % 32 != 0 || block > 256) return TODE_EINVAL;
  auto kern = !direct ? k_adjoint<Tab, AF, T>
              : r.tape->y_stage ? k_adjoint_steps<Tab, AF, T, true>
                                : k_adjoint_steps<Tab, AF, T, false>;
  int per_sm = 0;
  TODE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, 0));
  if (per_sm < 1) per_sm = 1;
  long long grid = (long long)r.num_sms * per_sm;
  const long long need = (threads + block - 1) / block;
  if (grid > need) grid = need;
  if (grid == 0) return TODE_OK;
  TODE_CUDA_TRY(cudaMemsetAsync(a.counter, 0, sizeof(int32_t), r.stream));
  TODE_CUDA_TRY(launch_order(r.B, StepsBin{r.n_acc, r.status}, order, order_part, r.stream));
  kern<<<(int)grid, block, 0, r.stream>>>(a);
  TODE_CUDA_TRY(cudaGetLastError());
  return TODE_OK;
}

// A strided tape makes the adjoint re-run the forward's attempts, so it must
// use the forward's lane grouping (linear_group): the FP32 error norm's
// butterfly order, and with it the recomputed mesh, depends on the group
// size.  A stride-1 tape with the accepted step sizes is reversed directly,
// and reversing a step gives the same bits for every grouping (each lane
// holds whole rows and columns), so D = 16 then takes 16 lanes with A's
// column in registers (measured fastest for the adjoint).
template <class Tab, typename T> tode_err simt_adjoint(const AdjReq& r) {
  if (r.f->kind == TODE_VDP) return launch_adjoint<Tab, VdpAdj<T>, T>(r);
  const bool direct = r.tape->stride == 1 && r.tape->h_acc != nullptr;
  if (direct && r.D == 16) return launch_adjoint<Tab, LinearAdj<T, 1, 16>, T>(r);
  switch (linear_group(r.D, r.o->group)) {
    case 1: return launch_adjoint<Tab, LinearAdj<T, 1, 1>, T>(r);
    case 2: return launch_adjoint<Tab, LinearAdj<T, 1, 2>, T>(r);
    case 4: return r.D == 4 ? launch_adjoint<Tab, LinearAdj<T, 1, 4>, T>(r)
                            : launch_adjoint<Tab, LinearAdj<T, 4, 4>, T>(r);
    case 8: return r.D == 8 ? launch_adjoint<Tab, LinearAdj<T, 1, 8>, T>(r)
                            : launch_adjoint<Tab, LinearAdj<T, 2, 8>, T>(r);
    case 16: return r.D == 16 ? launch_adjoint<Tab, LinearAdj<T, 1, 16>, T>(r)
                              : launch_adjoint<Tab, LinearAdj<T, 2, 16>, T>(r);
    default: return TODE_EUNSUPPORTED;
  }
}

// ---------------------------------------------------------------- t0, t1
// Gradients with respect to the integration bounds of the frozen map (every
// accepted step size but the last and every evaluation point's step held;
// t0 moves every mesh point before t1, the last step h = t1 - t_{N-1}
// absorbs the change).  For these autonomous fields the bounds enter only
// through the dense-output abscissae and the last step size, so
//   dL/dt1 = hbar = dL/dh of the last step (y_{N-1} held), and
//   dL/dt0 = -sum_tau <ybar_tau, dy/dt(tau)> - dL/dt1
// (translating t0 and t1 together shifts every output by -dy/dt).  The last
// step's hbar: with its stages Y_i, k_i and the reverse sweep's g_i,
//   hbar = <ybar_N, sum_i b_i k_i>
//        + sum_tau <ybar_tau, sum_i (b_i(theta) - theta b_i'(theta)) k_i>
//        + sum_i <g_i, sum_j a_ij k_j>.
// Backward instances run in tau = -t: hbar is dL/dtau1 there, and
// dL/dt1 = -hbar.  One lane group per instance; the last step comes from a
// stride-1 tape with the accepted step sizes.
template <typename T> struct TBoundsArgs {
  AdjArgs<T> a;
  const T* yp;   // [B][K][D] dy/dt at the points (the forward's yp_eval), or NULL
  double* gt0;   // [B] or NULL
  double* gt1;   // [B]
};

template <int G> __device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(Grp<G>::mask(), v, o, G);
  return v;
}

template <class Tab, class AF, typename T, bool YS>
__global__ void __launch_bounds__(128) k_t_bounds(TBoundsArgs<T> ta) {
  constexpr int R = AF::R, G = AF::G;
  const AdjArgs<T>& a = ta.a;
  const int D = a.D;
  const int g = Grp<G>::rank();
  const long long groups = (long long)gridDim.x * blockDim.x / G;
  for (long long gi = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G; gi < a.B;
       gi += groups) {
    const int i = (int)gi;
    const int N = a.n_acc[i];
    const bool bad = a.status[i] != ST_SUCCESS || N > a.tape.slots;
    const bool rev = reversed_at(a.t0, a.t1, i);
    // -sum_tau <ybar_tau, dy/dt(tau)> over every point (the forward's dy/dt)
    double tsum = 0.0;
    if (ta.gt0 && a.gye && ta.yp) {
      for (int q = 0; q < a.K; ++q)
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const size_t o = ((size_t)i * a.K + q) * D + g * R + r;
          tsum += (double)a.gye[o] * (double)ta.yp[o];
        }
      tsum = group_sum<G>(tsum);
    }
    double hbar = 0.0;
    if (!bad && N > 0) {
      AF F;
      F.load(a.fparam, i, rev ? T(-1) : T(1));
      AdjSlot<T, R> sl;
      adj_load_slot<YS, T, R, G>(a, i, D, N - 1, sl);
      const double t = sl.t;
      const T h = sl.h;
      const double hd = (double)h;
      // the stage inputs (recorded, or recomputed from y and k1) and k_i = f(Y_i)
      T Y[7][R];
      Stages<T, R> KS;
      T (&k)[7][R] = KS.k;
#pragma unroll
      for (int r = 0; r < R; ++r) Y[0][r] = sl.y[r];
      if constexpr (YS) {
#pragma unroll
        for (int q6 = 0; q6 < 6; ++q6)
#pragma unroll
          for (int r = 0; r < R; ++r) Y[q6 + 1][r] = sl.ys[q6][r];
      }
      T A[7][6], bw[7];
      double cs[7];
#pragma unroll
      for (int s = 0; s < 7; ++s) {
        cs[s] = Tab::c(s + 1);
        bw[s] = T(Tab::b(s + 1));
#pragma unroll
        for (int l = 0; l < 6; ++l) A[s][l] = T(Tab::a(s + 1, l + 1));
      }
#pragma unroll
      for (int s = 0; s < 7; ++s) {
        if constexpr (!YS) {
          if (s > 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
              T acc = T(0);
#pragma unroll
              for (int l = 0; l < s; ++l) acc = madd(A[s][l], k[l][r], acc);
              Y[s][r] = madd(h, acc, sl.y[r]);
            }
          }
        }
        F.eval(t + cs[s] * hd, Y[s], k[s]);
      }
      T yb[R], kb[7][R];
#pragma unroll
      for (int r = 0; r < R; ++r) yb[r] = a.gyf ? a.gyf[(size_t)i * D + g * R + r] : T(0);
      double part = 0.0;  // this lane's share of hbar
#pragma unroll
      for (int r = 0; r < R; ++r) {
        T sb = T(0);
#pragma unroll
        for (int s = 0; s < 7; ++s) sb = madd(bw[s], k[s][r], sb);
        part += (double)yb[r] * (double)sb;
      }
#pragma unroll
      for (int s = 0; s < 7; ++s)
#pragma unroll
        for (int r = 0; r < R; ++r) kb[s][r] = h * bw[s] * yb[r];
      // the points in the last step, from the last backwards
      AdjCursor<T, R> c;
      adj_cursor_start<T, R, G>(c, a, i, D);
      const long long kt = tkey(t), kn = tkey(flip(a.t1[i], c.m));
      while (true) {
        const double tq = c.tq;
        const long long kq = tkey(tq);
        if (!(kq > kt)) break;
        if (a.gye) {
          T w[7], dv[R];
          T th;
          if (kq == kn) {
            th = T(1);
#pragma unroll
            for (int s = 0; s < 7; ++s) w[s] = bw[s];
          } else {
            if constexpr (Comp<T>::on) th = T(tq - t) / h;
            else th = T((tq - t) / hd);
            dense_weights<Tab, T>(th, w);
          }
          dense_deriv<Tab, T, R>(th, T(1), KS, dv);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            T sw = T(0);
#pragma unroll
            for (int s = 0; s < 7; ++s) sw = madd(w[s], k[s][r], sw);
            part += (double)c.gq[r] * ((double)sw - (double)th * (double)dv[r]);
          }
#pragma unroll
          for (int s = 0; s < 7; ++s)
#pragma unroll
            for (int r = 0; r < R; ++r) kb[s][r] = madd(h * w[s], c.gq[r], kb[s][r]);
        }
        adj_cursor_next<T, R, G>(c, a, i, D);
      }
      // reverse stage sweep: g_i, and <g_i, sum_j a_ij k_j>
#pragma unroll
      for (int s = 6; s >= 1; --s) {
        T gs[R];
        F.vjp(Y[s], kb[s], gs);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          T sa = T(0);
#pragma unroll
          for (int l = 0; l < s; ++l) sa = madd(A[s][l], k[l][r], sa);
          part += (double)gs[r] * (double)sa;
        }
#pragma unroll
        for (int l = 0; l < s; ++l)
#pragma unroll
          for (int r = 0; r < R; ++r) kb[l][r] = madd(h * A[s][l], gs[r], kb[l][r]);
      }
      hbar = group_sum<G>(part);
    }
    if (g == 0) {
      const double nan = __longlong_as_double(0x7ff8000000000000LL);
      const double g1 = bad ? nan : (N > 0 ? (rev ? -hbar : hbar) : 0.0);
      ta.gt1[i] = g1;
      if (ta.gt0) ta.gt0[i] = bad ? nan : -tsum - g1;
    }
  }
}

template <class Tab, class AF, typename T>
tode_err launch_t_bounds(const AdjReq& r, const void* yp,
                                                         double* gt0, double* gt1) {
  TBoundsArgs<T> ta{};
  AdjArgs<T>& a = ta.a;
  a.B = r.B;
  a.D = r.D;
  a.K = r.K;
  a.t0 = r.t0;
  a.t1 = r.t1;
  a.te = r.te;
  a.n_acc = r.n_acc;
  a.status = r.status;
  a.tape = make_tape<T>(r.tape, r.B, r.D);
  a.gye = (const T*)r.gye;
  a.gyf = (const T*)r.gyf;
  a.fparam = (const T*)(r.f->kind == TODE_VDP ? r.f->mu : r.f->A);
  ta.yp = (const T*)yp;
  ta.gt0 = gt0;
  ta.gt1 = gt1;
  const long long threads = (long long)r.B * AF::G;
  long long grid = (threads + 127) / 128;
  if (grid > (long long)r.num_sms * 16) grid = (long long)r.num_sms * 16;
  if (grid == 0) return TODE_OK;
  if (r.tape->y_stage) k_t_bounds<Tab, AF, T, true><<<(int)grid, 128, 0, r.stream>>>(ta);
  else k_t_bounds<Tab, AF, T, false><<<(int)grid, 128, 0, r.stream>>>(ta);
  TODE_CUDA_TRY(cudaGetLastError());
  return TODE_OK;
}

template <class Tab, typename T>
tode_err simt_t_bounds(const AdjReq& r, const void* yp, double* gt0,
                                            double* gt1) {
  if (r.f->kind == TODE_VDP) return launch_t_bounds<Tab, VdpAdj<T>, T>(r, yp, gt0, gt1);
  switch (r.D) {  // one column of A per lane, as the direct adjoint takes it
    case 1: return launch_t_bounds<Tab, LinearAdj<T, 1, 1>, T>(r, yp, gt0, gt1);
    case 2: return launch_t_bounds<Tab, LinearAdj<T, 1, 2>, T>(r, yp, gt0, gt1);
    case 4: return launch_t_bounds<Tab, LinearAdj<T, 1, 4>, T>(r, yp, gt0, gt1);
    case 8: return launch_t_bounds<Tab, LinearAdj<T, 1, 8>, T>(r, yp, gt0, gt1);
    case 16: return launch_t_bounds<Tab, LinearAdj<T, 1, 16>, T>(r, yp, gt0, gt1);
    case 32: return launch_t_bounds<Tab, LinearAdj<T, 2, 16>, T>(r, yp, gt0, gt1);
    default: return TODE_EUNSUPPORTED;
  }
}

}  // namespace tode
