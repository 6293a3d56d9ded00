// tode_core.cuh -- device-side Dormand-Prince 5(4) step routine shared by the
// plain (one launch per step) and fused (persistent, work-stealing) forms.
//
// One instance is owned by a group of G adjacent lanes; lane g of the group
// holds components g*R .. g*R+R-1 of the state (D = G*R).  Every decision
// (accept/reject, step size, dense-output cursor) is computed identically on
// all lanes of the group, so the group's control flow is uniform and the
// plain and fused forms run bit-identical arithmetic.
//
// Method (torchode): independent per-instance state (Sec. 3), dopri5 with
// FSAL/SSAL and Horner dense output (Sec. 3, App. A), PI controller of
// Soderlind's family (Sec. 3, App. C), per-instance status (App. B).
// Tableau: Dormand & Prince 1980; dense output: the continuous extension of
// Hairer-Norsett-Wanner Sec. II.6 expanded into quartic weights b_i(theta);
// starting step: HNW Sec. II.4.
//
// FP64 instantiations are compiled with -fmad=false and evaluate every sum
// left to right, so their accept/reject sequences are reproducible bit for bit
// by any IEEE-754 implementation that follows the same order.
#pragma once
#include "tode_internal.h"
#include <cuda_runtime.h>
#include <stdint.h>

namespace tode {

// ---------------------------------------------------------------- tableau
struct DP5 {
  static constexpr double c2 = 1.0 / 5.0, c3 = 3.0 / 10.0, c4 = 4.0 / 5.0, c5 = 8.0 / 9.0;
  static constexpr double a21 = 1.0 / 5.0;
  static constexpr double a31 = 3.0 / 40.0, a32 = 9.0 / 40.0;
  static constexpr double a41 = 44.0 / 45.0, a42 = -56.0 / 15.0, a43 = 32.0 / 9.0;
  static constexpr double a51 = 19372.0 / 6561.0, a52 = -25360.0 / 2187.0,
                          a53 = 64448.0 / 6561.0, a54 = -212.0 / 729.0;
  static constexpr double a61 = 9017.0 / 3168.0, a62 = -355.0 / 33.0, a63 = 46732.0 / 5247.0,
                          a64 = 49.0 / 176.0, a65 = -5103.0 / 18656.0;
  // 5th-order weights = last stage row (FSAL/SSAL)
  static constexpr double b1 = 35.0 / 384.0, b3 = 500.0 / 1113.0, b4 = 125.0 / 192.0,
                          b5 = -2187.0 / 6784.0, b6 = 11.0 / 84.0;
  // embedded 4th-order weights
  static constexpr double bh1 = 5179.0 / 57600.0, bh3 = 7571.0 / 16695.0, bh4 = 393.0 / 640.0,
                          bh5 = -92097.0 / 339200.0, bh6 = 187.0 / 2100.0, bh7 = 1.0 / 40.0;
  // error weights, formed in double arithmetic from the two weight rows
  static constexpr double e1 = b1 - bh1, e3 = b3 - bh3, e4 = b4 - bh4, e5 = b5 - bh5,
                          e6 = b6 - bh6, e7 = 0.0 - bh7;
  // dense output b_i(theta) = theta*(q_i0 + theta*(q_i1 + theta*(q_i2 + theta*q_i3)))
  static constexpr double q10 = 1.0, q11 = -8048581381.0 / 2820520608.0,
                          q12 = 8663915743.0 / 2820520608.0,
                          q13 = -12715105075.0 / 11282082432.0;
  static constexpr double q31 = 131558114200.0 / 32700410799.0,
                          q32 = -68118460800.0 / 10900136933.0,
                          q33 = 87487479700.0 / 32700410799.0;
  static constexpr double q41 = -1754552775.0 / 470086768.0,
                          q42 = 14199869525.0 / 1410260304.0,
                          q43 = -10690763975.0 / 1880347072.0;
  static constexpr double q51 = 127303824393.0 / 49829197408.0,
                          q52 = -318862633887.0 / 49829197408.0,
                          q53 = 701980252875.0 / 199316789632.0;
  static constexpr double q61 = -282668133.0 / 205662961.0, q62 = 2019193451.0 / 616988883.0,
                          q63 = -1453857185.0 / 822651844.0;
  static constexpr double q71 = 40617522.0 / 29380423.0, q72 = -110615467.0 / 29380423.0,
                          q73 = 69997945.0 / 29380423.0;

  // The interface both pairs share (1-based indices as in the tableau; zero
  // entries fold away in unrolled loops): c_i, a_ij (stage rows 2..7, row 7
  // = b by FSAL), e_i = b_i - bhat_i, and the dense-output coefficients q_im
  // with b_i(theta) = theta*(q_i0 + theta*(q_i1 + theta*(q_i2 + theta*q_i3))).
  __host__ __device__ static constexpr double c(int i) {
    return i == 2 ? c2 : i == 3 ? c3 : i == 4 ? c4 : i == 5 ? c5 : i >= 6 ? 1.0 : 0.0;
  }
  __host__ __device__ static constexpr double a(int i, int j) {
    switch (i * 8 + j) {
      case 17: return a21;
      case 25: return a31; case 26: return a32;
      case 33: return a41; case 34: return a42; case 35: return a43;
      case 41: return a51; case 42: return a52; case 43: return a53; case 44: return a54;
      case 49: return a61; case 50: return a62; case 51: return a63; case 52: return a64;
      case 53: return a65;
      case 57: return b1; case 59: return b3; case 60: return b4; case 61: return b5;
      case 62: return b6;
      default: return 0.0;
    }
  }
  __host__ __device__ static constexpr double b(int i) { return a(7, i); }
  __host__ __device__ static constexpr double e(int i) {
    return i == 1 ? e1 : i == 3 ? e3 : i == 4 ? e4 : i == 5 ? e5 : i == 6 ? e6 : i == 7 ? e7
                                                                                        : 0.0;
  }
  __host__ __device__ static constexpr double q(int i, int m) {
    switch (i * 4 + m) {
      case 4: return q10; case 5: return q11; case 6: return q12; case 7: return q13;
      case 13: return q31; case 14: return q32; case 15: return q33;
      case 17: return q41; case 18: return q42; case 19: return q43;
      case 21: return q51; case 22: return q52; case 23: return q53;
      case 25: return q61; case 26: return q62; case 27: return q63;
      case 29: return q71; case 30: return q72; case 31: return q73;
      default: return 0.0;
    }
  }
};

// Tsitouras 5(4) pair (tsit5; the torchode paper names it in App. A as
// available beside dopri5): Ch. Tsitouras, Comput. Math. Appl. 62 (2011),
// the table and its continuous extension of order 4, decimals as published.
// FSAL: the 7th stage row is the 5th-order weight row and c7 = 1, b7 = 0.
struct TS5 {
  __host__ __device__ static constexpr double c(int i) {
    return i == 2 ? 0.161 : i == 3 ? 0.327 : i == 4 ? 0.9 : i == 5 ? 0.9800255409045097
                                                                   : i >= 6 ? 1.0 : 0.0;
  }
  __host__ __device__ static constexpr double a(int i, int j) {
    switch (i * 8 + j) {
      case 17: return 0.161;
      case 25: return -0.008480655492356989; case 26: return 0.335480655492357;
      case 33: return 2.897153057105493; case 34: return -6.359448489975075;
      case 35: return 4.3622954328695815;
      case 41: return 5.325864828439257; case 42: return -11.748883564062828;
      case 43: return 7.4955393428898365; case 44: return -0.09249506636175525;
      case 49: return 5.86145544294642; case 50: return -12.92096931784711;
      case 51: return 8.159367898576159; case 52: return -0.071584973281401;
      case 53: return -0.028269050394068383;
      case 57: return 0.09646076681806523; case 58: return 0.01;
      case 59: return 0.4798896504144996; case 60: return 1.379008574103742;
      case 61: return -3.290069515436081; case 62: return 2.324710524099774;
      default: return 0.0;
    }
  }
  __host__ __device__ static constexpr double b(int i) { return a(7, i); }
  __host__ __device__ static constexpr double e(int i) {
    switch (i) {
      case 1: return -0.00178001105222577714;
      case 2: return -0.0008164344596567469;
      case 3: return 0.007880878010261995;
      case 4: return -0.1447110071732629;
      case 5: return 0.5823571654525552;
      case 6: return -0.45808210592918697;
      case 7: return 0.015151515151515152;
      default: return 0.0;
    }
  }
  // The continuous extension as published, in factored form:
  //   b_1 = k1 theta (theta - r1) (theta^2 + p1 theta + s1),
  //   b_2, b_3 = k theta^2 (theta^2 + p theta + s),
  //   b_4..b_7 = k theta^2 (theta - u) (theta - v),
  // multiplied out here into the Horner coefficients q_i0..q_i3.
  static constexpr double k1 = -1.0530884977290216, r1 = 1.3299890189751412,
                          p1 = -1.4364028541716351, s1 = 0.7139816917074209;
  __host__ __device__ static constexpr double kq(int i) {
    return i == 2 ? 0.1017 : i == 3 ? 2.490627285651252793 : i == 4 ? -16.54810288924490272
         : i == 5 ? 47.37952196281928122 : i == 6 ? -34.87065786149660974 : 2.5;
  }
  // b_2, b_3: theta^2 + p theta + s;  b_4..b_7: roots u, v
  __host__ __device__ static constexpr double pq(int i) {
    return i == 2 ? -2.1966568338249754 : i == 3 ? -2.38535645472061657
         : i == 4 ? -(1.21712927295533244 + 0.61620406037800089)
         : i == 5 ? -(1.203071208372362603 + 0.658047292653547382)
         : i == 6 ? -(1.2 + 0.666666666666666667) : -(1.0 + 0.6);
  }
  __host__ __device__ static constexpr double sq(int i) {
    return i == 2 ? 1.2949852507374631 : i == 3 ? 1.57803468208092486
         : i == 4 ? 1.21712927295533244 * 0.61620406037800089
         : i == 5 ? 1.203071208372362603 * 0.658047292653547382
         : i == 6 ? 1.2 * 0.666666666666666667 : 1.0 * 0.6;
  }
  __host__ __device__ static constexpr double q(int i, int m) {
    if (i == 1) {
      // k1 theta (theta^3 + (p1 - r1) theta^2 + (s1 - r1 p1) theta - r1 s1)
      return m == 0 ? -(k1 * r1 * s1) : m == 1 ? k1 * (s1 - r1 * p1) : m == 2 ? k1 * (p1 - r1)
                                                                              : k1;
    }
    if (i < 2 || i > 7) return 0.0;
    // k theta^2 (theta^2 + p theta + s) = theta (0 + theta (k s + theta (k p + theta k)))
    return m == 0 ? 0.0 : m == 1 ? kq(i) * sq(i) : m == 2 ? kq(i) * pq(i) : kq(i);
  }
};

enum : int { ST_SUCCESS = 0, ST_MAX_STEPS = 1, ST_DT_UNDERFLOW = 2, ST_NONFINITE = 3,
             ST_INVALID = 4, ST_RUNNING = -1 };
enum : int { FL_PREV_REJ = 1, FL_REVERSE = 2 };

// Integration backward in time (t1 < t0) runs in tau = -t: every time the
// solver holds (t, t0, t1, the evaluation points, the tape's t) is -t and
// every step size stays positive, while the fields return -f (and their
// transposed products take -v).  IEEE rounding is symmetric under negation,
// so this is bit for bit the method with negative steps.  The sign is one
// bit (FL_REVERSE in the instance's flags) applied by xor, off the FP64 pipe.
constexpr unsigned long long SIGN_BIT = 0x8000000000000000ULL;
__device__ __forceinline__ unsigned long long rev_mask(int flags) {
  return (flags & FL_REVERSE) ? SIGN_BIT : 0ULL;
}
__device__ __forceinline__ double flip(double x, unsigned long long m) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)m);
}
// The direction of instance i from its raw t0, t1 (NaN: forward, and invalid).
__device__ __forceinline__ bool reversed_at(const double* t0, const double* t1, int i) {
  return t1[i] < t0[i];
}

// ---------------------------------------------------------------- scalar helpers
// a*b + c.  Both translation units are built with -fmad=false, so nothing is
// contracted behind the source's back: FP32 multiply-adds are written as
// explicit fused operations (identical in every kernel that inlines this
// routine), FP64 keeps a separate multiply and add (the oracle's arithmetic).
__device__ __forceinline__ float madd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double madd(double a, double b, double c) { return a * b + c; }

template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return (a > b) ? a : b; }
template <typename T> __device__ __forceinline__ T tmin(T a, T b) { return (b < a) ? b : a; }
__device__ __forceinline__ bool finite_(double x) { return isfinite(x); }
__device__ __forceinline__ bool finite_(float x) { return isfinite(x); }
__device__ __forceinline__ double nan_(double) { return __longlong_as_double(0x7ff8000000000000LL); }
__device__ __forceinline__ float nan_(float) { return __int_as_float(0x7fc00000); }

// Times are compared through order-preserving integer keys of their FP64
// bit patterns (integer ALU instead of the narrow FP64 pipe): for finite x, y
// key(x) < key(y) iff x < y and key(x) == key(y) iff x == y (-0 maps to +0).
__device__ __forceinline__ long long tkey(double x) {
  long long b = __double_as_longlong(x);
  if (b == (long long)0x8000000000000000ULL) b = 0;
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool tfinite(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

// FP64 x^y of the controller and the starting step: exp(y ln x) through one
// fixed sequence of IEEE-754 double operations, so that the FP64 path's step
// sizes are reproducible bit for bit on any IEEE machine running the same
// sequence (a platform pow may differ by an ulp, and the embedded error
// estimate amplifies such a difference about 1e4-fold through cancellation).
//   ln x : x = 2^e m, m in [sqrt(1/2), sqrt(2)), s = (m-1)/(m+1),
//          ln m = 2 s (1 + s^2/3 + ... + s^22/23)   (Horner in s^2),
//          ln x = e ln2_hi + (e ln2_lo + ln m)       (ln 2 split after 32 bits)
//   exp z: k = floor(z/ln2 + 1/2), r = (z - k ln2_hi) - k ln2_lo,
//          exp r = sum_{j<=14} r^j/j! (Horner), scaled by 2^k exactly.
// Only the -fmad=false translation unit for FP64 calls it.
__device__ __forceinline__ double spec_ln(double x) {
  const double ln2_hi = 0x1.62e42fee00000p-1, ln2_lo = 0x1.a39ef35793c76p-33;
  long long u = __double_as_longlong(x);
  int e = (int)((u >> 52) & 0x7ff);
  if (e == 0) {
    x = x * 18014398509481984.0;  // 2^54
    u = __double_as_longlong(x);
    e = (int)((u >> 52) & 0x7ff) - 54;
  }
  e -= 1023;
  double m = __longlong_as_double((u & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
  if (m > 0x1.6a09e667f3bcdp+0) {
    m = m * 0.5;
    e = e + 1;
  }
  const double s = (m - 1.0) / (m + 1.0);
  const double w = s * s;
  double p = 1.0 / 23.0;
  p = 1.0 / 21.0 + w * p;
  p = 1.0 / 19.0 + w * p;
  p = 1.0 / 17.0 + w * p;
  p = 1.0 / 15.0 + w * p;
  p = 1.0 / 13.0 + w * p;
  p = 1.0 / 11.0 + w * p;
  p = 1.0 / 9.0 + w * p;
  p = 1.0 / 7.0 + w * p;
  p = 1.0 / 5.0 + w * p;
  p = 1.0 / 3.0 + w * p;
  p = 1.0 + w * p;
  const double lnm = 2.0 * (s * p);
  const double de = (double)e;
  return de * ln2_hi + (de * ln2_lo + lnm);
}
__device__ __forceinline__ double spec_exp(double z) {
  const double ln2_hi = 0x1.62e42fee00000p-1, ln2_lo = 0x1.a39ef35793c76p-33;
  if (z > 700.0) return __longlong_as_double(0x7ff0000000000000LL);
  if (z < -700.0) return 0.0;
  const double k = floor(z * 0x1.71547652b82fep+0 + 0.5);
  const double r = (z - k * ln2_hi) - k * ln2_lo;
  double p = 1.0 / 87178291200.0;
  p = 1.0 / 6227020800.0 + r * p;
  p = 1.0 / 479001600.0 + r * p;
  p = 1.0 / 39916800.0 + r * p;
  p = 1.0 / 3628800.0 + r * p;
  p = 1.0 / 362880.0 + r * p;
  p = 1.0 / 40320.0 + r * p;
  p = 1.0 / 5040.0 + r * p;
  p = 1.0 / 720.0 + r * p;
  p = 1.0 / 120.0 + r * p;
  p = 1.0 / 24.0 + r * p;
  p = 1.0 / 6.0 + r * p;
  p = 0.5 + r * p;
  p = 1.0 + r * p;
  p = 1.0 + r * p;
  return p * __longlong_as_double((long long)((int)k + 1023) << 52);
}
__device__ __forceinline__ double ctl_pow(double x, double y) {
  if (x != x || y != y || x < 0.0) return __longlong_as_double(0x7ff8000000000000LL);
  if (x == 0.0) return (y > 0.0) ? 0.0 : __longlong_as_double(0x7ff0000000000000LL);
  if (isinf(x)) return (y > 0.0) ? __longlong_as_double(0x7ff0000000000000LL) : 0.0;
  if (x == 1.0 || y == 0.0) return 1.0;
  return spec_exp(y * spec_ln(x));
}
// FP32 controller power: no cross-machine reproducibility is asked of FP32.
__device__ __forceinline__ float ctl_pow(float x, float e) { return exp2f(e * __log2f(x)); }

// ---------------------------------------------------------------- group ops
// Group of G lanes (G divides 32).  mask() is the group's lane mask.
template <int G> struct Grp {
  __device__ __forceinline__ static unsigned mask() {
    if constexpr (G == 32) return 0xffffffffu;
    const int lane = threadIdx.x & 31;
    return ((1u << G) - 1u) << (lane - (lane % G));
  }
  __device__ __forceinline__ static int rank() { return (threadIdx.x & 31) % G; }
  template <typename T> __device__ __forceinline__ static T bcast(T v, int src) {
    if constexpr (G == 1) return v;
    else return __shfl_sync(mask(), v, src, G);
  }
};

// Sum over the D = G*R components in index order 0..D-1 (FP64: the exact
// left-to-right order; FP32: per-lane partial sums then a butterfly, which
// gives the same bits on every lane because IEEE addition commutes).
template <typename T, int R, int G>
__device__ __forceinline__ T group_sum(const T (&v)[R]) {
  if constexpr (sizeof(T) == 8) {
    T s = T(0);
    if constexpr (G == 1) {
#pragma unroll
      for (int r = 0; r < R; ++r) s = s + v[r];
    } else {
#pragma unroll
      for (int j = 0; j < G * R; ++j) s = s + Grp<G>::bcast(v[j % R], j / R);
    }
    return s;
  } else {
    T s = T(0);
#pragma unroll
    for (int r = 0; r < R; ++r) s = s + v[r];
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) s = s + __shfl_xor_sync(Grp<G>::mask(), s, off, G);
    return s;
  }
}

// Weighted RMS norm sqrt(sum_j (v_j / sc_j)^2 / D), per instance (HNW II.4).
template <typename T, int R, int G>
__device__ __forceinline__ T rms_norm(const T (&v)[R], const T (&sc)[R]) {
  T q2[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    T q = v[r] / sc[r];
    q2[r] = q * q;
  }
  return sqrt(group_sum<T, R, G>(q2) / T(G * R));
}

// ---------------------------------------------------------------- per-instance state
// FP32 state is accumulated with compensated (Kahan) summation: the state is
// y + ylo with |ylo| <= ulp(y)/2, so thousands of FP32 steps do not lose the
// rounding of every state update.  FP64 state is summed plainly.
template <typename T> struct Comp {
  static constexpr bool on = sizeof(T) == 4;
};

template <typename T, int R> struct Inst {
  T y[R];
  T ylo[R];      // compensation term (FP32 only; 0 in FP64)
  T k1[R];       // FSAL stage
  double t, t0, t1;
  T h;           // step size proposed for the next attempt
  T h_last;      // step size the last attempt used (clipped at t1)
  T rem;         // FP32 state: t1 - t rounded down to float (last-step test)
  T hmin;        // FP32 state: step-size underflow threshold 1e-14 max(|t0|,|t1|)
  T err_prev, err_prev2;  // error estimates of the last two accepted steps
  T rtol, atol;
  int n_acc, n_rej, cursor, status, flags;
  // the evaluation times at the cursor and after it (+inf past the last),
  // held in registers so that the end-of-step test loads nothing
  double tq, tq2;
};

struct SolveOpts {
  double safety, fac_min, fac_max, beta1, beta2, beta3, h0;
  int max_steps;
  // the same controller constants rounded to FP32 once on the host (an FP32
  // kernel then does no double-to-float conversion per attempt)
  float safety_f, fac_min_f, fac_max_f, beta1_f, beta2_f, beta3_f;
};
inline void opts_round_f32(SolveOpts& s) {
  s.safety_f = (float)s.safety;
  s.fac_min_f = (float)s.fac_min;
  s.fac_max_f = (float)s.fac_max;
  s.beta1_f = (float)s.beta1;
  s.beta2_f = (float)s.beta2;
  s.beta3_f = (float)s.beta3;
}
// controller constant in the state type
template <typename T> __device__ __forceinline__ T opt_v(double d, float f) {
  if constexpr (sizeof(T) == 4) return f;
  else return T(d);
}

// Output pointers for one instance.
template <typename T> struct InstOut {
  const double* te;  // [K]
  T* ye;             // [K][D]
  T* yp;             // [K][D] or NULL: dy/dt of the dense output at the points
  int K;
};

// Evaluation time q of the instance in the direction of integration (m:
// its rev_mask), +inf past the last one.
template <typename T>
__device__ __forceinline__ double te_at(const InstOut<T>& out, int q, unsigned long long m) {
  return q < out.K ? flip(out.te[q], m) : __longlong_as_double(0x7ff0000000000000LL);
}
// Moves the cursor past the point just written: the register pair shifts and
// the time after the next one is loaded (its latency overlaps the attempt).
template <typename T, int R>
__device__ __forceinline__ void advance_cursor(Inst<T, R>& s, const InstOut<T>& out) {
  s.cursor++;
  s.tq = s.tq2;
  s.tq2 = te_at(out, s.cursor + 1, rev_mask(s.flags));
}

// True when b_i(theta) vanishes identically (dopri5's stage 2).
template <class Tab> __host__ __device__ constexpr bool dense_zero(int i) {
  return Tab::q(i, 0) == 0.0 && Tab::q(i, 1) == 0.0 && Tab::q(i, 2) == 0.0 &&
         Tab::q(i, 3) == 0.0;
}

// Dense-output weights b_i(theta), each by Horner's rule.
template <class Tab, typename T> __device__ __forceinline__ void dense_weights(T th, T (&w)[7]) {
#pragma unroll
  for (int i = 1; i <= 7; ++i)
    w[i - 1] = th * madd(th, madd(th, madd(th, T(Tab::q(i, 3)), T(Tab::q(i, 2))),
                                  T(Tab::q(i, 1))),
                         T(Tab::q(i, 0)));
}

// Derivatives b_i'(theta) of the dense-output weights, each by Horner's rule.
template <class Tab, typename T> __device__ __forceinline__ void dense_dweights(T th, T (&w)[7]) {
#pragma unroll
  for (int i = 1; i <= 7; ++i)
    w[i - 1] = madd(th, madd(th, madd(th, T(4) * T(Tab::q(i, 3)), T(3) * T(Tab::q(i, 2))),
                             T(2) * T(Tab::q(i, 1))),
                    T(Tab::q(i, 0)));
}

// The stage derivatives k_1..k_7 of one step, as one indexable set.
template <typename T, int R> struct Stages {
  T k[7][R];
};

// Dense output of one evaluation point:  y + h * sum_i b_i(theta) k_i
// (+ the state's compensation term in FP32).
template <class Tab, typename T, int R>
__device__ __forceinline__ void dense_point(T theta, T h, const T (&y)[R], const T (&ylo)[R],
                                            const Stages<T, R>& K, T (&out)[R]) {
  T w[7];
  dense_weights<Tab, T>(theta, w);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    T s = w[0] * K.k[0][r];
#pragma unroll
    for (int i = 2; i <= 7; ++i)
      if (!dense_zero<Tab>(i)) s = madd(w[i - 1], K.k[i - 1][r], s);
    if constexpr (Comp<T>::on) out[r] = y[r] + madd(h, s, ylo[r]);
    else out[r] = madd(h, s, y[r]);
  }
}

// d/dt of the dense output at theta: sum_i b_i'(theta) k_i with b_i' the
// derivatives of the same quartics (the step size cancels), times dir to
// turn the solver's tau = dir t back into t.
template <class Tab, typename T, int R>
__device__ __forceinline__ void dense_deriv(T th, T dir, const Stages<T, R>& K, T (&out)[R]) {
  T w[7];
#pragma unroll
  for (int i = 1; i <= 7; ++i) {
    if (Tab::q(i, 0) != 0.0)
      w[i - 1] = madd(th, madd(th, madd(th, T(4) * T(Tab::q(i, 3)), T(3) * T(Tab::q(i, 2))),
                               T(2) * T(Tab::q(i, 1))),
                      T(Tab::q(i, 0)));
    else
      w[i - 1] = th * madd(th, madd(th, T(4) * T(Tab::q(i, 3)), T(3) * T(Tab::q(i, 2))),
                           T(2) * T(Tab::q(i, 1)));
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    T v = w[0] * K.k[0][r];
#pragma unroll
    for (int i = 2; i <= 7; ++i)
      if (!dense_zero<Tab>(i)) v = madd(w[i - 1], K.k[i - 1][r], v);
    out[r] = dir * v;
  }
}

// Write one evaluation point's R components of lane `g`.
template <typename T, int R, int G>
__device__ __forceinline__ void store_point(T* dst, const T (&v)[R]) {
  const int g = Grp<G>::rank();
#pragma unroll
  for (int r = 0; r < R; ++r) dst[g * R + r] = v[r];
}

// ---------------------------------------------------------------- tape / trace
// R consecutive components of one lane at p (p aligned to R * sizeof(T)
// when that is 8 or 16 bytes): one vector access instead of R.
template <typename T, int R> __device__ __forceinline__ void st_row(T* p, const T (&v)[R]) {
  if constexpr (R == 2 && sizeof(T) == 4) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else if constexpr (R == 4 && sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 2 && sizeof(T) == 8) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) p[r] = v[r];
  }
}
template <typename T, int R> __device__ __forceinline__ void ld_row(const T* p, T (&v)[R]) {
  if constexpr (R == 2 && sizeof(T) == 4) {
    const float2 u = *reinterpret_cast<const float2*>(p);
    v[0] = u.x, v[1] = u.y;
  } else if constexpr (R == 4 && sizeof(T) == 4) {
    const float4 u = *reinterpret_cast<const float4*>(p);
    v[0] = u.x, v[1] = u.y, v[2] = u.z, v[3] = u.w;
  } else if constexpr (R == 2 && sizeof(T) == 8) {
    const double2 u = *reinterpret_cast<const double2*>(p);
    v[0] = u.x, v[1] = u.y;
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = p[r];
  }
}

template <typename T> struct TapeDev {
  int slots, stride, B, D;
  T* y;
  T* ylo;  // FP32 only
  T* k1;   // FSAL stage at the slot
  double* t;
  T* h;
  T* err_prev;
  T* err_prev2;
  int32_t* flags;
  T* h_acc;   // optional: size of the accepted step that starts at the slot
  T* ystage;  // optional: its stage inputs Y_2..Y_7, [B][slots][6][D]
};
struct TraceDev {
  int cap;
  double* t;
  double* h;
  double* err;
  int32_t* acc;
  int32_t* len;
};

template <typename T, int R, int G>
__device__ __forceinline__ void tape_store(const TapeDev<T>& tp, int i, const Inst<T, R>& s) {
  if (tp.slots == 0 || (s.n_acc % tp.stride) != 0) return;
  const int j = s.n_acc / tp.stride;
  if (j >= tp.slots) return;
  const size_t o = (size_t)i * tp.slots + j;  // instance-major: [B][slots]
  const int g = Grp<G>::rank();
  st_row<T, R>(tp.y + o * tp.D + g * R, s.y);
  // a stride-1 tape with the accepted step sizes may leave out what only a
  // re-run needs (k1 too when it records the stage inputs)
  if (tp.k1) st_row<T, R>(tp.k1 + o * tp.D + g * R, s.k1);
  if constexpr (Comp<T>::on) {
    if (tp.ylo) st_row<T, R>(tp.ylo + o * tp.D + g * R, s.ylo);
  }
  if (g == 0) {
    tp.t[o] = s.t;
    if (tp.h) tp.h[o] = s.h;
    if (tp.err_prev) tp.err_prev[o] = s.err_prev;
    if (tp.err_prev2) tp.err_prev2[o] = s.err_prev2;
    if (tp.flags) tp.flags[o] = s.flags;
  }
}

// After an accepted attempt: the size of that step (n = n_acc - 1) and, when
// the tape keeps them, its stage inputs into its slot, so that a stride-1
// adjoint can reverse straight from the tape.
template <typename T, int R, int G>
__device__ __forceinline__ void tape_store_hacc(const TapeDev<T>& tp, int i, const Inst<T, R>& s,
                                                const T (&ys)[6][R]) {
  const int n = s.n_acc - 1;
  if (tp.slots == 0 || !tp.h_acc || (n % tp.stride) != 0) return;
  const int j = n / tp.stride;
  if (j >= tp.slots) return;
  if (Grp<G>::rank() == 0) tp.h_acc[(size_t)i * tp.slots + j] = s.h_last;
  if (tp.ystage && tp.stride == 1) {
    T* dst = tp.ystage + ((size_t)i * tp.slots + j) * 6 * tp.D + Grp<G>::rank() * R;
#pragma unroll
    for (int q = 0; q < 6; ++q) st_row<T, R>(dst + q * tp.D, ys[q]);
  }
}

// ---------------------------------------------------------------- init (a1, a2)
// Loads the instance, validates its times, writes evaluation points at t0,
// evaluates k1 = f(t0, y0) and picks the first step (given h0 or the HNW
// Sec. II.4 heuristic, which costs one more evaluation).  Returns false if
// the instance is already finished (invalid input or t1 == t0).
template <class Field, typename T, int R, int G>
__device__ bool inst_init(const Field& F, Inst<T, R>& s, const SolveOpts& o, int i, int D,
                          const T* y0, const double* t0p, const double* t1p, double rtol,
                          double atol, const InstOut<T>& out) {
  const int g = Grp<G>::rank();
  const bool rev = reversed_at(t0p, t1p, i);
  const unsigned long long msk = rev ? SIGN_BIT : 0ULL;
  s.t0 = flip(t0p[i], msk);
  s.t1 = flip(t1p[i], msk);
  s.t = s.t0;
  s.rtol = T(rtol);
  s.atol = T(atol);
  s.n_acc = s.n_rej = 0;
  s.cursor = 0;
  s.flags = rev ? FL_REVERSE : 0;
  s.err_prev = T(1);
  s.err_prev2 = T(1);
  s.h = T(0);
  s.h_last = T(0);
  s.rem = T(0);
  s.hmin = T(0);
  s.status = ST_RUNNING;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    s.y[r] = y0[(size_t)i * D + g * R + r];
    s.ylo[r] = T(0);
    s.k1[r] = T(0);
  }
  // validity of the time arguments (Sec. 3: per-instance bounds and points):
  // t0 <= te[0] <= ... <= te[K-1] <= t1, all finite; the group's lanes check
  // the points in parallel (point q against its predecessor)
  bool ok = tfinite(s.t0) && tfinite(s.t1) && !(s.t1 < s.t0);
  const long long k0 = tkey(s.t0), k1 = tkey(s.t1);
  {
    bool okl = true;
    for (int q = g; q < out.K; q += G) {
      const double v = flip(out.te[q], msk);
      const long long kv = tkey(v);
      const long long kp = q > 0 ? tkey(flip(out.te[q - 1], msk)) : k0;
      okl = okl && tfinite(v) && kv >= kp && kv <= k1;
    }
    if constexpr (G > 1) okl = __all_sync(Grp<G>::mask(), okl) != 0;
    ok = ok && okl;
  }
  if (!ok) {
    s.status = ST_INVALID;
    T nanv[R];
#pragma unroll
    for (int r = 0; r < R; ++r) nanv[r] = nan_(T(0));
    for (int q = 0; q < out.K; ++q) store_point<T, R, G>(out.ye + (size_t)q * D, nanv);
    if (out.yp)
      for (int q = 0; q < out.K; ++q) store_point<T, R, G>(out.yp + (size_t)q * D, nanv);
    return false;
  }
  s.tq = te_at(out, 0, msk);
  s.tq2 = te_at(out, 1, msk);
  while (tkey(s.tq) == k0) {  // points at t0 are y0 itself
    store_point<T, R, G>(out.ye + (size_t)s.cursor * D, s.y);
    advance_cursor(s, out);
  }
  if (out.yp && s.cursor > 0) {  // and their derivative f(t0, y0)
    T f0[R];
    F.eval(s.t, s.y, f0);
    const T dir = rev ? T(-1) : T(1);
#pragma unroll
    for (int r = 0; r < R; ++r) f0[r] = dir * f0[r];
    for (int q = 0; q < s.cursor; ++q) store_point<T, R, G>(out.yp + (size_t)q * D, f0);
  }
  if (k1 == k0) {
    s.status = ST_SUCCESS;
    return false;
  }
  if constexpr (Comp<T>::on) {
    s.rem = __double2float_rd(s.t1 - s.t0);
    s.hmin = T(1e-14 * tmax(fabs(s.t0), fabs(s.t1)));
  }
  F.eval(s.t, s.y, s.k1);
  if (o.h0 > 0.0) {
    s.h = T(o.h0);
    return true;
  }
  // starting step size, HNW Sec. II.4
  T sc[R], w[R], f1[R];
#pragma unroll
  for (int r = 0; r < R; ++r) sc[r] = madd(s.rtol, T(fabs(s.y[r])), s.atol);
  const T d0 = rms_norm<T, R, G>(s.y, sc);
  const T d1 = rms_norm<T, R, G>(s.k1, sc);
  const T h0 = (d0 < T(1e-5) || d1 < T(1e-5)) ? T(1e-6) : T(0.01) * (d0 / d1);
#pragma unroll
  for (int r = 0; r < R; ++r) w[r] = madd(h0, s.k1[r], s.y[r]);
  F.eval(s.t + (double)h0, w, f1);
#pragma unroll
  for (int r = 0; r < R; ++r) f1[r] = f1[r] - s.k1[r];
  const T d2 = rms_norm<T, R, G>(f1, sc) / h0;
  const T m = (d1 > d2) ? d1 : d2;
  const T h1 = (m <= T(1e-15)) ? tmax(T(1e-6), h0 * T(1e-3)) : ctl_pow(T(0.01) / m, T(1.0 / 5.0));
  T h = tmin(T(100) * h0, h1);
  h = tmin(h, T(s.t1 - s.t0));
  if (!(h > T(0) && finite_(h))) h = T(s.t1 - s.t0);
  s.h = h;
  return true;
}

// ---------------------------------------------------------------- stages (a3, a4)
// The six new stages of one attempt of the pair Tab from (t, y, K.k[0] = k1)
// with step h: the stage inputs Y_2..Y_7 into ys (Y_7 is the new solution
// y1, SSAL), K.k[1..6] = k2..k7, the increment inc = h sum_i b_i k_i and
// y1 = y + inc.  Each stage input is y + h (a_i1 k1 + a_i2 k2 + ...), the
// sum taken left to right; zero coefficients are skipped.  LAST = false
// leaves out the evaluation at y1 (k7, FSAL: the next step's k1).
template <class Tab, class Field, typename T, int R, bool LAST = true>
__device__ __forceinline__ void attempt_stages(const Field& F, double t, T h, const T (&y)[R],
                                               Stages<T, R>& K, T (&ys)[6][R], T (&y1)[R],
                                               T (&inc)[R]) {
  const double hd = (double)h;
#pragma unroll
  for (int i = 2; i <= 7; ++i) {
    T Y[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      T a = T(Tab::a(i, 1)) * K.k[0][r];
#pragma unroll
      for (int j = 2; j < i; ++j)
        if (Tab::a(i, j) != 0.0) a = madd(T(Tab::a(i, j)), K.k[j - 1][r], a);
      if (i < 7) {
        Y[r] = madd(h, a, y[r]);
      } else {
        inc[r] = h * a;
        Y[r] = y[r] + inc[r];  // SSAL: the 7th stage input is the new solution
        y1[r] = Y[r];
      }
      ys[i - 2][r] = Y[r];
    }
    if (i < 7 || LAST) F.eval(t + Tab::c(i) * hd, Y, K.k[i - 1]);
  }
}

// Embedded error estimate e = h sum_i (b_i - bhat_i) k_i and the norm's
// weights atol + rtol max(|y|, |y1|) (a4, a5); returns whether this lane's
// components of y1 are finite.
template <class Tab, typename T, int R>
__device__ __forceinline__ bool error_terms(T h, const T (&y)[R], const T (&y1)[R],
                                            const Stages<T, R>& K, T rtol, T atol, T (&ev)[R],
                                            T (&sc)[R]) {
  bool fin = true;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    T a = T(Tab::e(1)) * K.k[0][r];
#pragma unroll
    for (int i = 2; i <= 7; ++i)
      if (Tab::e(i) != 0.0) a = madd(T(Tab::e(i)), K.k[i - 1][r], a);
    ev[r] = h * a;
    sc[r] = madd(rtol, T(tmax(fabs(y[r]), fabs(y1[r]))), atol);
    fin = fin && finite_(y1[r]);
  }
  return fin;
}

// ---------------------------------------------------------------- one attempt (a3..a9)
// Returns true while the instance is still running.
// YP: the solve also writes dy/dt at the points (out.yp); a separate
// instantiation, so that solves without it keep the leaner kernel.
template <class Tab, class Field, typename T, int R, int G, bool YP = false>
__device__ bool inst_attempt(const Field& F, Inst<T, R>& s, const SolveOpts& o, int i, int D,
                             const InstOut<T>& out, const TraceDev& tr, T (&ys)[6][R]) {
  T h = s.h;
  bool last = false;
  if constexpr (Comp<T>::on) {
    // FP32 state: compare with t1 - t rounded down, so a step that is not
    // flagged last never passes t1 by more than FP64 rounding
    if (h >= s.rem) {
      h = s.rem;
      last = true;
    }
  } else if (s.t + (double)h >= s.t1) {
    h = T(s.t1 - s.t);
    last = true;
  }
  s.h_last = h;
  const double hd = (double)h;
  Stages<T, R> K;
#pragma unroll
  for (int r = 0; r < R; ++r) K.k[0][r] = s.k1[r];
  T y1[R], inc[R], ev[R], sc[R];
  attempt_stages<Tab, Field, T, R>(F, s.t, h, s.y, K, ys, y1, inc);
  const bool fin_local = error_terms<Tab, T, R>(h, s.y, y1, K, s.rtol, s.atol, ev, sc);
  const T err = rms_norm<T, R, G>(ev, sc);
  bool finite = finite_(err);
  if constexpr (G > 1) finite = finite && (__all_sync(Grp<G>::mask(), fin_local) != 0);
  else finite = finite && fin_local;
  const bool accept = finite && err <= T(1);

  const int att = s.n_acc + s.n_rej;
  if (tr.cap > 0 && att < tr.cap && Grp<G>::rank() == 0) {
    const size_t q = (size_t)i * tr.cap + att;
    tr.t[q] = flip(s.t, rev_mask(s.flags));  // the caller's time and signed step
    tr.h[q] = flip(hd, rev_mask(s.flags));
    tr.err[q] = (double)err;
    tr.acc[q] = accept ? 1 : 0;
  }

  T h_next;
  if (accept) {
    double t_next = last ? s.t1 : s.t + hd;
    if constexpr (Comp<T>::on) {
      if (!last && tkey(t_next) >= tkey(s.t1)) {  // landed on t1 by rounding
        last = true;
        t_next = s.t1;
      }
    }
    const long long kn = tkey(t_next);
    // new state (FP32: compensated sum y + (inc + ylo))
    T yn[R], ylon[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if constexpr (Comp<T>::on) {
        const T u = inc[r] + s.ylo[r];
        yn[r] = s.y[r] + u;
        ylon[r] = (s.y[r] - yn[r]) + u;
      } else {
        yn[r] = y1[r];
        ylon[r] = T(0);
      }
    }
    while (true) {  // the points in (t, t_next]; +inf past the last point
      const double tq = s.tq;
      const long long kq = tkey(tq);
      if (kq > kn) break;
      T* dst = out.ye + (size_t)s.cursor * D;
      T theta = T(1);
      if (kq == kn) {
        store_point<T, R, G>(dst, yn);
      } else {
        // abscissa: the difference tq - t in FP64, the ratio in the state type
        if constexpr (Comp<T>::on) theta = T(tq - s.t) / h;
        else theta = T((tq - s.t) / hd);
        T v[R];
        dense_point<Tab, T, R>(theta, h, s.y, s.ylo, K, v);
        store_point<T, R, G>(dst, v);
      }
      if constexpr (YP) {
        T v[R];
        dense_deriv<Tab, T, R>(theta, (s.flags & FL_REVERSE) ? T(-1) : T(1), K, v);
        store_point<T, R, G>(out.yp + (size_t)s.cursor * D, v);
      }
      advance_cursor(s, out);
    }
    T fac;
    if (err == T(0)) {
      fac = opt_v<T>(o.fac_max, o.fac_max_f);
    } else {
      fac = opt_v<T>(o.safety, o.safety_f) * ctl_pow(err, -opt_v<T>(o.beta1, o.beta1_f));
      if (o.beta2 != 0.0) fac = fac * ctl_pow(s.err_prev, opt_v<T>(o.beta2, o.beta2_f));
      if (o.beta3 != 0.0) fac = fac * ctl_pow(s.err_prev2, -opt_v<T>(o.beta3, o.beta3_f));
    }
    fac = tmin(tmax(fac, opt_v<T>(o.fac_min, o.fac_min_f)), opt_v<T>(o.fac_max, o.fac_max_f));
    if (s.flags & FL_PREV_REJ) fac = tmin(fac, T(1));
    h_next = h * fac;
    s.err_prev2 = s.err_prev;
    s.err_prev = tmax(err, T(1e-4));
    s.flags &= ~FL_PREV_REJ;
    s.n_acc++;
    s.t = t_next;
    if constexpr (Comp<T>::on) {
      if (!last) s.rem = __double2float_rd(s.t1 - s.t);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      s.y[r] = yn[r];
      s.ylo[r] = ylon[r];
      s.k1[r] = K.k[6][r];  // FSAL
    }
    if (last) s.status = ST_SUCCESS;
  } else {
    const T fmin = opt_v<T>(o.fac_min, o.fac_min_f);
    const T fac =
        finite ? tmin(tmax(opt_v<T>(o.safety, o.safety_f) * ctl_pow(err, -opt_v<T>(o.beta1, o.beta1_f)),
                           fmin),
                      T(1))
               : fmin;
    h_next = h * fac;
    s.flags |= FL_PREV_REJ;
    s.n_rej++;
  }
  s.h = h_next;
  if (s.status == ST_RUNNING) {
    bool under;
    if constexpr (Comp<T>::on) {
      // FP32 state: 1e-14 max(|t0|,|t1|) bounds 1e-14 max(|t|,|t1|) and lies
      // above the FP64 spacing of t, so "t + h == t" cannot occur first
      under = !(h_next >= s.hmin) || !(h_next > T(0));
    } else {
      const double scale = tmax(fabs(s.t), fabs(s.t1));
      const double hn = (double)h_next;
      under = s.t + hn == s.t || hn < 1e-14 * scale || !(h_next > T(0));
    }
    if (under)
      s.status = finite ? ST_DT_UNDERFLOW : ST_NONFINITE;
    else if (s.n_acc + s.n_rej >= o.max_steps)
      s.status = ST_MAX_STEPS;
  }
  return s.status == ST_RUNNING;
}

// ---------------------------------------------------------------- finalize
template <typename T, int R, int G>
__device__ void inst_finalize(const Inst<T, R>& s, const SolveOpts& o, int i, int D,
                              const InstOut<T>& out, T* y_final, int32_t* n_acc, int32_t* n_rej,
                              int32_t* n_fe, int32_t* status, const TraceDev& tr) {
  const int g = Grp<G>::rank();
  const bool invalid = s.status == ST_INVALID;
  if (s.status != ST_SUCCESS && !invalid) {  // points a failed instance never reached
    T nanv[R];
#pragma unroll
    for (int r = 0; r < R; ++r) nanv[r] = nan_(T(0));
    for (int q = s.cursor; q < out.K; ++q) {
      store_point<T, R, G>(out.ye + (size_t)q * D, nanv);
      if (out.yp) store_point<T, R, G>(out.yp + (size_t)q * D, nanv);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) y_final[(size_t)i * D + g * R + r] = invalid ? nan_(T(0)) : s.y[r];
  if (g == 0) {
    const int att = s.n_acc + s.n_rej;
    n_acc[i] = s.n_acc;
    n_rej[i] = s.n_rej;
    const bool stepped = !invalid && tkey(s.t1) != tkey(s.t0);
    n_fe[i] = stepped ? ((o.h0 > 0.0 ? 1 : 2) + 6 * att) : 0;
    status[i] = s.status;
    if (tr.cap > 0) tr.len[i] = att < tr.cap ? att : tr.cap;
  }
}

// ---------------------------------------------------------------- work order
// One CTA counting-sorts the instances into a work queue by a bin number
// (bin 0 first).  Every instance is solved or reversed independently of the
// others, so the order changes no result; it only decides which instances
// share a warp and which start first.  The order inside a bin is arbitrary.

// The counters are per (bin, warp), bin-major, so that lanes of different
// warps never contend for one counter (the bins of a batch are few and
// crowded) and the queue stays ordered by bin.
constexpr int ORDER_CACHE = ORDER_SMALL_B;  // bins kept in shared memory for the second pass

template <class BinOf>
__global__ void __launch_bounds__(ORDER_THREADS) k_counting_order(int B, BinOf bin_of,
                                                                  int32_t* order) {
  constexpr int W = ORDER_THREADS / 32, PER = ORDER_BINS * W / ORDER_THREADS;
  __shared__ int cnt[ORDER_BINS * W];  // [bin][warp]
  __shared__ int warp_tot[W];
  __shared__ unsigned char bins[ORDER_CACHE];  // a small batch's bins, for the second pass
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const bool cached = B <= ORDER_CACHE;
#pragma unroll
  for (int k = 0; k < PER; ++k) cnt[t * PER + k] = 0;
  __syncthreads();
  // independent iterations: unrolled so that their loads overlap
#pragma unroll 8
  for (int i = t; i < B; i += ORDER_THREADS) {
    const int b = bin_of(i);
    if (cached) bins[i] = (unsigned char)b;
    atomicAdd(&cnt[b * W + w], 1);
  }
  __syncthreads();
  // exclusive prefix sum over the (bin, warp) counters, PER per thread
  int loc[PER], sum = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    loc[k] = sum;
    sum += cnt[t * PER + k];
  }
  int incl = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    int x = warp_tot[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += v;
    }
    warp_tot[lane] = x;  // inclusive over warps
  }
  __syncthreads();
  const int before = (w > 0 ? warp_tot[w - 1] : 0) + incl - sum;
#pragma unroll
  for (int k = 0; k < PER; ++k) cnt[t * PER + k] = before + loc[k];
  __syncthreads();
#pragma unroll 8
  for (int i = t; i < B; i += ORDER_THREADS) {
    const int b = cached ? (int)bins[i] : bin_of(i);
    order[atomicAdd(&cnt[b * W + w], 1)] = i;
  }
}

// Multi-CTA form for large batches: every CTA counts its instances per bin
// (k_order_count), one CTA turns the counts into queue offsets, bin-major
// and CTA-minor (k_order_offsets), and every CTA places its instances from
// its own offsets (k_order_place; the same grid-stride walk as the count).
template <class BinOf>
__global__ void __launch_bounds__(ORDER_THREADS) k_order_count(int B, BinOf bin_of, int* part) {
  __shared__ int cnt[ORDER_BINS];
  const int t = threadIdx.x;
  if (t < ORDER_BINS) cnt[t] = 0;
  __syncthreads();
  const long long stride = (long long)gridDim.x * ORDER_THREADS;
#pragma unroll 4
  for (long long i = (long long)blockIdx.x * ORDER_THREADS + t; i < B; i += stride)
    atomicAdd(&cnt[bin_of((int)i)], 1);
  __syncthreads();
  if (t < ORDER_BINS) part[(size_t)blockIdx.x * ORDER_BINS + t] = cnt[t];
}

template <int NB>
__global__ void __launch_bounds__(NB) k_order_offsets(int ctas, int* part) {
  static_assert(NB == ORDER_BINS, "one thread per bin");
  __shared__ int warp_tot[NB / 32];
  const int b = threadIdx.x, lane = b & 31, w = b >> 5;
  int total = 0;
  for (int c = 0; c < ctas; ++c) total += part[(size_t)c * ORDER_BINS + b];
  int incl = total;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  int before = 0;
  for (int k = 0; k < w; ++k) before += warp_tot[k];
  int run = before + incl - total;  // queue start of bin b
  for (int c = 0; c < ctas; ++c) {
    const size_t q = (size_t)c * ORDER_BINS + b;
    const int v = part[q];
    part[q] = run;
    run += v;
  }
}

template <class BinOf>
__global__ void __launch_bounds__(ORDER_THREADS) k_order_place(int B, BinOf bin_of,
                                                               const int* part, int32_t* order) {
  __shared__ int cur[ORDER_BINS];
  const int t = threadIdx.x;
  if (t < ORDER_BINS) cur[t] = part[(size_t)blockIdx.x * ORDER_BINS + t];
  __syncthreads();
  const long long stride = (long long)gridDim.x * ORDER_THREADS;
#pragma unroll 4
  for (long long i = (long long)blockIdx.x * ORDER_THREADS + t; i < B; i += stride)
    order[atomicAdd(&cur[bin_of((int)i)], 1)] = (int32_t)i;
}

// Fills order[0..B) (part: order_part_bytes(B) of scratch, unused for a
// small batch).
template <class BinOf>
inline cudaError_t launch_order(int B, BinOf bin_of, int32_t* order, int* part,
                                cudaStream_t st) {
  if (B <= ORDER_SMALL_B) {
    k_counting_order<<<1, ORDER_THREADS, 0, st>>>(B, bin_of, order);
    return cudaGetLastError();
  }
  const int g = order_ctas(B);
  k_order_count<<<g, ORDER_THREADS, 0, st>>>(B, bin_of, part);
  k_order_offsets<ORDER_BINS><<<1, ORDER_BINS, 0, st>>>(g, part);
  k_order_place<<<g, ORDER_THREADS, 0, st>>>(B, bin_of, part, order);
  return cudaGetLastError();
}

// Longest integration interval first: t1 - t0 binned by its binary exponent
// and two leading fraction bits (a quarter octave per bin, 2^-32 .. 2^32,
// clamped outside).  An ordering key only, so the length is taken in FP32
// from times truncated to FP32 on the integer pipe (no FP64 operation on the
// single SM that sorts).  Empty, reversed or non-finite intervals, which
// finish at initialisation, go last.
__device__ __forceinline__ float trunc_to_float(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int e = (int)((hi >> 20) & 0x7ffu);
  const unsigned sign = hi & 0x80000000u;
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | ((hi & 0xfffffu) ? 1u : 0u));
  const int ef = e - 1023 + 127;
  if (ef < 1) return __uint_as_float(sign);                 // below float's normal range: 0
  if (ef > 254) return __uint_as_float(sign | 0x7f7fffffu);  // above: the largest float
  return __uint_as_float(sign | ((unsigned)ef << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}
struct IntervalBin {
  const double* t0;
  const double* t1;
  __device__ __forceinline__ int operator()(int i) const {
    const float len = fabsf(trunc_to_float(t1[i]) - trunc_to_float(t0[i]));  // either direction
    if (!(len > 0.0f) || !(len <= 3.4e38f)) return ORDER_BINS - 1;
    const unsigned b = __float_as_uint(len);
    const int key = ((int)((b >> 23) & 0xffu) - 127 + 32) * 4 + (int)((b >> 21) & 3u);
    const int k = key < 0 ? 0 : (key > ORDER_BINS - 2 ? ORDER_BINS - 2 : key);
    return ORDER_BINS - 2 - k;
  }
};

// Most accepted steps first (the adjoint's sweep lengths, capped at
// ORDER_BINS - 1); instances that failed do no work.
struct StepsBin {
  const int32_t* n_acc;
  const int32_t* status;
  __device__ __forceinline__ int operator()(int i) const {
    const int n = status[i] == ST_SUCCESS ? n_acc[i] : 0;
    return ORDER_BINS - 1 - (n < 0 ? 0 : (n > ORDER_BINS - 1 ? ORDER_BINS - 1 : n));
  }
};

// ---------------------------------------------------------------- work stealing
// Hands the next instance index to every group of the calling lanes with one
// atomic per warp (lanes of a group always arrive together).
template <int G>
__device__ __forceinline__ int grab_instance(int32_t* counter, int first_wave) {
  if constexpr (G > 1) __syncwarp(Grp<G>::mask());
  const unsigned active = __activemask();
  const int lane = threadIdx.x & 31;
  const int leader = lane - (lane % G);
  const unsigned want = __ballot_sync(active, (lane % G) == 0);
  const int first = __ffs(want) - 1;
  int base = 0;
  if (lane == first) base = atomicAdd(counter, __popc(want));
  base = __shfl_sync(active, base, first < 0 ? 0 : first);
  int mine = first_wave + base + __popc(want & ((1u << leader) - 1u));
  if constexpr (G > 1) mine = __shfl_sync(Grp<G>::mask(), mine, 0, G);
  return mine;
}

}  // namespace tode
