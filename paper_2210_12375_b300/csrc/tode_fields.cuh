// tode_fields.cuh -- built-in SIMT vector fields evaluated by a lane group.
//
// Each field object is bound to one instance (its parameters are loaded into
// registers once) and evaluates f(t, Y) for the group's R components, times
// the instance's direction dir (-1 when it integrates backward in time: the
// solver then runs in tau = -t, where the field is -f).
#pragma once
#include "tode_core.cuh"

namespace tode {

// Van der Pol, Eq. 1 written as a first-order system (D = 2, G = 1, R = 2):
//   y1' = y2,  y2' = mu (1 - y1^2) y2 - y1.
template <typename T> struct VdpField {
  T mu, dir;
  __device__ __forceinline__ void load(const T* mu_all, int i, T d) {
    mu = mu_all[i];
    dir = d;
  }
  __device__ __forceinline__ void eval(double, const T (&y)[2], T (&f)[2]) const {
    f[0] = dir * y[1];
    // mu (1 - y1^2) y2 - y1 (FP64: the same operations as written out)
    f[1] = dir * madd(mu * madd(-y[0], y[0], T(1)), y[1], -y[0]);
  }
};

// y' = A_i y, D = G*R; lane g owns rows g*R .. g*R+R-1 of A_i and gathers
// the whole state from its group with shuffles.  The direction is folded
// into the rows at load ((dir A) y is dir (A y) bit for bit).
template <typename T, int R, int G> struct LinearField {
  static constexpr int D = G * R;
  T a[R][D];
  __device__ __forceinline__ void load(const T* A_all, int i, T dir) {
    const int g = Grp<G>::rank();
    const T* A = A_all + (size_t)i * D * D + (size_t)g * R * D;
    if constexpr (sizeof(T) == 4 && (D % 4) == 0) {
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < D; c += 4) {
          const float4 v = *reinterpret_cast<const float4*>(A + r * D + c);
          a[r][c] = dir * v.x;
          a[r][c + 1] = dir * v.y;
          a[r][c + 2] = dir * v.z;
          a[r][c + 3] = dir * v.w;
        }
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) a[r][c] = dir * A[r * D + c];
    }
  }
  __device__ __forceinline__ void gather(const T (&y)[R], T (&yall)[D]) const {
#pragma unroll
    for (int j = 0; j < D; ++j) yall[j] = Grp<G>::bcast(y[j % R], j / R);
  }
  __device__ __forceinline__ void eval(double, const T (&y)[R], T (&f)[R]) const {
    T yall[D];
    gather(y, yall);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if constexpr (sizeof(T) == 8 || D < 8) {
        // FP64: left-to-right sum (the oracle's order); small D: one chain
        T s = T(0);
#pragma unroll
        for (int c = 0; c < D; ++c) s = madd(a[r][c], yall[c], s);
        f[r] = s;
      } else {
        // four partial sums over the columns c = 0, 1, 2, 3 (mod 4), added as
        // (s0 + s1) + (s2 + s3); (s0, s1) and (s2, s3) run as FP32x2 pairs
        // over adjacent columns (each lane rounds as a scalar fused
        // multiply-add: the same bits, half the instructions)
        float2 p01 = make_float2(0.0f, 0.0f), p23 = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int c = 0; c < D; c += 4) {
          p01 = __ffma2_rn(make_float2(a[r][c], a[r][c + 1]), make_float2(yall[c], yall[c + 1]),
                           p01);
          p23 = __ffma2_rn(make_float2(a[r][c + 2], a[r][c + 3]),
                           make_float2(yall[c + 2], yall[c + 3]), p23);
        }
        f[r] = (p01.x + p01.y) + (p23.x + p23.y);
      }
    }
  }
};

}  // namespace tode
