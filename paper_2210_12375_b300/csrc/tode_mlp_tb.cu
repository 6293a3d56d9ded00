// tode_mlp_tb.cu -- gradients with respect to t0 and t1 for the MLP field
//   f(t, y) = W_L tanh( ... tanh(W_1 [y; t] + b_1) ... ) + b_L
// on the frozen map of a solve (every accepted step size but the last held,
// every evaluation point in its step; t0 translates the mesh points before
// t1 and the last step h = t1 - t_{N-1} absorbs the change).
//
//   dL/dt1 = hbar, the cotangent of the last step size:
//     hbar = <ybar_N, sum_i b_i k_i>
//          + sum_tau <ybar_tau, sum_i (b_i(theta) - theta b_i'(theta)) k_i>
//          + sum_i <g_i, sum_j a_ij k_j> + sum_i c_i <kbar_i, df/dt(Y_i)>
//   (the last term because the field sees its stage times t_n + c_i h);
//   dL/dt0 = S_t - dL/dt1 - sum_tau <ybar_tau, dy/dt(tau)>,
// where S_t, the derivative of L when every time of the instance (t0, t1 and
// the evaluation points) moves together, is the sum over all reversed stages
// of the time input's cotangent -- the tensor-core adjoint accumulates it
// (tode_adjoint's gparam for this field).  The last step is re-run here in
// FP32 on the CUDA cores from its recorded stage inputs: one CTA per
// instance, the network's layers as warp-per-output dot products (forward)
// and thread-per-input column sums (backward) over the BF16 weights read
// from global memory, the stage activations kept in shared memory.
// Backward instances run in tau = -t with the field -f(-tau, y) as the
// solver ran them: hbar is dL/dtau1 there, and dL/dt1 = -hbar.  The pair
// (dopri5 or tsit5) is the one the solve used.
#include <cuda_bf16.h>

#include <algorithm>

#include "tode_core.cuh"
#include "tode_internal.h"

namespace tode {
namespace {

constexpr int TB_THREADS = 256;

struct MlpTbArgs {
  int B, K, D, NL, Hmax;
  int widths[MLP_MAX_LAYERS + 1];
  const __nv_bfloat16* W[MLP_MAX_LAYERS];
  const float* b[MLP_MAX_LAYERS];
  const double* t0;
  const double* t1;
  const double* te;
  const int32_t* n_acc;
  const int32_t* status;
  int slots;
  const float* tp_y;
  const double* tp_t;
  const float* tp_h;
  const float* tp_ys;  // [B][slots][6][D]
  const float* gye;    // [B][K][D] or NULL
  const float* gyf;    // [B][D] or NULL
  const float* yp;     // [B][K][D] or NULL
  double* gt0;         // [B] or NULL: S_t on entry, dL/dt0 on exit
  double* gt1;         // [B]
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum over the CTA of one value per thread (every thread gets it)
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < TB_THREADS / 32; ++w) s += red[w];
  return s;
}

// Shared memory (floats): Y[7][D], k[7][D], kb[7][D], x[Hmax + D + 1],
// g0[Hmax + D + 1], g1[Hmax + D + 1], act[7][NL-1][Hmax], then 8 doubles.
template <class Tab>
__global__ void __launch_bounds__(TB_THREADS) k_mlp_t_last(MlpTbArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int D = a.D, NL = a.NL, Hm = a.Hmax, XW = a.Hmax + a.D + 1;
  float* sY = sm;
  float* sk = sY + 7 * D;
  float* skb = sk + 7 * D;
  float* sx = skb + 7 * D;
  float* sg0 = sx + XW;
  float* sg1 = sg0 + XW;
  float* sact = sg1 + XW;
  double* red = reinterpret_cast<double*>(sact + 7 * (NL - 1) * Hm + 1);
  red = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(red) + 7) & ~uintptr_t(7));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = TB_THREADS / 32;

  for (int i = blockIdx.x; i < a.B; i += gridDim.x) {
    const int N = a.n_acc[i];
    const bool bad = a.status[i] != ST_SUCCESS || N > a.slots;
    const bool rev = a.t1[i] < a.t0[i];
    const unsigned long long m = rev ? SIGN_BIT : 0ULL;
    const float dir = rev ? -1.0f : 1.0f;
    // sum_tau <ybar_tau, dy/dt(tau)> over every point (the forward's dy/dt)
    double tpart = 0.0;
    if (a.gt0 && a.gye && a.yp)
      for (int e = tid; e < a.K * D; e += TB_THREADS) {
        const size_t o = (size_t)i * a.K * D + e;
        tpart += (double)a.gye[o] * (double)a.yp[o];
      }
    const double tsum = block_sum(tpart, red);
    double part = 0.0;  // this thread's share of hbar
    if (!bad && N > 0) {
      const size_t o = (size_t)i * a.slots + (N - 1);
      const double tn = a.tp_t[o];  // the solver's time (tau for a backward row)
      const float h = a.tp_h[o];
      for (int e = tid; e < 7 * D; e += TB_THREADS) {
        const int s = e / D, r = e % D;
        sY[e] = s == 0 ? a.tp_y[o * D + r] : a.tp_ys[(o * 6 + (s - 1)) * D + r];
      }
      __syncthreads();
      // k_s = F(tau_s, Y_s) = dir * f(t_s, Y_s), the hidden activations kept
      for (int s = 0; s < 7; ++s) {
        const double tau = tn + Tab::c(s + 1) * (double)h;
        for (int e = tid; e < D; e += TB_THREADS) sx[e] = sY[s * D + e];
        if (tid == 0) sx[D] = (float)flip(tau, m);  // the network sees the caller's time
        __syncthreads();
        for (int l = 0; l < NL; ++l) {
          const int Kin = a.widths[l], Nout = a.widths[l + 1];
          const __nv_bfloat16* W = a.W[l];
          float* dst = l + 1 < NL ? sact + ((size_t)s * (NL - 1) + l) * Hm : sg0;
          for (int j = warp; j < Nout; j += NW) {
            float acc = 0.0f;
            for (int c = lane; c < Kin; c += 32)
              acc = fmaf(__bfloat162float(W[(size_t)j * Kin + c]), sx[c], acc);
            acc = warp_sum(acc);
            if (lane == 0) {
              const float z = acc + (a.b[l] ? a.b[l][j] : 0.0f);
              dst[j] = l + 1 < NL ? tanhf(z) : z;
            }
          }
          __syncthreads();
          if (l + 1 < NL) {
            for (int e = tid; e < Nout; e += TB_THREADS) sx[e] = dst[e];
            __syncthreads();
          }
        }
        for (int e = tid; e < D; e += TB_THREADS) sk[s * D + e] = dir * sg0[e];
        __syncthreads();
      }
      // ybar_N: the final-state cotangent, and the points in (t_{N-1}, t1]
      const long long kt = tkey(tn), kn = tkey(flip(a.t1[i], m));
      for (int r = tid; r < D; r += TB_THREADS) {
        const float yb = a.gyf ? a.gyf[(size_t)i * D + r] : 0.0f;
        float sb = 0.0f;
        for (int s = 0; s < 7; ++s) sb = fmaf((float)Tab::b(s + 1), sk[s * D + r], sb);
        part += (double)yb * (double)sb;
        for (int s = 0; s < 7; ++s) skb[s * D + r] = h * (float)Tab::b(s + 1) * yb;
        if (a.gye)
          for (int q = a.K - 1; q >= 0; --q) {
            const double tq = flip(a.te[(size_t)i * a.K + q], m);
            const long long kq = tkey(tq);
            if (!(kq > kt)) break;
            const float th = kq == kn ? 1.0f : float(tq - tn) / h;
            float w[7], wd[7];
            if (kq == kn) {
              for (int s = 0; s < 7; ++s) w[s] = (float)Tab::b(s + 1);
            } else {
              dense_weights<Tab, float>(th, w);
            }
            dense_dweights<Tab, float>(th, wd);
            float sw = 0.0f, dv = 0.0f;
            for (int s = 0; s < 7; ++s) {
              sw = fmaf(w[s], sk[s * D + r], sw);
              dv = fmaf(wd[s], sk[s * D + r], dv);
            }
            const float gq = a.gye[((size_t)i * a.K + q) * D + r];
            part += (double)gq * ((double)sw - (double)th * (double)dv);
            for (int s = 0; s < 7; ++s) skb[s * D + r] = fmaf(h * w[s], gq, skb[s * D + r]);
          }
      }
      __syncthreads();
      // reverse stage sweep, stages 7..2: g_s = J^T kbar_s through the network
      for (int s = 6; s >= 1; --s) {
        // cotangent of the network's output: dir * kbar_s (F = dir f)
        for (int e = tid; e < D; e += TB_THREADS) sg0[e] = dir * skb[s * D + e];
        __syncthreads();
        float* gin = sg0;
        float* gout = sg1;
        for (int l = NL - 1; l >= 0; --l) {
          const int Kin = a.widths[l], Nout = a.widths[l + 1];
          const __nv_bfloat16* W = a.W[l];
          const float* hl = l > 0 ? sact + ((size_t)s * (NL - 1) + (l - 1)) * Hm : nullptr;
          for (int c = tid; c < Kin; c += TB_THREADS) {
            float acc = 0.0f;
            for (int j = 0; j < Nout; ++j)
              acc = fmaf(__bfloat162float(W[(size_t)j * Kin + c]), gin[j], acc);
            gout[c] = hl ? acc * (1.0f - hl[c] * hl[c]) : acc;
          }
          __syncthreads();
          float* t = gin;
          gin = gout;
          gout = t;
        }
        // gin = [g_y (D); g_t]: the state's and the time input's cotangents
        if (tid == 0) part += (double)Tab::c(s + 1) * (double)dir * (double)gin[D];
        for (int r = tid; r < D; r += TB_THREADS) {
          const float g = gin[r];
          float sa = 0.0f;
          for (int l = 0; l < s; ++l) sa = fmaf((float)Tab::a(s + 1, l + 1), sk[l * D + r], sa);
          part += (double)g * (double)sa;
          for (int l = 0; l < s; ++l)
            skb[l * D + r] = fmaf(h * (float)Tab::a(s + 1, l + 1), g, skb[l * D + r]);
        }
        __syncthreads();
      }
    }
    const double hbar = block_sum(part, red);
    if (tid == 0) {
      const double nan = __longlong_as_double(0x7ff8000000000000LL);
      const double g1 = bad ? nan : (N > 0 ? (rev ? -hbar : hbar) : 0.0);
      a.gt1[i] = g1;
      if (a.gt0) a.gt0[i] = bad ? nan : a.gt0[i] - g1 - tsum;
    }
    __syncthreads();
  }
}

}  // namespace

size_t mlp_t_bounds_smem(const tode_field_desc* f) {
  int hm = 1;
  for (int l = 1; l < f->n_layers; ++l) hm = hm > f->widths[l] ? hm : f->widths[l];
  const int D = f->D;
  return sizeof(float) * ((size_t)21 * D + 3 * ((size_t)hm + D + 1) +
                          (size_t)7 * (f->n_layers - 1) * hm + 1) +
         16 + 8 * sizeof(double);
}

tode_err mlp_t_bounds(const AdjReq& r, const void* yp, double* gt0, double* gt1) {
  const tode_field_desc* f = r.f;
  if (f->n_layers < 2 || f->n_layers > MLP_MAX_LAYERS) return TODE_EUNSUPPORTED;
  MlpTbArgs a{};
  a.B = r.B;
  a.K = r.K;
  a.D = r.D;
  a.NL = f->n_layers;
  int hm = 1;
  for (int l = 0; l <= f->n_layers; ++l) a.widths[l] = f->widths[l];
  for (int l = 1; l < f->n_layers; ++l) hm = hm > f->widths[l] ? hm : f->widths[l];
  a.Hmax = hm;
  for (int l = 0; l < f->n_layers; ++l) {
    a.W[l] = (const __nv_bfloat16*)f->W[l];
    a.b[l] = f->b ? f->b[l] : nullptr;
  }
  a.t0 = r.t0;
  a.t1 = r.t1;
  a.te = r.te;
  a.n_acc = r.n_acc;
  a.status = r.status;
  a.slots = r.tape->slots;
  a.tp_y = (const float*)r.tape->y;
  a.tp_t = r.tape->t;
  a.tp_h = (const float*)r.tape->h_acc;
  a.tp_ys = (const float*)r.tape->y_stage;
  a.gye = r.K > 0 ? (const float*)r.gye : nullptr;
  a.gyf = (const float*)r.gyf;
  a.yp = r.K > 0 ? (const float*)yp : nullptr;
  a.gt0 = gt0;
  a.gt1 = gt1;
  const size_t smem = mlp_t_bounds_smem(f);
  if (smem > 227 * 1024) return TODE_EUNSUPPORTED;
  const void* kern = r.o->method == TODE_TSIT5 ? (const void*)k_mlp_t_last<TS5>
                                                : (const void*)k_mlp_t_last<DP5>;
  TODE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = std::min(r.B, std::max(1, r.num_sms) * 4);
  if (r.o->method == TODE_TSIT5)
    k_mlp_t_last<TS5><<<grid, TB_THREADS, smem, r.stream>>>(a);
  else
    k_mlp_t_last<DP5><<<grid, TB_THREADS, smem, r.stream>>>(a);
  TODE_CUDA_TRY(cudaGetLastError());
  return TODE_OK;
}

}  // namespace tode
