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
// FP32 on the CUDA cores from its recorded stage inputs: a CTA takes eight
// instances at a time, so that every weight it reads (BF16, from global
// memory, warp-per-output dot products forward and thread-per-input column
// sums backward) serves eight instances; a stage's activations are
// recomputed before its transposed sweep instead of kept for all stages.
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

constexpr int TB_NI = 8;  // instances per CTA pass: every weight read serves all of them

// One layer for the NI instances of the pass: out_ii[j] = act(sum_c W[j][c]
// in_ii[c] + b[j]), a warp per output j, its lanes over the inputs c (the
// weight row read once, coalesced, for all NI instances).
__device__ void tb_layer(const __nv_bfloat16* W, const float* b, int Kin, int Nout, bool hidden,
                         const float* in, int in_stride, float* out, int out_stride) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NI = TB_NI, NW = TB_THREADS / 32;
  for (int j = warp; j < Nout; j += NW) {
    float acc[NI];
#pragma unroll
    for (int ii = 0; ii < NI; ++ii) acc[ii] = 0.0f;
    for (int c = lane; c < Kin; c += 32) {
      const float w = __bfloat162float(W[(size_t)j * Kin + c]);
#pragma unroll
      for (int ii = 0; ii < NI; ++ii) acc[ii] = fmaf(w, in[ii * in_stride + c], acc[ii]);
    }
#pragma unroll
    for (int ii = 0; ii < NI; ++ii) {
      const float v = warp_sum(acc[ii]);
      if (lane == 0) {
        const float z = v + (b ? b[j] : 0.0f);
        out[ii * out_stride + j] = hidden ? tanhf(z) : z;
      }
    }
  }
}

// The transposed layer for the NI instances: gout_ii[c] = sum_j W[j][c]
// gin_ii[j] (times 1 - h_ii[c]^2 when h is given), a thread per input c
// (consecutive threads read consecutive weights).
__device__ void tb_layer_t(const __nv_bfloat16* W, int Kin, int Nout, const float* gin,
                           int gin_stride, const float* h, int h_stride, float* gout,
                           int gout_stride) {
  constexpr int NI = TB_NI;
  for (int c = threadIdx.x; c < Kin; c += TB_THREADS) {
    float acc[NI];
#pragma unroll
    for (int ii = 0; ii < NI; ++ii) acc[ii] = 0.0f;
    for (int j = 0; j < Nout; ++j) {
      const float w = __bfloat162float(W[(size_t)j * Kin + c]);
#pragma unroll
      for (int ii = 0; ii < NI; ++ii) acc[ii] = fmaf(w, gin[ii * gin_stride + j], acc[ii]);
    }
#pragma unroll
    for (int ii = 0; ii < NI; ++ii) {
      const float hv = h ? h[ii * h_stride + c] : 0.0f;
      gout[ii * gout_stride + c] = h ? acc[ii] * (1.0f - hv * hv) : acc[ii];
    }
  }
}

// Shared memory: Y, k, kbar [NI][7][D]; three layer buffers [NI][Hmax + D
// + 1]; the activations of one stage [NI][NL-1][Hmax]; then (doubles) the
// hbar and sum_tau <ybar, dy/dt> partials [NI][D] and the time terms [NI].
template <class Tab>
__global__ void __launch_bounds__(TB_THREADS) k_mlp_t_last(MlpTbArgs a) {
  extern __shared__ __align__(16) float sm[];
  constexpr int NI = TB_NI;
  __shared__ double s_tn[NI];
  __shared__ float s_h[NI], s_dir[NI];
  __shared__ int s_N[NI], s_bad[NI], s_live[NI], s_valid[NI];
  __shared__ unsigned long long s_m[NI];
  const int D = a.D, NL = a.NL, Hm = a.Hmax, XW = a.Hmax + a.D + 1, SD = 7 * a.D;
  float* sY = sm;
  float* sk = sY + NI * SD;
  float* skb = sk + NI * SD;
  float* sx = skb + NI * SD;
  float* sg0 = sx + NI * XW;
  float* sg1 = sg0 + NI * XW;
  float* sact = sg1 + NI * XW;
  const int AS = (NL - 1) * Hm;  // one instance's activations of a stage
  double* sPart = reinterpret_cast<double*>(
      (reinterpret_cast<uintptr_t>(sact + NI * AS) + 7) & ~uintptr_t(7));
  double* sT = sPart + NI * D;
  double* sTime = sT + NI * D;
  const int tid = threadIdx.x;

  // the layer inputs [Y_s; t_s] of stage s (0-based) for the pass
  auto stage_input = [&](int s) {
    for (int e = tid; e < NI * D; e += TB_THREADS) {
      const int ii = e / D, r = e % D;
      sx[ii * XW + r] = sY[ii * SD + s * D + r];
    }
    if (tid < NI) {
      const double tau = s_tn[tid] + Tab::c(s + 1) * (double)s_h[tid];
      sx[tid * XW + D] = s_live[tid] ? (float)flip(tau, s_m[tid]) : 0.0f;  // the caller's time
    }
    __syncthreads();
  };

  for (int base = blockIdx.x * NI; base < a.B; base += gridDim.x * NI) {
    if (tid < NI) {
      const int i = base + tid;
      const bool valid = i < a.B;
      const int N = valid ? a.n_acc[i] : 0;
      const bool bad = valid && (a.status[i] != ST_SUCCESS || N > a.slots);
      const bool rev = valid && a.t1[i] < a.t0[i];
      s_valid[tid] = valid;
      s_N[tid] = N;
      s_bad[tid] = bad;
      s_live[tid] = valid && !bad && N > 0;
      s_m[tid] = rev ? SIGN_BIT : 0ULL;
      s_dir[tid] = rev ? -1.0f : 1.0f;
      const size_t o = (size_t)(valid ? i : 0) * a.slots + (N > 0 ? N - 1 : 0);
      s_tn[tid] = s_live[tid] ? a.tp_t[o] : 0.0;  // the solver's time (tau if backward)
      s_h[tid] = s_live[tid] ? a.tp_h[o] : 0.0f;
      sTime[tid] = 0.0;
    }
    __syncthreads();
    for (int e = tid; e < NI * SD; e += TB_THREADS) {
      const int ii = e / SD, s = (e % SD) / D, r = e % D;
      float v = 0.0f;
      if (s_live[ii]) {
        const size_t o = (size_t)(base + ii) * a.slots + (s_N[ii] - 1);
        v = s == 0 ? a.tp_y[o * D + r] : a.tp_ys[(o * 6 + (s - 1)) * D + r];
      }
      sY[e] = v;
    }
    // sum_tau <ybar_tau, dy/dt(tau)> per (instance, component), the forward's dy/dt
    for (int e = tid; e < NI * D; e += TB_THREADS) {
      const int ii = e / D, r = e % D;
      double tp = 0.0;
      if (s_valid[ii] && a.gt0 && a.gye && a.yp)
        for (int q = 0; q < a.K; ++q) {
          const size_t o = ((size_t)(base + ii) * a.K + q) * D + r;
          tp += (double)a.gye[o] * (double)a.yp[o];
        }
      sT[e] = tp;
      sPart[e] = 0.0;
    }
    __syncthreads();
    // k_s = F(tau_s, Y_s) = dir * f(t_s, Y_s) for the 7 stages
    for (int s = 0; s < 7; ++s) {
      stage_input(s);
      float* in = sx;
      for (int l = 0; l < NL; ++l) {
        const bool last = l + 1 == NL;
        float* out = last ? sg0 : (in == sx ? sg1 : sx);
        tb_layer(a.W[l], a.b[l], a.widths[l], a.widths[l + 1], !last, in, XW, out, XW);
        __syncthreads();
        in = out;
      }
      for (int e = tid; e < NI * D; e += TB_THREADS) {
        const int ii = e / D, r = e % D;
        sk[ii * SD + s * D + r] = s_dir[ii] * sg0[ii * XW + r];
      }
      __syncthreads();
    }
    // ybar_N: the final-state cotangent, and the points in (t_{N-1}, t1]
    for (int e = tid; e < NI * D; e += TB_THREADS) {
      const int ii = e / D, r = e % D;
      if (!s_live[ii]) continue;
      const int i = base + ii;
      const float* k = sk + ii * SD;
      float* kb = skb + ii * SD;
      const double tn = s_tn[ii];
      const float h = s_h[ii];
      double part = 0.0;
      const float yb = a.gyf ? a.gyf[(size_t)i * D + r] : 0.0f;
      float sb = 0.0f;
      for (int s = 0; s < 7; ++s) sb = fmaf((float)Tab::b(s + 1), k[s * D + r], sb);
      part += (double)yb * (double)sb;
      for (int s = 0; s < 7; ++s) kb[s * D + r] = h * (float)Tab::b(s + 1) * yb;
      const long long kt = tkey(tn), kn = tkey(flip(a.t1[i], s_m[ii]));
      if (a.gye)
        for (int q = a.K - 1; q >= 0; --q) {
          const double tq = flip(a.te[(size_t)i * a.K + q], s_m[ii]);
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
            sw = fmaf(w[s], k[s * D + r], sw);
            dv = fmaf(wd[s], k[s * D + r], dv);
          }
          const float gq = a.gye[((size_t)i * a.K + q) * D + r];
          part += (double)gq * ((double)sw - (double)th * (double)dv);
          for (int s = 0; s < 7; ++s) kb[s * D + r] = fmaf(h * w[s], gq, kb[s * D + r]);
        }
      sPart[e] += part;
    }
    __syncthreads();
    // reverse stage sweep, stages 7..2: the stage's activations again, then
    // g_s = J^T kbar_s through the network
    for (int s = 6; s >= 1; --s) {
      stage_input(s);
      for (int l = 0; l + 1 < NL; ++l) {
        const float* in = l == 0 ? sx : sact + (l - 1) * Hm;
        const int ins = l == 0 ? XW : AS;
        tb_layer(a.W[l], a.b[l], a.widths[l], a.widths[l + 1], true, in, ins, sact + l * Hm, AS);
        __syncthreads();
      }
      // cotangent of the network's output: dir * kbar_s (F = dir f)
      for (int e = tid; e < NI * D; e += TB_THREADS) {
        const int ii = e / D, r = e % D;
        sg0[ii * XW + r] = s_dir[ii] * skb[ii * SD + s * D + r];
      }
      __syncthreads();
      float* gin = sg0;
      float* gout = sg1;
      for (int l = NL - 1; l >= 0; --l) {
        const float* hl = l > 0 ? sact + (l - 1) * Hm : nullptr;
        tb_layer_t(a.W[l], a.widths[l], a.widths[l + 1], gin, XW, hl, AS, gout, XW);
        __syncthreads();
        float* t = gin;
        gin = gout;
        gout = t;
      }
      // gin = [g_y (D); g_t]: the state's and the time input's cotangents
      if (tid < NI && s_live[tid])
        sTime[tid] += (double)Tab::c(s + 1) * (double)s_dir[tid] * (double)gin[tid * XW + D];
      for (int e = tid; e < NI * D; e += TB_THREADS) {
        const int ii = e / D, r = e % D;
        if (!s_live[ii]) continue;
        const float* k = sk + ii * SD;
        float* kb = skb + ii * SD;
        const float h = s_h[ii];
        const float g = gin[ii * XW + r];
        float sa = 0.0f;
        for (int l = 0; l < s; ++l) sa = fmaf((float)Tab::a(s + 1, l + 1), k[l * D + r], sa);
        sPart[e] += (double)g * (double)sa;
        for (int l = 0; l < s; ++l)
          kb[l * D + r] = fmaf(h * (float)Tab::a(s + 1, l + 1), g, kb[l * D + r]);
      }
      __syncthreads();
    }
    if (tid < NI && s_valid[tid]) {
      const int i = base + tid;
      double hbar = sTime[tid], tsum = 0.0;
      for (int r = 0; r < D; ++r) {  // the components in a fixed order
        hbar += sPart[tid * D + r];
        tsum += sT[tid * D + r];
      }
      const double nan = __longlong_as_double(0x7ff8000000000000LL);
      const bool bad = s_bad[tid];
      const double g1 = bad ? nan : (s_N[tid] > 0 ? (double)s_dir[tid] * hbar : 0.0);
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
  const size_t D = (size_t)f->D, NI = TB_NI;
  return sizeof(float) * (NI * 21 * D + 3 * NI * ((size_t)hm + D + 1) +
                          NI * (size_t)(f->n_layers - 1) * hm) +
         8 + sizeof(double) * (2 * NI * D + NI);
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
  const int passes = (r.B + TB_NI - 1) / TB_NI;
  const int grid = std::min(passes, std::max(1, r.num_sms) * 2);
  if (r.o->method == TODE_TSIT5)
    k_mlp_t_last<TS5><<<grid, TB_THREADS, smem, r.stream>>>(a);
  else
    k_mlp_t_last<DP5><<<grid, TB_THREADS, smem, r.stream>>>(a);
  TODE_CUDA_TRY(cudaGetLastError());
  return TODE_OK;
}

}  // namespace tode
