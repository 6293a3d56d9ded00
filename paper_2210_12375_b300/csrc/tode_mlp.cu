// tode_mlp.cu -- batched adaptive dopri5 with the MLP field
//   f(t, y) = W_L tanh( ... tanh(W_1 [y; t] + b_1) ... ) + b_L
// evaluated on the tensor cores (tcgen05.mma, BF16 operands, FP32 accumulation
// in tensor memory), FP32 state, FP64 time.
//
// One CTA owns a tile of 128 rows; every row is an independent instance with
// its own t, h, accept/reject decisions and evaluation points (torchode
// Sec. 3).  Rows couple only through the field evaluation, which is one GEMM
// chain for the whole tile, so the CTA advances in rounds: every round each
// row contributes one input [Y; t] and receives f(t, Y).  A row runs its own
// phase machine on top of that (two evaluations of the starting-step
// heuristic, then stages 2..7 of each attempt, FSAL k1 reused); when its
// instance finishes it takes the next one from the global queue, so a
// finished row never waits for the rest of its tile (work stealing at row
// granularity).
//
// Threads: 256 per CTA, two per row (threads r and r + 128 share TMEM lane r
// and each owns D/2 state components and H/2 hidden columns).  Shared memory
// holds the weights (loaded once by bulk copy from a core-matrix image that
// k_mlp_weight_image builds), the BF16 input tile and the BF16 hidden tile.
// The input [Y; t] is always split into two BF16 terms (hi + lo, two MMAs
// into the same accumulator), so the state enters the field with ~16
// significant bits; hidden activations are split too when SPLIT is set, with
// tanh from exp (hi/lo resolution), else rounded to BF16 with tanh.approx.
#include "tode_core.cuh"
#include "tode_internal.h"
#include "tode_tc.cuh"

#include <cuda_bf16.h>

namespace tode {

constexpr int MLP_MAX_LAYERS = 4;

struct MlpArgs {
  int B, K;
  const float* y0;
  const double* t0;
  const double* t1;
  const double* te;
  const double* rtol_b;
  const double* atol_b;
  double rtol, atol;
  float* ye;
  float* yf;
  int32_t *n_acc, *n_rej, *n_fe, *status;
  SolveOpts o;
  TraceDev trace;
  const unsigned char* wimg;  // core-matrix images of all layers, back to back
  const float* bias[MLP_MAX_LAYERS];
  int32_t* counter;
  int32_t* err;
};

template <int D_, int H_, int NL_, bool SPLIT_> struct MlpCfg {
  static constexpr int D = D_, H = H_, NL = NL_;
  static constexpr bool SPLIT = SPLIT_;
  static constexpr int K0 = ((D + 1 + 15) / 16) * 16;  // [y; t] padded to 16
  static constexpr int C = D / 2;                        // state components per thread
  static constexpr int HC = H / 2;                       // hidden columns per thread
  static constexpr int TMEM_COLS = (H + D <= 256) ? 256 : 512;
  static constexpr int ACC_COL = 0, OUT_COL = H;
  // layer l: N_l x K_l
  __host__ __device__ static constexpr int N_of(int l) { return l == NL - 1 ? D : H; }
  __host__ __device__ static constexpr int K_of(int l) { return l == 0 ? K0 : H; }
  __host__ __device__ static constexpr int W_bytes(int l) { return N_of(l) * K_of(l) * 2; }
  __host__ __device__ static constexpr int W_off(int l) {
    int o = 0;
    for (int j = 0; j < l; ++j) o += W_bytes(j);
    return o;
  }
  static constexpr int WIMG_BYTES = W_off(NL);
  static constexpr int BIAS_FLOATS = (NL - 1) * H + D;
  // shared-memory carve (bytes)
  static constexpr int S_W = 0;
  static constexpr int S_XH = S_W + ((WIMG_BYTES + 1023) / 1024) * 1024;
  static constexpr int S_XL = S_XH + 128 * K0 * 2;
  static constexpr int S_HH = S_XL + 128 * K0 * 2;
  static constexpr int S_HL = S_HH + 128 * H * 2;
  static constexpr int S_BIAS = S_HL + (SPLIT ? 128 * H * 2 : 0);
  static constexpr int S_RED = S_BIAS + BIAS_FLOATS * 4;
  static constexpr int S_FIN = S_RED + 2 * 128 * 2 * 4;
  static constexpr int S_NXT = S_FIN + 2 * 128 * 4;
  static constexpr int S_END = S_NXT + 128 * 4;
  static_assert(D % 32 == 0 && H % 32 == 0 && NL >= 2 && NL <= MLP_MAX_LAYERS, "shape");
  static_assert(H <= 256 && D <= 256, "one MMA per layer and K slice");
};

enum : int { PH_IDLE = 0, PH_INIT0 = 1, PH_INIT1 = 2, PH_STAGE = 3 };  // PH_STAGE + s - 2

__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// tanh(x) = sign(x) (1 - e) / (1 + e), e = exp(-2|x|); absolute error ~1e-7
__device__ __forceinline__ float tanh_acc(float x) {
  const float e = __expf(-2.0f * fabsf(x));
  return copysignf(__fdividef(1.0f - e, 1.0f + e), x);
}

// Stores 16 consecutive values of a row as BF16 (hi, and lo = x - hi) into
// core-matrix tiles with K columns, starting at column k0 (a multiple of 8).
template <bool LO>
__device__ __forceinline__ void store_row16(unsigned char* th, unsigned char* tl, int row, int k0,
                                            int K, const float (&v)[16]) {
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float a = v[c * 8 + 2 * j], b = v[c * 8 + 2 * j + 1];
      const __nv_bfloat162 h2 = __floats2bfloat162_rn(a, b);
      hw[j] = *reinterpret_cast<const uint32_t*>(&h2);
      if (LO) {
        const __nv_bfloat162 l2 =
            __floats2bfloat162_rn(a - __low2float(h2), b - __high2float(h2));
        lw[j] = *reinterpret_cast<const uint32_t*>(&l2);
      }
    }
    const uint32_t off = tc::cm_offset(row, k0 + 8 * c, K);
    *reinterpret_cast<uint4*>(th + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    if (LO) *reinterpret_cast<uint4*>(tl + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
}

// Per-row solver state (identical scalars in both threads of the row).
struct MlpRow {
  int inst, phase, cursor, status, flags, n_acc, n_rej;
  double t, t0, t1;
  float h, h0h, err_prev, rtol, atol, rem, hmin;
  bool last;
};

template <class Cfg>
__global__ void __launch_bounds__(256, 1) k_mlp_fused(MlpArgs a) {
  constexpr int D = Cfg::D, H = Cfg::H, NL = Cfg::NL, K0 = Cfg::K0, C = Cfg::C;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar_mma, mbar_w;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  unsigned char* sW = sm + Cfg::S_W;
  unsigned char* sXh = sm + Cfg::S_XH;
  unsigned char* sXl = sm + Cfg::S_XL;
  unsigned char* sHh = sm + Cfg::S_HH;
  unsigned char* sHl = sm + Cfg::S_HL;
  float* sBias = reinterpret_cast<float*>(sm + Cfg::S_BIAS);
  float* sRed = reinterpret_cast<float*>(sm + Cfg::S_RED);  // [half][row][2]
  int* sFin = reinterpret_cast<int*>(sm + Cfg::S_FIN);      // [half][row]
  int* sNxt = reinterpret_cast<int*>(sm + Cfg::S_NXT);      // [row]

  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & 127, half = tid >> 7;
  const int coff = half * C;  // first state component of this thread
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;

  // ---- set-up: barriers, weights (bulk copy), biases, tensor memory
  if (tid == 0) {
    tc::mbar_init(&mbar_mma, 1);
    tc::mbar_init(&mbar_w, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    tc::mbar_expect_tx(&mbar_w, (uint32_t)Cfg::WIMG_BYTES);
#pragma unroll
    for (int l = 0; l < NL; ++l)
      tc::bulk_g2s(sW + Cfg::W_off(l), a.wimg + Cfg::W_off(l), (uint32_t)Cfg::W_bytes(l), &mbar_w);
  }
  {
    int o = 0;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const int n = Cfg::N_of(l);
      for (int j = tid; j < n; j += 256) sBias[o + j] = a.bias[l] ? a.bias[l][j] : 0.0f;
      o += n;
    }
  }
  // zero the input tiles once (padding columns stay zero)
  for (int j = tid; j < 128 * K0 * 2 / 16; j += 256) {
    reinterpret_cast<uint4*>(sXh)[j] = make_uint4(0, 0, 0, 0);
    reinterpret_cast<uint4*>(sXl)[j] = make_uint4(0, 0, 0, 0);
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base_s, Cfg::TMEM_COLS);
    tc::tmem_relinquish();
  }
  const bool w_ok = tc::mbar_wait(&mbar_w, 0);
  if (!w_ok) atomicExch(&abort_s, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_base_s;
  uint32_t mma_parity = 0;

  MlpRow s;
  s.inst = -1;
  s.phase = PH_IDLE;
  float y[C], ylo[C], k[7][C];
#pragma unroll
  for (int r = 0; r < C; ++r) {
    y[r] = ylo[r] = 0.0f;
#pragma unroll
    for (int j = 0; j < 7; ++j) k[j][r] = 0.0f;
  }
  bool need_grab = true;

  while (true) {
    // ---- hand out instances to rows that need one (one atomic per row)
    if (need_grab && half == 0) sNxt[row] = atomicAdd(a.counter, 1);
    __syncthreads();
    if (need_grab) {
      need_grab = false;
      const int i = sNxt[row];
      if (i >= a.B) {
        s.phase = PH_IDLE;
        s.inst = -1;
      } else {
        // load and validate the instance (Sec. 3: per-instance bounds / points)
        s.inst = i;
        s.t0 = a.t0[i];
        s.t1 = a.t1[i];
        s.t = s.t0;
        s.rtol = (float)(a.rtol_b ? a.rtol_b[i] : a.rtol);
        s.atol = (float)(a.atol_b ? a.atol_b[i] : a.atol);
        s.n_acc = s.n_rej = 0;
        s.cursor = 0;
        s.flags = 0;
        s.err_prev = 1.0f;
        s.h = s.h0h = 0.0f;
        s.last = false;
        s.status = ST_RUNNING;
#pragma unroll
        for (int r = 0; r < C; ++r) {
          y[r] = a.y0[(size_t)i * D + coff + r];
          ylo[r] = 0.0f;
        }
        const double* te = a.te + (size_t)i * a.K;
        bool ok = tfinite(s.t0) && tfinite(s.t1) && !(s.t1 < s.t0);
        const long long k0 = tkey(s.t0), k1 = tkey(s.t1);
        long long kprev = k0;
        for (int q = 0; q < a.K && ok; ++q) {
          const long long kv = tkey(te[q]);
          ok = tfinite(te[q]) && kv >= kprev && kv <= k1;
          kprev = kv;
        }
        float* ye = a.ye + (size_t)i * a.K * D + coff;
        bool done = false;
        if (!ok) {
          s.status = ST_INVALID;
          for (int q = 0; q < a.K; ++q)
#pragma unroll
            for (int r = 0; r < C; ++r) ye[(size_t)q * D + r] = nan_(0.0f);
          done = true;
        } else {
          while (s.cursor < a.K && tkey(te[s.cursor]) == k0) {
#pragma unroll
            for (int r = 0; r < C; ++r) ye[(size_t)s.cursor * D + r] = y[r];
            s.cursor++;
          }
          if (k1 == k0) {
            s.status = ST_SUCCESS;
            done = true;
          } else {
            s.rem = __double2float_rd(s.t1 - s.t0);
            s.hmin = (float)(1e-14 * tmax(fabs(s.t0), fabs(s.t1)));
            s.phase = PH_INIT0;
          }
        }
        if (done) {
          // finalize immediately, take another instance next round
#pragma unroll
          for (int r = 0; r < C; ++r)
            a.yf[(size_t)i * D + coff + r] = s.status == ST_INVALID ? nan_(0.0f) : y[r];
          if (half == 0) {
            a.n_acc[i] = a.n_rej[i] = a.n_fe[i] = 0;
            a.status[i] = s.status;
            if (a.trace.cap > 0) a.trace.len[i] = 0;
          }
          s.phase = PH_IDLE;
          need_grab = true;
        }
      }
    }
    // all rows idle and the queue exhausted -> done
    const bool any_work = __syncthreads_or(s.phase != PH_IDLE || need_grab) != 0;
    if (!any_work || abort_s) break;
    if (__syncthreads_or(need_grab && s.phase == PH_IDLE && s.inst >= 0) != 0) {
      // some row finished without work this round: refill first
      continue;
    }

    // ---- this row's field input [Y; t] for the round
    using Cc = DP5;
    float Y[16];
    float tin = 0.0f;
    const int stage = s.phase - PH_STAGE + 2;  // 2..7 in stage phases
    if (s.phase == PH_INIT0 || s.phase == PH_IDLE) {
#pragma unroll
      for (int r = 0; r < C; ++r) Y[r] = y[r];
      tin = (float)s.t;
    } else if (s.phase == PH_INIT1) {
#pragma unroll
      for (int r = 0; r < C; ++r) Y[r] = madd(s.h0h, k[0][r], y[r]);
      tin = (float)(s.t + (double)s.h0h);
    } else {
      if (stage == 2) {  // a new attempt starts: clip at t1
        float h = s.h;
        s.last = false;
        if (h >= s.rem) {
          h = s.rem;
          s.last = true;
        }
        s.h = h;
      }
      const float h = s.h;
      double cs = 0.0;
#pragma unroll
      for (int r = 0; r < C; ++r) {
        float acc;
        switch (stage) {
          case 2:
            acc = float(Cc::a21) * k[0][r];
            break;
          case 3:
            acc = float(Cc::a31) * k[0][r];
            acc = madd(float(Cc::a32), k[1][r], acc);
            break;
          case 4:
            acc = float(Cc::a41) * k[0][r];
            acc = madd(float(Cc::a42), k[1][r], acc);
            acc = madd(float(Cc::a43), k[2][r], acc);
            break;
          case 5:
            acc = float(Cc::a51) * k[0][r];
            acc = madd(float(Cc::a52), k[1][r], acc);
            acc = madd(float(Cc::a53), k[2][r], acc);
            acc = madd(float(Cc::a54), k[3][r], acc);
            break;
          case 6:
            acc = float(Cc::a61) * k[0][r];
            acc = madd(float(Cc::a62), k[1][r], acc);
            acc = madd(float(Cc::a63), k[2][r], acc);
            acc = madd(float(Cc::a64), k[3][r], acc);
            acc = madd(float(Cc::a65), k[4][r], acc);
            break;
          default:  // 7: the new solution (SSAL)
            acc = float(Cc::b1) * k[0][r];
            acc = madd(float(Cc::b3), k[2][r], acc);
            acc = madd(float(Cc::b4), k[3][r], acc);
            acc = madd(float(Cc::b5), k[4][r], acc);
            acc = madd(float(Cc::b6), k[5][r], acc);
            break;
        }
        Y[r] = (stage == 7) ? y[r] + h * acc : madd(h, acc, y[r]);
      }
      switch (stage) {
        case 2: cs = Cc::c2; break;
        case 3: cs = Cc::c3; break;
        case 4: cs = Cc::c4; break;
        case 5: cs = Cc::c5; break;
        default: cs = 1.0; break;
      }
      tin = (float)(s.t + cs * (double)h);
    }
    store_row16<true>(sXh, sXl, row, coff, K0, Y);
    if (half == 1) {  // the time input, hi + lo, in column D
      const __nv_bfloat16 th = __float2bfloat16_rn(tin);
      const __nv_bfloat16 tl = __float2bfloat16_rn(tin - __bfloat162float(th));
      *reinterpret_cast<__nv_bfloat16*>(sXh + tc::cm_offset(row, D, K0)) = th;
      *reinterpret_cast<__nv_bfloat16*>(sXl + tc::cm_offset(row, D, K0)) = tl;
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    // ---- the GEMM chain: hidden layers, then the output layer
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const int Kl = Cfg::K_of(l), Nl = Cfg::N_of(l);
      const uint32_t dcol = (l == NL - 1) ? Cfg::OUT_COL : Cfg::ACC_COL;
      if (tid == 0) {
        const uint32_t idesc = tc::idesc_bf16_f32(128, Nl);
        const uint32_t wa = tc::smem_u32(sW + Cfg::W_off(l));
        const uint32_t ah = tc::smem_u32(l == 0 ? sXh : sHh);
        const uint32_t al = tc::smem_u32(l == 0 ? sXl : sHl);
        const bool lo = (l == 0) || Cfg::SPLIT;
        for (int kk = 0; kk < Kl / 16; ++kk) {
          const uint64_t db = tc::smem_desc(wa + kk * 256, 128, Kl * 16);
          tc::mma_bf16(tbase + dcol, tc::smem_desc(ah + kk * 256, 128, Kl * 16), db, idesc,
                       kk > 0);
          if (lo)
            tc::mma_bf16(tbase + dcol, tc::smem_desc(al + kk * 256, 128, Kl * 16), db, idesc,
                         true);
        }
        tc::mma_commit(&mbar_mma);
      }
      const bool ok = tc::mbar_wait(&mbar_mma, mma_parity);
      mma_parity ^= 1u;
      if (!ok) atomicExch(&abort_s, 1);
      tc::fence_after_sync();
      if (l < NL - 1) {
        // hidden epilogue: bias, tanh, BF16 (split) into the hidden tile
        const float* bl = sBias + l * H;
#pragma unroll
        for (int c = 0; c < Cfg::HC; c += 16) {
          const int col = half * Cfg::HC + c;
          float v[16];
          tc::tmem_ld16(tbase + lane_base + Cfg::ACC_COL + col, v);
          tc::tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float z = v[j] + bl[col + j];
            v[j] = Cfg::SPLIT ? tanh_acc(z) : tanh_fast(z);
          }
          store_row16<Cfg::SPLIT>(sHh, sHl, row, col, H, v);
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
      }
    }
    // ---- output: f for this thread's components
    float f[16];
    {
      float v[16];
      tc::tmem_ld16(tbase + lane_base + Cfg::OUT_COL + coff, v);
      tc::tmem_wait_ld();
      const float* bo = sBias + (NL - 1) * H;
#pragma unroll
      for (int r = 0; r < C; ++r) f[r] = v[r] + bo[coff + r];
    }

    // ---- consume: partial sums of this thread's components
    float p0 = 0.0f, p1 = 0.0f;
    int fin = 1;
    float inc[16];
    if (s.phase == PH_INIT0) {
#pragma unroll
      for (int r = 0; r < C; ++r) {
        k[0][r] = f[r];
        const float sc = madd(s.rtol, fabsf(y[r]), s.atol);
        const float q0 = y[r] / sc, q1 = f[r] / sc;
        p0 = madd(q0, q0, p0);
        p1 = madd(q1, q1, p1);
      }
    } else if (s.phase == PH_INIT1) {
#pragma unroll
      for (int r = 0; r < C; ++r) {
        const float sc = madd(s.rtol, fabsf(y[r]), s.atol);
        const float q = (f[r] - k[0][r]) / sc;
        p0 = madd(q, q, p0);
      }
    } else if (s.phase >= PH_STAGE) {
#pragma unroll
      for (int j = 1; j < 7; ++j)
        if (j == stage - 1) {
#pragma unroll
          for (int r = 0; r < C; ++r) k[j][r] = f[r];
        }
      if (stage == 7) {
#pragma unroll
        for (int r = 0; r < C; ++r) {
          float acc = float(Cc::b1) * k[0][r];
          acc = madd(float(Cc::b3), k[2][r], acc);
          acc = madd(float(Cc::b4), k[3][r], acc);
          acc = madd(float(Cc::b5), k[4][r], acc);
          acc = madd(float(Cc::b6), k[5][r], acc);
          inc[r] = s.h * acc;
          const float y1 = y[r] + inc[r];
          float e = float(Cc::e1) * k[0][r];
          e = madd(float(Cc::e3), k[2][r], e);
          e = madd(float(Cc::e4), k[3][r], e);
          e = madd(float(Cc::e5), k[4][r], e);
          e = madd(float(Cc::e6), k[5][r], e);
          e = madd(float(Cc::e7), k[6][r], e);
          e = s.h * e;
          const float sc = madd(s.rtol, tmax(fabsf(y[r]), fabsf(y1)), s.atol);
          const float q = e / sc;
          p0 = madd(q, q, p0);
          fin = fin && isfinite(y1);
        }
      }
    }
    sRed[(half * 128 + row) * 2 + 0] = p0;
    sRed[(half * 128 + row) * 2 + 1] = p1;
    sFin[half * 128 + row] = fin;
    __syncthreads();
    const float s0 = sRed[row * 2 + 0] + sRed[(128 + row) * 2 + 0];
    const float s1 = sRed[row * 2 + 1] + sRed[(128 + row) * 2 + 1];
    const bool fin_all = sFin[row] && sFin[128 + row];

    const int i = s.inst;
    if (s.phase == PH_INIT0) {
      if (a.o.h0 > 0.0) {
        s.h = (float)a.o.h0;
        s.phase = PH_STAGE;
      } else {
        // starting step, HNW Sec. II.4
        const float d0 = sqrtf(s0 / float(D)), d1 = sqrtf(s1 / float(D));
        s.h0h = (d0 < 1e-5f || d1 < 1e-5f) ? 1e-6f : 0.01f * (d0 / d1);
        s.err_prev = d1;  // parked until the second evaluation
        s.phase = PH_INIT1;
      }
    } else if (s.phase == PH_INIT1) {
      const float d1 = s.err_prev;
      const float d2 = sqrtf(s0 / float(D)) / s.h0h;
      const float m = (d1 > d2) ? d1 : d2;
      const float h1 = (m <= 1e-15f) ? tmax(1e-6f, s.h0h * 1e-3f) : ctl_pow(0.01f / m, 0.2f);
      float h = tmin(100.0f * s.h0h, h1);
      h = tmin(h, (float)(s.t1 - s.t0));
      if (!(h > 0.0f && isfinite(h))) h = (float)(s.t1 - s.t0);
      s.h = h;
      s.err_prev = 1.0f;
      s.phase = PH_STAGE;
    } else if (s.phase >= PH_STAGE && stage < 7) {
      s.phase += 1;
    } else if (s.phase >= PH_STAGE) {
      // ---- end of an attempt: accept/reject, dense output, controller
      const float h = s.h;
      const double hd = (double)h;
      const float err = sqrtf(s0 / float(D));
      const bool finite = isfinite(err) && fin_all;
      const bool accept = finite && err <= 1.0f;
      const int att = s.n_acc + s.n_rej;
      if (a.trace.cap > 0 && att < a.trace.cap && half == 0) {
        const size_t q = (size_t)i * a.trace.cap + att;
        a.trace.t[q] = s.t;
        a.trace.h[q] = hd;
        a.trace.err[q] = (double)err;
        a.trace.acc[q] = accept ? 1 : 0;
      }
      float h_next;
      if (accept) {
        bool last = s.last;
        double t_next = last ? s.t1 : s.t + hd;
        if (!last && tkey(t_next) >= tkey(s.t1)) {
          last = true;
          t_next = s.t1;
        }
        const long long kn = tkey(t_next);
        float yn[16], ylon[16];
#pragma unroll
        for (int r = 0; r < C; ++r) {
          const float u = inc[r] + ylo[r];
          yn[r] = y[r] + u;
          ylon[r] = (y[r] - yn[r]) + u;
        }
        const double* te = a.te + (size_t)i * a.K;
        float* ye = a.ye + (size_t)i * a.K * D + coff;
        while (s.cursor < a.K) {
          const double tq = te[s.cursor];
          const long long kq = tkey(tq);
          if (kq > kn) break;
          float* dst = ye + (size_t)s.cursor * D;
          if (kq == kn) {
#pragma unroll
            for (int r = 0; r < C; ++r) dst[r] = yn[r];
          } else {
            const float th = float(tq - s.t) / h;
            float w[7];
            dense_weights<float>(th, w);
#pragma unroll
            for (int r = 0; r < C; ++r) {
              float acc = w[0] * k[0][r];
              acc = madd(w[2], k[2][r], acc);
              acc = madd(w[3], k[3][r], acc);
              acc = madd(w[4], k[4][r], acc);
              acc = madd(w[5], k[5][r], acc);
              acc = madd(w[6], k[6][r], acc);
              dst[r] = y[r] + madd(h, acc, ylo[r]);
            }
          }
          s.cursor++;
        }
        float fac;
        if (err == 0.0f) {
          fac = (float)a.o.fac_max;
        } else {
          fac = (float)a.o.safety * ctl_pow(err, (float)-a.o.beta1);
          if (a.o.beta2 != 0.0) fac = fac * ctl_pow(s.err_prev, (float)a.o.beta2);
        }
        fac = tmin(tmax(fac, (float)a.o.fac_min), (float)a.o.fac_max);
        if (s.flags & FL_PREV_REJ) fac = tmin(fac, 1.0f);
        h_next = h * fac;
        s.err_prev = tmax(err, 1e-4f);
        s.flags &= ~FL_PREV_REJ;
        s.n_acc++;
        s.t = t_next;
#pragma unroll
        for (int r = 0; r < C; ++r) {
          y[r] = yn[r];
          ylo[r] = ylon[r];
          k[0][r] = k[6][r];  // FSAL
        }
        if (last) s.status = ST_SUCCESS;
        else s.rem = __double2float_rd(s.t1 - s.t);
      } else {
        const float fac =
            finite ? tmin(tmax((float)a.o.safety * ctl_pow(err, (float)-a.o.beta1),
                               (float)a.o.fac_min),
                          1.0f)
                   : (float)a.o.fac_min;
        h_next = h * fac;
        s.flags |= FL_PREV_REJ;
        s.n_rej++;
      }
      s.h = h_next;
      if (s.status == ST_RUNNING) {
        if (!(h_next >= s.hmin) || !(h_next > 0.0f))
          s.status = finite ? ST_DT_UNDERFLOW : ST_NONFINITE;
        else if (s.n_acc + s.n_rej >= a.o.max_steps)
          s.status = ST_MAX_STEPS;
      }
      if (s.status == ST_RUNNING) {
        s.phase = PH_STAGE;  // next attempt, FSAL k1 in hand
      } else {
#pragma unroll
        for (int r = 0; r < C; ++r) a.yf[(size_t)i * D + coff + r] = y[r];
        if (half == 0) {
          const int at = s.n_acc + s.n_rej;
          a.n_acc[i] = s.n_acc;
          a.n_rej[i] = s.n_rej;
          a.n_fe[i] = (a.o.h0 > 0.0 ? 1 : 2) + 6 * at;
          a.status[i] = s.status;
          if (a.trace.cap > 0) a.trace.len[i] = at < a.trace.cap ? at : a.trace.cap;
        }
        s.phase = PH_IDLE;
        need_grab = true;
      }
    }
  }
  if (abort_s && tid == 0) atomicExch(a.err, 1);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, Cfg::TMEM_COLS);
}

// W_l [N][K_in] BF16 row-major -> core-matrix image with K padded to K_l.
__global__ void k_mlp_weight_image(const uint16_t* __restrict__ W, int N, int Kin, int Kp,
                                   unsigned char* img) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * Kp) return;
  const int n = e / Kp, kk = e % Kp;
  const uint16_t v = kk < Kin ? W[(size_t)n * Kin + kk] : (uint16_t)0;
  *reinterpret_cast<uint16_t*>(img + tc::cm_offset(n, kk, Kp)) = v;
}

// ---------------------------------------------------------------- host side
using Cfg32 = MlpCfg<32, 128, 3, false>;
using Cfg32s = MlpCfg<32, 128, 3, true>;

bool mlp_supported(const tode_field_desc* f) {
  if (!f || f->kind != TODE_MLP || !f->widths || f->n_layers != 3) return false;
  return f->D == 32 && f->widths[0] == 33 && f->widths[1] == 128 && f->widths[2] == 128 &&
         f->widths[3] == 32;
}

size_t mlp_workspace_bytes(const tode_field_desc* f) {
  (void)f;
  return align256(256) + align256((size_t)Cfg32::WIMG_BYTES);
}

template <class Cfg> static tode_err launch_mlp(const SolveReq& r) {
  MlpArgs a{};
  a.B = r.B;
  a.K = r.K;
  a.y0 = (const float*)r.y0;
  a.t0 = r.t0;
  a.t1 = r.t1;
  a.te = r.te;
  a.rtol_b = r.o->rtol_b;
  a.atol_b = r.o->atol_b;
  a.rtol = r.o->rtol;
  a.atol = r.o->atol;
  a.ye = (float*)r.ye;
  a.yf = (float*)r.yf;
  a.n_acc = r.n_acc;
  a.n_rej = r.n_rej;
  a.n_fe = r.n_fe;
  a.status = r.status;
  a.o.safety = r.o->safety;
  a.o.fac_min = r.o->fac_min;
  a.o.fac_max = r.o->fac_max;
  a.o.beta1 = r.o->beta1;
  a.o.beta2 = r.o->beta2;
  a.o.h0 = r.o->h0;
  a.o.max_steps = r.o->max_steps;
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
  for (int l = 0; l < MLP_MAX_LAYERS; ++l) a.bias[l] = l < Cfg::NL ? r.f->b[l] : nullptr;
  char* p = r.ws;
  a.counter = (int32_t*)p;
  a.err = (int32_t*)(p + 128);
  p += align256(256);
  unsigned char* img = (unsigned char*)p;
  a.wimg = img;
  const cudaStream_t st = r.stream;
  for (int l = 0; l < Cfg::NL; ++l) {
    const int N = Cfg::N_of(l), Kp = Cfg::K_of(l), Kin = r.f->widths[l];
    const int n = N * Kp;
    k_mlp_weight_image<<<(n + 255) / 256, 256, 0, st>>>((const uint16_t*)r.f->W[l], N, Kin, Kp,
                                                         img + Cfg::W_off(l));
  }
  TODE_CUDA_TRY(cudaGetLastError());
  TODE_CUDA_TRY(cudaMemsetAsync(r.ws, 0, 256, st));  // queue counter and error flag
  TODE_CUDA_TRY(cudaFuncSetAttribute(k_mlp_fused<Cfg>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     Cfg::S_END));
  long long grid = (r.B + 127) / 128;
  if (grid > r.num_sms) grid = r.num_sms;
  k_mlp_fused<Cfg><<<(int)grid, 256, Cfg::S_END, st>>>(a);
  TODE_CUDA_TRY(cudaGetLastError());
  return TODE_OK;
}

tode_err mlp_solve(const SolveReq& r, bool split) {
  if (r.o->form != TODE_FUSED) return TODE_EUNSUPPORTED;
  if (r.tape) return TODE_EUNSUPPORTED;
  return split ? launch_mlp<Cfg32s>(r) : launch_mlp<Cfg32>(r);
}

}  // namespace tode
