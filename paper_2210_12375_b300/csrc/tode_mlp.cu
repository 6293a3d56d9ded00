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
// k_mlp_images builds), the BF16 input tile and the BF16 hidden tile.
// The input [Y; t] is always split into two BF16 terms (hi + lo, two MMAs
// into the same accumulator), so the state enters the field with ~16
// significant bits; hidden activations are split too when SPLIT is set, with
// tanh from exp (hi/lo resolution), else rounded to BF16 with tanh.approx.
#include "tode_core.cuh"
#include "tode_internal.h"
#include "tode_tc.cuh"

#include <cuda.h>  // CUtensorMap and its encoder type (through the runtime entry point)
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

namespace tode {


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
  float* yp;  // [B][K][D] dy/dt at the points, or NULL
  float* yf;
  int32_t *n_acc, *n_rej, *n_fe, *status;
  SolveOpts o;
  TraceDev trace;
  const unsigned char* wimg;  // core-matrix images of all layers, back to back
  const float* bias[MLP_MAX_LAYERS];
  int32_t* counter;
  int32_t* err;
  // checkpoint tape (every accepted step; slots == 0: none)
  int slots;
  float* tp_y;
  float* tp_k1;
  double* tp_t;
  float* tp_h;
  float* tp_ys;  // [B][slots][6][D]: stage inputs Y_2..Y_7 of the accepted step
  // plain form: solver state between launches, and the "some instance is
  // still running" flag the host polls
  float* wy;
  float* wylo;
  float* wk1;
  double* wt;
  float* wh;
  float* wep;
  float* wep2;
  int32_t* wcur;
  int32_t* wfl;
  int32_t* active;
  // work order: the instance at queue position q (nullptr: q itself)
  const int32_t* order;
  // checkpoint tape of a budgeted solve (ck_stride > 1; the stage tape is
  // then off): slot j = the solver state at the start of accepted step
  // j * ck_stride (y, its compensation term, FSAL k1, t, the proposed step,
  // the controller's error history, the flags)
  int ck_stride, ck_slots;
  float* ck_y;
  float* ck_ylo;
  float* ck_k1;
  double* ck_t;
  float* ck_h;
  float* ck_ep;
  float* ck_ep2;
  int32_t* ck_fl;
  // re-solve of segment rs_seg (>= 0) of every instance from the checkpoint
  // tape: accepted steps rs_seg * ck_stride .. of the first solve (rs_nacc)
  // into the stage tape, no outputs; per instance the segment's steps and
  // its bounds in the caller's time (rs_n, rs_t0, rs_t1)
  int rs_seg;
  const int32_t* rs_nacc;
  int32_t* rs_n;
  double* rs_t0;
  double* rs_t1;
};

// Kernel modes of the MLP solver body: the fused persistent form, and the
// plain form's initialising launch and per-attempt launch.
enum : int { MLP_FUSED = 0, MLP_PLAIN_INIT = 1, MLP_PLAIN_STEP = 2 };

// Tile geometry and weight residency of the MLP solver, one struct per
// network family.
//
// MlpCfg: 128-row tiles, two threads per row, all weights resident in shared
// memory (the D = 32, H = 128 network: 49 KB of BF16 weights); M = 128 MMAs,
// row r of the tile in tensor-memory lane r.
template <int D_, int H_, int NL_, bool SPLIT_> struct MlpCfg {
  static constexpr int D = D_, H = H_, NL = NL_;
  static constexpr bool SPLIT = SPLIT_, STREAM = false, STACKED = false;
  static constexpr int ROWS = 128, TPR = 2, NT = 256;  // rows per tile, threads per row
  static constexpr int K0 = ((D + 1 + 15) / 16) * 16;  // [y; t] padded to 16
  static constexpr int C = D / TPR;                      // state components per thread
  static constexpr int HC = H / TPR;                     // hidden columns per thread
  static constexpr int TMEM_COLS = (H + D <= 256) ? 256 : 512;
  static constexpr int ACC_COL = 0, OUT_COL = H;
  __device__ static int row_of(int tid) { return tid & 127; }
  __device__ static int sub_of(int tid) { return tid >> 7; }
  // 16 hidden-accumulator columns [sub*HC + c, +16) of this thread's row
  __device__ static void hid_ld(uint32_t tbase, int tid, int c, float (&v)[16]) {
    const uint32_t lanes = (uint32_t)(32 * ((tid >> 5) & 3)) << 16;
    tc::tmem_ld16(tbase + lanes + ACC_COL + sub_of(tid) * HC + c, v);
  }
  // the output layer's columns of this thread's components
  __device__ static void out_ld(uint32_t tbase, int tid, float (&v)[C]) {
    const uint32_t lanes = (uint32_t)(32 * ((tid >> 5) & 3)) << 16;
    tc::tmem_ld16(tbase + lanes + OUT_COL + sub_of(tid) * C, v);
  }
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
  static constexpr int WREP = 1, WIMG_STRIDE = ((WIMG_BYTES + 255) / 256) * 256;
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
  // stage derivatives k2..k6 of every thread: [stage][float4][thread]
  static constexpr bool KSMEM = true;
  static constexpr int S_K = S_NXT + 128 * 4;
  static constexpr int S_END = S_K + 5 * 4 * NT * 16;
  static_assert(S_END <= 232448 - 1024, "shared memory");
  static_assert(D % 32 == 0 && H % 32 == 0 && NL >= 2 && NL <= MLP_MAX_LAYERS, "shape");
  static_assert(H <= 256 && D <= 256, "one MMA per layer and K slice");
};

// MlpWideCfg: the wide network (D = 64, H = 512, 1.2 MB of BF16 weights) on
// full-rate M = 128 MMAs.  A tile holds 64 instances, and its activation
// tiles stack each instance's two BF16 terms as adjacent rows: row 2r = hi,
// row 2r + 1 = lo of instance r.  One M = 128 MMA then forms both partial
// products (an M = 64 MMA runs at half the tensor rate: measured 128 cycles
// for either shape), the accumulator's lanes 2r and 2r + 1 hold them, and the
// epilogue adds the two with one lane shuffle.  The weights stream through
// shared memory in stages of 32 KB (consecutive K chunks of one layer, one
// bulk copy and one barrier each: per-copy completion, not bytes, paced the
// 16 KB ring) through a 2-slot ring.
//
// Thread map (256 threads): warp w reads tensor-memory lane quarter w % 4
// (stacked rows 32(w%4) .. +31 = instances 16(w%4) .. +15) and column half
// w / 4; lane L holds instance 16(w%4) + L/2, the hi (even L) or lo (odd L)
// product.  An instance's 16-component slices: sub = 2 (w / 4) + (L & 1).
template <int D_, int H_, int NL_> struct MlpWideCfg {
  static constexpr int D = D_, H = H_, NL = NL_;
  static constexpr bool SPLIT = true, STREAM = true, STACKED = true;
  static constexpr int ROWS = 64, TPR = 4, NT = 256;
  static constexpr int K0 = ((D + 1 + 15) / 16) * 16;
  static constexpr int C = D / TPR;
  static constexpr int HC = H / TPR;
  static constexpr int TMEM_COLS = 512;
  static constexpr int ACC_COL = 0, OUT_COL = 0;
  static_assert(C == 16 && H == 512 && D == 64, "shape");
  __device__ static int row_of(int tid) { return 16 * ((tid >> 5) & 3) + ((tid & 31) >> 1); }
  __device__ static int sub_of(int tid) { return 2 * (tid >> 7) + (tid & 1); }
  __host__ __device__ static constexpr int N_of(int l) { return l == NL - 1 ? D : H; }
  __host__ __device__ static constexpr int K_of(int l) { return l == 0 ? K0 : H; }
  __host__ __device__ static constexpr int W_bytes(int l) { return N_of(l) * K_of(l) * 2; }
  __host__ __device__ static constexpr int W_off(int l) {
    int o = 0;
    for (int j = 0; j < l; ++j) o += W_bytes(j);
    return o;
  }
  static constexpr int WIMG_BYTES = W_off(NL);
  // one weight image for all CTAs: more copies only spread the same reads
  // over more L2 lines (measured on the whole wide step: 16 copies 30.9 ms,
  // 8: 30.7, 4: 30.5, 2: 30.5, 1: 30.4)
  static constexpr int WREP = 1, WIMG_STRIDE = ((WIMG_BYTES + 255) / 256) * 256;
  static constexpr int BIAS_FLOATS = (NL - 1) * H + D;
  // weight stages: consecutive 16-column K chunks of one layer, up to 32 KB
  static constexpr int KC = 16, NSL = 2, SLOT_BYTES = 32768;
  __host__ __device__ static constexpr int chunk_bytes(int l) { return N_of(l) * KC * 2; }
  __host__ __device__ static constexpr int chunks(int l) { return K_of(l) / KC; }
  __host__ __device__ static constexpr int per_stage(int l) { return SLOT_BYTES / chunk_bytes(l); }
  __host__ __device__ static constexpr int stages(int l) {
    return (chunks(l) + per_stage(l) - 1) / per_stage(l);
  }
  __host__ __device__ static constexpr int first_stage(int l) {
    int s = 0;
    for (int j = 0; j < l; ++j) s += stages(j);
    return s;
  }
  static constexpr int STAGES = first_stage(NL);  // per round
  // stage g of the repeating round schedule: layer, first chunk, chunks, source
  __device__ static void stage_of(uint32_t g, int& l, int& c0, int& nc, int& off, int& bytes) {
    int st = (int)(g % (uint32_t)STAGES);
    l = 0;
    while (st >= stages(l)) st -= stages(l++);
    c0 = st * per_stage(l);
    nc = chunks(l) - c0 < per_stage(l) ? chunks(l) - c0 : per_stage(l);
    bytes = nc * chunk_bytes(l);
    off = W_off(l) + c0 * chunk_bytes(l);
  }
  // shared-memory carve (bytes): stacked [128][K] activation tiles
  static constexpr int S_XH = 0, S_XL = 0;  // one stacked tile
  static constexpr int S_HH = S_XH + 2 * ROWS * K0 * 2, S_HL = S_HH;
  static constexpr int S_W = S_HH + 2 * ROWS * H * 2;  // the ring
  static constexpr int S_BIAS = S_W + NSL * SLOT_BYTES;
  static constexpr int S_RED = S_BIAS + BIAS_FLOATS * 4;
  static constexpr int S_FIN = S_RED + TPR * ROWS * 2 * 4;
  static constexpr int S_NXT = S_FIN + TPR * ROWS * 4;
  static constexpr bool KSMEM = false;
  static constexpr int S_K = 0;
  static constexpr int S_END = S_NXT + ROWS * 4;
  static_assert(S_END <= 232448 - 1024, "shared memory");
  static_assert(SLOT_BYTES % chunk_bytes(0) == 0 && SLOT_BYTES % chunk_bytes(NL - 1) == 0, "stages");
};

// Stores 16 consecutive values of instance r as BF16 hi (stacked row 2r) and
// lo (row 2r + 1) into a stacked core-matrix tile with K columns, from
// column k0 (a multiple of 8).
__device__ __forceinline__ void store_row16_stk(unsigned char* t, int r, int k0, int K,
                                                const float (&v)[16]) {
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float a = v[c * 8 + 2 * j], b = v[c * 8 + 2 * j + 1];
      const __nv_bfloat162 h2 = __floats2bfloat162_rn(a, b);
      hw[j] = *reinterpret_cast<const uint32_t*>(&h2);
      const float2 d = __ffma2_rn(make_float2(__low2float(h2), __high2float(h2)),
                                  make_float2(-1.0f, -1.0f), make_float2(a, b));
      const __nv_bfloat162 l2 = __floats2bfloat162_rn(d.x, d.y);
      lw[j] = *reinterpret_cast<const uint32_t*>(&l2);
    }
    *reinterpret_cast<uint4*>(t + tc::cm_offset(2 * r, k0 + 8 * c, K)) =
        make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(t + tc::cm_offset(2 * r + 1, k0 + 8 * c, K)) =
        make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
}

// Lanes L and L ^ 1 of a warp hold the hi and lo products of one instance
// for the same 16 accumulator columns; returns their sum over the 8 columns
// this lane keeps (even lane: columns 0-7, odd lane: 8-15), hi + lo.
__device__ __forceinline__ void combine_pair8(const float (&v)[16], int odd, float (&z)[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float send = odd ? v[j] : v[8 + j];
    const float recv = __shfl_xor_sync(0xffffffffu, send, 1);
    z[j] = odd ? recv + v[8 + j] : v[j] + recv;  // hi + lo
  }
}

// The same pair sum over 32 columns [0,16) and [16,32) of the lane's row:
// the even lane keeps columns 0-15, the odd lane 16-31.
__device__ __forceinline__ void combine_pair16(const float (&v0)[16], const float (&v1)[16],
                                               int odd, float (&z)[16]) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const float send = odd ? v0[j] : v1[j];
    const float recv = __shfl_xor_sync(0xffffffffu, send, 1);
    z[j] = odd ? recv + v1[j] : v0[j] + recv;  // hi + lo
  }
}

// Eight values as BF16 hi and lo 16-byte rows.
__device__ __forceinline__ void split8(const float (&v)[8], uint4& hi, uint4& lo) {
  uint32_t hw[4], lw[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float a = v[2 * j], b = v[2 * j + 1];
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(a, b);
    hw[j] = *reinterpret_cast<const uint32_t*>(&h2);
    const float2 d = __ffma2_rn(make_float2(__low2float(h2), __high2float(h2)),
                                make_float2(-1.0f, -1.0f), make_float2(a, b));
    const __nv_bfloat162 l2 = __floats2bfloat162_rn(d.x, d.y);
    lw[j] = *reinterpret_cast<const uint32_t*>(&l2);
  }
  hi = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  lo = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

// Writes a lane's 8 hi and 8 lo values into a stacked tile (rows 2r, 2r+1),
// the even lane's hi with the odd lane's lo in one store so that the warp's
// rows cover all eight 16-byte bank groups.
__device__ __forceinline__ void store_pair8(unsigned char* t, int r, int col, int K, int odd,
                                            const uint4& hi, const uint4& lo) {
  const uint4 first = odd ? lo : hi, second = odd ? hi : lo;
  *reinterpret_cast<uint4*>(t + tc::cm_offset(2 * r + odd, col, K)) = first;
  *reinterpret_cast<uint4*>(t + tc::cm_offset(2 * r + 1 - odd, col, K)) = second;
}

enum : int { PH_IDLE = 0, PH_INIT0 = 1, PH_INIT1 = 2, PH_STAGE = 3 };  // PH_STAGE + s - 2
// row flag beside FL_PREV_REJ / FL_REVERSE: an instance with t1 = t0 whose
// points need dy/dt = f(t0, y0) runs one evaluation round and ends there
constexpr int FL_YP_ONLY = 4;

__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// tanh of two values as 1 - 2 / (1 + e^(2x)): one ex2 of 2x log2(e) and one
// reciprocal (MUFU), the rest in FP32x2 pairs; no sign fix-up is needed
// (e^(2x) -> inf gives 1, -> 0 gives -1, x = 0 gives 0 exactly).  Absolute
// error ~2e-7, below the hi + lo split of the activation (~16 bits).
__device__ __forceinline__ float ex2_mufu(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_mufu(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float2 tanh_acc2(float2 z) {
  constexpr float k2log2e = 2.8853900817779268f;  // 2 / ln 2
  const float2 s = __fmul2_rn(z, make_float2(k2log2e, k2log2e));
  const float2 d = __fadd2_rn(make_float2(ex2_mufu(s.x), ex2_mufu(s.y)), make_float2(1.0f, 1.0f));
  return __ffma2_rn(make_float2(rcp_mufu(d.x), rcp_mufu(d.y)), make_float2(-2.0f, -2.0f),
                    make_float2(1.0f, 1.0f));
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
        // (a, b) - hi: the product hi * -1 is exact, so one rounding as a - hi
        const float2 d = __ffma2_rn(make_float2(__low2float(h2), __high2float(h2)),
                                    make_float2(-1.0f, -1.0f), make_float2(a, b));
        const __nv_bfloat162 l2 = __floats2bfloat162_rn(d.x, d.y);
        lw[j] = *reinterpret_cast<const uint32_t*>(&l2);
      }
    }
    const uint32_t off = tc::cm_offset(row, k0 + 8 * c, K);
    *reinterpret_cast<uint4*>(th + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    if (LO) *reinterpret_cast<uint4*>(tl + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
}

// a_{s,j} of the tableau (stage 7 row = b), as float; s = 2..7, j = 1..6
__device__ __forceinline__ float dp_a(int s, int j) {
  using C = DP5;
  switch (s * 8 + j) {
    case 17: return float(C::a21);
    case 25: return float(C::a31);
    case 26: return float(C::a32);
    case 33: return float(C::a41);
    case 34: return float(C::a42);
    case 35: return float(C::a43);
    case 41: return float(C::a51);
    case 42: return float(C::a52);
    case 43: return float(C::a53);
    case 44: return float(C::a54);
    case 49: return float(C::a61);
    case 50: return float(C::a62);
    case 51: return float(C::a63);
    case 52: return float(C::a64);
    case 53: return float(C::a65);
    case 57: return float(C::b1);
    case 59: return float(C::b3);
    case 60: return float(C::b4);
    case 61: return float(C::b5);
    case 62: return float(C::b6);
    default: return 0.0f;
  }
}
// a_{s,j} of the pair Tab as float (dopri5: dp_a, the same values)
template <class Tab> __device__ __forceinline__ float tab_a(int s, int j) {
  if constexpr (std::is_same<Tab, DP5>::value) {
    return dp_a(s, j);
  } else {
#define TODE_TA(S, J) \
  case S * 8 + J: return float(Tab::a(S, J));
    switch (s * 8 + j) {
      TODE_TA(2, 1)
      TODE_TA(3, 1) TODE_TA(3, 2)
      TODE_TA(4, 1) TODE_TA(4, 2) TODE_TA(4, 3)
      TODE_TA(5, 1) TODE_TA(5, 2) TODE_TA(5, 3) TODE_TA(5, 4)
      TODE_TA(6, 1) TODE_TA(6, 2) TODE_TA(6, 3) TODE_TA(6, 4) TODE_TA(6, 5)
      TODE_TA(7, 1) TODE_TA(7, 2) TODE_TA(7, 3) TODE_TA(7, 4) TODE_TA(7, 5) TODE_TA(7, 6)
      default: return 0.0f;
    }
#undef TODE_TA
  }
}
// the pair keeps k_2 in its solution, error or dense output (tsit5; dopri5
// drops it)
template <class Tab> __host__ __device__ constexpr bool tab_k2() {
  return Tab::b(2) != 0.0 || Tab::e(2) != 0.0 || Tab::q(2, 0) != 0.0 || Tab::q(2, 1) != 0.0 ||
         Tab::q(2, 2) != 0.0 || Tab::q(2, 3) != 0.0;
}
// Per-row solver state (identical scalars in both threads of the row).
struct MlpRow {
  int inst, phase, cursor, status, flags, n_acc, n_rej, target;
  double t, t0, t1;
  float h, h0h, err_prev, err_prev2, rtol, atol, rem, hmin;
  bool last;
};

// The solver body shared by the fused form and the plain form.  Fused: a
// persistent grid, each row takes instances from a global counter and
// integrates them to their end.  Plain: tile c of ROWS instances belongs to
// CTA c mod grid; the initialising launch runs the starting-step rounds, every
// later launch one attempt (six stage rounds) per running instance, with the
// state parked in the workspace in between.  Tab: the Runge-Kutta pair
// (dopri5 or tsit5; the same seven-stage FSAL structure).
template <class Cfg, int MODE, class Tab>
__device__ __forceinline__ void mlp_solver(const MlpArgs a) {
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
  float* sRed = reinterpret_cast<float*>(sm + Cfg::S_RED);  // [sub][row][2]
  int* sFin = reinterpret_cast<int*>(sm + Cfg::S_FIN);      // [sub][row]
  int* sNxt = reinterpret_cast<int*>(sm + Cfg::S_NXT);      // [row]
  constexpr int ROWS = Cfg::ROWS, TPR = Cfg::TPR, NT = Cfg::NT;
  static_assert(C == 16, "16 state components per thread");
  // streamed weights: a ring of chunk buffers with full / empty barriers
  __shared__ __align__(8) uint64_t mbar_full[4], mbar_empty[4];
  uint32_t g_chunk = 0;  // chunks (stacked configs: stages) consumed so far

  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = Cfg::row_of(tid), sub = Cfg::sub_of(tid);
  const int coff = sub * C;  // first state component of this thread
  const unsigned char* wimg = a.wimg + (size_t)(blockIdx.x % Cfg::WREP) * Cfg::WIMG_STRIDE;

  // ---- set-up: barriers, weights (bulk copy), biases, tensor memory
  if (tid == 0) {
    tc::mbar_init(&mbar_mma, 1);
    tc::mbar_init(&mbar_w, 1);
    if constexpr (Cfg::STREAM)
      for (int b = 0; b < 4; ++b) {
        tc::mbar_init(&mbar_full[b], 1);
        tc::mbar_init(&mbar_empty[b], 1);
      }
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    if constexpr (Cfg::STACKED) {
      static_assert(Cfg::NSL <= 4, "ring barriers");
      for (int b = 0; b < Cfg::NSL; ++b) {  // the ring starts with stages 0 .. NSL-1
        int l_, c0_, nc_, off, bytes;
        Cfg::stage_of((uint32_t)b, l_, c0_, nc_, off, bytes);
        tc::mbar_expect_tx(&mbar_full[b], (uint32_t)bytes);
        tc::bulk_g2s(sW + b * Cfg::SLOT_BYTES, wimg + off, (uint32_t)bytes, &mbar_full[b]);
      }
    } else {
      tc::mbar_expect_tx(&mbar_w, (uint32_t)Cfg::WIMG_BYTES);
#pragma unroll
      for (int l = 0; l < NL; ++l)
        tc::bulk_g2s(sW + Cfg::W_off(l), wimg + Cfg::W_off(l), (uint32_t)Cfg::W_bytes(l),
                     &mbar_w);
    }
  }
  {
    int o = 0;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const int n = Cfg::N_of(l);
      for (int j = tid; j < n; j += NT) sBias[o + j] = a.bias[l] ? a.bias[l][j] : 0.0f;
      o += n;
    }
  }
  // zero the input tiles once (padding columns stay zero)
  if constexpr (Cfg::STACKED) {
    for (int j = tid; j < 2 * ROWS * K0 * 2 / 16; j += NT)
      reinterpret_cast<uint4*>(sXh)[j] = make_uint4(0, 0, 0, 0);
  } else {
    for (int j = tid; j < ROWS * K0 * 2 / 16; j += NT) {
      reinterpret_cast<uint4*>(sXh)[j] = make_uint4(0, 0, 0, 0);
      reinterpret_cast<uint4*>(sXl)[j] = make_uint4(0, 0, 0, 0);
    }
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base_s, Cfg::TMEM_COLS);
    tc::tmem_relinquish();
  }
  if constexpr (!Cfg::STREAM) {
    const bool w_ok = tc::mbar_wait(&mbar_w, 0);
    if (!w_ok) atomicExch(&abort_s, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_base_s;
  uint32_t mma_parity = 0;

  MlpRow s;
  s.inst = -1;
  s.target = -1;
  s.phase = PH_IDLE;
  // k1 (FSAL) in registers; k2..k6 of the attempt in shared memory when the
  // config has room (else in the thread's local array); k7 is the last f
  float y[C], ylo[C], k1[C];
#pragma unroll
  for (int r = 0; r < C; ++r) y[r] = ylo[r] = k1[r] = 0.0f;
  float kloc[Cfg::KSMEM ? 1 : 5][C];
  float4* sK = reinterpret_cast<float4*>(sm + Cfg::S_K);
  auto kput = [&](int j, const float (&v)[16]) {  // stage j = 2..6
    if constexpr (Cfg::KSMEM) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        sK[((j - 2) * 4 + q) * NT + tid] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
#pragma unroll
      for (int r = 0; r < C; ++r) kloc[j - 2][r] = v[r];
    }
  };
  auto kget = [&](int j, float (&v)[16]) {
    if constexpr (Cfg::KSMEM) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 u = sK[((j - 2) * 4 + q) * NT + tid];
        v[4 * q] = u.x, v[4 * q + 1] = u.y, v[4 * q + 2] = u.z, v[4 * q + 3] = u.w;
      }
    } else {
#pragma unroll
      for (int r = 0; r < C; ++r) v[r] = kloc[j - 2][r];
    }
  };
  bool need_grab = MODE == MLP_FUSED;  // fused: this row takes the next instance
  bool need_load = MODE != MLP_FUSED;  // plain: this row loads its instance of the tile
  int tile = blockIdx.x;

  // load and validate instance i, write its points at t0 and pick the phase
  auto start_instance = [&](const int i) {
    // load and validate the instance (Sec. 3: per-instance bounds / points)
    s.inst = i;
    s.target = -1;
    // backward in time (t1 < t0): the row runs in tau = -t with the field
    // -f(-tau, y) (its times through a sign xor, see tode_core.cuh)
    const unsigned long long m = (a.t1[i] < a.t0[i]) ? SIGN_BIT : 0ULL;
    if (a.rs_seg >= 0) {
      // re-solve: the segment's first accepted step from its checkpoint,
      // the same state the first solve had there (bit for bit)
      const int first = a.rs_seg * a.ck_stride, N = a.rs_nacc[i];
      const int n_seg = N - first < a.ck_stride ? N - first : a.ck_stride;
      if (n_seg <= 0 || a.rs_seg >= a.ck_slots) {
        if (sub == 0) {
          a.rs_n[i] = 0;
          a.rs_t0[i] = a.rs_t1[i] = a.t1[i];
        }
        s.phase = PH_IDLE;
        if (MODE == MLP_FUSED) need_grab = true;
        return;
      }
      const size_t o = (size_t)i * a.ck_slots + a.rs_seg;
      s.t0 = flip(a.t0[i], m);
      s.t1 = flip(a.t1[i], m);
      s.t = a.ck_t[o];
      s.rtol = (float)(a.rtol_b ? a.rtol_b[i] : a.rtol);
      s.atol = (float)(a.atol_b ? a.atol_b[i] : a.atol);
      s.n_acc = s.n_rej = 0;
      s.cursor = 0;
      s.flags = a.ck_fl[o];
      s.err_prev = a.ck_ep[o];
      s.err_prev2 = a.ck_ep2 ? a.ck_ep2[o] : 1.0f;
      s.h = a.ck_h[o];
      s.h0h = 0.0f;
      s.last = false;
      s.status = ST_RUNNING;
      s.target = n_seg;
      s.rem = __double2float_rd(s.t1 - s.t);
      s.hmin = (float)(1e-14 * tmax(fabs(s.t0), fabs(s.t1)));
#pragma unroll
      for (int r = 0; r < C; ++r) {
        y[r] = a.ck_y[o * D + coff + r];
        ylo[r] = a.ck_ylo[o * D + coff + r];
        k1[r] = a.ck_k1[o * D + coff + r];
      }
      if (sub == 0) {
        a.rs_n[i] = n_seg;
        a.rs_t0[i] = flip(s.t, m);
      }
      s.phase = PH_STAGE;
      return;
    }
    s.t0 = flip(a.t0[i], m);
    s.t1 = flip(a.t1[i], m);
    s.t = s.t0;
    s.rtol = (float)(a.rtol_b ? a.rtol_b[i] : a.rtol);
    s.atol = (float)(a.atol_b ? a.atol_b[i] : a.atol);
    s.n_acc = s.n_rej = 0;
    s.cursor = 0;
    s.flags = m ? FL_REVERSE : 0;
    s.err_prev = 1.0f;
    s.err_prev2 = 1.0f;
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
      const long long kv = tkey(flip(te[q], m));
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
      if (a.yp)
        for (int q = 0; q < a.K; ++q)
#pragma unroll
          for (int r = 0; r < C; ++r) a.yp[((size_t)i * a.K + q) * D + coff + r] = nan_(0.0f);
      done = true;
    } else {
      while (s.cursor < a.K && tkey(flip(te[s.cursor], m)) == k0) {
#pragma unroll
        for (int r = 0; r < C; ++r) ye[(size_t)s.cursor * D + r] = y[r];
        s.cursor++;
      }
      if (k1 == k0 && a.yp && s.cursor > 0) {
        // no step, but the points' dy/dt = f(t0, y0) takes one evaluation
        s.status = ST_SUCCESS;
        s.flags |= FL_YP_ONLY;
        s.phase = PH_INIT0;
      } else if (k1 == k0) {
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
      if (sub == 0) {
        a.n_acc[i] = a.n_rej[i] = a.n_fe[i] = 0;
        a.status[i] = s.status;
        if (a.trace.cap > 0) a.trace.len[i] = 0;
      }
      s.phase = PH_IDLE;
      if (MODE == MLP_FUSED) need_grab = true;
    }
  };
  // plain form: park the row's solver state for the next launch
  auto park = [&]() {
    const int i = s.inst;
#pragma unroll
    for (int r = 0; r < C; ++r) {
      const size_t o = (size_t)i * D + coff + r;
      a.wy[o] = y[r];
      a.wylo[o] = ylo[r];
      a.wk1[o] = k1[r];
    }
    if (sub == 0) {
      a.wt[i] = s.t;
      a.wh[i] = s.h;
      a.wep[i] = s.err_prev;
      a.wep2[i] = s.err_prev2;
      a.wcur[i] = s.cursor;
      a.wfl[i] = s.flags;
      a.n_acc[i] = s.n_acc;
      a.n_rej[i] = s.n_rej;
      a.status[i] = ST_RUNNING;
      *a.active = 1;
    }
    s.phase = PH_IDLE;
  };
  // plain form: resume a parked instance at the start of its next attempt
  auto resume = [&](const int i) {
    s.inst = i;
    s.target = -1;
    s.flags = a.wfl[i];
    s.t0 = flip(a.t0[i], rev_mask(s.flags));
    s.t1 = flip(a.t1[i], rev_mask(s.flags));
    s.t = a.wt[i];  // parked in the row's own time
    s.rtol = (float)(a.rtol_b ? a.rtol_b[i] : a.rtol);
    s.atol = (float)(a.atol_b ? a.atol_b[i] : a.atol);
    s.n_acc = a.n_acc[i];
    s.n_rej = a.n_rej[i];
    s.cursor = a.wcur[i];
    s.err_prev = a.wep[i];
    s.err_prev2 = a.wep2[i];
    s.h = a.wh[i];
    s.h0h = 0.0f;
    s.last = false;
    s.status = ST_RUNNING;
    s.rem = __double2float_rd(s.t1 - s.t);  // functions of (t, t0, t1), as in the fused form
    s.hmin = (float)(1e-14 * tmax(fabs(s.t0), fabs(s.t1)));
#pragma unroll
    for (int r = 0; r < C; ++r) {
      const size_t o = (size_t)i * D + coff + r;
      y[r] = a.wy[o];
      ylo[r] = a.wylo[o];
      k1[r] = a.wk1[o];
    }
    s.phase = PH_STAGE;
  };

  while (true) {
    if (MODE == MLP_FUSED) {
      // ---- hand out instances to rows that need one (one atomic per row)
      if (need_grab && sub == 0) sNxt[row] = atomicAdd(a.counter, 1);
      __syncthreads();
      if (need_grab) {
        need_grab = false;
        const int q = sNxt[row];
        const int i = q >= a.B ? a.B : (a.order ? a.order[q] : q);
        if (i >= a.B) {
          s.phase = PH_IDLE;
          s.inst = -1;
        } else {
          start_instance(i);
        }
      }
    } else if (need_load) {
      need_load = false;
      const int q = tile * ROWS + row;
      const int i = q >= a.B ? a.B : (a.order ? a.order[q] : q);
      s.phase = PH_IDLE;
      s.inst = -1;
      if (i < a.B) {
        if (MODE == MLP_PLAIN_INIT) start_instance(i);
        else if (a.status[i] == ST_RUNNING) resume(i);
      }
    }
    // all rows idle and the queue exhausted (fused) or the tile done (plain)
    const bool any_work = __syncthreads_or(s.phase != PH_IDLE || need_grab) != 0;
    if (abort_s) break;
    if (!any_work) {
      if (MODE == MLP_FUSED) break;
      tile += gridDim.x;
      if ((long long)tile * ROWS >= a.B) break;
      need_load = true;
      continue;
    }
    if (MODE == MLP_FUSED &&
        __syncthreads_or(need_grab && s.phase == PH_IDLE && s.inst >= 0) != 0) {
      // some row finished without work this round: refill first
      continue;
    }

    // ---- this row's field input [Y; t] for the round
    float Y[16];
    float tin = 0.0f;
    const int stage = s.phase - PH_STAGE + 2;  // 2..7 in stage phases
    if (s.phase == PH_INIT0 || s.phase == PH_IDLE) {
#pragma unroll
      for (int r = 0; r < C; ++r) Y[r] = y[r];
      tin = (float)flip(s.t, rev_mask(s.flags));  // the network sees the caller's time
    } else if (s.phase == PH_INIT1) {
#pragma unroll
      for (int r = 0; r < C; ++r) Y[r] = madd(s.h0h, k1[r], y[r]);
      tin = (float)flip(s.t + (double)s.h0h, rev_mask(s.flags));
    } else {
      if (stage == 2) {  // a new attempt starts: clip at t1
        if (a.ck_stride > 1 && !(s.flags & FL_PREV_REJ) && s.n_acc % a.ck_stride == 0 &&
            s.n_acc / a.ck_stride < a.ck_slots && a.rs_seg < 0) {
          // checkpoint: the state the first attempt of this step starts from
          const size_t o = (size_t)s.inst * a.ck_slots + s.n_acc / a.ck_stride;
#pragma unroll
          for (int r = 0; r < C; ++r) {
            a.ck_y[o * D + coff + r] = y[r];
            a.ck_ylo[o * D + coff + r] = ylo[r];
            a.ck_k1[o * D + coff + r] = k1[r];
          }
          if (sub == 0) {
            a.ck_t[o] = s.t;
            a.ck_h[o] = s.h;
            a.ck_ep[o] = s.err_prev;
            if (a.ck_ep2) a.ck_ep2[o] = s.err_prev2;
            a.ck_fl[o] = s.flags;
          }
        }
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
      // Y_s = y + h sum_j a_sj k_j, the terms in the order j = 1, 2, ...
      // (dopri5's stage-7 row is b, which has no k2 term)
      float acc[16];
      const float a1 = tab_a<Tab>(stage, 1);
#pragma unroll
      for (int r = 0; r < C; ++r) acc[r] = a1 * k1[r];
      for (int j = 2; j < stage && j <= 6; ++j) {
        if (stage == 7 && j == 2 && Tab::a(7, 2) == 0.0) continue;
        float kj[16];
        kget(j, kj);
        const float c = tab_a<Tab>(stage, j);
#pragma unroll
        for (int r = 0; r < C; ++r) acc[r] = madd(c, kj[r], acc[r]);
      }
#pragma unroll
      for (int r = 0; r < C; ++r) Y[r] = (stage == 7) ? y[r] + h * acc[r] : madd(h, acc[r], y[r]);
      if constexpr (std::is_same<Tab, DP5>::value) {
        switch (stage) {
          case 2: cs = DP5::c2; break;
          case 3: cs = DP5::c3; break;
          case 4: cs = DP5::c4; break;
          case 5: cs = DP5::c5; break;
          default: cs = 1.0; break;
        }
      } else {
        switch (stage) {
          case 2: cs = Tab::c(2); break;
          case 3: cs = Tab::c(3); break;
          case 4: cs = Tab::c(4); break;
          case 5: cs = Tab::c(5); break;
          case 6: cs = Tab::c(6); break;
          default: cs = Tab::c(7); break;
        }
      }
      tin = (float)flip(s.t + cs * (double)h, rev_mask(s.flags));
    }
    if constexpr (Cfg::STACKED) store_row16_stk(sXh, row, coff, K0, Y);
    else store_row16<true>(sXh, sXl, row, coff, K0, Y);
    if (s.phase >= PH_STAGE && s.n_acc < a.slots) {
      // tape: the stage inputs of this attempt (a retry after a rejection
      // overwrites them; the accepted attempt's stay)
      float4* dst = reinterpret_cast<float4*>(
          a.tp_ys + (((size_t)s.inst * a.slots + s.n_acc) * 6 + (stage - 2)) * D + coff);
#pragma unroll
      for (int q = 0; q < C / 4; ++q)
        dst[q] = make_float4(Y[4 * q], Y[4 * q + 1], Y[4 * q + 2], Y[4 * q + 3]);
    }
    if (sub == TPR - 1) {  // the time input, hi + lo, in column D
      const __nv_bfloat16 th = __float2bfloat16_rn(tin);
      const __nv_bfloat16 tl = __float2bfloat16_rn(tin - __bfloat162float(th));
      const int rh = Cfg::STACKED ? 2 * row : row, rl = Cfg::STACKED ? 2 * row + 1 : row;
      *reinterpret_cast<__nv_bfloat16*>(sXh + tc::cm_offset(rh, D, K0)) = th;
      *reinterpret_cast<__nv_bfloat16*>(sXl + tc::cm_offset(rl, D, K0)) = tl;
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
      if (tid == 0 && !abort_s) {
        const uint32_t ah = tc::smem_u32(l == 0 ? sXh : sHh);
        const uint32_t al = tc::smem_u32(l == 0 ? sXl : sHl);
        if constexpr (Cfg::STACKED) {
          // the layer's stages: per K chunk one M = 128 MMA per N half over
          // the stacked tile (hi and lo rows together), then a commit that
          // frees the stage's slot; thread 32 refills it (below)
          constexpr int NSL = Cfg::NSL;
          const int nh = Nl > 256 ? Nl / 256 : 1, nw = Nl > 256 ? 256 : Nl;
          const uint32_t idesc = tc::idesc_bf16_f32(128, nw);
          const int cb = Cfg::chunk_bytes(l);
          bool ok = true;
          for (int st = 0; st < Cfg::stages(l) && ok; ++st) {
            const uint32_t g = g_chunk + (uint32_t)st;
            const int b = (int)(g % NSL);
            ok = tc::mbar_wait(&mbar_full[b], (g / NSL) & 1u);
            if (!ok) break;
            int l_, c0, nc, off_, bytes_;
            Cfg::stage_of(g, l_, c0, nc, off_, bytes_);
            const uint32_t wb = tc::smem_u32(sW + b * Cfg::SLOT_BYTES);
            for (int c = 0; c < nc; ++c) {
              const int kc = c0 + c;
              const uint64_t da = tc::smem_desc(ah + kc * 256, 128, Kl * 16);
              for (int j = 0; j < nh; ++j) {
                const uint64_t db = tc::smem_desc(wb + c * cb + j * (256 / 8) * 256, 128, 256);
                tc::mma_bf16(tbase + 256 * j, da, db, idesc, kc > 0);
              }
            }
            tc::mma_commit(&mbar_empty[b]);
          }
          if (!ok) atomicExch(&abort_s, 1);
        } else {
          const uint32_t idesc = tc::idesc_bf16_f32(128, Nl);
          const uint32_t wa = tc::smem_u32(sW + Cfg::W_off(l));
          const bool lo = (l == 0) || Cfg::SPLIT;
          for (int kk = 0; kk < Kl / 16; ++kk) {
            const uint64_t db = tc::smem_desc(wa + kk * 256, 128, Kl * 16);
            tc::mma_bf16(tbase + dcol, tc::smem_desc(ah + kk * 256, 128, Kl * 16), db, idesc,
                         kk > 0);
            if (lo)
              tc::mma_bf16(tbase + dcol, tc::smem_desc(al + kk * 256, 128, Kl * 16), db, idesc,
                           true);
          }
        }
        tc::mma_commit(&mbar_mma);
      }
      if constexpr (Cfg::STACKED) {
        if (tid == 32 && !abort_s) {
          // producer: the slot of stage g takes stage g + NSL once the MMAs
          // that read it are done (a thread of its own, so the issuer never
          // waits on a copy it could have started earlier)
          constexpr int NSL = Cfg::NSL;
          bool ok = true;
          for (int st = 0; st < Cfg::stages(l) && ok; ++st) {
            const uint32_t g = g_chunk + (uint32_t)st;
            const int b = (int)(g % NSL);
            ok = tc::mbar_wait(&mbar_empty[b], (g / NSL) & 1u);
            if (!ok) break;
            int l2, c2, n2, off, bytes;
            Cfg::stage_of(g + NSL, l2, c2, n2, off, bytes);
            tc::mbar_expect_tx(&mbar_full[b], (uint32_t)bytes);
            tc::bulk_g2s(sW + b * Cfg::SLOT_BYTES, wimg + off, (uint32_t)bytes, &mbar_full[b]);
          }
          if (!ok) atomicExch(&abort_s, 1);
        }
        g_chunk += (uint32_t)Cfg::stages(l);
        __syncwarp();  // the other lanes of warps 0 and 1 wait for the issuer / producer here
      }
      const bool ok = Cfg::STACKED ? tc::mbar_wait_sleep(&mbar_mma, mma_parity)
                                   : tc::mbar_wait(&mbar_mma, mma_parity);
      mma_parity ^= 1u;
      if (!ok) atomicExch(&abort_s, 1);
      tc::fence_after_sync();
      if constexpr (Cfg::STACKED) {
        if (l < NL - 1) {
          // hidden epilogue on the stacked accumulator: the pair sum of the
          // hi and lo rows, bias, tanh, BF16 hi + lo into the stacked tile
          const float* bl = sBias + l * H;
          const int lane = tid & 31, odd = lane & 1, hf = warp >> 2;
          const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
#pragma unroll 1
          for (int c = 0; c < 256; c += 32) {
            float v0[16], v1[16];
            tc::tmem_ld16(tbase + lanes + 256 * hf + c, v0);
            tc::tmem_ld16(tbase + lanes + 256 * hf + c + 16, v1);
            tc::tmem_wait_ld();
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              float z[8];
              combine_pair8(u == 0 ? v0 : v1, odd, z);
              const int col = 256 * hf + c + 16 * u + 8 * odd;
              const float4 b0 = *reinterpret_cast<const float4*>(bl + col);
              const float4 b1 = *reinterpret_cast<const float4*>(bl + col + 4);
              const float2 t0 = tanh_acc2(__fadd2_rn(make_float2(z[0], z[1]), make_float2(b0.x, b0.y)));
              const float2 t1 = tanh_acc2(__fadd2_rn(make_float2(z[2], z[3]), make_float2(b0.z, b0.w)));
              const float2 t2 = tanh_acc2(__fadd2_rn(make_float2(z[4], z[5]), make_float2(b1.x, b1.y)));
              const float2 t3 = tanh_acc2(__fadd2_rn(make_float2(z[6], z[7]), make_float2(b1.z, b1.w)));
              const float hv[8] = {t0.x, t0.y, t1.x, t1.y, t2.x, t2.y, t3.x, t3.y};
              uint4 hi, lo;
              split8(hv, hi, lo);
              store_pair8(sHh, row, col, H, odd, hi, lo);
            }
          }
          tc::fence_proxy_async();
          tc::fence_before_sync();
          __syncthreads();
          tc::fence_after_sync();
        }
      } else if (l < NL - 1) {
        // hidden epilogue: bias, tanh, BF16 (split) into the hidden tile
        const float* bl = sBias + l * H;
        // the accumulator loads of up to four 16-column chunks in flight
        // together, one wait, then bias + tanh + split per chunk (the wide
        // network, short of registers, takes one chunk at a time)
        constexpr int NLD = Cfg::STREAM ? 1 : (Cfg::HC / 16 < 4 ? Cfg::HC / 16 : 4);
#pragma unroll
        for (int c0 = 0; c0 < Cfg::HC; c0 += 16 * NLD) {
          float v[NLD][16];
#pragma unroll
          for (int u = 0; u < NLD; ++u) Cfg::hid_ld(tbase, tid, c0 + 16 * u, v[u]);
          tc::tmem_wait_ld();
#pragma unroll
          for (int u = 0; u < NLD; ++u) {
            const int col = sub * Cfg::HC + c0 + 16 * u;
            const float4* b4 = reinterpret_cast<const float4*>(bl + col);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float4 bq = b4[q];
              const float2 z0 = __fadd2_rn(make_float2(v[u][4 * q], v[u][4 * q + 1]),
                                           make_float2(bq.x, bq.y));
              const float2 z1 = __fadd2_rn(make_float2(v[u][4 * q + 2], v[u][4 * q + 3]),
                                           make_float2(bq.z, bq.w));
              if constexpr (Cfg::SPLIT) {
                const float2 t0 = tanh_acc2(z0), t1 = tanh_acc2(z1);
                v[u][4 * q] = t0.x, v[u][4 * q + 1] = t0.y;
                v[u][4 * q + 2] = t1.x, v[u][4 * q + 3] = t1.y;
              } else {
                v[u][4 * q] = tanh_fast(z0.x), v[u][4 * q + 1] = tanh_fast(z0.y);
                v[u][4 * q + 2] = tanh_fast(z1.x), v[u][4 * q + 3] = tanh_fast(z1.y);
              }
            }
            store_row16<Cfg::SPLIT>(sHh, sHl, row, col, H, v[u]);
          }
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
      }
    }
    // ---- output: f for this thread's components
    float f[16];
    if constexpr (Cfg::STACKED) {
      // output columns [32 hf, 32 hf + 32) of the lane's stacked row, pair-summed
      float v0[16], v1[16], z[16];
      const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
      tc::tmem_ld16(tbase + lanes + 32 * (warp >> 2), v0);
      tc::tmem_ld16(tbase + lanes + 32 * (warp >> 2) + 16, v1);
      tc::tmem_wait_ld();
      combine_pair16(v0, v1, tid & 1, z);
      const float* bo = sBias + (NL - 1) * H;
#pragma unroll
      for (int r = 0; r < C; ++r) f[r] = z[r] + bo[coff + r];
    } else {
      float v[16];
      Cfg::out_ld(tbase, tid, v);
      tc::tmem_wait_ld();
      const float* bo = sBias + (NL - 1) * H;
#pragma unroll
      for (int r = 0; r < C; ++r) f[r] = v[r] + bo[coff + r];
    }
    if (s.flags & FL_REVERSE) {  // the row's field in tau = -t is -f
#pragma unroll
      for (int r = 0; r < C; ++r) f[r] = -f[r];
    }

    // ---- consume: partial sums of this thread's components
    float p0 = 0.0f, p1 = 0.0f;
    int fin = 1;
    float inc[16];
    float k3[16], k4[16], k5[16], k6[16];  // stage 7: the attempt's k3..k6
    constexpr bool K2 = tab_k2<Tab>();
    float k2[K2 ? 16 : 1];  // and k2 where the pair uses it
    if (s.phase == PH_INIT0) {
#pragma unroll
      for (int r = 0; r < C; ++r) {
        k1[r] = f[r];
        const float sc = madd(s.rtol, fabsf(y[r]), s.atol);
        const float q0 = y[r] / sc, q1 = f[r] / sc;
        p0 = madd(q0, q0, p0);
        p1 = madd(q1, q1, p1);
      }
      if (a.yp) {  // points at t0: dy/dt = f(t0, y0) in the caller's time
        const float dir = (s.flags & FL_REVERSE) ? -1.0f : 1.0f;
        for (int q = 0; q < s.cursor; ++q)
#pragma unroll
          for (int r = 0; r < C; ++r)
            a.yp[((size_t)s.inst * a.K + q) * D + coff + r] = dir * k1[r];
      }
    } else if (s.phase == PH_INIT1) {
#pragma unroll
      for (int r = 0; r < C; ++r) {
        const float sc = madd(s.rtol, fabsf(y[r]), s.atol);
        const float q = (f[r] - k1[r]) / sc;
        p0 = madd(q, q, p0);
      }
    } else if (s.phase >= PH_STAGE) {
      if (stage < 7) kput(stage, f);
      if (stage == 7) {
        if constexpr (K2) kget(2, k2);
        kget(3, k3);
        kget(4, k4);
        kget(5, k5);
        kget(6, k6);
#pragma unroll
        for (int r = 0; r < C; ++r) {
          float acc = float(Tab::b(1)) * k1[r];
          if constexpr (K2) acc = madd(float(Tab::b(2)), k2[r], acc);
          acc = madd(float(Tab::b(3)), k3[r], acc);
          acc = madd(float(Tab::b(4)), k4[r], acc);
          acc = madd(float(Tab::b(5)), k5[r], acc);
          acc = madd(float(Tab::b(6)), k6[r], acc);
          inc[r] = s.h * acc;
          const float y1 = y[r] + inc[r];
          float e = float(Tab::e(1)) * k1[r];
          if constexpr (K2) e = madd(float(Tab::e(2)), k2[r], e);
          e = madd(float(Tab::e(3)), k3[r], e);
          e = madd(float(Tab::e(4)), k4[r], e);
          e = madd(float(Tab::e(5)), k5[r], e);
          e = madd(float(Tab::e(6)), k6[r], e);
          e = madd(float(Tab::e(7)), f[r], e);
          e = s.h * e;
          const float sc = madd(s.rtol, tmax(fabsf(y[r]), fabsf(y1)), s.atol);
          const float q = e / sc;
          p0 = madd(q, q, p0);
          fin = fin && isfinite(y1);
        }
      }
    }
    sRed[(sub * ROWS + row) * 2 + 0] = p0;
    sRed[(sub * ROWS + row) * 2 + 1] = p1;
    sFin[sub * ROWS + row] = fin;
    __syncthreads();
    float s0 = sRed[row * 2 + 0], s1 = sRed[row * 2 + 1];
    bool fin_all = sFin[row] != 0;
#pragma unroll
    for (int u = 1; u < TPR; ++u) {  // the row's threads in a fixed order
      s0 += sRed[(u * ROWS + row) * 2 + 0];
      s1 += sRed[(u * ROWS + row) * 2 + 1];
      fin_all = fin_all && sFin[u * ROWS + row] != 0;
    }

    const int i = s.inst;
    if (s.phase == PH_INIT0 && (s.flags & FL_YP_ONLY)) {
      // t1 = t0: the evaluation was for dy/dt only; the instance ends here
#pragma unroll
      for (int r = 0; r < C; ++r) a.yf[(size_t)i * D + coff + r] = y[r];
      if (sub == 0) {
        a.n_acc[i] = a.n_rej[i] = a.n_fe[i] = 0;
        a.status[i] = ST_SUCCESS;
        if (a.trace.cap > 0) a.trace.len[i] = 0;
      }
      s.phase = PH_IDLE;
      if (MODE == MLP_FUSED) need_grab = true;
    } else if (s.phase == PH_INIT0) {
      if (a.o.h0 > 0.0) {
        s.h = (float)a.o.h0;
        s.phase = PH_STAGE;
        if (MODE == MLP_PLAIN_INIT) park();
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
      s.err_prev2 = 1.0f;
      s.phase = PH_STAGE;
      if (MODE == MLP_PLAIN_INIT) park();
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
      if (a.trace.cap > 0 && att < a.trace.cap && sub == 0) {
        const size_t q = (size_t)i * a.trace.cap + att;
        a.trace.t[q] = flip(s.t, rev_mask(s.flags));  // the caller's time and signed step
        a.trace.h[q] = flip(hd, rev_mask(s.flags));
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
        if (s.n_acc < a.slots) {  // tape: the state this accepted step started from
          const size_t o = (size_t)i * a.slots + s.n_acc;
#pragma unroll
          for (int r = 0; r < C; ++r) {
            a.tp_y[o * D + coff + r] = y[r];
            if (a.tp_k1) a.tp_k1[o * D + coff + r] = k1[r];
          }
          if (sub == 0) {
            a.tp_t[o] = s.t;
            a.tp_h[o] = h;
          }
        }
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
          const double tq = flip(te[s.cursor], rev_mask(s.flags));
          const long long kq = tkey(tq);
          if (kq > kn) break;
          float* dst = ye + (size_t)s.cursor * D;
          const float th = kq == kn ? 1.0f : float(tq - s.t) / h;
          if (kq == kn) {
#pragma unroll
            for (int r = 0; r < C; ++r) dst[r] = yn[r];
          } else {
            float w[7];
            dense_weights<Tab, float>(th, w);
#pragma unroll
            for (int r = 0; r < C; ++r) {
              float acc = w[0] * k1[r];
              if constexpr (K2) acc = madd(w[1], k2[r], acc);
              acc = madd(w[2], k3[r], acc);
              acc = madd(w[3], k4[r], acc);
              acc = madd(w[4], k5[r], acc);
              acc = madd(w[5], k6[r], acc);
              acc = madd(w[6], f[r], acc);
              dst[r] = y[r] + madd(h, acc, ylo[r]);
            }
          }
          if (a.yp) {  // dy/dt = sum_i b_i'(theta) k_i (the step size cancels)
            float w[7];
            dense_dweights<Tab, float>(th, w);
            const float dir = (s.flags & FL_REVERSE) ? -1.0f : 1.0f;
            float* dp = a.yp + ((size_t)i * a.K + s.cursor) * D + coff;
#pragma unroll
            for (int r = 0; r < C; ++r) {
              float acc = w[0] * k1[r];
              if constexpr (K2) acc = madd(w[1], k2[r], acc);
              acc = madd(w[2], k3[r], acc);
              acc = madd(w[3], k4[r], acc);
              acc = madd(w[4], k5[r], acc);
              acc = madd(w[5], k6[r], acc);
              acc = madd(w[6], f[r], acc);
              dp[r] = dir * acc;
            }
          }
          s.cursor++;
        }
        float fac;
        if (err == 0.0f) {
          fac = a.o.fac_max_f;
        } else {
          fac = a.o.safety_f * ctl_pow(err, -a.o.beta1_f);
          if (a.o.beta2 != 0.0) fac = fac * ctl_pow(s.err_prev, a.o.beta2_f);
          if (a.o.beta3 != 0.0) fac = fac * ctl_pow(s.err_prev2, -a.o.beta3_f);
        }
        fac = tmin(tmax(fac, a.o.fac_min_f), a.o.fac_max_f);
        if (s.flags & FL_PREV_REJ) fac = tmin(fac, 1.0f);
        h_next = h * fac;
        s.err_prev2 = s.err_prev;
        s.err_prev = tmax(err, 1e-4f);
        s.flags &= ~FL_PREV_REJ;
        s.n_acc++;
        s.t = t_next;
#pragma unroll
        for (int r = 0; r < C; ++r) {
          y[r] = yn[r];
          ylo[r] = ylon[r];
          k1[r] = f[r];  // FSAL: k1 <- k7
        }
        if (last) s.status = ST_SUCCESS;
        else s.rem = __double2float_rd(s.t1 - s.t);
        if (s.target >= 0 && s.n_acc >= s.target) s.status = ST_SUCCESS;  // segment re-solved
      } else {
        const float fac =
            finite ? tmin(tmax(a.o.safety_f * ctl_pow(err, -a.o.beta1_f),
                               a.o.fac_min_f),
                          1.0f)
                   : a.o.fac_min_f;
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
        if (MODE == MLP_PLAIN_STEP) park();
      } else if (s.target >= 0) {  // a re-solved segment: its end, no outputs
        if (sub == 0) a.rs_t1[i] = flip(s.t, rev_mask(s.flags));
        s.phase = PH_IDLE;
        if (MODE == MLP_FUSED) need_grab = true;
      } else {
        if (s.status != ST_SUCCESS) {  // points the failed instance never reached
          float* ye = a.ye + (size_t)i * a.K * D + coff;
          for (int q = s.cursor; q < a.K; ++q)
#pragma unroll
            for (int r = 0; r < C; ++r) ye[(size_t)q * D + r] = nan_(0.0f);
          if (a.yp)
            for (int q = s.cursor; q < a.K; ++q)
#pragma unroll
              for (int r = 0; r < C; ++r)
                a.yp[((size_t)i * a.K + q) * D + coff + r] = nan_(0.0f);
        }
#pragma unroll
        for (int r = 0; r < C; ++r) a.yf[(size_t)i * D + coff + r] = y[r];
        if (sub == 0) {
          const int at = s.n_acc + s.n_rej;
          a.n_acc[i] = s.n_acc;
          a.n_rej[i] = s.n_rej;
          a.n_fe[i] = (a.o.h0 > 0.0 ? 1 : 2) + 6 * at;
          a.status[i] = s.status;
          if (a.trace.cap > 0) a.trace.len[i] = at < a.trace.cap ? at : a.trace.cap;
        }
        s.phase = PH_IDLE;
        if (MODE == MLP_FUSED) need_grab = true;
      }
    }
  }
  if constexpr (Cfg::STACKED) {
    if (tid == 0) {
      // the ring's copies still in flight land before the CTA exits
      // (stages g_chunk .. g_chunk + NSL - 1 were issued and not consumed)
      constexpr uint32_t NSL = Cfg::NSL;
      const uint32_t first = g_chunk, last = g_chunk + NSL - 1;
      for (uint32_t x = first; x <= last; ++x)
        if (!tc::mbar_wait(&mbar_full[x % NSL], (x / NSL) & 1u)) atomicExch(&abort_s, 1);
    }
  }
  if (abort_s && tid == 0) atomicExch(a.err, 1);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, Cfg::TMEM_COLS);
}

template <class Cfg, class Tab = DP5>
__global__ void __launch_bounds__(256, 1) k_mlp_fused(MlpArgs a) {
  mlp_solver<Cfg, MLP_FUSED, Tab>(a);
}
template <class Cfg, class Tab = DP5>
__global__ void __launch_bounds__(256, 1) k_mlp_plain_init(MlpArgs a) {
  mlp_solver<Cfg, MLP_PLAIN_INIT, Tab>(a);
}
template <class Cfg, class Tab = DP5>
__global__ void __launch_bounds__(256, 1) k_mlp_plain_step(MlpArgs a) {
  mlp_solver<Cfg, MLP_PLAIN_STEP, Tab>(a);
}

// The BF16 weights W_l [N_l][K_in,l] (row-major) as core-matrix images with
// K padded to K_l, for all layers and all copies in one launch.  Layouts:
//   IMG_TILE     one [N_l][K_l] tile per layer (weights resident in shared memory)
//   IMG_CHUNKS   K_l/16 consecutive [N_l][16] tiles (the streamed K chunks)
//   IMG_CHUNKS2  IMG_CHUNKS split in two half images (`half` bytes apart) for
//                a CTA pair: an M = 256 product of width NW = min(N_l, 256)
//                takes columns [NW j, NW j + NW/2) from CTA 0 and the next
//                NW/2 from CTA 1, so half r of chunk c holds those rows of
//                every product j, as [N_l/2][16] (rows NW/2 j .. of product j)
//   IMG_TCHUNKS2 W_l^T in K chunks along the layer's outputs for a CTA pair:
//                half r of chunk c is an MN-major [16][K_l/2] tile of outputs
//                16c .. 16c+15, its inputs split as in IMG_CHUNKS2
enum : int { IMG_TILE = 0, IMG_CHUNKS = 1, IMG_CHUNKS2 = 2, IMG_TCHUNKS2 = 3 };
struct ImageJob {
  const uint16_t* W[MLP_MAX_LAYERS];
  int N[MLP_MAX_LAYERS], Kin[MLP_MAX_LAYERS], Kp[MLP_MAX_LAYERS];
  size_t off[MLP_MAX_LAYERS];      // layer offset inside one copy (one half)
  long long start[MLP_MAX_LAYERS + 1];  // element ranges of the layers
  int nl, reps, mode;
  size_t stride;  // bytes between copies
  size_t half;    // bytes between the two halves of a pair image
};
// (product, CTA, row inside the CTA's part) of index x along a pair
// product's N of width n_total
__device__ __forceinline__ void pair_split(int x, int n_total, int& r, int& xr) {
  const int nw = n_total < 256 ? n_total : 256, hw = nw / 2;
  const int j = x / nw, p = x - j * nw;
  r = p / hw;
  xr = j * hw + (p - r * hw);
}
__global__ void k_mlp_images(ImageJob j, unsigned char* img) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= j.start[j.nl]) return;
  int l = 0;
  while (e >= j.start[l + 1]) ++l;
  const long long x = e - j.start[l];
  const int Kp = j.Kp[l], N = j.N[l];
  const int n = (int)(x / Kp), k = (int)(x % Kp);
  const uint16_t v = k < j.Kin[l] ? j.W[l][(size_t)n * j.Kin[l] + k] : (uint16_t)0;
  size_t off;
  if (j.mode == IMG_TILE) {
    off = tc::cm_offset(n, k, Kp);
  } else if (j.mode == IMG_CHUNKS) {
    off = (size_t)(k / 16) * (size_t)N * 32u + tc::cm_offset(n, k % 16, 16);
  } else if (j.mode == IMG_CHUNKS2) {
    int r, nr;
    pair_split(n, N, r, nr);
    off = (size_t)r * j.half + (size_t)(k / 16) * (size_t)N * 16u + tc::cm_offset(nr, k % 16, 16);
  } else {
    int r, kr;
    pair_split(k, Kp, r, kr);
    off = (size_t)r * j.half + (size_t)(n / 16) * 16u * (size_t)Kp + tc::cm_offset(n % 16, kr, Kp / 2);
  }
  for (int r = 0; r < j.reps; ++r)
    *reinterpret_cast<uint16_t*>(img + (size_t)r * j.stride + j.off[l] + off) = v;
}

// Host side: the image job of a network config (W_off / T_off give the
// layer offsets of the chosen layout).
template <class Cfg>
static tode_err build_images(const tode_field_desc* f, unsigned char* img, int mode, int reps,
                             size_t stride, const size_t (&layer_off)[MLP_MAX_LAYERS],
                             cudaStream_t st, size_t half = 0) {
  ImageJob j{};
  j.nl = Cfg::NL;
  j.reps = reps;
  j.mode = mode;
  j.stride = stride;
  j.half = half;
  j.start[0] = 0;
  for (int l = 0; l < Cfg::NL; ++l) {
    j.W[l] = (const uint16_t*)f->W[l];
    j.N[l] = Cfg::N_of(l);
    j.Kin[l] = f->widths[l];
    j.Kp[l] = Cfg::K_of(l);
    j.off[l] = layer_off[l];
    j.start[l + 1] = j.start[l] + (long long)j.N[l] * j.Kp[l];
  }
  const long long n = j.start[Cfg::NL];
  k_mlp_images<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(j, img);
  TODE_CUDA_TRY(cudaGetLastError());
  return TODE_OK;
}

// ======================================================================
// Discrete adjoint of the MLP-field solve (torchode App. A: gradients by
// backpropagation through the solver), on the frozen mesh the forward
// recorded (every accepted step: y_n, FSAL k1, t_n, h_n).
//
// Rows of a 128-row tile reverse their own instances (assigned statically,
// row r of CTA c takes instances c*128 + r, c*128 + r + 128*grid, ..., so the
// weight gradients are summed in a fixed order).  Reversing one accepted step
// takes 7 rounds for every row (stages 7..1), so all rows of a tile stay in
// step; the forward recorded each accepted step's stage inputs Y_2..Y_7, so a
// round runs the hidden layers at Y_s and then the backward chain for the
// stage cotangent kbar_s.  A round, for the whole tile:
//   gh2 = kbar W3        dW3^T += h2^T kbar          (h2: split BF16 tile)
//   delta2 = gh2 (1 - h2^2)
//   gh1 = delta2 W2      dW2 += delta2^T h1, db2 += delta2^T 1
//   delta1 = gh1 (1 - h1^2)
//   gx = delta1 W1       dW1 += delta1^T [X | 1]     (the 1 column gives db1)
// Transposed operands are the same shared-memory tiles read MN-major; dW
// accumulates in tensor memory over the whole kernel and is written once
// per CTA as a partial, which k_mlp_grad_reduce sums over CTAs in order.
// Y_1 is the step's start, Y_2..Y_7 come from the tape.
// ======================================================================
template <class Cfg> struct MlpAdjLayout {
  static constexpr int D = Cfg::D, H = Cfg::H, K0 = Cfg::K0;
  static_assert(Cfg::NL == 3 && Cfg::SPLIT, "adjoint built for two hidden layers, split");
  static_assert(D == 32 && H == 128 && K0 == 48, "tensor-memory plan below");
  static constexpr int S_W = 0;
  static constexpr int S_XH = ((Cfg::WIMG_BYTES + 1023) / 1024) * 1024;
  static constexpr int S_XL = S_XH + 128 * K0 * 2;
  static constexpr int S_H1H = S_XL + 128 * K0 * 2;
  static constexpr int S_H1L = S_H1H + 128 * H * 2;
  static constexpr int S_H2H = S_H1L + 128 * H * 2;
  static constexpr int S_H2L = S_H2H + 128 * H * 2;
  static constexpr int S_D3H = S_H2L + 128 * H * 2;
  static constexpr int S_D3L = S_D3H + 128 * D * 2;
  static constexpr int S_ONES = S_D3L + 128 * D * 2;
  static constexpr int S_BIAS = S_ONES + 128 * 16 * 2;
  static constexpr int S_END = S_BIAS + Cfg::BIAS_FLOATS * 4;
  static_assert(S_END <= 232448 - 1024, "shared memory");
  // tensor memory columns: accumulators on 32-column boundaries
  //   R [0,128)  D1 [128,256)  D0 [256,304)  DB [320,336)  D2 [352,384)
  static constexpr uint32_t T_R = 0, T_D1 = 128, T_D0 = 256, T_DB = 320, T_D2 = 352,
                            T_COLS = 512;
  // per-CTA partial gradient block (floats)
  static constexpr int P_W0 = 0;                 // [H][K0]  (col D: t weight, col D+1: db1)
  static constexpr int P_W1 = P_W0 + H * K0;     // [H][H]
  static constexpr int P_B1 = P_W1 + H * H;      // [H]
  static constexpr int P_W2T = P_B1 + H;         // [H][D]   (dW3 transposed)
  static constexpr int P_B2 = P_W2T + H * D;     // [D]
  static constexpr int P_FLOATS = P_B2 + D;
};

struct MlpAdjArgs {
  int B, K;
  const double* t0;
  const double* t1;
  const double* te;
  const int32_t* n_acc;
  const int32_t* status;
  int slots;
  const float* tp_y;
  const float* tp_k1;
  const double* tp_t;
  const float* tp_h;
  const float* tp_ys;  // [B][slots][6][D]: Y_2..Y_7
  const float* gye;
  const float* gyf;
  float* gy0;
  const unsigned char* wimg;
  const float* bias[MLP_MAX_LAYERS];
  float* part;   // [grid][P_FLOATS]
  int32_t* overflow;
  int32_t* err;
  double* gts;   // [B] or NULL: each instance's time-translation sum (see tode.h)
};

constexpr int ADJ_ROUNDS = 7;  // one reverse round per stage, 7..1

__device__ __forceinline__ double dp_c(int s) {
  using C = DP5;
  return s == 2 ? C::c2 : s == 3 ? C::c3 : s == 4 ? C::c4 : s == 5 ? C::c5 : s >= 6 ? 1.0 : 0.0;
}
// c_s of the pair Tab (dopri5: dp_c)
template <class Tab> __device__ __forceinline__ double tab_c(int s) {
  if constexpr (std::is_same<Tab, DP5>::value) {
    return dp_c(s);
  } else {
    return s == 2 ? Tab::c(2) : s == 3 ? Tab::c(3) : s == 4 ? Tab::c(4) : s == 5 ? Tab::c(5)
         : s == 6 ? Tab::c(6) : s == 7 ? Tab::c(7) : 0.0;
  }
}
// o = k[j] for a runtime j (selects; keeps k in registers)
__device__ __forceinline__ void pick7(const float (&k)[7][16], int j, float (&o)[16]) {
#pragma unroll
  for (int r = 0; r < 16; ++r) o[r] = k[0][r];
#pragma unroll
  for (int u = 1; u < 7; ++u)
    if (u == j) {
#pragma unroll
      for (int r = 0; r < 16; ++r) o[r] = k[u][r];
    }
}

template <class Cfg, class Tab = DP5>
__global__ void __launch_bounds__(256, 1) k_mlp_adjoint(MlpAdjArgs a) {
  using L = MlpAdjLayout<Cfg>;
  constexpr int D = Cfg::D, H = Cfg::H, K0 = Cfg::K0, C = Cfg::C, HC = Cfg::HC;
  static_assert(C == 16, "16 state components per thread");
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar_mma, mbar_w;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  unsigned char* sW = sm + L::S_W;
  unsigned char* sXh = sm + L::S_XH;
  unsigned char* sXl = sm + L::S_XL;
  unsigned char* sH1h = sm + L::S_H1H;
  unsigned char* sH1l = sm + L::S_H1L;
  unsigned char* sH2h = sm + L::S_H2H;
  unsigned char* sH2l = sm + L::S_H2L;
  unsigned char* sD3h = sm + L::S_D3H;
  unsigned char* sD3l = sm + L::S_D3L;
  unsigned char* sOnes = sm + L::S_ONES;
  float* sBias = reinterpret_cast<float*>(sm + L::S_BIAS);

  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & 127, half = tid >> 7;
  const int coff = half * C;
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  const int grid = gridDim.x;

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
    for (int l = 0; l < 3; ++l)
      tc::bulk_g2s(sW + Cfg::W_off(l), a.wimg + Cfg::W_off(l), (uint32_t)Cfg::W_bytes(l), &mbar_w);
  }
  {
    int o = 0;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const int n = Cfg::N_of(l);
      for (int j = tid; j < n; j += 256) sBias[o + j] = a.bias[l] ? a.bias[l][j] : 0.0f;
      o += n;
    }
  }
  // input tiles: zero, with a constant 1 in column D+1 (hi) for db1
  for (int j = tid; j < 128 * K0 * 2 / 16; j += 256) {
    reinterpret_cast<uint4*>(sXh)[j] = make_uint4(0, 0, 0, 0);
    reinterpret_cast<uint4*>(sXl)[j] = make_uint4(0, 0, 0, 0);
  }
  // ones operand for db2: [K = 128 rows][N = 16], column 0 = 1
  for (int j = tid; j < 128 * 16; j += 256) {
    const int r = j / 16, c = j % 16;
    *reinterpret_cast<__nv_bfloat16*>(sOnes + tc::cm_offset(r, c, 16)) =
        __float2bfloat16_rn(c == 0 ? 1.0f : 0.0f);
  }
  __syncthreads();
  if (tid < 128)
    *reinterpret_cast<__nv_bfloat16*>(sXh + tc::cm_offset(tid, D + 1, K0)) =
        __float2bfloat16_rn(1.0f);
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base_s, L::T_COLS);
    tc::tmem_relinquish();
  }
  if (!tc::mbar_wait(&mbar_w, 0)) atomicExch(&abort_s, 1);
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_base_s;
  const uint32_t tl = tbase + lane_base;  // this warp's lane quarter
  // accumulator chunks in flight per wait in the hidden epilogue (2 and 4
  // measured no faster here: the round's registers are mostly the cotangents)
  constexpr int ADJ_NLD = 1;
  uint32_t parity = 0;
  bool dw_first = true;  // the next backward round starts the dW accumulators

  // ---- per-row reverse state
  int inst = blockIdx.x * 128 + row;
  bool act = false;
  int n = -1, N = 0, q = -1;
  bool bad = false;
  double tn = 0.0, tnext = 0.0;
  float h = 0.0f;
  unsigned long long rmask = 0;  // the instance runs backward in time: tau = -t, field -f
  float tsum = 0.0f;  // the time inputs' cotangents of the instance's stages (a.gts)
  float yb[16], db3[16], kb[7][16];
#pragma unroll
  for (int r = 0; r < C; ++r) {
    yb[r] = db3[r] = 0.0f;
#pragma unroll
    for (int j = 0; j < 7; ++j) kb[j][r] = 0.0f;
  }

  // step n of instance i: its time and size (the stage inputs come from the
  // tape round by round)
  auto load_step = [&](int i) {
    const size_t o = (size_t)i * a.slots + n;
    tn = a.tp_t[o];
    h = a.tp_h[o];
    tnext = (n == N - 1) ? flip(a.t1[i], rmask) : tn + (double)h;
    act = true;
  };
  // Y_s of the step being reversed: Y_1 = y_n, Y_2..Y_7 as the forward recorded
  auto load_stage = [&](int s_, float (&Yo)[16]) {
    const size_t o = (size_t)inst * a.slots + n;
    const float4* p = s_ == 1
        ? reinterpret_cast<const float4*>(a.tp_y + o * D + coff)
        : reinterpret_cast<const float4*>(a.tp_ys + (o * 6 + (s_ - 2)) * D + coff);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const float4 u = p[v];
      Yo[4 * v] = u.x, Yo[4 * v + 1] = u.y, Yo[4 * v + 2] = u.z, Yo[4 * v + 3] = u.w;
    }
  };
  // finish the current instance (if `finishing`) and move to the next one
  // that has a step to reverse
  auto next_work = [&](bool finishing) {
    while (true) {
      if (finishing) {
        const int i = inst;
        if (!bad && a.gye) {
          const long long k0 = tkey(flip(a.t0[i], rmask));
          for (; q >= 0; --q)
            if (tkey(flip(a.te[(size_t)i * a.K + q], rmask)) == k0)
#pragma unroll
              for (int r = 0; r < C; ++r) yb[r] += a.gye[((size_t)i * a.K + q) * D + coff + r];
        }
#pragma unroll
        for (int r = 0; r < C; ++r) a.gy0[(size_t)i * D + coff + r] = bad ? nan_(0.0f) : yb[r];
        if (a.gts && half == 0) a.gts[i] = bad ? (double)nan_(0.0f) : (double)tsum;
        inst += grid * 128;
        finishing = false;
      }
      if (inst >= a.B) {
        act = false;
        return;
      }
      const int i = inst;
      N = a.n_acc[i];
      bad = a.status[i] != ST_SUCCESS;
      rmask = (a.t1[i] < a.t0[i]) ? SIGN_BIT : 0ULL;
      if (!bad && N > a.slots) {
        bad = true;
        if (half == 0) atomicExch(a.overflow, 1);
      }
#pragma unroll
      for (int r = 0; r < C; ++r) yb[r] = a.gyf ? a.gyf[(size_t)i * D + coff + r] : 0.0f;
      tsum = 0.0f;
      q = a.K - 1;
      n = N - 1;
      if (bad || n < 0) {
        finishing = true;
        continue;
      }
      load_step(i);
      return;
    }
  };
  next_work(false);

  auto barrier = [&]() {
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  };
  auto wait_mma = [&]() {
    if (!tc::mbar_wait(&mbar_mma, parity)) atomicExch(&abort_s, 1);
    parity ^= 1u;
    tc::fence_after_sync();
  };
  // hidden epilogue: h = tanh(acc + b) into a split tile
  // (ADJ_NLD accumulator chunks in flight per wait, additions in FP32x2 pairs)
  auto hidden_epi = [&](const float* bl, unsigned char* th, unsigned char* tlo) {
#pragma unroll
    for (int c0 = 0; c0 < HC; c0 += 16 * ADJ_NLD) {
      float v[ADJ_NLD][16];
#pragma unroll
      for (int u = 0; u < ADJ_NLD; ++u) tc::tmem_ld16(tl + L::T_R + half * HC + c0 + 16 * u, v[u]);
      tc::tmem_wait_ld();
#pragma unroll
      for (int u = 0; u < ADJ_NLD; ++u) {
        const int col = half * HC + c0 + 16 * u;
        const float4* b4 = reinterpret_cast<const float4*>(bl + col);
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          const float4 bq = b4[q4];
          const float2 t0 = tanh_acc2(__fadd2_rn(make_float2(v[u][4 * q4], v[u][4 * q4 + 1]),
                                                 make_float2(bq.x, bq.y)));
          const float2 t1 = tanh_acc2(__fadd2_rn(make_float2(v[u][4 * q4 + 2], v[u][4 * q4 + 3]),
                                                 make_float2(bq.z, bq.w)));
          v[u][4 * q4] = t0.x, v[u][4 * q4 + 1] = t0.y;
          v[u][4 * q4 + 2] = t1.x, v[u][4 * q4 + 3] = t1.y;
        }
        store_row16<true>(th, tlo, row, col, H, v[u]);
      }
    }
  };
  // backward epilogue: delta = acc (1 - h^2) with h = hi + lo of the tile;
  // the split delta replaces h in place (row-local; its other readers are done)
  auto delta_epi = [&](unsigned char* th, unsigned char* tlo) {
#pragma unroll
    for (int c = 0; c < HC; c += 16) {
      const int col = half * HC + c;
      float v[16];
      tc::tmem_ld16(tl + L::T_R + col, v);
#pragma unroll
      for (int c8 = 0; c8 < 2; ++c8) {
        const uint32_t off = tc::cm_offset(row, col + 8 * c8, H);
        const uint4 hv = *reinterpret_cast<const uint4*>(th + off);
        const uint4 lv = *reinterpret_cast<const uint4*>(tlo + off);
        const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w}, lw[4] = {lv.x, lv.y, lv.z, lv.w};
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&hw[j]);
          const __nv_bfloat162 l2 = *reinterpret_cast<const __nv_bfloat162*>(&lw[j]);
          // x = hi + lo, then v * (1 - x^2), the pair's operations packed
          const float2 x = __fadd2_rn(make_float2(__low2float(h2), __high2float(h2)),
                                      make_float2(__low2float(l2), __high2float(l2)));
          const float2 g = __ffma2_rn(make_float2(-x.x, -x.y), x, make_float2(1.0f, 1.0f));
          const float2 d = __fmul2_rn(make_float2(v[8 * c8 + 2 * j], v[8 * c8 + 2 * j + 1]), g);
          v[8 * c8 + 2 * j] = d.x;
          v[8 * c8 + 2 * j + 1] = d.y;
        }
      }
      store_row16<true>(th, tlo, row, col, H, v);
    }
  };
  const float bw[7] = {float(Tab::b(1)), float(Tab::b(2)), float(Tab::b(3)), float(Tab::b(4)),
                       float(Tab::b(5)), float(Tab::b(6)), float(Tab::b(7))};
  const uint32_t idH = tc::idesc_bf16_f32(128, H);

  for (int rnd = 0;; ++rnd) {
    const int ph = rnd % ADJ_ROUNDS;
    if (ph == 0 && __syncthreads_or(act) == 0) break;
    const int s = 7 - ph;  // stage reversed this round (block-uniform)

    // ---- stage input [Y_s; t_s] and the cotangent kbar_s of this row
    float Y[16], d3[16];
    float tin = 0.0f;
    if (act && s == 7) {
      // kbar_i = h b_i ybar_{n+1} + sum_{tau in step} h b_i(theta_tau) ybar_tau
      const int i = inst;
#pragma unroll
      for (int j = 0; j < 7; ++j)
#pragma unroll
        for (int r = 0; r < C; ++r) kb[j][r] = h * bw[j] * yb[r];
      const long long kt = tkey(tn), kn = tkey(tnext);
      while (q >= 0) {
        const double tq = flip(a.te[(size_t)i * a.K + q], rmask);
        const long long kq = tkey(tq);
        if (!(kq > kt)) break;
        if (a.gye) {
          float gq[16], w[7];
#pragma unroll
          for (int r = 0; r < C; ++r) gq[r] = a.gye[((size_t)i * a.K + q) * D + coff + r];
          if (kq == kn) {
#pragma unroll
            for (int j = 0; j < 7; ++j) w[j] = bw[j];
          } else {
            dense_weights<Tab, float>(float(tq - tn) / h, w);
          }
#pragma unroll
          for (int j = 0; j < 7; ++j)
#pragma unroll
            for (int r = 0; r < C; ++r) kb[j][r] = madd(h * w[j], gq[r], kb[j][r]);
#pragma unroll
          for (int r = 0; r < C; ++r) yb[r] += gq[r];
        }
        q--;
      }
    }
    if (act) {
      load_stage(s, Y);
      tin = (float)flip(tn + tab_c<Tab>(s) * (double)h, rmask);  // the caller's time
      pick7(kb, s - 1, d3);
      if (rmask) {  // the field in tau is -f: its products take -kbar
#pragma unroll
        for (int r = 0; r < C; ++r) d3[r] = -d3[r];
      }
    } else {
#pragma unroll
      for (int r = 0; r < C; ++r) Y[r] = d3[r] = 0.0f;
    }
    store_row16<true>(sXh, sXl, row, coff, K0, Y);
    store_row16<true>(sD3h, sD3l, row, coff, D, d3);
    if (half == 1) {
      const __nv_bfloat16 th = __float2bfloat16_rn(tin);
      const __nv_bfloat16 tlo = __float2bfloat16_rn(tin - __bfloat162float(th));
      *reinterpret_cast<__nv_bfloat16*>(sXh + tc::cm_offset(row, D, K0)) = th;
      *reinterpret_cast<__nv_bfloat16*>(sXl + tc::cm_offset(row, D, K0)) = tlo;
    }
    barrier();

    // F0: acc = X W1^T (hi + lo)
    if (tid == 0) {
      const uint32_t wa = tc::smem_u32(sW + Cfg::W_off(0));
      for (int kk = 0; kk < K0 / 16; ++kk) {
        const uint64_t db = tc::smem_desc(wa + kk * 256, 128, K0 * 16);
        tc::mma_bf16(tbase + L::T_R, tc::smem_desc(tc::smem_u32(sXh) + kk * 256, 128, K0 * 16), db,
                     idH, kk > 0);
        tc::mma_bf16(tbase + L::T_R, tc::smem_desc(tc::smem_u32(sXl) + kk * 256, 128, K0 * 16), db,
                     idH, true);
      }
      tc::mma_commit(&mbar_mma);
    }
    wait_mma();
    hidden_epi(sBias, sH1h, sH1l);
    barrier();
    // F1: acc = h1 W2^T
    if (tid == 0) {
      const uint32_t wa = tc::smem_u32(sW + Cfg::W_off(1));
      for (int kk = 0; kk < H / 16; ++kk) {
        const uint64_t db = tc::smem_desc(wa + kk * 256, 128, H * 16);
        tc::mma_bf16(tbase + L::T_R, tc::smem_desc(tc::smem_u32(sH1h) + kk * 256, 128, H * 16), db,
                     idH, kk > 0);
        tc::mma_bf16(tbase + L::T_R, tc::smem_desc(tc::smem_u32(sH1l) + kk * 256, 128, H * 16), db,
                     idH, true);
      }
      tc::mma_commit(&mbar_mma);
    }
    wait_mma();
    hidden_epi(sBias + H, sH2h, sH2l);
    barrier();

    float fg[16];  // g = J_f(Y_s)^T kbar_s
    float tcot = 0.0f;  // and the time input's cotangent (a.gts only)
    {
      const bool acc0 = !dw_first;
      // B2: acc = kbar W3;  dW3^T += h2^T kbar  (split: hi*hi + lo*hi + hi*lo)
      if (tid == 0) {
        const uint32_t w3 = tc::smem_u32(sW + Cfg::W_off(2));
        const uint32_t dh = tc::smem_u32(sD3h), dl = tc::smem_u32(sD3l);
        const uint32_t idR = tc::idesc_bf16_f32(128, H, false, true);
        for (int kk = 0; kk < D / 16; ++kk) {
          const uint64_t db = tc::smem_desc_mn(w3 + kk * 2 * (H * 16), H * 16);
          tc::mma_bf16(tbase + L::T_R, tc::smem_desc(dh + kk * 256, 128, D * 16), db, idR, kk > 0);
          tc::mma_bf16(tbase + L::T_R, tc::smem_desc(dl + kk * 256, 128, D * 16), db, idR, true);
        }
        const uint32_t idT = tc::idesc_bf16_f32(128, D, true, true);
        const uint32_t hh = tc::smem_u32(sH2h), hl = tc::smem_u32(sH2l);
        for (int kk = 0; kk < 128 / 16; ++kk) {
          const uint64_t bh = tc::smem_desc_mn(dh + kk * 2 * (D * 16), D * 16);
          const uint64_t bl = tc::smem_desc_mn(dl + kk * 2 * (D * 16), D * 16);
          const uint64_t ah = tc::smem_desc_mn(hh + kk * 2 * (H * 16), H * 16);
          const uint64_t al = tc::smem_desc_mn(hl + kk * 2 * (H * 16), H * 16);
          tc::mma_bf16(tbase + L::T_D2, ah, bh, idT, acc0 || kk > 0);
          tc::mma_bf16(tbase + L::T_D2, al, bh, idT, true);
          tc::mma_bf16(tbase + L::T_D2, ah, bl, idT, true);
        }
        tc::mma_commit(&mbar_mma);
      }
      wait_mma();
      delta_epi(sH2h, sH2l);  // delta2 replaces h2
      barrier();
      // B1: acc = delta2 W2;  dW2 += delta2^T h1;  db2 += delta2^T 1
      if (tid == 0) {
        const uint32_t w2 = tc::smem_u32(sW + Cfg::W_off(1));
        const uint32_t dh = tc::smem_u32(sH2h), dl = tc::smem_u32(sH2l);
        const uint32_t idR = tc::idesc_bf16_f32(128, H, false, true);
        for (int kk = 0; kk < H / 16; ++kk) {
          const uint64_t db = tc::smem_desc_mn(w2 + kk * 2 * (H * 16), H * 16);
          tc::mma_bf16(tbase + L::T_R, tc::smem_desc(dh + kk * 256, 128, H * 16), db, idR, kk > 0);
          tc::mma_bf16(tbase + L::T_R, tc::smem_desc(dl + kk * 256, 128, H * 16), db, idR, true);
        }
        const uint32_t idT = tc::idesc_bf16_f32(128, H, true, true);
        const uint32_t idB = tc::idesc_bf16_f32(128, 16, true, true);
        const uint32_t hh = tc::smem_u32(sH1h), hl = tc::smem_u32(sH1l);
        for (int kk = 0; kk < 128 / 16; ++kk) {
          const uint64_t ah = tc::smem_desc_mn(dh + kk * 2 * (H * 16), H * 16);
          const uint64_t al = tc::smem_desc_mn(dl + kk * 2 * (H * 16), H * 16);
          const uint64_t bh = tc::smem_desc_mn(hh + kk * 2 * (H * 16), H * 16);
          const uint64_t bl = tc::smem_desc_mn(hl + kk * 2 * (H * 16), H * 16);
          const uint64_t b1 = tc::smem_desc_mn(tc::smem_u32(sOnes) + kk * 2 * (16 * 16), 16 * 16);
          const bool acc = acc0 || kk > 0;
          tc::mma_bf16(tbase + L::T_D1, ah, bh, idT, acc);
          tc::mma_bf16(tbase + L::T_D1, al, bh, idT, true);
          tc::mma_bf16(tbase + L::T_D1, ah, bl, idT, true);
          tc::mma_bf16(tbase + L::T_DB, ah, b1, idB, acc);
          tc::mma_bf16(tbase + L::T_DB, al, b1, idB, true);
        }
        tc::mma_commit(&mbar_mma);
      }
      wait_mma();
      delta_epi(sH1h, sH1l);  // delta1 replaces h1
      barrier();
      // B0: acc = delta1 W1;  dW1 += delta1^T [X | 1]
      if (tid == 0) {
        const uint32_t w1 = tc::smem_u32(sW + Cfg::W_off(0));
        const uint32_t dh = tc::smem_u32(sH1h), dl = tc::smem_u32(sH1l);
        const uint32_t idR = tc::idesc_bf16_f32(128, K0, false, true);
        for (int kk = 0; kk < H / 16; ++kk) {
          const uint64_t db = tc::smem_desc_mn(w1 + kk * 2 * (K0 * 16), K0 * 16);
          tc::mma_bf16(tbase + L::T_R, tc::smem_desc(dh + kk * 256, 128, H * 16), db, idR, kk > 0);
          tc::mma_bf16(tbase + L::T_R, tc::smem_desc(dl + kk * 256, 128, H * 16), db, idR, true);
        }
        const uint32_t idT = tc::idesc_bf16_f32(128, K0, true, true);
        const uint32_t xh = tc::smem_u32(sXh), xl = tc::smem_u32(sXl);
        for (int kk = 0; kk < 128 / 16; ++kk) {
          const uint64_t ah = tc::smem_desc_mn(dh + kk * 2 * (H * 16), H * 16);
          const uint64_t al = tc::smem_desc_mn(dl + kk * 2 * (H * 16), H * 16);
          const uint64_t bh = tc::smem_desc_mn(xh + kk * 2 * (K0 * 16), K0 * 16);
          const uint64_t bl = tc::smem_desc_mn(xl + kk * 2 * (K0 * 16), K0 * 16);
          const bool acc = acc0 || kk > 0;
          tc::mma_bf16(tbase + L::T_D0, ah, bh, idT, acc);
          tc::mma_bf16(tbase + L::T_D0, al, bh, idT, true);
          tc::mma_bf16(tbase + L::T_D0, ah, bl, idT, true);
        }
        tc::mma_commit(&mbar_mma);
      }
      wait_mma();
      tc::tmem_ld16(tl + L::T_R + coff, fg);
      // column D of the product: the cotangent of the field's time input
      if (a.gts) tcot = tc::tmem_ld1(tl + L::T_R + D);
      tc::tmem_wait_ld();
      dw_first = false;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (abort_s) break;

    // ---- consume (row-local)
    if (!act) continue;
    {
      float kbs[16];
      pick7(kb, s - 1, kbs);
#pragma unroll
      for (int r = 0; r < C; ++r) db3[r] += rmask ? -kbs[r] : kbs[r];
#pragma unroll
      for (int j = 0; j < 6; ++j) {  // kbar_j += h a_{s,j} g  (j < s)
        if (j + 1 >= s) continue;
        const float c = h * tab_a<Tab>(s, j + 1);
#pragma unroll
        for (int r = 0; r < C; ++r) kb[j][r] = madd(c, fg[r], kb[j][r]);
      }
#pragma unroll
      for (int r = 0; r < C; ++r) yb[r] += fg[r];
      tsum += tcot;
      if (s == 1) {  // step n reversed
        n -= 1;
        if (n >= 0) load_step(inst);
        else next_work(true);
      }
    }
  }

  // ---- per-CTA partial gradients: tensor-memory accumulators, db3 over rows
  float* P = a.part + (size_t)blockIdx.x * L::P_FLOATS;
  tc::fence_after_sync();
  {
    float v[16];
    // dW1 (and its t and bias columns): lane = output unit of layer 1
    for (int c = half * 32; c < (half ? K0 : 32); c += 16) {
      tc::tmem_ld16(tl + L::T_D0 + c, v);
      tc::tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j) P[L::P_W0 + row * K0 + c + j] = dw_first ? 0.0f : v[j];
    }
#pragma unroll
    for (int c = 0; c < HC; c += 16) {
      const int col = half * HC + c;
      tc::tmem_ld16(tl + L::T_D1 + col, v);
      tc::tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j) P[L::P_W1 + row * H + col + j] = dw_first ? 0.0f : v[j];
    }
    tc::tmem_ld16(tl + L::T_DB, v);
    tc::tmem_wait_ld();
    if (half == 0) P[L::P_B1 + row] = dw_first ? 0.0f : v[0];
    tc::tmem_ld16(tl + L::T_D2 + coff, v);
    tc::tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < 16; ++j) P[L::P_W2T + row * D + coff + j] = dw_first ? 0.0f : v[j];
  }
  // db3: sum the rows' accumulators in a fixed order (reuses the h2 tile)
  float* sDb = reinterpret_cast<float*>(sH2h);
  tc::fence_before_sync();
  __syncthreads();
#pragma unroll
  for (int r = 0; r < C; ++r) sDb[row * D + coff + r] = db3[r];
  __syncthreads();
  if (tid < D) {
    float acc = 0.0f;
    for (int rr = 0; rr < 128; ++rr) acc += sDb[rr * D + tid];
    P[L::P_B2 + tid] = acc;
  }
  if (abort_s && tid == 0) atomicExch(a.err, 1);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, L::T_COLS);
}

// ======================================================================
// Discrete adjoint of the wide MLP field (D = 64, three tanh layers of
// 512; App. A), on the stacked M = 128 tiles of MlpWideCfg.
//
// Rows of a 64-instance tile reverse their own instances, 7 lockstep
// rounds per accepted step (stages 7..1) from the recorded stage inputs.
// A round runs the hidden layers at Y_s (forward weight chunks) and then
// the backward chain for the stage cotangent kbar_s (transposed chunks):
//   gh3 = kbar W4     delta3 = gh3 (1 - h3^2)
//   gh2 = delta3 W3   delta2 = gh2 (1 - h2^2)
//   gh1 = delta2 W2   delta1 = gh1 (1 - h1^2)
//   gx  = delta1 W1   (the state part of the stage's cotangent)
// The weight gradients dW_l = delta_l^T act_l sum over every reversed
// (instance, step, stage).  Two 512 x 512 products do not fit in tensor
// memory, so every round stages its 64 rows of act_l (X = [Y; t; 1], h1,
// h2, h3) and delta_l (delta1..3, kbar) as BF16 hi + lo in the layout the
// tensor cores read -- MN-major core-matrix blocks of 64 rows x (up to) 128
// features -- and k_mlp_dw forms the products from them afterwards.  A row
// whose instance is done runs on zeros: its kbar and hence every delta is
// 0, so its staged rows add nothing.
//
// The chain runs on CTA pairs (2-CTA clusters): the pair's MMAs are
// M = 256 over both CTAs' stacked tiles, issued by CTA 0, and each CTA
// streams only its half of every weight chunk (IMG_CHUNKS2 / IMG_TCHUNKS2),
// so a stage carries twice the tensor work per byte an SM receives.  The
// halves come in as 2-D tensor-map copies of the cta_group::2 form: CTA 1's
// copy completes on CTA 0's barrier, which expects both halves' bytes; per
// product CTA 1 reports its tile written; CTA 0's commits arrive in both
// CTAs' barriers (a CTA refills its own slot).  Both CTAs
// run the same rounds: the pair stops when neither has a row left (the
// shorter tile's rows run on zeros meanwhile).
// ======================================================================
template <class Cfg> struct WideAdj {
  static constexpr int D = Cfg::D, H = Cfg::H, K0 = Cfg::K0, ROWS = Cfg::ROWS;
  static_assert(Cfg::NL == 4 && D == 64 && H == 512 && K0 == 80 && ROWS == 64, "network");
  // Three 32 KB slots: a slot's refill is requested when the pair's MMAs of
  // the stage before are done, and its copy plus the hand-off to CTA 0 must
  // land within the two stages of MMAs still queued (with two slots the
  // tensor pipe drained at every stage).
  static constexpr int NSL = 3, SLOT_BYTES = 32768;
  // shared memory: one stacked tile, [128][K0] input X, then h1, h2
  // ([128][H]), then the kbar tile [128][D], then delta3 .. delta1
  // ([128][H]); the weight ring; one hidden layer's biases (loaded while
  // that layer's product runs).  h3 lives only in its staged rows.
  static constexpr int S_H = 0;
  static constexpr int S_W = S_H + 2 * ROWS * H * 2;
  static constexpr int S_BIAS = S_W + NSL * SLOT_BYTES;
  static constexpr int S_END = S_BIAS + H * 4;
  static_assert(S_END <= 232448 - 1024, "shared memory");
  // the round's weight stream: segments 0-2 the forward chunks of layers
  // 0-2 ([N][16] K-major), segments 3-6 the transposed chunks of layers 3,
  // 2, 1, 0 ([16 outputs][K] MN-major); a CTA streams its half of each
  // chunk, from the half image that holds layer l at W_off(l) / 2
  static constexpr int NSEG = 7;
  static constexpr size_t HALF_BYTES = Cfg::WIMG_BYTES / 2;
  static_assert(HALF_BYTES % 16 == 0, "bulk copies");
  __host__ __device__ static constexpr int seg_layer(int q) { return q < 3 ? q : 6 - q; }
  __host__ __device__ static constexpr bool seg_tr(int q) { return q >= 3; }
  __host__ __device__ static constexpr int seg_chunk_bytes(int q) {  // one CTA's half
    return q < 3 ? Cfg::N_of(q) * 16 : 16 * Cfg::K_of(seg_layer(q));
  }
  __host__ __device__ static constexpr int seg_chunks(int q) {
    return q < 3 ? Cfg::K_of(q) / 16 : Cfg::N_of(seg_layer(q)) / 16;
  }
  __host__ __device__ static constexpr int seg_per_stage(int q) {
    return SLOT_BYTES / seg_chunk_bytes(q);
  }
  __host__ __device__ static constexpr int seg_stages(int q) {
    return (seg_chunks(q) + seg_per_stage(q) - 1) / seg_per_stage(q);
  }
  __host__ __device__ static constexpr int stages() {
    int s = 0;
    for (int q = 0; q < NSEG; ++q) s += seg_stages(q);
    return s;
  }
  __host__ __device__ static void stage_of(uint32_t g, int& q, int& c0, int& nc, int& off,
                                           int& bytes) {
    int st = (int)(g % (uint32_t)stages());
    q = 0;
    while (st >= seg_stages(q)) st -= seg_stages(q++);
    c0 = st * seg_per_stage(q);
    nc = seg_chunks(q) - c0 < seg_per_stage(q) ? seg_chunks(q) - c0 : seg_per_stage(q);
    bytes = nc * seg_chunk_bytes(q);
    off = Cfg::W_off(seg_layer(q)) / 2 + c0 * seg_chunk_bytes(q);
  }
  // staged tensors; each splits into planes of (up to) 128 features -- 256
  // for h1 and h2, the N = 256 operands of dW2 and dW3 -- and a plane holds
  // one block pair (hi, lo) per (chain CTA, reverse round)
  enum { T_X = 0, T_H1 = 1, T_H2 = 2, T_H3 = 3, T_D1 = 4, T_D2 = 5, T_D3 = 6, T_K = 7, NTEN = 8 };
  __host__ __device__ static constexpr int fb_width(int t) {
    return t == T_X ? K0 : t == T_K ? D : (t == T_H1 || t == T_H2) ? 256 : 128;
  }
  __host__ __device__ static constexpr int t_fb(int t) {
    return t == T_X || t == T_K ? 1 : H / fb_width(t);
  }
  __host__ __device__ static constexpr int blk_bytes(int t) { return ROWS * fb_width(t) * 2; }
  __host__ __device__ static constexpr int plane_first(int t) {
    int p = 0;
    for (int j = 0; j < t; ++j) p += t_fb(j);
    return p;
  }
  static constexpr int NPLANES = plane_first(NTEN);
  // byte offset of 8 features [m, m+8) of row r inside a block of width F
  __host__ __device__ static constexpr uint32_t blk_off(int r, int m, int F) {
    return (uint32_t)((r >> 3) * F * 16 + (m >> 3) * 128 + (r & 7) * 16);
  }
};

// the chain's weight stages as 2-D tensor-map boxes: both pair images (the
// forward chunks', then the transposed chunks', WREP copies each) as one
// [rows][64] BF16 tensor of 128-byte rows, one map per stage size
constexpr int WIDE_TMAPS = 4;
struct WideAdjArgs {
  CUtensorMap tmap[WIDE_TMAPS];  // boxes of tmap_rows[k] rows
  int tmap_rows[WIDE_TMAPS];
  int i0, B, K;                  // the slice: queue positions i0 .. i0+B-1
  const int32_t* order;          // queue position -> instance (most accepted steps first)
  const double* t0;
  const double* t1;
  const double* te;
  const int32_t* n_acc;
  const int32_t* status;
  int slots;
  const float* tp_y;
  const double* tp_t;
  const float* tp_h;
  const float* tp_ys;            // [B][slots][6][D]: Y_2..Y_7
  const float* gye;
  const float* gyf;
  float* gy0;
  const float* bias;             // layers 0-2's biases at l*H (16-byte aligned copy)
  unsigned char* plane[32];      // staging planes (WideAdj::NPLANES used)
  int cap;                       // reverse rounds per CTA the planes hold
  int32_t* rounds;               // [grid]: reverse rounds staged by each CTA
  int32_t* overflow;
  int32_t* err;
  double* gts;  // [B] or NULL: each instance's time-translation sum
};

// 8 floats from a BF16 hi + lo pair of 16-byte rows
__device__ __forceinline__ void unsplit8(const uint4& hi, const uint4& lo, float (&v)[8]) {
  const uint32_t hw[4] = {hi.x, hi.y, hi.z, hi.w}, lw[4] = {lo.x, lo.y, lo.z, lo.w};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&hw[j]);
    const __nv_bfloat162 l2 = *reinterpret_cast<const __nv_bfloat162*>(&lw[j]);
    v[2 * j] = __low2float(h2) + __low2float(l2);
    v[2 * j + 1] = __high2float(h2) + __high2float(l2);
  }
}

template <class Cfg, class Tab = DP5>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(256, 1)
    k_mlp_adjoint_wide(const __grid_constant__ WideAdjArgs a) {
  using L = WideAdj<Cfg>;
  constexpr int D = Cfg::D, H = Cfg::H, K0 = Cfg::K0, C = Cfg::C, ROWS = Cfg::ROWS;
  constexpr int NSL = L::NSL;
  extern __shared__ __align__(1024) unsigned char sm[];
  // mbar_full (CTA 0): both halves of a stage landed (CTA 1's copies
  // complete on CTA 0's barrier); mbar_tile (CTA 0): CTA 1's tile is written
  // for the next product; mbar_empty / mbar_mma: the pair's MMAs of a stage /
  // a product are done (arrive in both CTAs); mbar_fin: CTA 0's last MMAs
  // are done
  __shared__ __align__(8) uint64_t mbar_mma, mbar_full[NSL], mbar_empty[NSL], mbar_tile, mbar_fin;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  __shared__ int pair_flag[2];
  unsigned char* sH = sm + L::S_H;  // the stacked tile (also the input and kbar tiles)
  unsigned char* sW = sm + L::S_W;
  float* sBias = reinterpret_cast<float*>(sm + L::S_BIAS);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, odd = lane & 1, hf = warp >> 2;
  const int row = Cfg::row_of(tid), sub = Cfg::sub_of(tid);
  const int coff = sub * C;
  const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
  const uint32_t rank = tc::cluster_rank();
  // this CTA's half image: byte offsets in the tensor-map rows (the
  // transposed image follows the forward one)
  const size_t rep = (size_t)((blockIdx.x >> 1) % Cfg::WREP) * Cfg::WIMG_STRIDE + rank * L::HALF_BYTES;
  const size_t timg_off = (size_t)Cfg::WREP * Cfg::WIMG_STRIDE;
  uint32_t g_stage = 0;  // weight stages consumed so far
  uint32_t tile_par = 0;  // products issued so far (parity of mbar_tile)

  // this CTA's half of stage g into the slot; CTA 0 expects both halves
  auto issue_stage = [&](uint32_t g, int slot) {
    int q, c0, nc, off, bytes;
    L::stage_of(g, q, c0, nc, off, bytes);
    const int rows = bytes / 128;
    int m = 0;
    while (m + 1 < WIDE_TMAPS && a.tmap_rows[m] != rows) ++m;
    const size_t boff = (L::seg_tr(q) ? timg_off : 0) + rep + (size_t)off;
    uint32_t mb;
    if (rank == 0) {
      tc::mbar_expect_tx(&mbar_full[slot], 2u * (uint32_t)bytes);
      mb = tc::smem_u32(&mbar_full[slot]);
    } else {
      mb = tc::peer_addr(&mbar_full[slot], 0);
    }
    tc::tensor_g2s_pair(sW + slot * L::SLOT_BYTES, &a.tmap[m], 0, (int)(boff / 128), mb);
  };
  if (tid == 0) {
    tc::mbar_init(&mbar_mma, 1);
    for (int b = 0; b < NSL; ++b) {
      tc::mbar_init(&mbar_full[b], 1);
      tc::mbar_init(&mbar_empty[b], 1);
    }
    tc::mbar_init(&mbar_tile, 1);
    tc::mbar_init(&mbar_fin, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // both CTAs run and their barriers are initialised before any arrival or
  // copy crosses; the pair's tensor memory is allocated by a warp of each
  tc::cluster_sync();
  if (tid == 0)
    for (int b = 0; b < NSL; ++b) issue_stage((uint32_t)b, b);
  if (warp == 0) tc::tmem_alloc_pair(&tmem_base_s, 512);
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_base_s;
  uint32_t parity = 0;

  // ---- this row's instance (one per row and slice) and its reverse state
  const int pos = a.i0 + (int)blockIdx.x * ROWS + row;
  const int inst = pos < a.i0 + a.B ? a.order[pos] : -1;
  // backward in time: the row runs in tau = -t with the field -f
  const unsigned long long rmask = (inst >= 0 && a.t1[inst] < a.t0[inst]) ? SIGN_BIT : 0ULL;
  bool act = false, bad = false;
  int n = -1, N = 0, q = -1;
  double tn = 0.0, tnext = 0.0;
  float h = 0.0f;
  float tsum = 0.0f;  // the time inputs' cotangents of the instance's stages (a.gts)
  float yb[16], kb[7][16];
#pragma unroll
  for (int r = 0; r < C; ++r) {
    yb[r] = 0.0f;
#pragma unroll
    for (int j = 0; j < 7; ++j) kb[j][r] = 0.0f;
  }
  auto load_step = [&]() {
    const size_t o = (size_t)inst * a.slots + n;
    tn = a.tp_t[o];
    h = a.tp_h[o];
    tnext = (n == N - 1) ? flip(a.t1[inst], rmask) : tn + (double)h;
  };
  // Y_s of the step being reversed: Y_1 = y_n, Y_2..Y_7 as the forward recorded
  auto load_stage = [&](int s_, float (&Yo)[16]) {
    const size_t o = (size_t)inst * a.slots + n;
    const float4* p = s_ == 1
        ? reinterpret_cast<const float4*>(a.tp_y + o * D + coff)
        : reinterpret_cast<const float4*>(a.tp_ys + (o * 6 + (s_ - 2)) * D + coff);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const float4 u = p[v];
      Yo[4 * v] = u.x, Yo[4 * v + 1] = u.y, Yo[4 * v + 2] = u.z, Yo[4 * v + 3] = u.w;
    }
  };
  // the instance is done: cotangents of points at t0, then dL/dy0
  auto finish = [&]() {
    if (!bad && a.gye) {
      const long long k0 = tkey(flip(a.t0[inst], rmask));
      for (; q >= 0; --q)
        if (tkey(flip(a.te[(size_t)inst * a.K + q], rmask)) == k0)
#pragma unroll
          for (int r = 0; r < C; ++r) yb[r] += a.gye[((size_t)inst * a.K + q) * D + coff + r];
    }
#pragma unroll
    for (int r = 0; r < C; ++r) a.gy0[(size_t)inst * D + coff + r] = bad ? nan_(0.0f) : yb[r];
    if (a.gts && sub == 0) a.gts[inst] = bad ? (double)nan_(0.0f) : (double)tsum;
    act = false;
  };
  if (inst >= 0) {
    N = a.n_acc[inst];
    bad = a.status[inst] != ST_SUCCESS;
    if (!bad && N > a.slots) {
      bad = true;
      if (sub == 0) atomicExch(a.overflow, 1);
    }
#pragma unroll
    for (int r = 0; r < C; ++r) yb[r] = a.gyf ? a.gyf[(size_t)inst * D + coff + r] : 0.0f;
    q = a.K - 1;
    n = N - 1;
    act = true;
    if (bad || n < 0) finish();
    else load_step();
  }

  auto barrier = [&]() {
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  };
  auto wait_mma = [&]() {
    if (!abort_s && !tc::mbar_wait_sleep(&mbar_mma, parity)) atomicExch(&abort_s, 1);
    parity ^= 1u;
    tc::fence_after_sync();
  };
  // one product of the round (segment qs) on the pair.  CTA 0's thread 0
  // waits for CTA 1's tile, then issues M = 256 MMAs over both stacked tiles
  // (K-major, Ka columns) as both halves of each stage arrive (on CTA 0's
  // barrier); CTA 1's thread 0 reports its tile; thread 32 of each CTA
  // refills its own slot with the stage NSL ahead once the pair's MMAs of
  // the slot are done.  N > 256 runs as
  // products of 256 (tensor-memory columns 256 j); a CTA's half of a chunk
  // holds NW/2 columns of each (IMG_CHUNKS2 / IMG_TCHUNKS2).
  auto gemm = [&](int qs, uint32_t a_addr, int Ka, int Nl) {
    const bool tr = L::seg_tr(qs);
    if (tid == 0 && !abort_s) {
      bool ok = true;
      if (rank != 0) {
        tc::mbar_arrive_peer(&mbar_tile, 0);
      } else {
        const int nh = Nl > 256 ? Nl / 256 : 1, nw = Nl > 256 ? 256 : Nl, hw = nw / 2;
        const uint32_t idesc = tc::idesc_bf16_f32(256, nw, false, tr);
        const int cb = L::seg_chunk_bytes(qs);
        ok = tc::mbar_wait_cluster(&mbar_tile, tile_par);
        tc::fence_after_sync();
        for (int st = 0; st < L::seg_stages(qs) && ok; ++st) {
          const uint32_t g = g_stage + (uint32_t)st;
          const int b = (int)(g % NSL);
          ok = tc::mbar_wait_cluster(&mbar_full[b], (g / NSL) & 1u);
          if (!ok) break;
          int q_, c0, nc, off_, bytes_;
          L::stage_of(g, q_, c0, nc, off_, bytes_);
          const uint32_t wb = tc::smem_u32(sW + b * L::SLOT_BYTES);
          for (int c = 0; c < nc; ++c) {
            const int kc = c0 + c;
            const uint64_t da = tc::smem_desc(a_addr + kc * 256, 128, Ka * 16);
            for (int j = 0; j < nh; ++j) {
              const uint64_t db =
                  tr ? tc::smem_desc_mn(wb + c * cb + j * (hw / 8) * 128, (Nl / 2) * 16)
                     : tc::smem_desc(wb + c * cb + j * hw * 32, 128, 256);
              tc::mma_bf16_pair(tbase + 256 * j, da, db, idesc, kc > 0);
            }
          }
          tc::mma_commit_pair_both(&mbar_empty[b]);
        }
        tc::mma_commit_pair_both(&mbar_mma);
      }
      if (!ok) atomicExch(&abort_s, 1);
    } else if (tid == 32 && !abort_s) {
      bool ok = true;
      for (int st = 0; st < L::seg_stages(qs) && ok; ++st) {
        const uint32_t g = g_stage + (uint32_t)st;
        const int b = (int)(g % NSL);
        ok = tc::mbar_wait(&mbar_empty[b], (g / NSL) & 1u);
        if (ok) issue_stage(g + NSL, b);
      }
      if (!ok) atomicExch(&abort_s, 1);
    }
    g_stage += (uint32_t)L::seg_stages(qs);
    tile_par ^= 1u;
    __syncwarp();
  };
  size_t blk = 0;  // this round's staging block
  // stages 8 features (hi, lo) of tensor t for this row at column col
  auto stage8 = [&](int t, int col, const uint4& hi, const uint4& lo) {
    const int fw = L::fb_width(t);
    const int fb = col / fw, m = col - fb * fw;
    unsigned char* dst = a.plane[L::plane_first(t) + fb] + blk * 2 * (size_t)L::blk_bytes(t) +
                         L::blk_off(row, m, fw);
    if (t == L::T_H1 || t == L::T_H2 || t == L::T_H3) {  // read back by the delta epilogues
      *reinterpret_cast<uint4*>(dst) = hi;
      *reinterpret_cast<uint4*>(dst + L::blk_bytes(t)) = lo;
    } else {  // read only by the weight-gradient kernel: streamed past the L2
      __stcs(reinterpret_cast<uint4*>(dst), hi);
      __stcs(reinterpret_cast<uint4*>(dst + L::blk_bytes(t)), lo);
    }
  };
  auto stage16 = [&](int t, int col, const float (&v)[16]) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      float w8[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) w8[j] = v[8 * u + j];
      uint4 hi, lo;
      split8(w8, hi, lo);
      stage8(t, col + 8 * u, hi, lo);
    }
  };
  // hidden epilogue: h = tanh(acc + b), staged as act and (to_tile) written
  // into the stacked tile as the next product's A
  auto epi_hidden = [&](int t_act, bool to_tile) {
#pragma unroll 1
    for (int c = 0; c < 256; c += 32) {
      float v0[16], v1[16];
      tc::tmem_ld16(tbase + lanes + 256 * hf + c, v0);
      tc::tmem_ld16(tbase + lanes + 256 * hf + c + 16, v1);
      tc::tmem_wait_ld();
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        float z[8];
        combine_pair8(u == 0 ? v0 : v1, odd, z);
        const int col = 256 * hf + c + 16 * u + 8 * odd;
        const float4 b0 = *reinterpret_cast<const float4*>(sBias + col);
        const float4 b1 = *reinterpret_cast<const float4*>(sBias + col + 4);
        const float2 t0 = tanh_acc2(__fadd2_rn(make_float2(z[0], z[1]), make_float2(b0.x, b0.y)));
        const float2 t1 = tanh_acc2(__fadd2_rn(make_float2(z[2], z[3]), make_float2(b0.z, b0.w)));
        const float2 t2 = tanh_acc2(__fadd2_rn(make_float2(z[4], z[5]), make_float2(b1.x, b1.y)));
        const float2 t3 = tanh_acc2(__fadd2_rn(make_float2(z[6], z[7]), make_float2(b1.z, b1.w)));
        const float hv[8] = {t0.x, t0.y, t1.x, t1.y, t2.x, t2.y, t3.x, t3.y};
        uint4 hi, lo;
        split8(hv, hi, lo);
        if (to_tile) store_pair8(sH, row, col, H, odd, hi, lo);
        stage8(t_act, col, hi, lo);
      }
    }
  };
  // delta epilogue: delta = acc (1 - h^2), h from its staged rows in global
  // memory (fetched one iteration ahead, so that their latency overlaps the
  // previous columns' arithmetic); the split delta replaces the tile and is
  // staged
  auto epi_delta = [&](int t_h, int t_del) {
    const int fw = L::fb_width(t_h);
    auto ld_h = [&](int c, uint4 (&hh)[2], uint4 (&hl)[2]) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int col = 256 * hf + c + 16 * u + 8 * odd;
        const int fb = col / fw, m = col - fb * fw;
        const unsigned char* src = a.plane[L::plane_first(t_h) + fb] +
                                   blk * 2 * (size_t)L::blk_bytes(t_h) + L::blk_off(row, m, fw);
        hh[u] = *reinterpret_cast<const uint4*>(src);
        hl[u] = *reinterpret_cast<const uint4*>(src + L::blk_bytes(t_h));
      }
    };
    uint4 nh[2], nl[2];
    ld_h(0, nh, nl);
#pragma unroll 1
    for (int c = 0; c < 256; c += 32) {
      float v0[16], v1[16];
      tc::tmem_ld16(tbase + lanes + 256 * hf + c, v0);
      tc::tmem_ld16(tbase + lanes + 256 * hf + c + 16, v1);
      uint4 hh[2], hl[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) hh[u] = nh[u], hl[u] = nl[u];
      if (c + 32 < 256) ld_h(c + 32, nh, nl);
      tc::tmem_wait_ld();
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        float z[8], hv[8], dv[8];
        combine_pair8(u == 0 ? v0 : v1, odd, z);
        unsplit8(hh[u], hl[u], hv);
#pragma unroll
        for (int j = 0; j < 8; ++j) dv[j] = z[j] * madd(-hv[j], hv[j], 1.0f);
        const int col = 256 * hf + c + 16 * u + 8 * odd;
        uint4 hi, lo;
        split8(dv, hi, lo);
        store_pair8(sH, row, col, H, odd, hi, lo);
        stage8(t_del, col, hi, lo);
      }
    }
  };

  // layer l's biases into shared memory, by threads that neither issue nor
  // refill (the previous epilogue's reads ended at the barrier before the product)
  auto load_bias = [&](int l) {
    if (tid >= 64 && tid < 64 + H / 4)
      reinterpret_cast<float4*>(sBias)[tid - 64] =
          __ldg(reinterpret_cast<const float4*>(a.bias + (size_t)l * H) + (tid - 64));
  };
  const float bw[7] = {float(Tab::b(1)), float(Tab::b(2)), float(Tab::b(3)), float(Tab::b(4)),
                       float(Tab::b(5)), float(Tab::b(6)), float(Tab::b(7))};
  int k_round = 0;  // reverse rounds staged by this CTA (the same in both CTAs of the pair)
  int n_check = 0;
  for (int rnd = 0;; ++rnd) {
    const int ph = rnd % ADJ_ROUNDS;
    if (ph == 0) {
      // the pair goes on while either CTA has a row left and neither gave up
      // (abort_s is read after a barrier: block-uniform)
      const int mine = __syncthreads_or(act) ? 1 : 0;
      if (tid == 0) pair_flag[n_check & 1] = mine | (abort_s ? 2 : 0);
      tc::cluster_sync();
      const int f = pair_flag[n_check & 1] | tc::ld_peer_s32(&pair_flag[n_check & 1], rank ^ 1u);
      ++n_check;
      if (!(f & 1) || (f & 2)) break;
    }
    if (abort_s) continue;  // wind down to the pair's next check
    const int s = 7 - ph;   // the stage reversed this round (block-uniform)
    if (k_round >= a.cap) {  // cannot happen: the planes hold 7 rounds per tape slot
      if (tid == 0) {
        atomicExch(a.err, 2);
        abort_s = 1;
      }
      __syncthreads();
      continue;
    }
    blk = (size_t)blockIdx.x * a.cap + k_round;

    // ---- stage input [Y_s; t_s] and the cotangent kbar_s of this row
    float Y[16], kq[16];
    float tin = 0.0f;
    if (act && s == 7) {
#pragma unroll
      for (int j = 0; j < 7; ++j)
#pragma unroll
        for (int r = 0; r < C; ++r) kb[j][r] = h * bw[j] * yb[r];
      const long long kt = tkey(tn), kn = tkey(tnext);
      while (q >= 0) {
        const double tq = flip(a.te[(size_t)inst * a.K + q], rmask);
        const long long kk = tkey(tq);
        if (!(kk > kt)) break;
        if (a.gye) {
          float gq[16], w[7];
#pragma unroll
          for (int r = 0; r < C; ++r) gq[r] = a.gye[((size_t)inst * a.K + q) * D + coff + r];
          if (kk == kn) {
#pragma unroll
            for (int j = 0; j < 7; ++j) w[j] = bw[j];
          } else {
            dense_weights<Tab, float>(float(tq - tn) / h, w);
          }
#pragma unroll
          for (int j = 0; j < 7; ++j)
#pragma unroll
            for (int r = 0; r < C; ++r) kb[j][r] = madd(h * w[j], gq[r], kb[j][r]);
#pragma unroll
          for (int r = 0; r < C; ++r) yb[r] += gq[r];
        }
        q--;
      }
    }
    if (act) {
      load_stage(s, Y);
      tin = (float)flip(tn + tab_c<Tab>(s) * (double)h, rmask);  // the caller's time
      pick7(kb, s - 1, kq);
      if (rmask) {  // the field in tau is -f: its products take -kbar
#pragma unroll
        for (int r = 0; r < C; ++r) kq[r] = -kq[r];
      }
    } else {
#pragma unroll
      for (int r = 0; r < C; ++r) Y[r] = kq[r] = 0.0f;
    }
    store_row16_stk(sH, row, coff, K0, Y);  // the input tile [128][K0]
    stage16(L::T_X, coff, Y);
    stage16(L::T_K, coff, kq);
    if (sub == Cfg::TPR - 1) {
      // columns D.. of the input: the time (hi + lo) and zero padding, all
      // rewritten because the kbar tile of the last round shares the bytes;
      // staged as [t; 1; 0...], the constant input whose weight gradient is db1
      float tail[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) tail[j] = 0.0f;
      tail[0] = tin;
      store_row16_stk(sH, row, D, K0, tail);
      tail[1] = 1.0f;
      stage16(L::T_X, D, tail);
    }
    barrier();

    // ---- forward layers at Y_s
    gemm(0, tc::smem_u32(sH), K0, H);
    load_bias(0);
    wait_mma();
    __syncthreads();
    epi_hidden(L::T_H1, true);
    barrier();
    gemm(1, tc::smem_u32(sH), H, H);
    load_bias(1);
    wait_mma();
    __syncthreads();
    epi_hidden(L::T_H2, true);
    barrier();
    gemm(2, tc::smem_u32(sH), H, H);
    load_bias(2);
    wait_mma();
    __syncthreads();
    epi_hidden(L::T_H3, false);  // h3: staged only
    store_row16_stk(sH, row, coff, D, kq);       // the kbar tile [128][D]
    barrier();
    // ---- backward chain
    gemm(3, tc::smem_u32(sH), D, H);  // gh3 = kbar W4
    wait_mma();
    epi_delta(L::T_H3, L::T_D3);
    barrier();
    gemm(4, tc::smem_u32(sH), H, H);  // gh2 = delta3 W3
    wait_mma();
    epi_delta(L::T_H2, L::T_D2);
    barrier();
    gemm(5, tc::smem_u32(sH), H, H);  // gh1 = delta2 W2
    wait_mma();
    epi_delta(L::T_H1, L::T_D1);
    barrier();
    gemm(6, tc::smem_u32(sH), H, K0);  // gx = delta1 W1
    wait_mma();
    float fg[16];
    float tcot = 0.0f;  // the time input's cotangent (column D), hi + lo rows
    {
      float v0[16], v1[16];
      tc::tmem_ld16(tbase + lanes + 32 * hf, v0);
      tc::tmem_ld16(tbase + lanes + 32 * hf + 16, v1);
      if (a.gts) tcot = tc::tmem_ld1(tbase + lanes + D);
      tc::tmem_wait_ld();
      combine_pair16(v0, v1, odd, fg);
      if (a.gts) tcot += __shfl_xor_sync(0xffffffffu, tcot, 1);
    }
    k_round++;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (abort_s) continue;

    // ---- consume (row-local)
    if (!act) continue;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      if (j + 1 >= s) continue;
      const float cc = h * tab_a<Tab>(s, j + 1);
#pragma unroll
      for (int r = 0; r < C; ++r) kb[j][r] = madd(cc, fg[r], kb[j][r]);
    }
#pragma unroll
    for (int r = 0; r < C; ++r) yb[r] += fg[r];
    tsum += tcot;
    if (s == 1) {
      n -= 1;
      if (n >= 0) load_step();
      else finish();
    }
  }
  if (tid == 0) {
    a.rounds[blockIdx.x] = k_round;
    if (rank == 0) {
      // the ring's copies still in flight (stages g .. g + NSL - 1, both
      // CTAs' halves: they complete on CTA 0's barriers) land before either
      // CTA exits, and the pair's MMAs, which read both CTAs' shared memory,
      // are done
      for (uint32_t x = g_stage; x < g_stage + NSL; ++x)
        if (!tc::mbar_wait_cluster(&mbar_full[x % NSL], (x / NSL) & 1u)) atomicExch(&abort_s, 1);
      tc::mma_commit_pair_local(&mbar_fin);
      if (!tc::mbar_wait(&mbar_fin, 0)) atomicExch(&abort_s, 1);
    }
    if (abort_s) atomicExch(a.err, 1);
  }
  // neither CTA leaves while the other may still reach its shared memory
  tc::fence_before_sync();
  tc::cluster_sync();
  if (warp == 0) tc::tmem_dealloc_pair(tbase, 512);
}

// ---------------------------------------------------------------- dW, db
// The weight and bias gradients of the wide adjoint from the staged blocks:
//   dW_l[o][i] = sum over staged rows of delta_l[row][o] act_l[row][i]
// in three BF16 products per pair of split operands (hi*hi + lo*hi + hi*lo;
// the lo*lo term is below FP32 rounding of the sum), FP32 accumulation in
// tensor memory.  A job is one 128-feature block of the output's rows
// (M = 128); its work items split the chain CTAs (the K dimension) into
// parts, each accumulating its own partial in a fixed order, which
// k_mlp_dw_reduce sums part by part: deterministic.  A work item's copies
// stream through two A and two B slots (more slots for the jobs with small
// blocks measured slower: their extra bytes in flight evicted the blocks
// that the N = 256 jobs share through L2).  A partial is column-major
// ([column][128 output rows]), so that the accumulator's rows, one per
// thread, go out coalesced.
//   kind 0: D[o][i] += A^T B over nb operand blocks of width bw (dW)
//   kind 1: D[o][0] += A^T 1 (a bias: the delta's column sums)
//   kind 2: D[*][i] += 1^T B (the output bias from the kbar rows)
struct DwJob {
  int kind, ta, fa, tb, nb, bw;  // tensors / feature blocks of A and B
};
constexpr int DW_MAX_JOBS = 32;
constexpr int DW_PART_FLOATS = 128 * 512;
constexpr int DW_NA = 2, DW_NB = 2, DW_SLOT_A = 32768, DW_SLOT_B = 65536;
constexpr int DW_RING = DW_NA * DW_SLOT_A + DW_NB * DW_SLOT_B;
struct DwArgs {
  int njobs;
  DwJob job[DW_MAX_JOBS];
  int item0[DW_MAX_JOBS + 1];  // first work item of each job
  int chain_grid, cap;         // the chain kernel's CTAs and plane capacity
  const int32_t* rounds;       // [chain_grid]
  const unsigned char* plane[32];
  float* part;                 // [items][128][512]
  int32_t* err;
};

template <class Cfg>
__global__ void __launch_bounds__(128, 1) k_mlp_dw(DwArgs a) {
  using L = WideAdj<Cfg>;
  extern __shared__ __align__(1024) unsigned char sm[];
  constexpr int NA = DW_NA, NB = DW_NB, SLOT_A = DW_SLOT_A, SLOT_B = DW_SLOT_B;
  __shared__ __align__(8) uint64_t fullA[NA], emptyA[NA], fullB[NB], emptyB[NB], done;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int item = blockIdx.x;
  int j = 0;
  while (j + 1 < a.njobs && item >= a.item0[j + 1]) ++j;
  const DwJob jb = a.job[j];
  unsigned char* sA = sm;
  unsigned char* sB = sm + NA * SLOT_A;
  unsigned char* sOnes = sm + DW_RING;  // [128][16] K-major BF16 ones
  const int P = a.item0[j + 1] - a.item0[j], p = item - a.item0[j];
  const int c_lo = (int)((long long)a.chain_grid * p / P);
  const int c_hi = (int)((long long)a.chain_grid * (p + 1) / P);
  const bool hasA = jb.kind != 2, hasB = jb.kind != 1;
  const int nbp = jb.kind == 0 ? jb.nb : 1;  // B parts per block (one MMA group each)
  const int abytes = hasA ? 2 * L::blk_bytes(jb.ta) : 0;
  const int bbytes = hasB ? 2 * L::blk_bytes(jb.tb) : 0;
  const unsigned char* pa = hasA ? a.plane[L::plane_first(jb.ta) + jb.fa] : nullptr;

  if (tid == 0) {
    for (int b = 0; b < NA; ++b) {
      tc::mbar_init(&fullA[b], 1);
      tc::mbar_init(&emptyA[b], 1);
    }
    for (int b = 0; b < NB; ++b) {
      tc::mbar_init(&fullB[b], 1);
      tc::mbar_init(&emptyB[b], 1);
    }
    tc::mbar_init(&done, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int e = tid; e < 128 * 16 / 8; e += 128)
    reinterpret_cast<uint4*>(sOnes)[e] =
        make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base_s, 512);
    tc::tmem_relinquish();
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_base_s;
  // the blocks of this item: CTAs [c_lo, c_hi), rounds [0, rounds[c])
  int nblk = 0;
  for (int c = c_lo; c < c_hi; ++c) nblk += a.rounds[c];

  if (tid == 32) {
    // producer: the same sequence the MMA thread consumes (A of a block,
    // then its B parts); each ring slot is refilled once its MMAs are done
    int ia = 0, ib = 0;
    bool ok = true;
    for (int c = c_lo; c < c_hi && ok; ++c)
      for (int k = 0; k < a.rounds[c] && ok; ++k) {
        const size_t bk = (size_t)c * a.cap + k;
        if (hasA) {
          const int s = ia % NA;
          if (ia >= NA) ok = tc::mbar_wait(&emptyA[s], ((ia - NA) / NA) & 1u);
          if (!ok) break;
          tc::mbar_expect_tx(&fullA[s], (uint32_t)abytes);
          tc::bulk_g2s(sA + s * SLOT_A, pa + bk * abytes, (uint32_t)abytes, &fullA[s]);
          ++ia;
        }
        if (hasB)
          for (int u = 0; u < nbp && ok; ++u) {
            const int s = ib % NB;
            if (ib >= NB) ok = tc::mbar_wait(&emptyB[s], ((ib - NB) / NB) & 1u);
            if (!ok) break;
            const unsigned char* pb = a.plane[L::plane_first(jb.tb) + u];
            tc::mbar_expect_tx(&fullB[s], (uint32_t)bbytes);
            tc::bulk_g2s(sB + s * SLOT_B, pb + bk * bbytes, (uint32_t)bbytes, &fullB[s]);
            ++ib;
          }
      }
    if (!ok) atomicExch(&abort_s, 1);
  } else if (tid == 0) {
    const int FA = hasA ? L::fb_width(jb.ta) : 0, FB = hasB ? L::fb_width(jb.tb) : 0;
    const int ablk = hasA ? L::blk_bytes(jb.ta) : 0, bblk = hasB ? L::blk_bytes(jb.tb) : 0;
    const uint32_t ones = tc::smem_u32(sOnes);
    int ia = 0, ib = 0, blk_i = 0;
    bool ok = true;
    for (int c = c_lo; c < c_hi && ok; ++c)
      for (int k = 0; k < a.rounds[c] && ok; ++k, ++blk_i) {
        uint32_t aA = 0;
        if (hasA) {
          const int s = ia % NA;
          ok = tc::mbar_wait(&fullA[s], (ia / NA) & 1u);
          if (!ok) break;
          aA = tc::smem_u32(sA + s * SLOT_A);
        }
        for (int u = 0; u < nbp && ok; ++u) {
          uint32_t aB = 0;
          if (hasB) {
            const int s = ib % NB;
            ok = tc::mbar_wait(&fullB[s], (ib / NB) & 1u);
            if (!ok) break;
            aB = tc::smem_u32(sB + s * SLOT_B);
          }
          const uint32_t dcol = tbase + (uint32_t)(jb.kind == 0 ? u * jb.bw : 0);
          for (int ks = 0; ks < 4; ++ks) {  // 16 staged rows per K step
            const bool acc0 = blk_i > 0 || ks > 0;
            if (jb.kind == 0) {
              const uint32_t idesc = tc::idesc_bf16_f32(128, jb.bw, true, true);
              const uint64_t ah = tc::smem_desc_mn(aA + ks * 2 * FA * 16, FA * 16);
              const uint64_t al = tc::smem_desc_mn(aA + ablk + ks * 2 * FA * 16, FA * 16);
              const uint64_t bh = tc::smem_desc_mn(aB + ks * 2 * FB * 16, FB * 16);
              const uint64_t bl = tc::smem_desc_mn(aB + bblk + ks * 2 * FB * 16, FB * 16);
              tc::mma_bf16(dcol, ah, bh, idesc, acc0);
              tc::mma_bf16(dcol, al, bh, idesc, true);
              tc::mma_bf16(dcol, ah, bl, idesc, true);
            } else if (jb.kind == 1) {  // column sums: A^T times a ones operand (N = 16)
              const uint32_t idesc = tc::idesc_bf16_f32(128, 16, true, false);
              const uint64_t ah = tc::smem_desc_mn(aA + ks * 2 * FA * 16, FA * 16);
              const uint64_t al = tc::smem_desc_mn(aA + ablk + ks * 2 * FA * 16, FA * 16);
              const uint64_t b1 = tc::smem_desc(ones, 128, 256);
              tc::mma_bf16(dcol, ah, b1, idesc, acc0);
              tc::mma_bf16(dcol, al, b1, idesc, true);
            } else {  // a ones operand (M = 128) times B: every row holds B's column sums
              const uint32_t idesc = tc::idesc_bf16_f32(128, FB, false, true);
              const uint64_t a1 = tc::smem_desc(ones, 128, 256);
              const uint64_t bh = tc::smem_desc_mn(aB + ks * 2 * FB * 16, FB * 16);
              const uint64_t bl = tc::smem_desc_mn(aB + bblk + ks * 2 * FB * 16, FB * 16);
              tc::mma_bf16(dcol, a1, bh, idesc, acc0);
              tc::mma_bf16(dcol, a1, bl, idesc, true);
            }
          }
          if (hasB) {
            tc::mma_commit(&emptyB[ib % NB]);
            ++ib;
          }
        }
        if (hasA && ok) {
          tc::mma_commit(&emptyA[ia % NA]);
          ++ia;
        }
      }
    if (!ok) atomicExch(&abort_s, 1);
    tc::mma_commit(&done);
  }
  __syncwarp();
  if (!tc::mbar_wait_sleep(&done, 0)) atomicExch(&abort_s, 1);
  tc::fence_after_sync();
  // add the accumulator to this item's partial (rows = lanes, one per
  // thread; column-major, so a warp's 32 rows of a column are contiguous)
  const int ncols = jb.kind == 0 ? jb.nb * jb.bw : jb.kind == 1 ? 16 : L::fb_width(jb.tb);
  if (nblk > 0 && !abort_s) {
    float* dst = a.part + (size_t)item * DW_PART_FLOATS + tid;
    const uint32_t lanes = (uint32_t)(32 * warp) << 16;
    for (int c0 = 0; c0 < ncols; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tbase + lanes + c0, v);
      tc::tmem_wait_ld();
      float o[16];
#pragma unroll
      for (int e = 0; e < 16; ++e)
        if (c0 + e < ncols) o[e] = dst[(size_t)(c0 + e) * 128];
#pragma unroll
      for (int e = 0; e < 16; ++e)
        if (c0 + e < ncols) dst[(size_t)(c0 + e) * 128] = o[e] + v[e];
    }
  }
  if (abort_s && tid == 0) atomicExch(a.err, 3);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

// Gradients from the work items' partials, summed part by part in order:
// gW0 [512][65] and gb0 (dW1's constant column), gW1, gW2 [512][512],
// gW3 [64][512] (staged transposed), gb1, gb2, gb3.
struct DwReduceArgs {
  const float* part;
  int item0[DW_MAX_JOBS + 1];
  int jW[4], jb[4];  // first job of each gradient (4 consecutive row-block jobs; gb3: one)
  float* gW[4];
  float* gb[4];
};
__global__ void k_mlp_dw_reduce(DwReduceArgs a) {
  constexpr int H = 512, D = 64, IN0 = D + 1;
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  // partial element (row m, column nn) of each item of a job, in item order;
  // consecutive threads take consecutive rows m where the partial's rows are
  // the gradient's (the column-major partials read coalesced)
  auto sum = [&](int job, int m, int nn) {
    float s = 0.0f;
    for (int it = a.item0[job]; it < a.item0[job + 1]; ++it)
      s += a.part[(size_t)it * DW_PART_FLOATS + (size_t)nn * 128 + m];
    return s;
  };
  if (e < (long long)H * IN0) {  // gW0 [o][i], i < 65
    const int i = (int)(e / H), o = (int)(e % H);
    a.gW[0][(size_t)o * IN0 + i] = sum(a.jW[0] + o / 128, o % 128, i);
    return;
  }
  e -= (long long)H * IN0;
  if (e < H) {
    if (a.gb[0]) a.gb[0][e] = sum(a.jW[0] + (int)e / 128, (int)e % 128, IN0);
    return;
  }
  e -= H;
  for (int l = 1; l <= 2; ++l) {
    if (e < (long long)H * H) {
      const int i = (int)(e / H), o = (int)(e % H);
      a.gW[l][(size_t)o * H + i] = sum(a.jW[l] + o / 128, o % 128, i);
      return;
    }
    e -= (long long)H * H;
    if (e < H) {
      if (a.gb[l]) a.gb[l][e] = sum(a.jb[l] + (int)e / 128, (int)e % 128, 0);
      return;
    }
    e -= H;
  }
  if (e < (long long)D * H) {  // gW3 [o][i] from dW3^T [i][o]
    const int o = (int)(e / H), i = (int)(e % H);
    a.gW[3][e] = sum(a.jW[3] + i / 128, i % 128, o);
    return;
  }
  e -= (long long)D * H;
  if (e < D && a.gb[3]) a.gb[3][e] = sum(a.jb[3], 0, (int)e);
}

// Queue of instances, most accepted steps first, and by index within equal
// counts (stable: the same order on every call, so the weight-gradient sums
// run in a fixed order).  One CTA: per 1024-instance chunk every warp ranks
// its lanes per bin, the warps' bin counts are prefixed in warp order.
__global__ void __launch_bounds__(1024) k_order_steps_stable(int B, StepsBin bin_of,
                                                             int32_t* order) {
  __shared__ int cnt[32][ORDER_BINS];
  __shared__ int base[ORDER_BINS];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  if (t < ORDER_BINS) base[t] = 0;
  __syncthreads();
  for (int i = t; i < B; i += 1024) atomicAdd(&base[bin_of(i)], 1);
  __syncthreads();
  if (t == 0) {
    int run = 0;
    for (int b = 0; b < ORDER_BINS; ++b) {
      const int v = base[b];
      base[b] = run;
      run += v;
    }
  }
  __syncthreads();
  for (int c0 = 0; c0 < B; c0 += 1024) {
    const int i = c0 + t;
    const int b = i < B ? bin_of(i) : -1;
#pragma unroll
    for (int k = 0; k < ORDER_BINS / 32; ++k) cnt[w][lane + 32 * k] = 0;
    __syncwarp();
    const unsigned m = __match_any_sync(0xffffffffu, b);
    const int rank = __popc(m & ((1u << lane) - 1u));
    if (b >= 0 && rank == 0) cnt[w][b] = __popc(m);
    __syncthreads();
    if (t < ORDER_BINS) {
      int run = base[t];
      for (int k = 0; k < 32; ++k) {
        const int v = cnt[k][t];
        cnt[k][t] = run;
        run += v;
      }
      base[t] = run;
    }
    __syncthreads();
    if (b >= 0) order[cnt[w][b] + rank] = i;
    __syncthreads();
  }
}


// Sums the per-CTA partials in CTA order into the caller's gradients
// (layouts of the weights: W_l [out][in], b_l [out]).
template <class Cfg>
__global__ void k_mlp_grad_reduce(const float* part, int grid, float* gW0, float* gb0, float* gW1,
                                  float* gb1, float* gW2, float* gb2) {
  using L = MlpAdjLayout<Cfg>;
  constexpr int D = Cfg::D, H = Cfg::H, K0 = Cfg::K0, IN = D + 1;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  // eight interleaved partial sums over the CTAs, combined as a fixed tree
  // (the same order on every call: deterministic)
  auto sum = [&](int off) {
    float acc[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    int c = 0;
    for (; c + 8 <= grid; c += 8)
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] += part[(size_t)(c + u) * L::P_FLOATS + off];
    for (int u = 0; c < grid; ++c, ++u) acc[u] += part[(size_t)c * L::P_FLOATS + off];
    return ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
  };
  int k = e;
  if (k < H * IN) {
    const int o = k / IN, j = k % IN;
    gW0[k] = sum(L::P_W0 + o * K0 + j);
    return;
  }
  k -= H * IN;
  if (k < H) {
    if (gb0) gb0[k] = sum(L::P_W0 + k * K0 + IN);
    return;
  }
  k -= H;
  if (k < H * H) {
    gW1[k] = sum(L::P_W1 + k);
    return;
  }
  k -= H * H;
  if (k < H) {
    if (gb1) gb1[k] = sum(L::P_B1 + k);
    return;
  }
  k -= H;
  if (k < D * H) {
    const int o = k / H, j = k % H;  // W3 [out = D][in = H]
    gW2[k] = sum(L::P_W2T + j * D + o);
    return;
  }
  k -= D * H;
  if (k < D && gb2) gb2[k] = sum(L::P_B2 + k);
}

// ======================================================================
// Joint continuous adjoint of the D = 32, H = 128 MLP field (App. A, the
// CNF benchmark's "torchode-joint" backward pass): ONE adjoint equation for
// the whole batch, of size 2BD + P -- the state integrated back, its
// adjoint and the adjoint of the shared parameters -- solved backward from
// t1 to t0 with one step size, one RMS error norm over all its components
// and one accept/reject decision (the joint semantics of Sec. 4.1), by
// dopri5 with the solver's controller and starting-step heuristic:
//   dy/dt = f(t, y_b),  da_b/dt = -J_f(t, y_b)^T a_b,
//   dabar/dt = -G,  G = sum_b (df/dtheta)(t, y_b)^T a_b.
// A stage of a row is one augmented evaluation: the hidden layers and the
// output layer at [Y; t] (k_y = f), then the transposed chain with the
// cotangent A (k_a = -J^T A) and the tile's weight products, its part of G,
// in tensor memory (the round of k_mlp_adjoint with a fresh accumulator per
// stage).  A row owns its y and a; abar is one vector of P values.
//
// Per attempt two launches: k_mlp_jadj (128-row tiles; six stages; each
// CTA adds its stages' parts of G, weighted by -h b_i and -h e_i, into its
// own slots, and writes its rows' candidate and squared scaled errors) and
// k_mlp_jadj_decide (per parameter: the CTAs' slots summed in CTA order,
// abar's candidate and error; its last CTA -- a ticket, no CTA waits for
// another -- sums every partial in order, decides and runs the controller).
// The launches after an accepted attempt commit its candidate (rows: y, a,
// k7 as the next k1; abar: the vector and its k7).  Two launch pairs before
// the first attempt of a segment take the starting step.
// ======================================================================
enum : int { JA_EVAL = 0, JA_PROBE = 1, JA_STEP = 2 };

struct JadjCtl {
  double t, t_end;       // time (decreasing: backward) and the segment's end
  double h, h_use;       // proposed step (> 0) and the next attempt's, clipped at t_end
  double h0, d1;         // the starting-step heuristic between its launches
  double err_prev, err_prev2;
  int use_last, n_acc, n_rej, n_fe, status, pending, prev_rej;
  unsigned int ticket;
};

struct JadjArgs {
  int B;
  const unsigned char* wimg;
  const float* bias[3];
  float *y, *a, *yc, *ac;  // [B][D]: state and the attempt's candidate
  float* kst;              // [7][B][2D]: stage derivatives [k_y | k_a]; slot 0 = k1
  float* gpart;            // [grid][3][P]: each CTA's slots U, E, F
  double* epart;           // [grid][2]: the rows' squared scaled sums
  double *th, *thc, *kth1, *fsum;  // [P]: abar, its candidate, its k1, the candidate's k7
  double* dpart;           // [decide grid][2]
  JadjCtl* ctl;
  double rtol, atol, safety, fac_min, fac_max, beta1, beta2, beta3, nnorm;
  int max_steps;
  int32_t* err;
};

// The parameter vector's padding entries (input columns past [y; t; 1] of
// the first layer) are not part of the problem: no norm term.
template <class L> __host__ __device__ constexpr bool jadj_real(int p) {
  return !(p < L::P_W1 && (p % L::K0) >= L::D + 2);
}

template <class Cfg, class Tb = DP5>
__global__ void __launch_bounds__(256, 1) k_mlp_jadj(JadjArgs a, int mode) {
  using L = MlpAdjLayout<Cfg>;
  constexpr int D = Cfg::D, H = Cfg::H, K0 = Cfg::K0, C = Cfg::C, HC = Cfg::HC;
  constexpr int P = L::P_FLOATS;
  const JadjCtl c = *a.ctl;
  if (c.status != ST_RUNNING) return;  // block-uniform: the segment is over
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar_mma, mbar_w;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  __shared__ double red[8];
  unsigned char* sW = sm + L::S_W;
  unsigned char* sXh = sm + L::S_XH;
  unsigned char* sXl = sm + L::S_XL;
  unsigned char* sH1h = sm + L::S_H1H;
  unsigned char* sH1l = sm + L::S_H1L;
  unsigned char* sH2h = sm + L::S_H2H;
  unsigned char* sH2l = sm + L::S_H2L;
  unsigned char* sD3h = sm + L::S_D3H;
  unsigned char* sD3l = sm + L::S_D3L;
  unsigned char* sOnes = sm + L::S_ONES;
  float* sBias = reinterpret_cast<float*>(sm + L::S_BIAS);

  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & 127, half = tid >> 7;
  const int coff = half * C;
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  const int inst = blockIdx.x * 128 + row;
  const bool live = inst < a.B;

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
    for (int l = 0; l < 3; ++l)
      tc::bulk_g2s(sW + Cfg::W_off(l), a.wimg + Cfg::W_off(l), (uint32_t)Cfg::W_bytes(l), &mbar_w);
  }
  {
    int o = 0;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const int n = Cfg::N_of(l);
      for (int j = tid; j < n; j += 256) sBias[o + j] = a.bias[l] ? a.bias[l][j] : 0.0f;
      o += n;
    }
  }
  for (int j = tid; j < 128 * K0 * 2 / 16; j += 256) {
    reinterpret_cast<uint4*>(sXh)[j] = make_uint4(0, 0, 0, 0);
    reinterpret_cast<uint4*>(sXl)[j] = make_uint4(0, 0, 0, 0);
  }
  for (int j = tid; j < 128 * 16; j += 256) {
    const int r = j / 16, cc = j % 16;
    *reinterpret_cast<__nv_bfloat16*>(sOnes + tc::cm_offset(r, cc, 16)) =
        __float2bfloat16_rn(cc == 0 ? 1.0f : 0.0f);
  }
  __syncthreads();
  if (tid < 128)
    *reinterpret_cast<__nv_bfloat16*>(sXh + tc::cm_offset(tid, D + 1, K0)) =
        __float2bfloat16_rn(1.0f);
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base_s, L::T_COLS);
    tc::tmem_relinquish();
  }
  if (!tc::mbar_wait(&mbar_w, 0)) atomicExch(&abort_s, 1);
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_base_s;
  const uint32_t tl = tbase + lane_base;
  uint32_t parity = 0;

  // ---- this thread's components of its row: commit, then load
  const size_t BD = (size_t)a.B * D, KS = 2 * BD;  // KS: floats per stage slot
  const size_t ro = (size_t)inst * D + coff;       // y / a offset
  const size_t ko = (size_t)inst * 2 * D + coff;   // slot offset (y part; a part at +D)
  auto ld16 = [&](const float* p, float (&v)[16]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 u = reinterpret_cast<const float4*>(p)[q];
      v[4 * q] = u.x, v[4 * q + 1] = u.y, v[4 * q + 2] = u.z, v[4 * q + 3] = u.w;
    }
  };
  auto st16 = [&](float* p, const float (&v)[16]) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      reinterpret_cast<float4*>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  };
  float y[16], av[16];
  if (live) {
    if (mode == JA_STEP && c.pending) {  // the previous attempt was accepted
      float v[16];
      ld16(a.yc + ro, v);
      st16(a.y + ro, v);
      ld16(a.ac + ro, v);
      st16(a.a + ro, v);
      ld16(a.kst + 6 * KS + ko, v);
      st16(a.kst + ko, v);
      ld16(a.kst + 6 * KS + ko + D, v);
      st16(a.kst + ko + D, v);
    }
    ld16(a.y + ro, y);
    ld16(a.a + ro, av);
  } else {
#pragma unroll
    for (int r = 0; r < C; ++r) y[r] = av[r] = 0.0f;
  }

  auto barrier = [&]() {
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  };
  auto wait_mma = [&]() {
    if (!tc::mbar_wait(&mbar_mma, parity)) atomicExch(&abort_s, 1);
    parity ^= 1u;
    tc::fence_after_sync();
  };
  auto hidden_epi = [&](const float* bl, unsigned char* th, unsigned char* tlo) {
#pragma unroll
    for (int c0 = 0; c0 < HC; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tl + L::T_R + half * HC + c0, v);
      tc::tmem_wait_ld();
      const int col = half * HC + c0;
      const float4* b4 = reinterpret_cast<const float4*>(bl + col);
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        const float4 bq = b4[q4];
        const float2 t0 = tanh_acc2(__fadd2_rn(make_float2(v[4 * q4], v[4 * q4 + 1]),
                                               make_float2(bq.x, bq.y)));
        const float2 t1 = tanh_acc2(__fadd2_rn(make_float2(v[4 * q4 + 2], v[4 * q4 + 3]),
                                               make_float2(bq.z, bq.w)));
        v[4 * q4] = t0.x, v[4 * q4 + 1] = t0.y;
        v[4 * q4 + 2] = t1.x, v[4 * q4 + 3] = t1.y;
      }
      store_row16<true>(th, tlo, row, col, H, v);
    }
  };
  auto delta_epi = [&](unsigned char* th, unsigned char* tlo) {
#pragma unroll
    for (int c0 = 0; c0 < HC; c0 += 16) {
      const int col = half * HC + c0;
      float v[16];
      tc::tmem_ld16(tl + L::T_R + col, v);
#pragma unroll
      for (int c8 = 0; c8 < 2; ++c8) {
        const uint32_t off = tc::cm_offset(row, col + 8 * c8, H);
        const uint4 hv = *reinterpret_cast<const uint4*>(th + off);
        const uint4 lv = *reinterpret_cast<const uint4*>(tlo + off);
        const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w}, lw[4] = {lv.x, lv.y, lv.z, lv.w};
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&hw[j]);
          const __nv_bfloat162 l2 = *reinterpret_cast<const __nv_bfloat162*>(&lw[j]);
          const float2 x = __fadd2_rn(make_float2(__low2float(h2), __high2float(h2)),
                                      make_float2(__low2float(l2), __high2float(l2)));
          const float2 g = __ffma2_rn(make_float2(-x.x, -x.y), x, make_float2(1.0f, 1.0f));
          const float2 d = __fmul2_rn(make_float2(v[8 * c8 + 2 * j], v[8 * c8 + 2 * j + 1]), g);
          v[8 * c8 + 2 * j] = d.x;
          v[8 * c8 + 2 * j + 1] = d.y;
        }
      }
      store_row16<true>(th, tlo, row, col, H, v);
    }
  };
  const uint32_t idH = tc::idesc_bf16_f32(128, H);

  // ---- the stages of this launch
  float* S = a.gpart + (size_t)blockIdx.x * 3 * P;  // this CTA's slots U, E, F
  bool u_init = false, e_init = false, f_init = false;
  float Udb[16], Edb[16], Fdb[16];  // the output bias's part of G: sum over rows of A
#pragma unroll
  for (int r = 0; r < C; ++r) Udb[r] = Edb[r] = Fdb[r] = 0.0f;
  const double hsd = mode == JA_STEP ? -c.h_use : -c.h0;  // negative: backward in time
  const float hs = (float)hsd;
  const int nst = mode == JA_STEP ? 6 : 1;
  float sq0 = 0.0f, sq1 = 0.0f;  // this thread's squared scaled terms
#pragma unroll 1
  for (int st = 0; st < nst; ++st) {
    const int i = mode == JA_STEP ? st + 2 : 1;  // the tableau's stage
    const int slot = mode == JA_STEP ? i - 1 : (mode == JA_EVAL ? 0 : 1);
    float Y[16], A[16];
    double tin = c.t;
    if (live && mode == JA_PROBE) {
      float k0[16];
      ld16(a.kst + ko, k0);
#pragma unroll
      for (int r = 0; r < C; ++r) Y[r] = madd(hs, k0[r], y[r]);
      ld16(a.kst + ko + D, k0);
#pragma unroll
      for (int r = 0; r < C; ++r) A[r] = madd(hs, k0[r], av[r]);
      tin = c.t + hsd;
    } else if (live && mode == JA_STEP) {
      // Y_i = y + h (a_i1 k_1 + ... + a_i,i-1 k_i-1), the same for A
      float sy[16], sa[16], kk[16];
#pragma unroll
      for (int r = 0; r < C; ++r) sy[r] = sa[r] = 0.0f;
      for (int l = 1; l < i; ++l) {
        const float al = (float)Tb::a(i, l);
        if (al == 0.0f) continue;
        ld16(a.kst + (size_t)(l - 1) * KS + ko, kk);
#pragma unroll
        for (int r = 0; r < C; ++r) sy[r] = madd(al, kk[r], sy[r]);
        ld16(a.kst + (size_t)(l - 1) * KS + ko + D, kk);
#pragma unroll
        for (int r = 0; r < C; ++r) sa[r] = madd(al, kk[r], sa[r]);
      }
#pragma unroll
      for (int r = 0; r < C; ++r) {
        Y[r] = madd(hs, sy[r], y[r]);
        A[r] = madd(hs, sa[r], av[r]);
      }
      tin = c.t + Tb::c(i) * hsd;
      if (i == 7) {  // SSAL: the last stage input is the candidate
        st16(a.yc + ro, Y);
        st16(a.ac + ro, A);
      }
    } else {
#pragma unroll
      for (int r = 0; r < C; ++r) {
        Y[r] = live ? y[r] : 0.0f;
        A[r] = live ? av[r] : 0.0f;
      }
    }
    store_row16<true>(sXh, sXl, row, coff, K0, Y);
    store_row16<true>(sD3h, sD3l, row, coff, D, A);
    if (half == 1) {
      const float tf = live ? (float)tin : 0.0f;
      const __nv_bfloat16 th = __float2bfloat16_rn(tf);
      const __nv_bfloat16 tlo = __float2bfloat16_rn(tf - __bfloat162float(th));
      *reinterpret_cast<__nv_bfloat16*>(sXh + tc::cm_offset(row, D, K0)) = th;
      *reinterpret_cast<__nv_bfloat16*>(sXl + tc::cm_offset(row, D, K0)) = tlo;
    }
    barrier();

    // F0, F1: the hidden layers at [Y; t]
    if (tid == 0) {
      const uint32_t wa = tc::smem_u32(sW + Cfg::W_off(0));
      for (int kk = 0; kk < K0 / 16; ++kk) {
        const uint64_t db = tc::smem_desc(wa + kk * 256, 128, K0 * 16);
        tc::mma_bf16(tbase + L::T_R, tc::smem_desc(tc::smem_u32(sXh) + kk * 256, 128, K0 * 16), db,
                     idH, kk > 0);
        tc::mma_bf16(tbase + L::T_R, tc::smem_desc(tc::smem_u32(sXl) + kk * 256, 128, K0 * 16), db,
                     idH, true);
      }
      tc::mma_commit(&mbar_mma);
    }
    wait_mma();
    hidden_epi(sBias, sH1h, sH1l);
    barrier();
    if (tid == 0) {
      const uint32_t wa = tc::smem_u32(sW + Cfg::W_off(1));
      for (int kk = 0; kk < H / 16; ++kk) {
        const uint64_t db = tc::smem_desc(wa + kk * 256, 128, H * 16);
        tc::mma_bf16(tbase + L::T_R, tc::smem_desc(tc::smem_u32(sH1h) + kk * 256, 128, H * 16), db,
                     idH, kk > 0);
        tc::mma_bf16(tbase + L::T_R, tc::smem_desc(tc::smem_u32(sH1l) + kk * 256, 128, H * 16), db,
                     idH, true);
      }
      tc::mma_commit(&mbar_mma);
    }
    wait_mma();
    hidden_epi(sBias + H, sH2h, sH2l);
    barrier();
    // F2: the output layer, k_y = h2 W3^T + b3
    float ky[16], ka[16];
    if (tid == 0) {
      const uint32_t wa = tc::smem_u32(sW + Cfg::W_off(2));
      const uint32_t idD = tc::idesc_bf16_f32(128, D);
      for (int kk = 0; kk < H / 16; ++kk) {
        const uint64_t db = tc::smem_desc(wa + kk * 256, 128, H * 16);
        tc::mma_bf16(tbase + L::T_R, tc::smem_desc(tc::smem_u32(sH2h) + kk * 256, 128, H * 16), db,
                     idD, kk > 0);
        tc::mma_bf16(tbase + L::T_R, tc::smem_desc(tc::smem_u32(sH2l) + kk * 256, 128, H * 16), db,
                     idD, true);
      }
      tc::mma_commit(&mbar_mma);
    }
    wait_mma();
    tc::tmem_ld16(tl + L::T_R + coff, ky);
    tc::tmem_wait_ld();
#pragma unroll
    for (int r = 0; r < C; ++r) ky[r] += sBias[2 * H + coff + r];
    barrier();  // every lane's output read before B2 overwrites the accumulator
    // B2: acc = A W3;  G_W3^T = h2^T A  (split operands: hi*hi + lo*hi + hi*lo)
    if (tid == 0) {
      const uint32_t w3 = tc::smem_u32(sW + Cfg::W_off(2));
      const uint32_t dh = tc::smem_u32(sD3h), dl = tc::smem_u32(sD3l);
      const uint32_t idR = tc::idesc_bf16_f32(128, H, false, true);
      for (int kk = 0; kk < D / 16; ++kk) {
        const uint64_t db = tc::smem_desc_mn(w3 + kk * 2 * (H * 16), H * 16);
        tc::mma_bf16(tbase + L::T_R, tc::smem_desc(dh + kk * 256, 128, D * 16), db, idR, kk > 0);
        tc::mma_bf16(tbase + L::T_R, tc::smem_desc(dl + kk * 256, 128, D * 16), db, idR, true);
      }
      const uint32_t idT = tc::idesc_bf16_f32(128, D, true, true);
      const uint32_t hh = tc::smem_u32(sH2h), hl = tc::smem_u32(sH2l);
      for (int kk = 0; kk < 128 / 16; ++kk) {
        const uint64_t bh = tc::smem_desc_mn(dh + kk * 2 * (D * 16), D * 16);
        const uint64_t bl = tc::smem_desc_mn(dl + kk * 2 * (D * 16), D * 16);
        const uint64_t ah = tc::smem_desc_mn(hh + kk * 2 * (H * 16), H * 16);
        const uint64_t al = tc::smem_desc_mn(hl + kk * 2 * (H * 16), H * 16);
        tc::mma_bf16(tbase + L::T_D2, ah, bh, idT, kk > 0);
        tc::mma_bf16(tbase + L::T_D2, al, bh, idT, true);
        tc::mma_bf16(tbase + L::T_D2, ah, bl, idT, true);
      }
      tc::mma_commit(&mbar_mma);
    }
    wait_mma();
    delta_epi(sH2h, sH2l);  // delta2 replaces h2
    barrier();
    // B1: acc = delta2 W2;  G_W2 = delta2^T h1;  G_b2 = delta2^T 1
    if (tid == 0) {
      const uint32_t w2 = tc::smem_u32(sW + Cfg::W_off(1));
      const uint32_t dh = tc::smem_u32(sH2h), dl = tc::smem_u32(sH2l);
      const uint32_t idR = tc::idesc_bf16_f32(128, H, false, true);
      for (int kk = 0; kk < H / 16; ++kk) {
        const uint64_t db = tc::smem_desc_mn(w2 + kk * 2 * (H * 16), H * 16);
        tc::mma_bf16(tbase + L::T_R, tc::smem_desc(dh + kk * 256, 128, H * 16), db, idR, kk > 0);
        tc::mma_bf16(tbase + L::T_R, tc::smem_desc(dl + kk * 256, 128, H * 16), db, idR, true);
      }
      const uint32_t idT = tc::idesc_bf16_f32(128, H, true, true);
      const uint32_t idB = tc::idesc_bf16_f32(128, 16, true, true);
      const uint32_t hh = tc::smem_u32(sH1h), hl = tc::smem_u32(sH1l);
      for (int kk = 0; kk < 128 / 16; ++kk) {
        const uint64_t ah = tc::smem_desc_mn(dh + kk * 2 * (H * 16), H * 16);
        const uint64_t al = tc::smem_desc_mn(dl + kk * 2 * (H * 16), H * 16);
        const uint64_t bh = tc::smem_desc_mn(hh + kk * 2 * (H * 16), H * 16);
        const uint64_t bl = tc::smem_desc_mn(hl + kk * 2 * (H * 16), H * 16);
        const uint64_t b1 = tc::smem_desc_mn(tc::smem_u32(sOnes) + kk * 2 * (16 * 16), 16 * 16);
        tc::mma_bf16(tbase + L::T_D1, ah, bh, idT, kk > 0);
        tc::mma_bf16(tbase + L::T_D1, al, bh, idT, true);
        tc::mma_bf16(tbase + L::T_D1, ah, bl, idT, true);
        tc::mma_bf16(tbase + L::T_DB, ah, b1, idB, kk > 0);
        tc::mma_bf16(tbase + L::T_DB, al, b1, idB, true);
      }
      tc::mma_commit(&mbar_mma);
    }
    wait_mma();
    delta_epi(sH1h, sH1l);  // delta1 replaces h1
    barrier();
    // B0: acc = delta1 W1 (= J^T A, the t column too);  G_W1 = delta1^T [X | 1]
    if (tid == 0) {
      const uint32_t w1 = tc::smem_u32(sW + Cfg::W_off(0));
      const uint32_t dh = tc::smem_u32(sH1h), dl = tc::smem_u32(sH1l);
      const uint32_t idR = tc::idesc_bf16_f32(128, K0, false, true);
      for (int kk = 0; kk < H / 16; ++kk) {
        const uint64_t db = tc::smem_desc_mn(w1 + kk * 2 * (K0 * 16), K0 * 16);
        tc::mma_bf16(tbase + L::T_R, tc::smem_desc(dh + kk * 256, 128, H * 16), db, idR, kk > 0);
        tc::mma_bf16(tbase + L::T_R, tc::smem_desc(dl + kk * 256, 128, H * 16), db, idR, true);
      }
      const uint32_t idT = tc::idesc_bf16_f32(128, K0, true, true);
      const uint32_t xh = tc::smem_u32(sXh), xl = tc::smem_u32(sXl);
      for (int kk = 0; kk < 128 / 16; ++kk) {
        const uint64_t ah = tc::smem_desc_mn(dh + kk * 2 * (H * 16), H * 16);
        const uint64_t al = tc::smem_desc_mn(dl + kk * 2 * (H * 16), H * 16);
        const uint64_t bh = tc::smem_desc_mn(xh + kk * 2 * (K0 * 16), K0 * 16);
        const uint64_t bl = tc::smem_desc_mn(xl + kk * 2 * (K0 * 16), K0 * 16);
        tc::mma_bf16(tbase + L::T_D0, ah, bh, idT, kk > 0);
        tc::mma_bf16(tbase + L::T_D0, al, bh, idT, true);
        tc::mma_bf16(tbase + L::T_D0, ah, bl, idT, true);
      }
      tc::mma_commit(&mbar_mma);
    }
    wait_mma();
    tc::tmem_ld16(tl + L::T_R + coff, ka);
    tc::tmem_wait_ld();
#pragma unroll
    for (int r = 0; r < C; ++r) ka[r] = -ka[r];  // k_a = -J^T A
    if (live) {
      st16(a.kst + (size_t)slot * KS + ko, ky);
      st16(a.kst + (size_t)slot * KS + ko + D, ka);
    }

    // ---- this stage's part of G into the CTA's slots: U += (-h b_i) G,
    // E += (-h e_i) G, F = -G (the stage whose k is a next k1 or a probe)
    float wU = 0.0f, wE = 0.0f, wF = 0.0f;
    if (mode == JA_STEP) {
      wU = (float)(-hsd * Tb::b(i));
      wE = (float)(-hsd * Tb::e(i));
      if (i == 7) wF = -1.0f;
    } else {
      wF = -1.0f;
    }
    if (wU != 0.0f || wE != 0.0f || wF != 0.0f) {
      // 16 consecutive slot entries (64-byte aligned): both slots' old values
      // are loaded before anything is stored, so the loads overlap
      auto rmw16 = [&](int idx, const float (&v)[16]) {
        float4 u[4], e[4];
        float4* pu = reinterpret_cast<float4*>(S + idx);
        float4* pe = reinterpret_cast<float4*>(S + P + idx);
        float4* pf = reinterpret_cast<float4*>(S + 2 * P + idx);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          u[q] = (wU != 0.0f && u_init) ? pu[q] : make_float4(0.f, 0.f, 0.f, 0.f);
          e[q] = (wE != 0.0f && e_init) ? pe[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (wU != 0.0f)
            pu[q] = make_float4(madd(wU, v[4 * q], u[q].x), madd(wU, v[4 * q + 1], u[q].y),
                                madd(wU, v[4 * q + 2], u[q].z), madd(wU, v[4 * q + 3], u[q].w));
          if (wE != 0.0f)
            pe[q] = make_float4(madd(wE, v[4 * q], e[q].x), madd(wE, v[4 * q + 1], e[q].y),
                                madd(wE, v[4 * q + 2], e[q].z), madd(wE, v[4 * q + 3], e[q].w));
          if (wF != 0.0f)
            pf[q] = make_float4(wF * v[4 * q], wF * v[4 * q + 1], wF * v[4 * q + 2],
                                wF * v[4 * q + 3]);
        }
      };
      float v[16];
      // G_W1 (lane = hidden unit; its t and b1 columns included)
      for (int cc = half * 32; cc < (half ? K0 : 32); cc += 16) {
        tc::tmem_ld16(tl + L::T_D0 + cc, v);
        tc::tmem_wait_ld();
        rmw16(L::P_W0 + row * K0 + cc, v);
      }
#pragma unroll 1
      for (int cc = 0; cc < HC; cc += 16) {
        const int col = half * HC + cc;
        tc::tmem_ld16(tl + L::T_D1 + col, v);
        tc::tmem_wait_ld();
        rmw16(L::P_W1 + row * H + col, v);
      }
      tc::tmem_ld16(tl + L::T_DB, v);
      tc::tmem_wait_ld();
      if (half == 0) {
        const int idx = L::P_B1 + row;
        if (wU != 0.0f) S[idx] = madd(wU, v[0], u_init ? S[idx] : 0.0f);
        if (wE != 0.0f) S[P + idx] = madd(wE, v[0], e_init ? S[P + idx] : 0.0f);
        if (wF != 0.0f) S[2 * P + idx] = wF * v[0];
      }
      tc::tmem_ld16(tl + L::T_D2 + coff, v);
      tc::tmem_wait_ld();
      rmw16(L::P_W2T + row * D + coff, v);
#pragma unroll
      for (int r = 0; r < C; ++r) {
        Udb[r] = madd(wU, A[r], Udb[r]);
        Edb[r] = madd(wE, A[r], Edb[r]);
        if (wF != 0.0f) Fdb[r] = wF * A[r];
      }
      u_init = u_init || wU != 0.0f;
      e_init = e_init || wE != 0.0f;
      f_init = f_init || wF != 0.0f;
    }
    // the squared scaled terms of the starting-step norms
    if (live && mode == JA_EVAL) {
#pragma unroll
      for (int r = 0; r < C; ++r) {
        const float sy = (float)a.atol + (float)a.rtol * fabsf(y[r]);
        const float sa = (float)a.atol + (float)a.rtol * fabsf(av[r]);
        sq0 += (y[r] / sy) * (y[r] / sy) + (av[r] / sa) * (av[r] / sa);
        sq1 += (ky[r] / sy) * (ky[r] / sy) + (ka[r] / sa) * (ka[r] / sa);
      }
    } else if (live && mode == JA_PROBE) {
      float k0[16];
      ld16(a.kst + ko, k0);
#pragma unroll
      for (int r = 0; r < C; ++r) {
        const float sy = (float)a.atol + (float)a.rtol * fabsf(y[r]);
        const float dy = (ky[r] - k0[r]) / sy;
        sq0 += dy * dy;
      }
      ld16(a.kst + ko + D, k0);
#pragma unroll
      for (int r = 0; r < C; ++r) {
        const float sa = (float)a.atol + (float)a.rtol * fabsf(av[r]);
        const float da = (ka[r] - k0[r]) / sa;
        sq0 += da * da;
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (abort_s) break;
  }

  // ---- the attempt's error terms of this row: e = h sum_i e_i k_i,
  // scaled by atol + rtol max(|z|, |z1|) (z1 = the candidate)
  if (live && mode == JA_STEP && !abort_s) {
#pragma unroll 1
    for (int part = 0; part < 2; ++part) {
      float e[16], kk[16], z1[16];
#pragma unroll
      for (int r = 0; r < C; ++r) e[r] = 0.0f;
      for (int l = 1; l <= 7; ++l) {
        const float el = (float)Tb::e(l);
        if (el == 0.0f) continue;
        ld16(a.kst + (size_t)(l - 1) * KS + ko + part * D, kk);
#pragma unroll
        for (int r = 0; r < C; ++r) e[r] = madd(el, kk[r], e[r]);
      }
      ld16((part ? a.ac : a.yc) + ro, z1);
#pragma unroll
      for (int r = 0; r < C; ++r) {
        const float z = part ? av[r] : y[r];
        const float sc = madd((float)a.rtol, fmaxf(fabsf(z), fabsf(z1[r])), (float)a.atol);
        const float q = (hs * e[r]) / sc;
        sq0 += q * q;
      }
    }
  }
  // the output bias's part of G: the rows' sums, in row order (the h2 tile
  // is free now)
  float* sR = reinterpret_cast<float*>(sH2h);
  auto row_sum = [&](const float (&v)[16], bool init, float* dst) {
#pragma unroll
    for (int r = 0; r < C; ++r) sR[row * D + coff + r] = v[r];
    __syncthreads();
    if (tid < D) {
      float s = 0.0f;
      for (int rr = 0; rr < 128; ++rr) s += sR[rr * D + tid];
      dst[L::P_B2 + tid] = init ? s : 0.0f;
    }
    __syncthreads();
  };
  row_sum(Udb, u_init, S);
  row_sum(Edb, e_init, S + P);
  row_sum(Fdb, f_init, S + 2 * P);
  // slots no stage wrote hold zeros (their decide launch reads them)
  for (int p = tid; p < P; p += 256) {
    if (p >= L::P_B2) break;
    if (!u_init) S[p] = 0.0f;
    if (!e_init) S[P + p] = 0.0f;
    if (!f_init) S[2 * P + p] = 0.0f;
  }
  // this CTA's squared scaled sums, in a fixed order, in FP64
  {
    double v0 = sq0, v1 = sq1;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      v0 += __shfl_xor_sync(0xffffffffu, v0, off);
      v1 += __shfl_xor_sync(0xffffffffu, v1, off);
    }
    if ((tid & 31) == 0) red[warp] = v0;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < 8; ++w) s += red[w];
      a.epart[2 * blockIdx.x] = s;
    }
    __syncthreads();
    if ((tid & 31) == 0) red[warp] = v1;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < 8; ++w) s += red[w];
      a.epart[2 * blockIdx.x + 1] = s;
    }
  }
  if (abort_s && tid == 0) atomicExch(a.err, 1);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, L::T_COLS);
}

// Decide launch of the joint continuous adjoint (see k_mlp_jadj): per
// parameter the CTAs' slots in CTA order, abar's candidate and its squared
// scaled error term; then the last CTA's decision and controller, exactly
// the solver's (the oracle's orc_solve on the same augmented problem).
template <class Cfg, class Tb = DP5>
__global__ void __launch_bounds__(256) k_mlp_jadj_decide(JadjArgs a, int mode, int grid1) {
  using L = MlpAdjLayout<Cfg>;
  constexpr int P = L::P_FLOATS;
  __shared__ double red[8];
  __shared__ int last_s;
  const JadjCtl c = *a.ctl;
  if (c.status != ST_RUNNING) return;
  const int tid = threadIdx.x;
  const double hs = -c.h_use;
  double s0 = 0.0, s1 = 0.0;
  for (int p = blockIdx.x * 256 + tid; p < P; p += gridDim.x * 256) {
    if (mode == JA_STEP && c.pending) {  // commit the accepted candidate
      a.th[p] = a.thc[p];
      a.kth1[p] = a.fsum[p];
    }
    // the CTAs' slots in CTA order (eight rows of loads in flight, added
    // one by one in order), by compensated FP32 sums: B300's FP64 pipe is
    // narrow, and the compensation keeps the sums to a few FP32 roundings
    float su = 0.0f, cu = 0.0f, se = 0.0f, ce = 0.0f, sf = 0.0f, cf = 0.0f;
    auto kahan = [](float& s_, float& c_, float x) {
      const float yk = x - c_;
      const float tk = s_ + yk;
      c_ = (tk - s_) - yk;
      s_ = tk;
    };
    for (int b0 = 0; b0 < grid1; b0 += 8) {
      float u[8], e[8], f[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int b = b0 + q;
        const float* S = a.gpart + (size_t)b * 3 * P;
        const bool in = b < grid1;
        u[q] = (in && mode == JA_STEP) ? __ldcg(S + p) : 0.0f;
        e[q] = (in && mode == JA_STEP) ? __ldcg(S + P + p) : 0.0f;
        f[q] = in ? __ldcg(S + 2 * P + p) : 0.0f;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        kahan(su, cu, u[q]);
        kahan(se, ce, e[q]);
        kahan(sf, cf, f[q]);
      }
    }
    const double U = (double)su - (double)cu, E = (double)se - (double)ce,
                 Fs = (double)sf - (double)cf;
    const double th = a.th[p];
    if (!jadj_real<L>(p)) {
      if (mode == JA_STEP) {
        a.thc[p] = th;
        a.fsum[p] = 0.0;
      } else if (mode == JA_EVAL) {
        a.kth1[p] = 0.0;
      }
      continue;
    }
    if (mode == JA_EVAL) {
      a.kth1[p] = Fs;
      const double sc = a.atol + a.rtol * fabs(th);
      s0 += (th / sc) * (th / sc);
      s1 += (Fs / sc) * (Fs / sc);
    } else if (mode == JA_PROBE) {
      const double sc = a.atol + a.rtol * fabs(th);
      const double d = (Fs - a.kth1[p]) / sc;
      s0 += d * d;
    } else {
      const double k1 = a.kth1[p];
      const double thn = th + (U + hs * Tb::b(1) * k1);
      const double e = E + hs * Tb::e(1) * k1;
      a.thc[p] = thn;
      a.fsum[p] = Fs;
      const double sc = a.atol + a.rtol * fmax(fabs(th), fabs(thn));
      s0 += (e / sc) * (e / sc);
    }
  }
  // this CTA's partials in a fixed order
  auto cta_total = [&](double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0)
      for (int w = 0; w < 8; ++w) s += red[w];
    __syncthreads();
    return s;
  };
  const double p0 = cta_total(s0), p1 = cta_total(s1);
  if (tid == 0) {
    a.dpart[2 * blockIdx.x] = p0;
    a.dpart[2 * blockIdx.x + 1] = p1;
    __threadfence();
    last_s = atomicAdd(&a.ctl->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last_s) return;
  __threadfence();
  // ---- the last CTA: every partial (each thread a fixed subset, then the
  // fixed tree of cta_total), then thread 0's decision
  double q0 = 0.0, q1 = 0.0;
  for (int b = tid; b < (int)gridDim.x; b += 256) {
    q0 += __ldcg(a.dpart + 2 * b);
    q1 += __ldcg(a.dpart + 2 * b + 1);
  }
  for (int b = tid; b < grid1; b += 256) {
    q0 += __ldcg(a.epart + 2 * b);
    q1 += __ldcg(a.epart + 2 * b + 1);
  }
  const double t0 = cta_total(q0), t1 = cta_total(q1);
  if (tid != 0) return;
  JadjCtl n = c;
  n.ticket = 0;
  const double N = a.nnorm;
  auto clip = [&]() {
    const double rem = n.t - n.t_end;
    if (n.h >= rem) {
      n.h_use = rem;
      n.use_last = 1;
    } else {
      n.h_use = n.h;
      n.use_last = 0;
    }
  };
  if (mode == JA_EVAL) {
    const double d0 = sqrt(t0 / N), d1 = sqrt(t1 / N);
    n.h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * (d0 / d1);
    n.d1 = d1;
    n.n_fe += 1;
  } else if (mode == JA_PROBE) {
    const double d2 = sqrt(t0 / N) / c.h0;
    const double m = fmax(c.d1, d2);
    const double h1 = (m <= 1e-15) ? fmax(1e-6, c.h0 * 1e-3) : ctl_pow(0.01 / m, 1.0 / 5.0);
    double h = fmin(100.0 * c.h0, h1);
    h = fmin(h, c.t - c.t_end);
    if (!(h > 0.0 && isfinite(h))) h = c.t - c.t_end;
    n.h = h;
    n.n_fe += 1;
    clip();
  } else {
    const double err = sqrt(t0 / N);
    const bool finite = isfinite(err);
    const bool accept = finite && err <= 1.0;
    double h_next;
    n.n_fe += 6;
    if (accept) {
      n.t = c.use_last ? c.t_end : c.t + hs;
      double fac;
      if (err == 0.0) {
        fac = a.fac_max;
      } else {
        fac = a.safety * ctl_pow(err, -a.beta1);
        if (a.beta2 != 0.0) fac = fac * ctl_pow(c.err_prev, a.beta2);
        if (a.beta3 != 0.0) fac = fac * ctl_pow(c.err_prev2, -a.beta3);
      }
      fac = fmin(fmax(fac, a.fac_min), a.fac_max);
      if (c.prev_rej) fac = fmin(fac, 1.0);
      h_next = c.h_use * fac;
      n.err_prev2 = c.err_prev;
      n.err_prev = fmax(err, 1e-4);
      n.prev_rej = 0;
      n.n_acc += 1;
      n.pending = 1;
      if (c.use_last) n.status = ST_SUCCESS;
    } else {
      const double fac =
          finite ? fmin(fmax(a.safety * ctl_pow(err, -a.beta1), a.fac_min), 1.0) : a.fac_min;
      h_next = c.h_use * fac;
      n.prev_rej = 1;
      n.n_rej += 1;
      n.pending = 0;
    }
    n.h = h_next;
    if (n.status == ST_RUNNING) {
      const double scale = fmax(fabs(n.t), fabs(n.t_end));
      if (n.t - h_next == n.t || h_next < 1e-14 * scale || !(h_next > 0.0))
        n.status = finite ? ST_DT_UNDERFLOW : ST_NONFINITE;
      else if (n.n_acc + n.n_rej >= a.max_steps)
        n.status = ST_MAX_STEPS;
    }
    clip();
  }
  *a.ctl = n;
}

// Segment end: commit an accepted last candidate (rows and abar).
__global__ void k_mlp_jadj_commit(JadjArgs a, int P) {
  const JadjCtl c = *a.ctl;
  if (!c.pending) return;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long BD = (long long)a.B * 32;
  if (e < BD) {
    a.y[e] = a.yc[e];
    a.a[e] = a.ac[e];
  }
  if (e < P) a.th[e] = a.thc[e];
}

// a += the cotangent of evaluation point q (the loss jumps there).
__global__ void k_mlp_jadj_jump(float* av, const float* gye, int B, int K, int D, int q) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)B * D) return;
  const long long b = e / D, j = e % D;
  av[e] += gye[(b * K + q) * D + j];
}

// abar (the parameters' layout of the adjoint partials) into the layers'
// gradients, W[l] row-major [out][in] like the field's weights.
template <class Cfg>
__global__ void k_mlp_jadj_out(const double* th, float* gW0, float* gb0, float* gW1, float* gb1,
                               float* gW2, float* gb2) {
  using L = MlpAdjLayout<Cfg>;
  constexpr int D = Cfg::D, H = Cfg::H, K0 = Cfg::K0, IN = D + 1;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < H * IN) {
    gW0[k] = (float)th[L::P_W0 + (k / IN) * K0 + k % IN];
    return;
  }
  k -= H * IN;
  if (k < H) {
    if (gb0) gb0[k] = (float)th[L::P_W0 + k * K0 + IN];
    return;
  }
  k -= H;
  if (k < H * H) {
    gW1[k] = (float)th[L::P_W1 + k];
    return;
  }
  k -= H * H;
  if (k < H) {
    if (gb1) gb1[k] = (float)th[L::P_B1 + k];
    return;
  }
  k -= H;
  if (k < D * H) {
    gW2[k] = (float)th[L::P_W2T + (k % H) * D + k / H];
    return;
  }
  k -= D * H;
  if (k < D && gb2) gb2[k] = (float)th[L::P_B2 + k];
}

// ---------------------------------------------------------------- host side
// Opts a kernel into its dynamic shared memory once per device: the
// attribute is host-side state, and doing it once keeps later calls (for
// instance inside a CUDA-graph capture) free of it.
static tode_err smem_optin(const void* fn, int bytes, std::atomic<uint64_t>& done) {
  int dev = 0;
  TODE_CUDA_TRY(cudaGetDevice(&dev));
  const uint64_t bit = 1ull << (dev & 63);
  if (done.load() & bit) return TODE_OK;
  TODE_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.fetch_or(bit);
  return TODE_OK;
}

using Cfg32 = MlpCfg<32, 128, 3, false>;
using Cfg32s = MlpCfg<32, 128, 3, true>;
using Cfg64s = MlpWideCfg<64, 512, 4>;  // the wide network's solver (stacked M = 128 tiles)

// the two networks the MLP field is built for
static bool is_d32_h128(const tode_field_desc* f) {
  return f->n_layers == 3 && f->D == 32 && f->widths[0] == 33 && f->widths[1] == 128 &&
         f->widths[2] == 128 && f->widths[3] == 32;
}
static bool is_d64_h512(const tode_field_desc* f) {
  return f->n_layers == 4 && f->D == 64 && f->widths[0] == 65 && f->widths[1] == 512 &&
         f->widths[2] == 512 && f->widths[3] == 512 && f->widths[4] == 64;
}

bool mlp_supported(const tode_field_desc* f) {
  if (!f || f->kind != TODE_MLP || !f->widths) return false;
  return is_d32_h128(f) || is_d64_h512(f);
}

size_t mlp_workspace_bytes(const tode_field_desc* f, const tode_options* o) {
  const size_t img = is_d64_h512(f) ? (size_t)Cfg64s::WREP * Cfg64s::WIMG_STRIDE
                                    : (size_t)Cfg32::WREP * Cfg32::WIMG_STRIDE;
  // counters, images, the work order and its sort's per-CTA counts
  size_t b = align256(256) + img + align256((size_t)std::max(f->B, 1) * 4) +
             order_part_bytes(f->B);
  if (o->form == TODE_PLAIN) {  // parked solver state (must match launch_mlp)
    const size_t B = (size_t)f->B, D = (size_t)f->D;
    b += 3 * align256(B * D * 4) + align256(B * 8) + 5 * align256(B * 4);
  }
  return b;
}

template <class Cfg, class Tab = DP5> static tode_err launch_mlp(const SolveReq& r) {
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
  a.yp = (float*)r.yp;
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
  a.o.beta3 = r.o->beta3;
  a.o.h0 = r.o->h0;
  a.o.max_steps = r.o->max_steps;
  opts_round_f32(a.o);
  a.rs_seg = -1;
  auto set_ck = [&](const tode_tape* tp) {
    a.ck_stride = tp->stride;
    a.ck_slots = tp->slots;
    a.ck_y = (float*)tp->y;
    a.ck_ylo = (float*)tp->y_lo;
    a.ck_k1 = (float*)tp->k1;
    a.ck_t = tp->t;
    a.ck_h = (float*)tp->h;
    a.ck_ep = (float*)tp->err_prev;
    a.ck_ep2 = (float*)tp->err_prev2;
    a.ck_fl = tp->flags;
  };
  if (r.tape && r.tape->stride > 1) {  // checkpoints every stride steps, no stage tape
    a.slots = 0;
    set_ck(r.tape);
  } else if (r.tape) {
    a.slots = r.tape->slots;
    a.tp_y = (float*)r.tape->y;
    a.tp_k1 = (float*)r.tape->k1;
    a.tp_t = r.tape->t;
    a.tp_h = (float*)r.tape->h_acc;
    a.tp_ys = (float*)r.tape->y_stage;
  } else {
    a.slots = 0;
  }
  if (r.resolve) {  // one segment from the checkpoints into the stage tape
    set_ck(r.ck);
    a.rs_seg = r.rs_seg;
    a.rs_nacc = r.n_acc;
    a.rs_n = r.rs_n;
    a.rs_t0 = r.rs_t0;
    a.rs_t1 = r.rs_t1;
    a.K = 0;
    a.ye = a.yp = nullptr;
  }
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
  a.active = (int32_t*)(p + 64);
  a.err = (int32_t*)(p + 128);
  p += align256(256);
  unsigned char* img = (unsigned char*)p;
  a.wimg = img;
  p += (size_t)Cfg::WREP * Cfg::WIMG_STRIDE;
  int32_t* order = (int32_t*)p;
  p += align256((size_t)std::max(r.B, 1) * 4);
  int* order_part = (int*)p;
  p += order_part_bytes(r.B);
  a.order = nullptr;
  if (r.o->order == 1 && r.B > 0) {
    // the longest integration intervals first (rows refill from the queue,
    // so the long instances start early and the tail shortens)
    TODE_CUDA_TRY(launch_order(r.B, IntervalBin{r.t0, r.t1}, order, order_part, r.stream));
    a.order = order;
  }
  if (r.o->form == TODE_PLAIN) {
    const size_t B = (size_t)r.B, D = (size_t)r.D;
    a.wy = (float*)p;
    p += align256(B * D * 4);
    a.wylo = (float*)p;
    p += align256(B * D * 4);
    a.wk1 = (float*)p;
    p += align256(B * D * 4);
    a.wt = (double*)p;
    p += align256(B * 8);
    a.wh = (float*)p;
    p += align256(B * 4);
    a.wep = (float*)p;
    p += align256(B * 4);
    a.wep2 = (float*)p;
    p += align256(B * 4);
    a.wcur = (int32_t*)p;
    p += align256(B * 4);
    a.wfl = (int32_t*)p;
    p += align256(B * 4);
  }
  const cudaStream_t st = r.stream;
  {
    size_t loff[MLP_MAX_LAYERS] = {};
    for (int l = 0; l < Cfg::NL; ++l) loff[l] = Cfg::W_off(l);
    const tode_err e = build_images<Cfg>(r.f, img, Cfg::STREAM ? IMG_CHUNKS : IMG_TILE, Cfg::WREP,
                                         Cfg::WIMG_STRIDE, loff, st);
    if (e != TODE_OK) return e;
  }
  TODE_CUDA_TRY(cudaMemsetAsync(r.ws, 0, 256, st));  // queue counter and error flag
  {
    static std::atomic<uint64_t> done{0};
    const tode_err e = smem_optin((const void*)k_mlp_fused<Cfg, Tab>, Cfg::S_END, done);
    if (e != TODE_OK) return e;
  }
  long long grid = (r.B + Cfg::ROWS - 1) / Cfg::ROWS;
  if (grid > r.num_sms) grid = r.num_sms;
  if (grid == 0) return TODE_OK;
  if (r.o->form == TODE_PLAIN) {
    {
      static std::atomic<uint64_t> d0{0}, d1{0};
      tode_err e = smem_optin((const void*)k_mlp_plain_init<Cfg, Tab>, Cfg::S_END, d0);
      if (e == TODE_OK) e = smem_optin((const void*)k_mlp_plain_step<Cfg, Tab>, Cfg::S_END, d1);
      if (e != TODE_OK) return e;
    }
    k_mlp_plain_init<Cfg, Tab><<<(int)grid, Cfg::NT, Cfg::S_END, st>>>(a);
    TODE_CUDA_TRY(cudaGetLastError());
    const int poll = r.o->poll_every > 0 ? r.o->poll_every : 16;
    long long launched = 0;
    const long long limit = (long long)r.o->max_steps + 2LL * poll + 2;
    while (true) {
      for (int c = 0; c < poll - 1; ++c)
        k_mlp_plain_step<Cfg, Tab><<<(int)grid, Cfg::NT, Cfg::S_END, st>>>(a);
      TODE_CUDA_TRY(cudaMemsetAsync(a.active, 0, sizeof(int32_t), st));
      k_mlp_plain_step<Cfg, Tab><<<(int)grid, Cfg::NT, Cfg::S_END, st>>>(a);
      TODE_CUDA_TRY(cudaGetLastError());
      launched += poll;
      int32_t any = 0;
      TODE_CUDA_TRY(cudaMemcpyAsync(&any, a.active, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      TODE_CUDA_TRY(cudaStreamSynchronize(st));
      if (!any) break;
      // one attempt per launch for every running instance: max_steps bounds
      // the loop; this guard is never expected to fire
      if (launched > limit) return TODE_ETIMEOUT;
    }
    return TODE_OK;
  }
  k_mlp_fused<Cfg, Tab><<<(int)grid, Cfg::NT, Cfg::S_END, st>>>(a);
  TODE_CUDA_TRY(cudaGetLastError());
  return TODE_OK;
}

tode_err mlp_solve(const SolveReq& r, bool split) {
  if (r.o->form != TODE_FUSED && r.o->form != TODE_PLAIN) return TODE_EUNSUPPORTED;
  if (r.resolve && (r.o->form != TODE_FUSED || !split)) return TODE_EUNSUPPORTED;
  if (r.o->method == TODE_TSIT5) {  // the Tsitouras pair, split form
    if (!split) return TODE_EUNSUPPORTED;
    return is_d64_h512(r.f) ? launch_mlp<Cfg64s, TS5>(r) : launch_mlp<Cfg32s, TS5>(r);
  }
  if (is_d64_h512(r.f)) return split ? launch_mlp<Cfg64s>(r) : TODE_EUNSUPPORTED;
  return split ? launch_mlp<Cfg32s>(r) : launch_mlp<Cfg32>(r);
}

// ---- wide network: the staged adjoint's scratch and work items
struct WidePlan {
  int grid, cap, items;
  size_t off_img, off_timg, off_bias, off_order, off_rounds, off_plane[32], off_part, total;
};
// The dW/db jobs of the wide adjoint, in the order dW2, dW3, dW1 (with the
// constant input's column: db1), dW4^T, db2, db3, db4 -- four 128-row blocks
// each (db4: one) -- with their work items (the chain CTAs split in parts:
// ten for the 512 x 512 products, four otherwise: 148 items, one wave of
// one CTA per SM on a 148-SM B300, the heavy items' bytes close to the
// others').  jW[l] / jb[l]: the first job of gradient l.  Returns the
// number of work items.
static int wide_dw_jobs(DwArgs* a, int (&jW)[4], int (&jb)[4]) {
  using L = WideAdj<MlpWideCfg<64, 512, 4>>;
  int nj = 0, it = 0;
  auto add = [&](DwJob j, int parts) {
    if (a) {
      a->job[nj] = j;
      a->item0[nj] = it;
    }
    it += parts;
    ++nj;
  };
  jW[1] = nj;
  for (int mb = 0; mb < 4; ++mb) add(DwJob{0, L::T_D2, mb, L::T_H1, 2, 256}, 10);
  jW[2] = nj;
  for (int mb = 0; mb < 4; ++mb) add(DwJob{0, L::T_D3, mb, L::T_H2, 2, 256}, 10);
  jW[0] = jb[0] = nj;
  for (int mb = 0; mb < 4; ++mb) add(DwJob{0, L::T_D1, mb, L::T_X, 1, 80}, 4);
  jW[3] = nj;
  for (int mb = 0; mb < 4; ++mb) add(DwJob{0, L::T_H3, mb, L::T_K, 1, 64}, 4);
  jb[1] = nj;
  for (int mb = 0; mb < 4; ++mb) add(DwJob{1, L::T_D2, mb, 0, 0, 16}, 4);
  jb[2] = nj;
  for (int mb = 0; mb < 4; ++mb) add(DwJob{1, L::T_D3, mb, 0, 0, 16}, 4);
  jb[3] = nj;
  add(DwJob{2, 0, 0, L::T_K, 1, 64}, 4);
  if (a) {
    a->njobs = nj;
    a->item0[nj] = it;
  }
  return it;
}
static WidePlan wide_plan(int B, int slots, int num_sms) {
  using Cfg = Cfg64s;
  using L = WideAdj<Cfg>;
  WidePlan p{};
  p.grid = (int)std::min<long long>((B + 63) / 64, num_sms);
  p.grid += p.grid & 1;  // CTA pairs
  p.cap = 7 * std::max(slots, 1);  // one instance per row per slice
  const size_t nblk = (size_t)std::max(p.grid, 1) * p.cap;
  size_t o = align256(256);
  p.off_img = o;
  o += (size_t)Cfg::WREP * Cfg::WIMG_STRIDE;
  p.off_timg = o;
  o += (size_t)Cfg::WREP * Cfg::WIMG_STRIDE;
  p.off_bias = o;
  o += align256((size_t)3 * Cfg::H * 4);
  p.off_order = o;
  o += align256((size_t)std::max(B, 1) * 4);
  p.off_rounds = o;
  o += align256((size_t)std::max(p.grid, 1) * 4);
  for (int t = 0; t < L::NTEN; ++t)
    for (int fb = 0; fb < L::t_fb(t); ++fb) {
      p.off_plane[L::plane_first(t) + fb] = o;
      o += align256(nblk * 2 * (size_t)L::blk_bytes(t));
    }
  int jW[4], jb[4];
  p.items = wide_dw_jobs(nullptr, jW, jb);
  p.off_part = o;
  o += (size_t)p.items * DW_PART_FLOATS * 4;
  p.total = o;
  return p;
}

// The wide adjoint's slices hold mult x (SMs x 64) instances (tode_options
// ctas_per_sm, 1..4; default 1): larger slices mean fewer, larger weight-
// gradient passes and more staging memory; the chain CTAs past one per SM
// queue for a free SM.  Results do not depend on it.
static int wide_slice_mult(const tode_options* o) {
  return (o && o->ctas_per_sm > 0) ? std::min(o->ctas_per_sm, 4) : 1;
}

size_t mlp_adjoint_scratch_bytes(const tode_field_desc* f, const tode_options* o, int slots,
                                 int num_sms) {
  using L = MlpAdjLayout<Cfg32s>;
  if (is_d64_h512(f)) return wide_plan(f->B, slots, num_sms * wide_slice_mult(o)).total;
  if (!is_d32_h128(f)) return 0;
  const long long grid = std::min<long long>((f->B + 127) / 128, num_sms);
  return align256(256) + align256((size_t)Cfg32s::WIMG_BYTES) +
         align256((size_t)grid * L::P_FLOATS * 4);
}

static constexpr int DW_SMEM = DW_RING + 4096;  // the copy ring, the ones tile

// The tensor maps of the chain's weight stream: the distinct stage sizes of
// a round (in 128-byte rows, at most WIDE_TMAPS), each a box of that many
// rows over both pair images.  The encoder comes from the driver through the
// runtime's entry-point query (the library links only the runtime).
template <class Cfg>
static tode_err wide_tensor_maps(const unsigned char* img, WideAdjArgs& a) {
  using L = WideAdj<Cfg>;
  static std::atomic<void*> encoder{nullptr};
  void* fn = encoder.load();
  if (!fn) {
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return TODE_ECUDA;
    }
    encoder.store(fn);
  }
  int n = 0;
  for (int g = 0; g < L::stages(); ++g) {
    int q, c0, nc, off, bytes;
    L::stage_of((uint32_t)g, q, c0, nc, off, bytes);
    if (bytes % 128 != 0 || off % 128 != 0) return TODE_EINVAL;
    const int rows = bytes / 128;
    int m = 0;
    while (m < n && a.tmap_rows[m] != rows) ++m;
    if (m == n) {
      if (n == WIDE_TMAPS || rows > 256) return TODE_EINVAL;
      a.tmap_rows[n++] = rows;
    }
  }
  for (int m = n; m < WIDE_TMAPS; ++m) a.tmap_rows[m] = a.tmap_rows[0];
  static_assert(Cfg::WIMG_STRIDE % 128 == 0 && L::HALF_BYTES % 128 == 0, "128-byte rows");
  const cuuint64_t dims[2] = {64, (cuuint64_t)2 * Cfg::WREP * Cfg::WIMG_STRIDE / 128};
  const cuuint64_t strides[1] = {128};
  const cuuint32_t estr[2] = {1, 1};
  for (int m = 0; m < WIDE_TMAPS; ++m) {
    const cuuint32_t box[2] = {64, (cuuint32_t)a.tmap_rows[m]};
    const CUresult r = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn)(
        &a.tmap[m], CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<unsigned char*>(img), dims,
        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return TODE_ECUDA;
  }
  return TODE_OK;
}

template <class Tab> static tode_err mlp_wide_adjoint(const AdjReq& r) {
  using Cfg = Cfg64s;
  using L = WideAdj<Cfg>;
  const cudaStream_t st = r.stream;
  const WidePlan p = wide_plan(r.B, r.tape->slots, r.num_sms * wide_slice_mult(r.o));
  if (r.scratch_bytes < p.total) return TODE_EWORKSPACE;
  char* base = r.scratch;
  WideAdjArgs a{};
  a.K = r.K;
  a.order = (const int32_t*)(base + p.off_order);
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
  a.gye = (const float*)r.gye;
  a.gyf = (const float*)r.gyf;
  a.gy0 = (float*)r.gy0;
  a.bias = (const float*)(base + p.off_bias);
  a.err = (int32_t*)(base + 128);
  a.overflow = r.overflow;
  a.gts = (double*)r.gparam;  // MLP field: the time-translation sums, or NULL
  a.cap = p.cap;
  a.rounds = (int32_t*)(base + p.off_rounds);
  unsigned char* img = (unsigned char*)base + p.off_img;
  unsigned char* timg = (unsigned char*)base + p.off_timg;
  {
    const tode_err e = wide_tensor_maps<Cfg>(img, a);
    if (e != TODE_OK) return e;
  }
  for (int q = 0; q < L::NPLANES; ++q) a.plane[q] = (unsigned char*)base + p.off_plane[q];
  DwArgs d{};
  int jW[4], jb[4];
  wide_dw_jobs(&d, jW, jb);
  d.cap = p.cap;
  d.rounds = a.rounds;
  for (int q = 0; q < L::NPLANES; ++q) d.plane[q] = a.plane[q];
  d.part = (float*)(base + p.off_part);
  d.err = a.err;
  // weight images for the CTA pairs (forward and transposed chunks, two
  // halves of WIMG_BYTES / 2 each, WREP copies)
  {
    size_t woff[MLP_MAX_LAYERS] = {};
    for (int l = 0; l < Cfg::NL; ++l) woff[l] = Cfg::W_off(l) / 2;
    tode_err e = build_images<Cfg>(r.f, img, IMG_CHUNKS2, Cfg::WREP, Cfg::WIMG_STRIDE, woff, st,
                                   L::HALF_BYTES);
    if (e == TODE_OK)
      e = build_images<Cfg>(r.f, timg, IMG_TCHUNKS2, Cfg::WREP, Cfg::WIMG_STRIDE, woff, st,
                            L::HALF_BYTES);
    if (e != TODE_OK) return e;
  }
  TODE_CUDA_TRY(cudaMemsetAsync(base, 0, 256, st));
  TODE_CUDA_TRY(cudaMemsetAsync(d.part, 0, (size_t)p.items * DW_PART_FLOATS * 4, st));
  // the hidden layers' biases, contiguous and aligned for vector loads (none: 0)
  TODE_CUDA_TRY(cudaMemsetAsync(base + p.off_bias, 0, (size_t)3 * Cfg::H * 4, st));
  for (int l = 0; l < 3; ++l)
    if (r.f->b[l])
      TODE_CUDA_TRY(cudaMemcpyAsync(base + p.off_bias + (size_t)l * Cfg::H * 4, r.f->b[l],
                                    (size_t)Cfg::H * 4, cudaMemcpyDeviceToDevice, st));
  // the queue: most accepted steps first, so the rows of a tile reverse
  // instances of similar length (stable: a fixed order every call)
  k_order_steps_stable<<<1, 1024, 0, st>>>(r.B, StepsBin{r.n_acc, r.status},
                                           (int32_t*)(base + p.off_order));
  TODE_CUDA_TRY(cudaGetLastError());
  {
    static std::atomic<uint64_t> d0{0}, d1{0};
    tode_err e = smem_optin((const void*)k_mlp_adjoint_wide<Cfg, Tab>, L::S_END, d0);
    if (e == TODE_OK) e = smem_optin((const void*)k_mlp_dw<Cfg>, DW_SMEM, d1);
    if (e != TODE_OK) return e;
  }
  // a slice's pairs all resident at once (one pair per two SMs the cluster
  // scheduler can place, times the slice multiplier)
  int grid = p.grid;
  {
    static std::atomic<int> pairs_cached{0};
    int pairs = pairs_cached.load();
    if (pairs <= 0) {
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(2);
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes = L::S_END;
      TODE_CUDA_TRY(cudaOccupancyMaxActiveClusters(&pairs, (const void*)k_mlp_adjoint_wide<Cfg, Tab>,
                                                   &cfg));
      if (pairs <= 0) return TODE_ECUDA;
      pairs_cached.store(pairs);
    }
    grid = std::min(grid, 2 * pairs * wide_slice_mult(r.o));
  }
  const int slice = grid * 64;
  for (int i0 = 0; i0 < r.B; i0 += slice) {
    a.i0 = i0;
    a.B = std::min(slice, r.B - i0);
    int cg = (a.B + 63) / 64;
    cg += cg & 1;  // CTA pairs: an odd tile count gets an idle partner
    k_mlp_adjoint_wide<Cfg, Tab><<<cg, 256, L::S_END, st>>>(a);
    TODE_CUDA_TRY(cudaGetLastError());
    d.chain_grid = cg;
    k_mlp_dw<Cfg><<<p.items, 128, DW_SMEM, st>>>(d);
    TODE_CUDA_TRY(cudaGetLastError());
  }
  DwReduceArgs ra{};
  ra.part = d.part;
  for (int j = 0; j <= d.njobs; ++j) ra.item0[j] = d.item0[j];
  for (int l = 0; l < 4; ++l) {
    ra.jW[l] = jW[l];
    ra.jb[l] = jb[l];
    ra.gW[l] = r.gW[l];
    ra.gb[l] = r.gb ? r.gb[l] : nullptr;
  }
  const long long total = 512LL * 65 + 512 + 2 * (512LL * 512 + 512) + 64LL * 512 + 64;
  k_mlp_dw_reduce<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(ra);
  TODE_CUDA_TRY(cudaGetLastError());
  return TODE_OK;
}

template <class Tab> static tode_err mlp_adjoint_tab(const AdjReq& r) {
  using Cfg = Cfg32s;
  using L = MlpAdjLayout<Cfg>;
  if (is_d64_h512(r.f)) {
    if (r.tape->stride != 1 || !r.tape->h_acc || !r.tape->y || !r.tape->t || !r.tape->y_stage)
      return TODE_EINVAL;
    if (!r.gW || !r.gW[0] || !r.gW[1] || !r.gW[2] || !r.gW[3]) return TODE_EINVAL;
    return mlp_wide_adjoint<Tab>(r);
  }
  if (!is_d32_h128(r.f)) return TODE_EUNSUPPORTED;
  if (r.tape->stride != 1 || !r.tape->h_acc || !r.tape->y || !r.tape->t || !r.tape->y_stage)
    return TODE_EINVAL;
  if (!r.gW || !r.gW[0] || !r.gW[1] || !r.gW[2]) return TODE_EINVAL;
  const cudaStream_t st = r.stream;
  const long long grid = std::min<long long>((r.B + 127) / 128, r.num_sms);
  MlpAdjArgs a{};
  a.B = r.B;
  a.K = r.K;
  a.t0 = r.t0;
  a.t1 = r.t1;
  a.te = r.te;
  a.n_acc = r.n_acc;
  a.status = r.status;
  a.slots = r.tape->slots;
  a.tp_y = (const float*)r.tape->y;
  a.tp_k1 = (const float*)r.tape->k1;
  a.tp_t = r.tape->t;
  a.tp_h = (const float*)r.tape->h_acc;
  a.tp_ys = (const float*)r.tape->y_stage;
  a.gye = (const float*)r.gye;
  a.gyf = (const float*)r.gyf;
  a.gy0 = (float*)r.gy0;
  for (int l = 0; l < MLP_MAX_LAYERS; ++l) a.bias[l] = l < 3 ? r.f->b[l] : nullptr;
  char* p = r.scratch;
  a.err = (int32_t*)(p + 128);
  p += align256(256);
  unsigned char* img = (unsigned char*)p;
  a.wimg = img;
  p += align256((size_t)Cfg::WIMG_BYTES);
  a.part = (float*)p;
  a.overflow = r.overflow;
  a.gts = (double*)r.gparam;  // MLP field: the time-translation sums, or NULL
  {
    size_t loff[MLP_MAX_LAYERS] = {};
    for (int l = 0; l < Cfg::NL; ++l) loff[l] = Cfg::W_off(l);
    const tode_err e = build_images<Cfg>(r.f, img, IMG_TILE, 1, Cfg::WIMG_STRIDE, loff, st);
    if (e != TODE_OK) return e;
  }
  TODE_CUDA_TRY(cudaMemsetAsync(r.scratch, 0, 256, st));
  {
    static std::atomic<uint64_t> done{0};
    const tode_err e = smem_optin((const void*)k_mlp_adjoint<Cfg, Tab>, L::S_END, done);
    if (e != TODE_OK) return e;
  }
  k_mlp_adjoint<Cfg, Tab><<<(int)grid, 256, L::S_END, st>>>(a);
  TODE_CUDA_TRY(cudaGetLastError());
  const int total = Cfg::H * (Cfg::D + 1) + Cfg::H + Cfg::H * Cfg::H + Cfg::H +
                    Cfg::D * Cfg::H + Cfg::D;
  k_mlp_grad_reduce<Cfg><<<(total + 255) / 256, 256, 0, st>>>(
      a.part, (int)grid, r.gW[0], r.gb ? r.gb[0] : nullptr, r.gW[1], r.gb ? r.gb[1] : nullptr,
      r.gW[2], r.gb ? r.gb[2] : nullptr);
  TODE_CUDA_TRY(cudaGetLastError());
  return TODE_OK;
}

tode_err mlp_adjoint(const AdjReq& r) {
  return r.o->method == TODE_TSIT5 ? mlp_adjoint_tab<TS5>(r) : mlp_adjoint_tab<DP5>(r);
}


// ---------------------------------------------------------------- joint continuous adjoint
// Workspace: control block, weight image, the rows' state and candidate,
// the stage slots, the CTAs' parameter slots, abar and its companions.
struct JadjWs {
  JadjCtl* ctl;
  int32_t* err;
  unsigned char* img;
  float *y, *a, *yc, *ac, *kst, *gpart;
  double *epart, *th, *thc, *kth1, *fsum, *dpart;
  size_t bytes;
};
static JadjWs jadj_carve(char* base, int B) {
  using L = MlpAdjLayout<Cfg32s>;
  constexpr int D = 32, P = L::P_FLOATS;
  const size_t BD = (size_t)B * D;
  const int grid1 = (B + 127) / 128, grid2 = (P + 255) / 256;
  JadjWs w{};
  size_t o = 0;
  auto take = [&](size_t n) {
    char* q = base ? base + o : nullptr;
    o += align256(n);
    return q;
  };
  char* c = take(256);
  w.ctl = (JadjCtl*)c;
  w.err = c ? (int32_t*)(c + 128) : nullptr;
  w.img = (unsigned char*)take((size_t)Cfg32s::WIMG_BYTES);
  w.y = (float*)take(BD * 4);
  w.a = (float*)take(BD * 4);
  w.yc = (float*)take(BD * 4);
  w.ac = (float*)take(BD * 4);
  w.kst = (float*)take(7 * 2 * BD * 4);
  w.gpart = (float*)take((size_t)grid1 * 3 * P * 4);
  w.epart = (double*)take((size_t)grid1 * 2 * 8);
  w.th = (double*)take((size_t)P * 8);
  w.thc = (double*)take((size_t)P * 8);
  w.kth1 = (double*)take((size_t)P * 8);
  w.fsum = (double*)take((size_t)P * 8);
  w.dpart = (double*)take((size_t)grid2 * 2 * 8);
  w.bytes = o;
  return w;
}
static_assert(sizeof(JadjCtl) <= 128, "joint adjoint control block");

size_t mlp_jadj_workspace_bytes(const tode_field_desc* f) {
  if (!is_d32_h128(f)) return 0;
  return jadj_carve(nullptr, f->B).bytes;
}

template <class Tb> static tode_err mlp_joint_adjoint_tab(const JadjReq& r) {
  using Cfg = Cfg32s;
  using L = MlpAdjLayout<Cfg>;
  constexpr int D = 32, P = L::P_FLOATS;
  if (!is_d32_h128(r.f)) return TODE_EUNSUPPORTED;
  const cudaStream_t st = r.stream;
  const int B = r.B, K = r.K;
  const int grid1 = (B + 127) / 128, grid2 = (P + 255) / 256;
  const JadjWs w = jadj_carve(r.ws, B);
  JadjArgs a{};
  a.B = B;
  a.wimg = w.img;
  for (int l = 0; l < 3; ++l) a.bias[l] = r.f->b[l];
  a.y = w.y;
  a.a = w.a;
  a.yc = w.yc;
  a.ac = w.ac;
  a.kst = w.kst;
  a.gpart = w.gpart;
  a.epart = w.epart;
  a.th = w.th;
  a.thc = w.thc;
  a.kth1 = w.kth1;
  a.fsum = w.fsum;
  a.dpart = w.dpart;
  a.ctl = w.ctl;
  a.err = w.err;
  const tode_options* o = r.o;
  a.rtol = o->rtol;
  a.atol = o->atol;
  a.safety = o->safety;
  a.fac_min = o->fac_min;
  a.fac_max = o->fac_max;
  a.beta1 = o->beta1;
  a.beta2 = o->beta2;
  a.beta3 = o->beta3;
  a.max_steps = o->max_steps;
  // the norm's components: y and a of every row, the network's parameters
  a.nnorm = 2.0 * B * D + (double)(Cfg::H * (D + 1) + Cfg::H + Cfg::H * Cfg::H + Cfg::H +
                                   D * Cfg::H + D);
  {
    size_t loff[MLP_MAX_LAYERS] = {};
    for (int l = 0; l < Cfg::NL; ++l) loff[l] = Cfg::W_off(l);
    const tode_err e = build_images<Cfg>(r.f, w.img, IMG_TILE, 1, Cfg::WIMG_STRIDE, loff, st);
    if (e != TODE_OK) return e;
  }
  {
    static std::atomic<uint64_t> done{0};
    const tode_err e = smem_optin((const void*)k_mlp_jadj<Cfg, Tb>, L::S_END, done);
    if (e != TODE_OK) return e;
  }
  const size_t BD = (size_t)B * D;
  TODE_CUDA_TRY(cudaMemsetAsync(w.ctl, 0, 256, st));
  TODE_CUDA_TRY(cudaMemsetAsync(w.th, 0, (size_t)P * 8, st));
  TODE_CUDA_TRY(cudaMemcpyAsync(w.y, r.y1, BD * 4, cudaMemcpyDeviceToDevice, st));
  if (r.gyf)
    TODE_CUDA_TRY(cudaMemcpyAsync(w.a, r.gyf, BD * 4, cudaMemcpyDeviceToDevice, st));
  else
    TODE_CUDA_TRY(cudaMemsetAsync(w.a, 0, BD * 4, st));
  const unsigned jb = (unsigned)((BD + 255) / 256);
  auto jump = [&](int q) -> tode_err {
    if (r.gye) {
      k_mlp_jadj_jump<<<jb, 256, 0, st>>>(w.a, r.gye, B, K, D, q);
      TODE_CUDA_TRY(cudaGetLastError());
    }
    return TODE_OK;
  };
  auto pair = [&](int mode) -> tode_err {
    k_mlp_jadj<Cfg, Tb><<<grid1, 256, L::S_END, st>>>(a, mode);
    TODE_CUDA_TRY(cudaGetLastError());
    k_mlp_jadj_decide<Cfg, Tb><<<grid2, 256, 0, st>>>(a, mode, grid1);
    TODE_CUDA_TRY(cudaGetLastError());
    return TODE_OK;
  };
  // cotangents of the points at t1 start a
  int k = K - 1;
  while (k >= 0 && r.te[k] == r.t1) {
    const tode_err e = jump(k--);
    if (e != TODE_OK) return e;
  }
  int32_t n_acc = 0, n_rej = 0, n_fe = 0, status = ST_SUCCESS;
  double start = r.t1;
  const int poll = 4;
  while (true) {
    const double end = (k >= 0 && r.te[k] > r.t0) ? r.te[k] : r.t0;
    if (end != start) {
      JadjCtl h{};
      h.t = start;
      h.t_end = end;
      h.err_prev = h.err_prev2 = 1.0;
      h.status = ST_RUNNING;
      TODE_CUDA_TRY(cudaMemcpyAsync(w.ctl, &h, sizeof(h), cudaMemcpyHostToDevice, st));
      TODE_CUDA_TRY(cudaStreamSynchronize(st));  // h is reused below
      tode_err e = pair(JA_EVAL);
      if (e == TODE_OK) e = pair(JA_PROBE);
      if (e != TODE_OK) return e;
      long long launched = 0;
      const long long limit = (long long)o->max_steps + 2LL * poll + 2;
      while (true) {
        for (int q = 0; q < poll; ++q) {
          e = pair(JA_STEP);
          if (e != TODE_OK) return e;
        }
        launched += poll;
        TODE_CUDA_TRY(cudaMemcpyAsync(&h, w.ctl, sizeof(h), cudaMemcpyDeviceToHost, st));
        TODE_CUDA_TRY(cudaStreamSynchronize(st));
        if (h.status != ST_RUNNING) break;
        // one attempt per launch pair, so max_steps bounds the loop
        if (launched > limit) return TODE_ETIMEOUT;
      }
      k_mlp_jadj_commit<<<(unsigned)((std::max<size_t>(BD, P) + 255) / 256), 256, 0, st>>>(a, P);
      TODE_CUDA_TRY(cudaGetLastError());
      n_acc += h.n_acc;
      n_rej += h.n_rej;
      n_fe += h.n_fe;
      if (h.status != ST_SUCCESS) {
        status = h.status;
        break;
      }
    }
    while (k >= 0 && r.te[k] == end) {
      const tode_err e = jump(k--);
      if (e != TODE_OK) return e;
    }
    start = end;
    if (end == r.t0) break;
  }
  TODE_CUDA_TRY(cudaMemcpyAsync(r.gy0, w.a, BD * 4, cudaMemcpyDeviceToDevice, st));
  if (r.y0) TODE_CUDA_TRY(cudaMemcpyAsync(r.y0, w.y, BD * 4, cudaMemcpyDeviceToDevice, st));
  const int total = Cfg::H * (D + 1) + Cfg::H + Cfg::H * Cfg::H + Cfg::H + D * Cfg::H + D;
  k_mlp_jadj_out<Cfg><<<(total + 255) / 256, 256, 0, st>>>(
      w.th, r.gW[0], r.gb ? r.gb[0] : nullptr, r.gW[1], r.gb ? r.gb[1] : nullptr, r.gW[2],
      r.gb ? r.gb[2] : nullptr);
  TODE_CUDA_TRY(cudaGetLastError());
  int32_t flag = 0;
  TODE_CUDA_TRY(cudaMemcpyAsync(&flag, w.err, 4, cudaMemcpyDeviceToHost, st));
  TODE_CUDA_TRY(cudaStreamSynchronize(st));
  r.stats[0] = n_acc;
  r.stats[1] = n_rej;
  r.stats[2] = n_fe;
  r.stats[3] = status;
  return flag ? TODE_ETIMEOUT : TODE_OK;
}

// the pair of the joint continuous adjoint's steps (dopri5 or tsit5)
tode_err mlp_joint_adjoint(const JadjReq& r) {
  return r.o->method == TODE_TSIT5 ? mlp_joint_adjoint_tab<TS5>(r) : mlp_joint_adjoint_tab<DP5>(r);
}

}  // namespace tode
