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

#include <cuda_bf16.h>

#include <cublas_v2.h>

#include <algorithm>
#include <atomic>
#include <mutex>

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

// MlpBigCfg: the wide network (H = 512; 1.2 MB of BF16 weights).  Split
// activations of 128 rows would need 256 KB, so a tile has 64 rows (M = 64
// MMAs: row m of the tile lands in tensor-memory lane (m/16)*32 + m%16), four
// threads per row.  The weights are streamed through shared memory in
// 16-column K chunks (a 4-stage ring of bulk copies on mbarriers) every round.
template <int D_, int H_, int NL_> struct MlpBigCfg {
  static constexpr int D = D_, H = H_, NL = NL_;
  static constexpr bool SPLIT = true, STREAM = true, STACKED = false;
  static constexpr int ROWS = 64, TPR = 4, NT = 256;
  static constexpr int K0 = ((D + 1 + 15) / 16) * 16;
  static constexpr int C = D / TPR;
  static constexpr int HC = H / TPR;
  static constexpr int TMEM_COLS = 512;
  static constexpr int ACC_COL = 0, OUT_COL = 0;  // the output reuses the hidden accumulator
  static_assert(C == 16 && H == 512 && D <= 256 && HC % 16 == 0, "shape");
  // warp w reads lane quarter w%4 (rows 16*(w%4) .. +15 in lanes 0-15); lanes
  // 0-15 and 16-31 of the warp take different column ranges of the same rows
  __device__ static int row_of(int tid) { return 16 * ((tid >> 5) & 3) + (tid & 15); }
  __device__ static int sub_of(int tid) { return 2 * (tid >> 7) + ((tid >> 4) & 1); }
  __device__ static void hid_ld(uint32_t tbase, int tid, int c, float (&v)[16]) {
    const uint32_t lanes = (uint32_t)(32 * ((tid >> 5) & 3)) << 16;
    tc::tmem_ld16x2<HC>(tbase + lanes + ACC_COL + (tid >> 7) * 2 * HC + c, v);
  }
  __device__ static void out_ld(uint32_t tbase, int tid, float (&v)[C]) {
    const uint32_t lanes = (uint32_t)(32 * ((tid >> 5) & 3)) << 16;
    tc::tmem_ld16x2<C>(tbase + lanes + OUT_COL + (tid >> 7) * 2 * C, v);
  }
  // layer l: N_l x K_l, image = K chunks of [N_l][16] core-matrix tiles
  __host__ __device__ static constexpr int N_of(int l) { return l == NL - 1 ? D : H; }
  __host__ __device__ static constexpr int K_of(int l) { return l == 0 ? K0 : H; }
  __host__ __device__ static constexpr int W_bytes(int l) { return N_of(l) * K_of(l) * 2; }
  __host__ __device__ static constexpr int W_off(int l) {
    int o = 0;
    for (int j = 0; j < l; ++j) o += W_bytes(j);
    return o;
  }
  static constexpr int WIMG_BYTES = W_off(NL);
  // every CTA streams the same chunks at about the same time; CTAs read one
  // of WREP copies of the image so the requests spread over the L2 slices
  static constexpr int WREP = 16, WIMG_STRIDE = ((WIMG_BYTES + 255) / 256) * 256;
  static constexpr int BIAS_FLOATS = (NL - 1) * H + D;
  static constexpr int KC = 16, NS = 4;                       // chunk K, ring stages
  static constexpr int STAGE_BYTES = H * KC * 2;             // the largest chunk
  __host__ __device__ static constexpr int chunks(int l) { return K_of(l) / KC; }
  __host__ __device__ static constexpr int chunks_per_round() {
    int n = 0;
    for (int l = 0; l < NL; ++l) n += chunks(l);
    return n;
  }
  // global chunk index -> image offset and size
  __device__ static void chunk_src(uint32_t g, int& off, int& bytes) {
    int c = (int)(g % (uint32_t)chunks_per_round());
    int l = 0;
    while (c >= chunks(l)) c -= chunks(l++);
    bytes = N_of(l) * KC * 2;
    off = W_off(l) + c * bytes;
  }
  // shared-memory carve (bytes)
  static constexpr int S_XH = 0;
  static constexpr int S_XL = S_XH + ROWS * K0 * 2;
  static constexpr int S_HH = S_XL + ROWS * K0 * 2;
  static constexpr int S_HL = S_HH + ROWS * H * 2;
  static constexpr int S_W = S_HL + ROWS * H * 2;  // the chunk ring
  static constexpr int S_BIAS = S_W + NS * STAGE_BYTES;
  static constexpr int S_RED = S_BIAS + BIAS_FLOATS * 4;
  static constexpr int S_FIN = S_RED + TPR * ROWS * 2 * 4;
  static constexpr int S_NXT = S_FIN + TPR * ROWS * 4;
  static constexpr bool KSMEM = false;  // no room: the stage derivatives stay in the thread
  static constexpr int S_K = 0;
  static constexpr int S_END = S_NXT + ROWS * 4;
  static_assert(S_END <= 232448 - 1024, "shared memory");
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
  static constexpr int WREP = 16, WIMG_STRIDE = ((WIMG_BYTES + 255) / 256) * 256;
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

// tanh_acc of two values, the additions packed in pairs (FP32x2 operations
// round each lane as the scalar ones: the same results, half the additions).
__device__ __forceinline__ float2 tanh_acc2(float2 z) {
  const float2 e = make_float2(__expf(-2.0f * fabsf(z.x)), __expf(-2.0f * fabsf(z.y)));
  const float2 num = __ffma2_rn(e, make_float2(-1.0f, -1.0f), make_float2(1.0f, 1.0f));  // 1 - e
  const float2 den = __fadd2_rn(e, make_float2(1.0f, 1.0f));                           // 1 + e
  return make_float2(copysignf(__fdividef(num.x, den.x), z.x),
                     copysignf(__fdividef(num.y, den.y), z.y));
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
// Per-row solver state (identical scalars in both threads of the row).
struct MlpRow {
  int inst, phase, cursor, status, flags, n_acc, n_rej;
  double t, t0, t1;
  float h, h0h, err_prev, err_prev2, rtol, atol, rem, hmin;
  bool last;
};

// The solver body shared by the fused form and the plain form.  Fused: a
// persistent grid, each row takes instances from a global counter and
// integrates them to their end.  Plain: tile c of ROWS instances belongs to
// CTA c mod grid; the initialising launch runs the starting-step rounds, every
// later launch one attempt (six stage rounds) per running instance, with the
// state parked in the workspace in between.
template <class Cfg, int MODE>
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
    } else if constexpr (Cfg::STREAM) {
      static_assert(Cfg::NS <= 4, "ring barriers");
      for (int b = 0; b < Cfg::NS; ++b) {  // the ring starts with chunks 0 .. NS-1
        int off, bytes;
        Cfg::chunk_src((uint32_t)b, off, bytes);
        tc::mbar_expect_tx(&mbar_full[b], (uint32_t)bytes);
        tc::bulk_g2s(sW + b * Cfg::STAGE_BYTES, wimg + off, (uint32_t)bytes, &mbar_full[b]);
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
    s.t0 = a.t0[i];
    s.t1 = a.t1[i];
    s.t = s.t0;
    s.rtol = (float)(a.rtol_b ? a.rtol_b[i] : a.rtol);
    s.atol = (float)(a.atol_b ? a.atol_b[i] : a.atol);
    s.n_acc = s.n_rej = 0;
    s.cursor = 0;
    s.flags = 0;
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
    s.t0 = a.t0[i];
    s.t1 = a.t1[i];
    s.t = a.wt[i];
    s.rtol = (float)(a.rtol_b ? a.rtol_b[i] : a.rtol);
    s.atol = (float)(a.atol_b ? a.atol_b[i] : a.atol);
    s.n_acc = a.n_acc[i];
    s.n_rej = a.n_rej[i];
    s.cursor = a.wcur[i];
    s.flags = a.wfl[i];
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
        const int i = sNxt[row];
        if (i >= a.B) {
          s.phase = PH_IDLE;
          s.inst = -1;
        } else {
          start_instance(i);
        }
      }
    } else if (need_load) {
      need_load = false;
      const int i = tile * ROWS + row;
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
      for (int r = 0; r < C; ++r) Y[r] = madd(s.h0h, k1[r], y[r]);
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
      // Y_s = y + h sum_j a_sj k_j, the terms in the order j = 1, 2, ...
      // (the stage-7 row is b, which has no k2 term)
      float acc[16];
      const float a1 = dp_a(stage, 1);
#pragma unroll
      for (int r = 0; r < C; ++r) acc[r] = a1 * k1[r];
      for (int j = 2; j < stage && j <= 6; ++j) {
        if (stage == 7 && j == 2) continue;
        float kj[16];
        kget(j, kj);
        const float c = dp_a(stage, j);
#pragma unroll
        for (int r = 0; r < C; ++r) acc[r] = madd(c, kj[r], acc[r]);
      }
#pragma unroll
      for (int r = 0; r < C; ++r) Y[r] = (stage == 7) ? y[r] + h * acc[r] : madd(h, acc[r], y[r]);
      switch (stage) {
        case 2: cs = Cc::c2; break;
        case 3: cs = Cc::c3; break;
        case 4: cs = Cc::c4; break;
        case 5: cs = Cc::c5; break;
        default: cs = 1.0; break;
      }
      tin = (float)(s.t + cs * (double)h);
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
        } else if constexpr (Cfg::STREAM) {
          // K chunk c of layer l sits in ring slot g % NS; after issuing chunk
          // g, the slot of chunk g-1 is refilled with chunk g-1+NS once its
          // MMAs are done
          constexpr int NS = Cfg::NS;
          const int nh = Nl > 256 ? Nl / 256 : 1, nw = Nl > 256 ? 256 : Nl;
          const uint32_t idesc = tc::idesc_bf16_f32(ROWS, nw);
          bool ok = true;
          for (int c = 0; c < Kl / Cfg::KC && ok; ++c, ++g_chunk) {
            const int b = (int)(g_chunk % NS);
            ok = tc::mbar_wait(&mbar_full[b], (g_chunk / NS) & 1u);
            if (!ok) break;
            const uint32_t wb = tc::smem_u32(sW + b * Cfg::STAGE_BYTES);
            const uint64_t dh = tc::smem_desc(ah + c * 256, 128, Kl * 16);
            const uint64_t dl = tc::smem_desc(al + c * 256, 128, Kl * 16);
            for (int j = 0; j < nh; ++j) {
              const uint64_t db = tc::smem_desc(wb + j * (256 / 8) * 256, 128, 256);
              tc::mma_bf16(tbase + dcol + 256 * j, dh, db, idesc, c > 0);
              tc::mma_bf16(tbase + dcol + 256 * j, dl, db, idesc, true);
            }
            tc::mma_commit(&mbar_empty[b]);
            if (g_chunk >= 1) {
              const uint32_t gp = g_chunk - 1;
              const int pb = (int)(gp % NS);
              ok = tc::mbar_wait(&mbar_empty[pb], (gp / NS) & 1u);
              if (!ok) break;
              int off, bytes;
              Cfg::chunk_src(gp + NS, off, bytes);
              tc::mbar_expect_tx(&mbar_full[pb], (uint32_t)bytes);
              tc::bulk_g2s(sW + pb * Cfg::STAGE_BYTES, wimg + off, (uint32_t)bytes,
                           &mbar_full[pb]);
            }
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

    // ---- consume: partial sums of this thread's components
    float p0 = 0.0f, p1 = 0.0f;
    int fin = 1;
    float inc[16];
    float k3[16], k4[16], k5[16], k6[16];  // stage 7: the attempt's k3..k6
    if (s.phase == PH_INIT0) {
#pragma unroll
      for (int r = 0; r < C; ++r) {
        k1[r] = f[r];
        const float sc = madd(s.rtol, fabsf(y[r]), s.atol);
        const float q0 = y[r] / sc, q1 = f[r] / sc;
        p0 = madd(q0, q0, p0);
        p1 = madd(q1, q1, p1);
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
        kget(3, k3);
        kget(4, k4);
        kget(5, k5);
        kget(6, k6);
#pragma unroll
        for (int r = 0; r < C; ++r) {
          float acc = float(Cc::b1) * k1[r];
          acc = madd(float(Cc::b3), k3[r], acc);
          acc = madd(float(Cc::b4), k4[r], acc);
          acc = madd(float(Cc::b5), k5[r], acc);
          acc = madd(float(Cc::b6), k6[r], acc);
          inc[r] = s.h * acc;
          const float y1 = y[r] + inc[r];
          float e = float(Cc::e1) * k1[r];
          e = madd(float(Cc::e3), k3[r], e);
          e = madd(float(Cc::e4), k4[r], e);
          e = madd(float(Cc::e5), k5[r], e);
          e = madd(float(Cc::e6), k6[r], e);
          e = madd(float(Cc::e7), f[r], e);
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
    if (s.phase == PH_INIT0) {
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
              float acc = w[0] * k1[r];
              acc = madd(w[2], k3[r], acc);
              acc = madd(w[3], k4[r], acc);
              acc = madd(w[4], k5[r], acc);
              acc = madd(w[5], k6[r], acc);
              acc = madd(w[6], f[r], acc);
              dst[r] = y[r] + madd(h, acc, ylo[r]);
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
      } else {
        if (s.status != ST_SUCCESS) {  // points the failed instance never reached
          float* ye = a.ye + (size_t)i * a.K * D + coff;
          for (int q = s.cursor; q < a.K; ++q)
#pragma unroll
            for (int r = 0; r < C; ++r) ye[(size_t)q * D + r] = nan_(0.0f);
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
  } else if constexpr (Cfg::STREAM) {
    if (tid == 0) {
      // the ring's copies still in flight land before the CTA exits
      const uint32_t first = g_chunk, last = g_chunk == 0 ? Cfg::NS - 1 : g_chunk + Cfg::NS - 2;
      for (uint32_t x = first; x <= last; ++x)
        if (!tc::mbar_wait(&mbar_full[x % Cfg::NS], (x / Cfg::NS) & 1u)) atomicExch(&abort_s, 1);
    }
  }
  if (abort_s && tid == 0) atomicExch(a.err, 1);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, Cfg::TMEM_COLS);
}

template <class Cfg>
__global__ void __launch_bounds__(256, 1) k_mlp_fused(MlpArgs a) {
  mlp_solver<Cfg, MLP_FUSED>(a);
}
template <class Cfg>
__global__ void __launch_bounds__(256, 1) k_mlp_plain_init(MlpArgs a) {
  mlp_solver<Cfg, MLP_PLAIN_INIT>(a);
}
template <class Cfg>
__global__ void __launch_bounds__(256, 1) k_mlp_plain_step(MlpArgs a) {
  mlp_solver<Cfg, MLP_PLAIN_STEP>(a);
}

// The BF16 weights W_l [N_l][K_in,l] (row-major) as core-matrix images with
// K padded to K_l, for all layers and all copies in one launch.  Layouts:
//   IMG_TILE    one [N_l][K_l] tile per layer (weights resident in shared memory)
//   IMG_CHUNKS  K_l/16 consecutive [N_l][16] tiles (the streamed K chunks)
//   IMG_TCHUNKS N_l/16 consecutive MN-major [16][K_l] tiles: W_l^T in K chunks
//               along the layer's outputs (the transposed products)
enum : int { IMG_TILE = 0, IMG_CHUNKS = 1, IMG_TCHUNKS = 2 };
struct ImageJob {
  const uint16_t* W[MLP_MAX_LAYERS];
  int N[MLP_MAX_LAYERS], Kin[MLP_MAX_LAYERS], Kp[MLP_MAX_LAYERS];
  size_t off[MLP_MAX_LAYERS];      // layer offset inside one copy
  long long start[MLP_MAX_LAYERS + 1];  // element ranges of the layers
  int nl, reps, mode;
  size_t stride;  // bytes between copies
};
__global__ void k_mlp_images(ImageJob j, unsigned char* img) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= j.start[j.nl]) return;
  int l = 0;
  while (e >= j.start[l + 1]) ++l;
  const long long x = e - j.start[l];
  const int Kp = j.Kp[l], N = j.N[l];
  const int n = (int)(x / Kp), k = (int)(x % Kp);
  const uint16_t v = k < j.Kin[l] ? j.W[l][(size_t)n * j.Kin[l] + k] : (uint16_t)0;
  uint32_t off;
  if (j.mode == IMG_TILE) off = tc::cm_offset(n, k, Kp);
  else if (j.mode == IMG_CHUNKS) off = (uint32_t)(k / 16) * (uint32_t)N * 32u + tc::cm_offset(n, k % 16, 16);
  else off = (uint32_t)(n / 16) * 16u * (uint32_t)Kp * 2u + tc::cm_offset(n % 16, k, Kp);
  for (int r = 0; r < j.reps; ++r)
    *reinterpret_cast<uint16_t*>(img + (size_t)r * j.stride + j.off[l] + off) = v;
}

// Host side: the image job of a network config (W_off / T_off give the
// layer offsets of the chosen layout).
template <class Cfg>
static tode_err build_images(const tode_field_desc* f, unsigned char* img, int mode, int reps,
                             size_t stride, const size_t (&layer_off)[MLP_MAX_LAYERS],
                             cudaStream_t st) {
  ImageJob j{};
  j.nl = Cfg::NL;
  j.reps = reps;
  j.mode = mode;
  j.stride = stride;
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
};

constexpr int ADJ_ROUNDS = 7;  // one reverse round per stage, 7..1

__device__ __forceinline__ double dp_c(int s) {
  using C = DP5;
  return s == 2 ? C::c2 : s == 3 ? C::c3 : s == 4 ? C::c4 : s == 5 ? C::c5 : s >= 6 ? 1.0 : 0.0;
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

template <class Cfg>
__global__ void __launch_bounds__(256, 1) k_mlp_adjoint(MlpAdjArgs a) {
  using L = MlpAdjLayout<Cfg>;
  using Cc = DP5;
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
    tnext = (n == N - 1) ? a.t1[i] : tn + (double)h;
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
          const long long k0 = tkey(a.t0[i]);
          for (; q >= 0; --q)
            if (tkey(a.te[(size_t)i * a.K + q]) == k0)
#pragma unroll
              for (int r = 0; r < C; ++r) yb[r] += a.gye[((size_t)i * a.K + q) * D + coff + r];
        }
#pragma unroll
        for (int r = 0; r < C; ++r) a.gy0[(size_t)i * D + coff + r] = bad ? nan_(0.0f) : yb[r];
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
      if (!bad && N > a.slots) {
        bad = true;
        if (half == 0) atomicExch(a.overflow, 1);
      }
#pragma unroll
      for (int r = 0; r < C; ++r) yb[r] = a.gyf ? a.gyf[(size_t)i * D + coff + r] : 0.0f;
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
  const float bw[7] = {float(Cc::b1), 0.0f, float(Cc::b3), float(Cc::b4), float(Cc::b5),
                       float(Cc::b6), 0.0f};
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
        const double tq = a.te[(size_t)i * a.K + q];
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
            dense_weights<float>(float(tq - tn) / h, w);
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
      tin = (float)(tn + dp_c(s) * (double)h);
      pick7(kb, s - 1, d3);
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
      for (int r = 0; r < C; ++r) db3[r] += kbs[r];
#pragma unroll
      for (int j = 0; j < 6; ++j) {  // kbar_j += h a_{s,j} g  (j < s)
        if (j + 1 >= s) continue;
        const float c = h * dp_a(s, j + 1);
#pragma unroll
        for (int r = 0; r < C; ++r) kb[j][r] = madd(c, fg[r], kb[j][r]);
      }
#pragma unroll
      for (int r = 0; r < C; ++r) yb[r] += fg[r];
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
// 512; App. A).  Same schedule as k_mlp_adjoint -- rows reverse their own
// instances, 7 lockstep rounds per accepted step, stage inputs from the tape
// -- on 64-row tiles with the weights streamed through a chunk ring.  The reverse rounds need the
// transposed weights too (W_l^T, K chunks along the layer's outputs).
//
// The weight gradients do not fit in tensor memory (two 512 x 512 layers),
// so every reverse round writes the rows of its layer inputs (X, h1, h2, h3)
// and of its pre-activation cotangents (delta1, delta2, delta3, kbar), as
// BF16 hi + lo, to a staging area; dW_l = delta_l^T act_l and the bias sums
// are then plain GEMMs over the staged rows (mlp_wide_dw).
// ======================================================================
template <class Cfg> struct WideAdjLayout {
  static constexpr int D = Cfg::D, H = Cfg::H, K0 = Cfg::K0, ROWS = Cfg::ROWS;
  static_assert(Cfg::NL == 4 && D == 64 && H == 512 && K0 == 80 && ROWS == 64, "network");
  static constexpr int NS = 3;                         // ring stages
  static constexpr int STAGE_BYTES = 16 * H * 2;      // the largest chunk (16 x 512)
  static constexpr int S_XH = 0;
  static constexpr int S_XL = S_XH + ROWS * K0 * 2;
  static constexpr int S_HH = S_XL + ROWS * K0 * 2;   // the hidden / delta tile
  static constexpr int S_HL = S_HH + ROWS * H * 2;
  static constexpr int S_KH = S_HL + ROWS * H * 2;    // kbar tile
  static constexpr int S_KL = S_KH + ROWS * D * 2;
  static constexpr int S_W = S_KL + ROWS * D * 2;     // chunk ring
  static constexpr int S_BIAS = S_W + NS * STAGE_BYTES;
  static constexpr int S_END = S_BIAS + Cfg::BIAS_FLOATS * 4;
  static_assert(S_END <= 232448 - 1024, "shared memory");
  // transposed image: layer l, chunk c = outputs [16c, 16c+16) as an MN-major
  // [16][IN_l] core-matrix tile
  __host__ __device__ static constexpr int IN_of(int l) { return Cfg::K_of(l); }
  __host__ __device__ static constexpr int T_bytes(int l) { return Cfg::N_of(l) * IN_of(l) * 2; }
  __host__ __device__ static constexpr int T_off(int l) {
    int o = 0;
    for (int j = 0; j < l; ++j) o += T_bytes(j);
    return o;
  }
  static constexpr int TIMG_BYTES = T_off(Cfg::NL);
  static constexpr int TIMG_STRIDE = ((TIMG_BYTES + 255) / 256) * 256;
  // chunk schedule of a reverse round: forward layers 0..2, then the
  // transposed layers 3, 2, 1, 0
  static constexpr int REV_CHUNKS = 5 + 32 + 32 + 4 + 32 + 32 + 32;
  // global chunk index -> (transposed?, layer, chunk) -> image offset, bytes
  __device__ static void chunk_src(uint32_t g, bool& tr, int& off, int& bytes) {
    int p = (int)(g % (uint32_t)REV_CHUNKS);
    const int cnt[7] = {5, 32, 32, 4, 32, 32, 32};
    const int lay[7] = {0, 1, 2, 3, 2, 1, 0};
    int k = 0;
    while (p >= cnt[k]) p -= cnt[k++];
    const int l = lay[k];
    if (k < 3) {
      tr = false;
      bytes = Cfg::N_of(l) * 32;
      off = Cfg::W_off(l) + p * bytes;
    } else {
      tr = true;
      bytes = 16 * IN_of(l) * 2;
      off = T_off(l) + p * bytes;
    }
  }
};

struct WideAdjArgs {
  int i0, B, K;  // the slice: instances i0 .. i0+B-1 of the batch
  const double* t0;
  const double* t1;
  const double* te;
  const int32_t* n_acc;
  const int32_t* status;
  int slots, Btot;
  const float* tp_y;
  const float* tp_k1;
  const double* tp_t;
  const float* tp_h;
  const float* gye;
  const float* gyf;
  float* gy0;
  const unsigned char* wimg;  // forward chunk image (copies WIMG_STRIDE apart)
  const unsigned char* timg;  // transposed chunk image (copies TIMG_STRIDE apart)
  const float* bias[MLP_MAX_LAYERS];
  // staging: rows (c*cap + round)*64 + row; hi and lo planes
  uint16_t* sa[4][2];  // X [80], h1, h2, h3 [512]
  uint16_t* sg[4][2];  // delta1, delta2, delta3 [512], kbar [64]
  int cap;             // reverse rounds per CTA
  const float* tp_ys;  // [Btot][slots][6][D]: Y_2..Y_7
  int32_t* overflow;
  int32_t* err;
};

// Stores 16 values of a row as BF16 hi / lo into two row-major planes.
__device__ __forceinline__ void stage_row16(uint16_t* hp, uint16_t* lp, size_t off,
                                            const float (&v)[16]) {
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float a0 = v[c * 8 + 2 * j], b0 = v[c * 8 + 2 * j + 1];
      const __nv_bfloat162 h2 = __floats2bfloat162_rn(a0, b0);
      const __nv_bfloat162 l2 = __floats2bfloat162_rn(a0 - __low2float(h2), b0 - __high2float(h2));
      hw[j] = *reinterpret_cast<const uint32_t*>(&h2);
      lw[j] = *reinterpret_cast<const uint32_t*>(&l2);
    }
    *reinterpret_cast<uint4*>(hp + off + 8 * c) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(lp + off + 8 * c) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
}
// 16 values hi + lo of a staged row, as floats
__device__ __forceinline__ void unstage_row16(const uint16_t* hp, const uint16_t* lp, size_t off,
                                              float (&v)[16]) {
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const uint4 h = *reinterpret_cast<const uint4*>(hp + off + 8 * c);
    const uint4 l = *reinterpret_cast<const uint4*>(lp + off + 8 * c);
    const uint32_t hw[4] = {h.x, h.y, h.z, h.w}, lw[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&hw[j]);
      const __nv_bfloat162 l2 = *reinterpret_cast<const __nv_bfloat162*>(&lw[j]);
      v[c * 8 + 2 * j] = __low2float(h2) + __low2float(l2);
      v[c * 8 + 2 * j + 1] = __high2float(h2) + __high2float(l2);
    }
  }
}

template <class Cfg>
__global__ void __launch_bounds__(256, 1) k_mlp_adjoint_wide(WideAdjArgs a) {
  using L = WideAdjLayout<Cfg>;
  using Cc = DP5;
  constexpr int D = Cfg::D, H = Cfg::H, K0 = Cfg::K0, C = Cfg::C, HC = Cfg::HC, ROWS = 64;
  constexpr int NS = L::NS;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar_mma, mbar_full[NS], mbar_empty[NS];
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  unsigned char* sXh = sm + L::S_XH;
  unsigned char* sXl = sm + L::S_XL;
  unsigned char* sHh = sm + L::S_HH;
  unsigned char* sHl = sm + L::S_HL;
  unsigned char* sKh = sm + L::S_KH;
  unsigned char* sKl = sm + L::S_KL;
  unsigned char* sW = sm + L::S_W;
  float* sBias = reinterpret_cast<float*>(sm + L::S_BIAS);

  const int tid = threadIdx.x;
  const int row = Cfg::row_of(tid), sub = Cfg::sub_of(tid);
  const int coff = sub * C;
  const int grid = gridDim.x;
  const unsigned char* wimg = a.wimg + (size_t)(blockIdx.x % Cfg::WREP) * Cfg::WIMG_STRIDE;
  const unsigned char* timg = a.timg + (size_t)(blockIdx.x % Cfg::WREP) * L::TIMG_STRIDE;
  uint32_t g_chunk = 0;

  if (tid == 0) {
    tc::mbar_init(&mbar_mma, 1);
    for (int b = 0; b < NS; ++b) {
      tc::mbar_init(&mbar_full[b], 1);
      tc::mbar_init(&mbar_empty[b], 1);
    }
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue_copy = [&](uint32_t g, int slot) {
    bool tr;
    int off, bytes;
    L::chunk_src(g, tr, off, bytes);
    tc::mbar_expect_tx(&mbar_full[slot], (uint32_t)bytes);
    tc::bulk_g2s(sW + slot * L::STAGE_BYTES, (tr ? timg : wimg) + off, (uint32_t)bytes,
                 &mbar_full[slot]);
  };
  if (tid == 0)
    for (int b = 0; b < NS; ++b) issue_copy((uint32_t)b, b);
  {
    int o = 0;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int n = Cfg::N_of(l);
      for (int j = tid; j < n; j += 256) sBias[o + j] = a.bias[l] ? a.bias[l][j] : 0.0f;
      o += n;
    }
  }
  for (int j = tid; j < ROWS * K0 * 2 / 16; j += 256) {
    reinterpret_cast<uint4*>(sXh)[j] = make_uint4(0, 0, 0, 0);
    reinterpret_cast<uint4*>(sXl)[j] = make_uint4(0, 0, 0, 0);
  }
  __syncthreads();
  if (tid < ROWS)  // the constant 1 column (D + 1) gives db1 through dW1
    *reinterpret_cast<__nv_bfloat16*>(sXh + tc::cm_offset(tid, D + 1, K0)) =
        __float2bfloat16_rn(1.0f);
  if ((tid >> 5) == 0) {
    tc::tmem_alloc(&tmem_base_s, 512);
    tc::tmem_relinquish();
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_base_s;
  uint32_t parity = 0;

  // ---- per-row reverse state (as in k_mlp_adjoint)
  int inst = a.i0 + blockIdx.x * ROWS + row;
  const int iend = a.i0 + a.B;
  bool act = false;
  int n = -1, N = 0, q = -1;
  bool bad = false;
  double tn = 0.0, tnext = 0.0;
  float h = 0.0f;
  float yb[16], kb[7][16];
#pragma unroll
  for (int r = 0; r < C; ++r) {
    yb[r] = 0.0f;
#pragma unroll
    for (int j = 0; j < 7; ++j) kb[j][r] = 0.0f;
  }
  auto load_step = [&](int i) {
    const size_t o = (size_t)i * a.slots + n;
    tn = a.tp_t[o];
    h = a.tp_h[o];
    tnext = (n == N - 1) ? a.t1[i] : tn + (double)h;
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
  auto next_work = [&](bool finishing) {
    while (true) {
      if (finishing) {
        const int i = inst;
        if (!bad && a.gye) {
          const long long k0 = tkey(a.t0[i]);
          for (; q >= 0; --q)
            if (tkey(a.te[(size_t)i * a.K + q]) == k0)
#pragma unroll
              for (int r = 0; r < C; ++r) yb[r] += a.gye[((size_t)i * a.K + q) * D + coff + r];
        }
#pragma unroll
        for (int r = 0; r < C; ++r) a.gy0[(size_t)i * D + coff + r] = bad ? nan_(0.0f) : yb[r];
        inst += grid * ROWS;
        finishing = false;
      }
      if (inst >= iend) {
        act = false;
        return;
      }
      const int i = inst;
      N = a.n_acc[i];
      bad = a.status[i] != ST_SUCCESS;
      if (!bad && N > a.slots) {
        bad = true;
        if (sub == 0) atomicExch(a.overflow, 1);
      }
#pragma unroll
      for (int r = 0; r < C; ++r) yb[r] = a.gyf ? a.gyf[(size_t)i * D + coff + r] : 0.0f;
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
  // one GEMM of the round through the ring: A = the layer's input tile (K
  // major, hi and lo), B = the next K chunks; N = 512 as two halves of 256
  // or one MMA of width nw.  Transposed chunks are MN-major [16][IN] tiles.
  auto gemm = [&](uint32_t ah, uint32_t al, int Ka, int nchunks, int Nl, bool tr) {
    if (tid != 0 || abort_s) return;
    const int nh = Nl > 256 ? Nl / 256 : 1, nw = Nl > 256 ? 256 : Nl;
    const uint32_t idesc = tc::idesc_bf16_f32(ROWS, nw, false, tr);
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c, ++g_chunk) {
      const int b = (int)(g_chunk % NS);
      ok = tc::mbar_wait(&mbar_full[b], (g_chunk / NS) & 1u);
      if (!ok) break;
      const uint32_t wb = tc::smem_u32(sW + b * L::STAGE_BYTES);
      const uint64_t dh = tc::smem_desc(ah + c * 256, 128, Ka * 16);
      const uint64_t dl = tc::smem_desc(al + c * 256, 128, Ka * 16);
      for (int j = 0; j < nh; ++j) {
        const uint64_t db = tr ? tc::smem_desc_mn(wb + j * (256 / 8) * 128, Nl * 16)
                               : tc::smem_desc(wb + j * (256 / 8) * 256, 128, 256);
        tc::mma_bf16(tbase + 256 * j, dh, db, idesc, c > 0);
        tc::mma_bf16(tbase + 256 * j, dl, db, idesc, true);
      }
      tc::mma_commit(&mbar_empty[b]);
      if (g_chunk >= 1) {
        const uint32_t gp = g_chunk - 1;
        const int pb = (int)(gp % NS);
        ok = tc::mbar_wait(&mbar_empty[pb], (gp / NS) & 1u);
        if (!ok) break;
        issue_copy(gp + NS, pb);
      }
    }
    if (!ok) atomicExch(&abort_s, 1);
    tc::mma_commit(&mbar_mma);
  };
  // hidden epilogue: h = tanh(acc + b) into the tile; reverse rounds also
  // stage the row
  auto hidden_epi = [&](const float* bl, bool stage, uint16_t* shp, uint16_t* slp, size_t srow) {
#pragma unroll
    for (int c = 0; c < HC; c += 16) {
      const int col = sub * HC + c;
      float v[16];
      Cfg::hid_ld(tbase, tid, c, v);
      tc::tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = tanh_acc(v[j] + bl[col + j]);
      store_row16<true>(sHh, sHl, row, col, H, v);
      if (stage) stage_row16(shp, slp, srow * H + col, v);
    }
  };
  // delta epilogue: delta = acc (1 - h^2); h from the tile (own layer) or
  // from the staged row; the split delta replaces the tile, and is staged
  auto delta_epi = [&](bool h_in_tile, const uint16_t* hhp, const uint16_t* hlp, uint16_t* shp,
                       uint16_t* slp, size_t srow) {
#pragma unroll
    for (int c = 0; c < HC; c += 16) {
      const int col = sub * HC + c;
      float v[16], hv[16];
      Cfg::hid_ld(tbase, tid, c, v);
      if (h_in_tile) {
#pragma unroll
        for (int c8 = 0; c8 < 2; ++c8) {
          const uint32_t off = tc::cm_offset(row, col + 8 * c8, H);
          const uint4 hh = *reinterpret_cast<const uint4*>(sHh + off);
          const uint4 ll = *reinterpret_cast<const uint4*>(sHl + off);
          const uint32_t hw[4] = {hh.x, hh.y, hh.z, hh.w}, lw[4] = {ll.x, ll.y, ll.z, ll.w};
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&hw[j]);
            const __nv_bfloat162 l2 = *reinterpret_cast<const __nv_bfloat162*>(&lw[j]);
            hv[8 * c8 + 2 * j] = __low2float(h2) + __low2float(l2);
            hv[8 * c8 + 2 * j + 1] = __high2float(h2) + __high2float(l2);
          }
        }
      } else {
        unstage_row16(hhp, hlp, srow * H + col, hv);
      }
      tc::tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] *= madd(-hv[j], hv[j], 1.0f);
      store_row16<true>(sHh, sHl, row, col, H, v);
      stage_row16(shp, slp, srow * H + col, v);
    }
  };
  const float bw[7] = {float(Cc::b1), 0.0f, float(Cc::b3), float(Cc::b4), float(Cc::b5),
                       float(Cc::b6), 0.0f};
  int rev_round = 0;  // reverse rounds staged by this CTA

  for (int rnd = 0;; ++rnd) {
    const int ph = rnd % ADJ_ROUNDS;
    if (ph == 0 && __syncthreads_or(act) == 0) break;
    if (abort_s) break;
    const int s = 7 - ph;  // stage reversed this round (block-uniform)
    if (rev_round >= a.cap) {  // cannot happen: the staging is sized for it
      if (tid == 0) atomicExch(a.err, 2);
      break;
    }
    const size_t srow = ((size_t)blockIdx.x * a.cap + rev_round) * ROWS + row;

    // ---- stage input [Y_s; t_s] and the cotangent kbar_s of this row
    float Y[16], d3[16];
    float tin = 0.0f;
    if (act && s == 7) {
      const int i = inst;
#pragma unroll
      for (int j = 0; j < 7; ++j)
#pragma unroll
        for (int r = 0; r < C; ++r) kb[j][r] = h * bw[j] * yb[r];
      const long long kt = tkey(tn), kn = tkey(tnext);
      while (q >= 0) {
        const double tq = a.te[(size_t)i * a.K + q];
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
            dense_weights<float>(float(tq - tn) / h, w);
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
      tin = (float)(tn + dp_c(s) * (double)h);
      pick7(kb, s - 1, d3);
    } else {
#pragma unroll
      for (int r = 0; r < C; ++r) Y[r] = d3[r] = 0.0f;
    }
    store_row16<true>(sXh, sXl, row, coff, K0, Y);
    if (sub == Cfg::TPR - 1) {
      const __nv_bfloat16 th = __float2bfloat16_rn(tin);
      const __nv_bfloat16 tlo = __float2bfloat16_rn(tin - __bfloat162float(th));
      *reinterpret_cast<__nv_bfloat16*>(sXh + tc::cm_offset(row, D, K0)) = th;
      *reinterpret_cast<__nv_bfloat16*>(sXl + tc::cm_offset(row, D, K0)) = tlo;
    }
    store_row16<true>(sKh, sKl, row, coff, D, d3);
    // staged rows: X = [Y; t; 1; 0...] and kbar
    stage_row16(a.sa[0][0], a.sa[0][1], srow * K0 + coff, Y);
    stage_row16(a.sg[3][0], a.sg[3][1], srow * D + coff, d3);
    if (sub == Cfg::TPR - 1) {
      float tail[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) tail[j] = 0.0f;
      tail[0] = tin;
      tail[1] = 1.0f;
      stage_row16(a.sa[0][0], a.sa[0][1], srow * K0 + D, tail);
    }
    barrier();

    // ---- forward layers at Y_s
    gemm(tc::smem_u32(sXh), tc::smem_u32(sXl), K0, K0 / 16, H, false);
    wait_mma();
    hidden_epi(sBias, true, a.sa[1][0], a.sa[1][1], srow);
    barrier();
    gemm(tc::smem_u32(sHh), tc::smem_u32(sHl), H, H / 16, H, false);
    wait_mma();
    hidden_epi(sBias + H, true, a.sa[2][0], a.sa[2][1], srow);
    barrier();
    gemm(tc::smem_u32(sHh), tc::smem_u32(sHl), H, H / 16, H, false);
    wait_mma();
    hidden_epi(sBias + 2 * H, true, a.sa[3][0], a.sa[3][1], srow);
    barrier();

    float fg[16];
    {
      // gh3 = kbar W3 -> delta3 (h3 in the tile)
      gemm(tc::smem_u32(sKh), tc::smem_u32(sKl), D, D / 16, H, true);
      wait_mma();
      delta_epi(true, nullptr, nullptr, a.sg[2][0], a.sg[2][1], srow);
      barrier();
      // gh2 = delta3 W2 -> delta2 (h2 staged)
      gemm(tc::smem_u32(sHh), tc::smem_u32(sHl), H, H / 16, H, true);
      wait_mma();
      delta_epi(false, a.sa[2][0], a.sa[2][1], a.sg[1][0], a.sg[1][1], srow);
      barrier();
      // gh1 = delta2 W1 -> delta1 (h1 staged)
      gemm(tc::smem_u32(sHh), tc::smem_u32(sHl), H, H / 16, H, true);
      wait_mma();
      delta_epi(false, a.sa[1][0], a.sa[1][1], a.sg[0][0], a.sg[0][1], srow);
      barrier();
      // gx = delta1 W0: the state part of the cotangent
      gemm(tc::smem_u32(sHh), tc::smem_u32(sHl), H, H / 16, K0, true);
      wait_mma();
      Cfg::out_ld(tbase, tid, fg);
      tc::tmem_wait_ld();
      rev_round++;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (abort_s) break;

    // ---- consume (row-local; as in k_mlp_adjoint)
    if (!act) continue;
    {
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        if (j + 1 >= s) continue;
        const float c = h * dp_a(s, j + 1);
#pragma unroll
        for (int r = 0; r < C; ++r) kb[j][r] = madd(c, fg[r], kb[j][r]);
      }
#pragma unroll
      for (int r = 0; r < C; ++r) yb[r] += fg[r];
      if (s == 1) {
        n -= 1;
        if (n >= 0) load_step(inst);
        else next_work(true);
      }
    }
  }
  if (tid == 0) {  // the ring's copies still in flight land before the CTA exits
    const uint32_t first = g_chunk, last = g_chunk == 0 ? NS - 1 : g_chunk + NS - 2;
    for (uint32_t x = first; x <= last; ++x)
      if (!tc::mbar_wait(&mbar_full[x % NS], (x / NS) & 1u)) atomicExch(&abort_s, 1);
  }
  if (abort_s && tid == 0) atomicExch(a.err, 1);
  tc::fence_before_sync();
  __syncthreads();
  if ((tid >> 5) == 0) tc::tmem_dealloc(tbase, 512);
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
using Cfg64w = MlpBigCfg<64, 512, 4>;
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
  const size_t img = is_d64_h512(f) ? (size_t)Cfg64w::WREP * Cfg64w::WIMG_STRIDE
                                    : (size_t)Cfg32::WREP * Cfg32::WIMG_STRIDE;
  size_t b = align256(256) + img;
  if (o->form == TODE_PLAIN) {  // parked solver state (must match launch_mlp)
    const size_t B = (size_t)f->B, D = (size_t)f->D;
    b += 3 * align256(B * D * 4) + align256(B * 8) + 5 * align256(B * 4);
  }
  return b;
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
  a.o.beta3 = r.o->beta3;
  a.o.h0 = r.o->h0;
  a.o.max_steps = r.o->max_steps;
  opts_round_f32(a.o);
  if (r.tape) {
    a.slots = r.tape->slots;
    a.tp_y = (float*)r.tape->y;
    a.tp_k1 = (float*)r.tape->k1;
    a.tp_t = r.tape->t;
    a.tp_h = (float*)r.tape->h_acc;
    a.tp_ys = (float*)r.tape->y_stage;
  } else {
    a.slots = 0;
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
    const tode_err e = smem_optin((const void*)k_mlp_fused<Cfg>, Cfg::S_END, done);
    if (e != TODE_OK) return e;
  }
  long long grid = (r.B + Cfg::ROWS - 1) / Cfg::ROWS;
  if (grid > r.num_sms) grid = r.num_sms;
  if (grid == 0) return TODE_OK;
  if (r.o->form == TODE_PLAIN) {
    {
      static std::atomic<uint64_t> d0{0}, d1{0};
      tode_err e = smem_optin((const void*)k_mlp_plain_init<Cfg>, Cfg::S_END, d0);
      if (e == TODE_OK) e = smem_optin((const void*)k_mlp_plain_step<Cfg>, Cfg::S_END, d1);
      if (e != TODE_OK) return e;
    }
    k_mlp_plain_init<Cfg><<<(int)grid, Cfg::NT, Cfg::S_END, st>>>(a);
    TODE_CUDA_TRY(cudaGetLastError());
    const int poll = r.o->poll_every > 0 ? r.o->poll_every : 16;
    long long launched = 0;
    const long long limit = (long long)r.o->max_steps + 2LL * poll + 2;
    while (true) {
      for (int c = 0; c < poll - 1; ++c)
        k_mlp_plain_step<Cfg><<<(int)grid, Cfg::NT, Cfg::S_END, st>>>(a);
      TODE_CUDA_TRY(cudaMemsetAsync(a.active, 0, sizeof(int32_t), st));
      k_mlp_plain_step<Cfg><<<(int)grid, Cfg::NT, Cfg::S_END, st>>>(a);
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
  k_mlp_fused<Cfg><<<(int)grid, Cfg::NT, Cfg::S_END, st>>>(a);
  TODE_CUDA_TRY(cudaGetLastError());
  return TODE_OK;
}

tode_err mlp_solve(const SolveReq& r, bool split) {
  if (r.o->form != TODE_FUSED && r.o->form != TODE_PLAIN) return TODE_EUNSUPPORTED;
  if (r.tape && r.tape->stride != 1) return TODE_EUNSUPPORTED;
  if (is_d64_h512(r.f)) return split ? launch_mlp<Cfg64s>(r) : TODE_EUNSUPPORTED;
  return split ? launch_mlp<Cfg32s>(r) : launch_mlp<Cfg32>(r);
}

// ---- wide network: scratch plan of the staged adjoint
struct WidePlan {
  int grid, cap;       // CTAs, reverse rounds per CTA per slice
  size_t rows;         // staged rows per slice
  size_t off_timg, off_stage[8], off_dw0, off_ones, off_cublas, total;
};
static constexpr size_t WIDE_CUBLAS_WS = 32u << 20;
static WidePlan wide_plan(int B, int slots, int num_sms) {
  using Cfg = Cfg64w;
  using L = WideAdjLayout<Cfg>;
  WidePlan p{};
  p.grid = (int)std::min<long long>((B + 63) / 64, num_sms);
  p.cap = 7 * std::max(slots, 1);  // one instance per row per slice
  p.rows = (size_t)p.grid * p.cap * 64;
  size_t o = align256(256) + (size_t)Cfg::WREP * Cfg::WIMG_STRIDE;
  p.off_timg = o;
  o += (size_t)Cfg::WREP * L::TIMG_STRIDE;
  const int width[8] = {Cfg::K0, Cfg::H, Cfg::H, Cfg::H, Cfg::H, Cfg::H, Cfg::H, Cfg::D};
  for (int q = 0; q < 8; ++q) {  // sa[0..3], sg[0..3]; hi then lo planes
    p.off_stage[q] = o;
    o += 2 * align256(p.rows * width[q] * 2);
  }
  p.off_dw0 = o;
  o += align256((size_t)Cfg::H * Cfg::K0 * 4);
  p.off_ones = o;
  o += align256(p.rows * 2);
  p.off_cublas = o;
  o += WIDE_CUBLAS_WS;
  p.total = o;
  return p;
}

size_t mlp_adjoint_scratch_bytes(const tode_field_desc* f, int slots, int num_sms) {
  using L = MlpAdjLayout<Cfg32s>;
  if (is_d64_h512(f)) return wide_plan(f->B, slots, num_sms).total;
  if (!is_d32_h128(f)) return 0;
  const long long grid = std::min<long long>((f->B + 127) / 128, num_sms);
  return align256(256) + align256((size_t)Cfg32s::WIMG_BYTES) +
         align256((size_t)grid * L::P_FLOATS * 4);
}

__global__ void k_fill_bf16_one(uint16_t* p, size_t n) {
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e < n) p[e] = 0x3F80;  // BF16 1.0
}
// gW0 [H][65] from the padded [H][80] accumulator
__global__ void k_copy_cols(const float* src, int rows, int ld, int cols, float* dst) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < rows * cols) dst[e] = src[(size_t)(e / cols) * ld + e % cols];
}

// one cuBLAS handle per device, created on first use
static cublasHandle_t cublas_for_device(int dev) {
  static std::mutex mu;
  static cublasHandle_t handles[64] = {};
  std::lock_guard<std::mutex> g(mu);
  if (dev < 0 || dev >= 64) return nullptr;
  if (!handles[dev] && cublasCreate(&handles[dev]) != CUBLAS_STATUS_SUCCESS) handles[dev] = nullptr;
  return handles[dev];
}

static tode_err mlp_wide_adjoint(const AdjReq& r) {
  using Cfg = Cfg64w;
  using L = WideAdjLayout<Cfg>;
  const cudaStream_t st = r.stream;
  const WidePlan p = wide_plan(r.B, r.tape->slots, r.num_sms);
  if (r.scratch_bytes < p.total) return TODE_EWORKSPACE;
  int dev = 0;
  TODE_CUDA_TRY(cudaGetDevice(&dev));
  cublasHandle_t hb = cublas_for_device(dev);
  if (!hb) return TODE_ECUDA;
  char* base = r.scratch;
  WideAdjArgs a{};
  a.K = r.K;
  a.t0 = r.t0;
  a.t1 = r.t1;
  a.te = r.te;
  a.n_acc = r.n_acc;
  a.status = r.status;
  a.slots = r.tape->slots;
  a.Btot = r.B;
  a.tp_y = (const float*)r.tape->y;
  a.tp_k1 = (const float*)r.tape->k1;
  a.tp_t = r.tape->t;
  a.tp_h = (const float*)r.tape->h_acc;
  a.gye = (const float*)r.gye;
  a.gyf = (const float*)r.gyf;
  a.gy0 = (float*)r.gy0;
  for (int l = 0; l < MLP_MAX_LAYERS; ++l) a.bias[l] = r.f->b[l];
  a.err = (int32_t*)(base + 128);
  a.overflow = r.overflow;
  a.cap = p.cap;
  a.tp_ys = (const float*)r.tape->y_stage;
  unsigned char* img = (unsigned char*)base + align256(256);
  unsigned char* timg = (unsigned char*)base + p.off_timg;
  a.wimg = img;
  a.timg = timg;
  const int width[8] = {Cfg::K0, Cfg::H, Cfg::H, Cfg::H, Cfg::H, Cfg::H, Cfg::H, Cfg::D};
  uint16_t* planes[8][2];
  for (int q = 0; q < 8; ++q) {
    planes[q][0] = (uint16_t*)(base + p.off_stage[q]);
    planes[q][1] = (uint16_t*)(base + p.off_stage[q] + align256(p.rows * width[q] * 2));
  }
  for (int j = 0; j < 4; ++j)
    for (int k = 0; k < 2; ++k) {
      a.sa[j][k] = planes[j][k];
      a.sg[j][k] = planes[4 + j][k];
    }
  float* dw0 = (float*)(base + p.off_dw0);
  uint16_t* ones = (uint16_t*)(base + p.off_ones);
  // weight images (forward chunks and transposed chunks, WREP copies each)
  {
    size_t woff[MLP_MAX_LAYERS] = {}, toff[MLP_MAX_LAYERS] = {};
    for (int l = 0; l < Cfg::NL; ++l) {
      woff[l] = Cfg::W_off(l);
      toff[l] = L::T_off(l);
    }
    tode_err e = build_images<Cfg>(r.f, img, IMG_CHUNKS, Cfg::WREP, Cfg::WIMG_STRIDE, woff, st);
    if (e == TODE_OK)
      e = build_images<Cfg>(r.f, timg, IMG_TCHUNKS, Cfg::WREP, L::TIMG_STRIDE, toff, st);
    if (e != TODE_OK) return e;
  }
  k_fill_bf16_one<<<(unsigned)((p.rows + 255) / 256), 256, 0, st>>>(ones, p.rows);
  TODE_CUDA_TRY(cudaGetLastError());
  TODE_CUDA_TRY(cudaMemsetAsync(base, 0, 256, st));
  TODE_CUDA_TRY(cudaMemsetAsync(dw0, 0, (size_t)Cfg::H * Cfg::K0 * 4, st));
  for (int l = 1; l < 4; ++l)
    TODE_CUDA_TRY(cudaMemsetAsync(r.gW[l], 0, (size_t)Cfg::N_of(l) * Cfg::K_of(l) * 4, st));
  if (r.gb)
    for (int l = 0; l < 4; ++l)
      if (r.gb[l]) TODE_CUDA_TRY(cudaMemsetAsync(r.gb[l], 0, (size_t)Cfg::N_of(l) * 4, st));
  {
    static std::atomic<uint64_t> done{0};
    const tode_err e = smem_optin((const void*)k_mlp_adjoint_wide<Cfg>, L::S_END, done);
    if (e != TODE_OK) return e;
  }
  if (cublasSetStream(hb, st) != CUBLAS_STATUS_SUCCESS ||
      cublasSetWorkspace(hb, base + p.off_cublas, WIDE_CUBLAS_WS) != CUBLAS_STATUS_SUCCESS)
    return TODE_ECUDA;
  const float one = 1.0f;
  // dW_l (row-major [out][in]) += delta_l^T act_l: in cuBLAS's column-major
  // terms C[in x out] += act[in x R] * delta[out x R]^T
  auto gemm = [&](const uint16_t* act_p, int in, const uint16_t* del_p, int out, float* C) {
    return cublasGemmEx(hb, CUBLAS_OP_N, CUBLAS_OP_T, in, out, (int)p.rows, &one, act_p,
                        CUDA_R_16BF, in, del_p, CUDA_R_16BF, out, &one, C, CUDA_R_32F, in,
                        CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT) == CUBLAS_STATUS_SUCCESS;
  };
  auto colsum = [&](const uint16_t* del_p, int out, float* C) {  // db += delta^T 1
    return cublasGemmEx(hb, CUBLAS_OP_N, CUBLAS_OP_N, out, 1, (int)p.rows, &one, del_p,
                        CUDA_R_16BF, out, ones, CUDA_R_16BF, (int)p.rows, &one, C, CUDA_R_32F,
                        out, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT) == CUBLAS_STATUS_SUCCESS;
  };
  const int slice = p.grid * 64;
  for (int i0 = 0; i0 < r.B; i0 += slice) {
    for (int q = 0; q < 8; ++q)
      TODE_CUDA_TRY(cudaMemsetAsync(planes[q][0], 0, 2 * align256(p.rows * width[q] * 2), st));
    a.i0 = i0;
    a.B = std::min(slice, r.B - i0);
    k_mlp_adjoint_wide<Cfg><<<p.grid, 256, L::S_END, st>>>(a);
    TODE_CUDA_TRY(cudaGetLastError());
    for (int l = 0; l < 4; ++l) {
      const int in = Cfg::K_of(l), out = Cfg::N_of(l);
      float* C = l == 0 ? dw0 : r.gW[l];
      bool ok = gemm(planes[l][0], in, planes[4 + l][0], out, C) &&  // hi * hi
                gemm(planes[l][1], in, planes[4 + l][0], out, C) &&  // lo * hi
                gemm(planes[l][0], in, planes[4 + l][1], out, C);    // hi * lo
      if (ok && r.gb && r.gb[l])
        ok = colsum(planes[4 + l][0], out, r.gb[l]) && colsum(planes[4 + l][1], out, r.gb[l]);
      if (!ok) return TODE_ECUDA;
    }
  }
  k_copy_cols<<<(Cfg::H * (Cfg::D + 1) + 255) / 256, 256, 0, st>>>(dw0, Cfg::H, Cfg::K0, Cfg::D + 1,
                                                                   r.gW[0]);
  TODE_CUDA_TRY(cudaGetLastError());
  return TODE_OK;
}

tode_err mlp_adjoint(const AdjReq& r) {
  using Cfg = Cfg32s;
  using L = MlpAdjLayout<Cfg>;
  if (is_d64_h512(r.f)) {
    if (r.tape->stride != 1 || !r.tape->h_acc || !r.tape->y || !r.tape->t || !r.tape->y_stage)
      return TODE_EINVAL;
    if (!r.gW || !r.gW[0] || !r.gW[1] || !r.gW[2] || !r.gW[3]) return TODE_EINVAL;
    return mlp_wide_adjoint(r);
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
  {
    size_t loff[MLP_MAX_LAYERS] = {};
    for (int l = 0; l < Cfg::NL; ++l) loff[l] = Cfg::W_off(l);
    const tode_err e = build_images<Cfg>(r.f, img, IMG_TILE, 1, Cfg::WIMG_STRIDE, loff, st);
    if (e != TODE_OK) return e;
  }
  TODE_CUDA_TRY(cudaMemsetAsync(r.scratch, 0, 256, st));
  {
    static std::atomic<uint64_t> done{0};
    const tode_err e = smem_optin((const void*)k_mlp_adjoint<Cfg>, L::S_END, done);
    if (e != TODE_OK) return e;
  }
  k_mlp_adjoint<Cfg><<<(int)grid, 256, L::S_END, st>>>(a);
  TODE_CUDA_TRY(cudaGetLastError());
  const int total = Cfg::H * (Cfg::D + 1) + Cfg::H + Cfg::H * Cfg::H + Cfg::H +
                    Cfg::D * Cfg::H + Cfg::D;
  k_mlp_grad_reduce<Cfg><<<(total + 255) / 256, 256, 0, st>>>(
      a.part, (int)grid, r.gW[0], r.gb ? r.gb[0] : nullptr, r.gW[1], r.gb ? r.gb[1] : nullptr,
      r.gW[2], r.gb ? r.gb[2] : nullptr);
  TODE_CUDA_TRY(cudaGetLastError());
  return TODE_OK;
}

}  // namespace tode
