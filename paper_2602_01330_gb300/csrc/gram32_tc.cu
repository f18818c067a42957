// Bond-32 transfer-chain Gram on tensor cores with split-BF16 operands (bf16x3).
//
// Same contraction as gram32.cu (§II-C, Eqs. 8-10, block-structured, h = 16): per site,
// pair and (s, t), G = E_t B with B = A_s[t](x_j), then E'_s += C G with C = A_s[t](x_i)^dagger.
// Each complex 16 x 16 x 16 product Z = X Y is one real GEMM of the block form
//     [Xr | Xi] (16 x 32) . [[Yr, Yi], [-Yi, Yr]] (32 x 32) = [Zr | Zi] (16 x 32),
// run as m16n8k16 BF16 MMAs with FP32 accumulation. Every FP32 operand v is split into
// v = hi + lo (both BF16) and each product is lo.hi + hi.lo + hi.hi (bf16x3), which keeps
// about 16 significant bits per product; the lo.lo term is dropped.
//
// Dataflow: one warp per pair, everything between sites in registers. An m16n8 accumulator
// tile of a matrix X holds, lane by lane, exactly the B-operand fragment of X^T (lane 4g + t
// has X[g][2t], X[g][2t+1] and the same for row g + 8; the B fragment wants Y[2t][g],
// Y[2t+1][g]). So the step order is chosen to always consume an accumulator as the B
// operand of a transposed product:
//   step 1:  G^T = B^T E_t^T     (A operand B^T from shared memory, B operand from E_t's
//                                  accumulators),
//   step 2:  E'_s += C G          (A operand C from shared memory, B operand from G^T's
//                                  accumulators),
// and E'_s is again in accumulator form for the next site. No intermediate goes through
// shared memory. A sample's operand is stored once, X = [Re A^T | Im A^T] split into BF16
// hi / lo: step 1 uses it as B^T, step 2 as C = conj(A)^T by negating the other factor's
// matching rows (put_chunk, mma_block_side).
//
// Operand staging, one site per stage of a shared-memory ring, by warps separate from the
// pair warps so that it runs under their MMAs:
//   split operands (dk_mps_split32, the faster form): one copy warp moves each sample's
//     10 KB image with one bulk copy;
//   complex64 site tensors: four staging warps load them from HBM (one site ahead, in
//     registers) and split them.
#include <math.h>

#include "common.cuh"
#include "gram_common.cuh"
#include "internal.h"
#include "transfer.cuh"

namespace dk {
namespace tc32 {

using u32 = uint32_t;
using u16 = uint16_t;

constexpr int SAMPLE_FLOATS = 32 * 32 * 2;  // compact site tensor, complex64
constexpr int CHUNKS = SAMPLE_FLOATS / 4;    // 16-byte chunks per sample-site
// Operand tiles are row-major BF16 with 80-byte rows (32 values + 8 pad), so that the 8
// rows of an ldmatrix phase hit 8 different 16-byte bank groups.
constexpr int ROW = 40;                      // u16 per padded row
constexpr int COP = 16 * ROW;                // one operand (16 x 32) in u16
constexpr int SBUF = 4 * 2 * COP;            // one sample: 4 (s, t) blocks x hi / lo

__device__ __forceinline__ void mma16816(float (&d)[4], const u32 (&a)[4], u32 b0, u32 b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(u32 (&r)[4], const u16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}

// (x, y) -> packed BF16 pairs hi and lo with x ~ hi + lo (low half = x): hi = round(x, y)
// to BF16, the residuals x - hi and y - hi (exact in FP32: the upper half of hi's word, and
// the lower half shifted up, are hi's values as FP32) rounded to BF16 again. Six instructions
// in inline PTX, so that the compiler keeps them where the schedule places them.
__device__ __forceinline__ void split2(float x, float y, u32& hi, u32& lo) {
  asm volatile(
      "{\n\t.reg .b32 hx, hy;\n\t.reg .f32 rx, ry;\n\t"
      "cvt.rn.bf16x2.f32 %0, %3, %2;\n\t"
      "shl.b32 hx, %0, 16;\n\t"
      "and.b32 hy, %0, 0xffff0000;\n\t"
      "sub.f32 rx, %2, hx;\n\t"
      "sub.f32 ry, %3, hy;\n\t"
      "cvt.rn.bf16x2.f32 %1, ry, rx;\n\t}"
      : "=r"(hi), "=r"(lo)
      : "f"(x), "f"(y));
}
constexpr u32 NEG2 = 0x80008000u;  // flips the sign of both BF16 halves

// Operand of block (s, t) of a sample: X[p][k] = Re A[k][p] (k < 16), Im A[k-16][p]
// (k >= 16), A[a][p] the compact element (s, j = p, l = 16 t + a): the B^T operand of a
// column sample (transpose) as it is, and the C operand of a row sample (conjugate transpose)
// with its k >= 16 half negated, which mma_block applies to the other factor instead (CONJ).
// A 16-byte chunk holds elements l, l+1 of compact row r = 16 s + p.
__device__ __forceinline__ void put_chunk(u16* buf, int chunk, float4 v) {
  const int r = chunk >> 4, q = chunk & 15;
  const int s = r >> 4, p = r & 15;
  const int l = 2 * q, t = l >> 4, a = l & 15;
  u16* hi = buf + (s * 2 + t) * 2 * COP;
  u16* lo = hi + COP;
  u32 h, w;
  split2(v.x, v.z, h, w);  // Re at a, a+1
  *reinterpret_cast<u32*>(hi + p * ROW + a) = h;
  *reinterpret_cast<u32*>(lo + p * ROW + a) = w;
  split2(v.y, v.w, h, w);  // Im at a, a+1
  *reinterpret_cast<u32*>(hi + p * ROW + 16 + a) = h;
  *reinterpret_cast<u32*>(lo + p * ROW + 16 + a) = w;
}

// Thread u (0..511 over a sample's chunks) -> chunk 16 r + q, r = 16 s + p, q = 8 t + q'.
// A warp takes q' = 0..7 and p in {0, 2, 4, 6} (+1, +8): its stores into one (s, t) operand
// start at banks 20 p + q' mod 32 = {0, 8, 16, 24} + q' (a padded row is 20 banks), so they
// are conflict-free, and its global reads are four runs of 128 contiguous bytes.
__device__ __forceinline__ int chunk_of(int u) {
  const int qq = u & 7, psel = (u >> 3) & 3, par = (u >> 5) & 1, t = (u >> 6) & 1, phi = (u >> 7) & 1,
            s = (u >> 8) & 1;
  const int p = 2 * psel + par + 8 * phi;
  return 16 * (16 * s + p) + 8 * t + qq;
}

// Accumulator state of one complex 16 x 16 matrix X: v[nt][4], nt 0..1 = real part columns
// 0-7 / 8-15, nt 2..3 = imaginary part (m16n8 accumulator layout).
struct Frag {
  float v[2][4][4];  // two bond blocks
};

// B-operand words of Y = X^T (or of the block matrix built from it) taken from X's
// accumulators: w[c][h][tile] = X component c (0 Re, 1 Im), rows g (h = 0) or g + 8 (h = 1),
// columns 2t, 2t+1 of column tile `tile`, split into BF16 hi / lo.
struct BFrag {
  u32 hi[2][2][2], lo[2][2][2];
};

__device__ __forceinline__ void to_bfrag(const float (&x)[4][4], BFrag& f) {
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int tile = 0; tile < 2; ++tile)
        split2(x[2 * c + tile][2 * h], x[2 * c + tile][2 * h + 1], f.hi[c][h][tile], f.lo[c][h][tile]);
}

// Step q (0..7) of to_bfrag, in the same (c, h, tile) order: the same words, one split2.
__device__ __forceinline__ void to_bfrag_step(const float (&x)[4][4], BFrag& f, int q) {
  const int c = q >> 2, h = (q >> 1) & 1, tile = q & 1;
  split2(x[2 * c + tile][2 * h], x[2 * c + tile][2 * h + 1], f.hi[c][h][tile], f.lo[c][h][tile]);
}

// acc += [Xr | Xi] . [[Yr, Yi], [-Yi, Yr]] for X (16 x 16 complex) from shared memory
// (xh: hi operand, lo operand COP further) and Y given by f (Y = the transpose of the matrix
// whose accumulators made f). k-step kk = 0 takes the rows [Yr | Yi], kk = 1 [-Yi | Yr]; with
// CONJ, X is used as [Xr | -Xi] (the conjugate of the stored matrix) by negating the kk = 1
// rows instead, [Yi | -Yr]: the same products, so the same sums. The MMAs are issued
// term-major over the four independent n-tile accumulators. With SIDE, the conversion
// sf = to_bfrag(sx) of an independent matrix is spread over the block, one split2 after every
// third MMA, so that the warp issues it between MMAs instead of in a burst of its own.
template <bool CONJ, bool SIDE>
__device__ __forceinline__ void mma_block_side(float (&acc)[4][4], const u16* xh, const BFrag& f, int lane,
                                               const float (&sx)[4][4], BFrag& sf) {
  int n = 0;
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    u32 ahi[4], alo[4];
    const u16* rowp = xh + (lane & 15) * ROW + 16 * kk + 8 * (lane >> 4);
    ldsm_x4(ahi, rowp);
    ldsm_x4(alo, rowp + COP);
    u32 bh[4][2], bl[4][2];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int c = (nt >> 1) ^ kk, h = nt & 1;
      const u32 sg = (kk == 1 && ((nt < 2) != CONJ)) ? NEG2 : 0u;
      bh[nt][0] = f.hi[c][h][0] ^ sg;
      bh[nt][1] = f.hi[c][h][1] ^ sg;
      bl[nt][0] = f.lo[c][h][0] ^ sg;
      bl[nt][1] = f.lo[c][h][1] ^ sg;
    }
#pragma unroll
    for (int term = 0; term < 3; ++term)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt, ++n) {
        if (term == 0) mma16816(acc[nt], alo, bh[nt][0], bh[nt][1]);
        else if (term == 1) mma16816(acc[nt], ahi, bl[nt][0], bl[nt][1]);
        else mma16816(acc[nt], ahi, bh[nt][0], bh[nt][1]);
        if (SIDE && n % 3 == 2) to_bfrag_step(sx, sf, n / 3);
      }
  }
}

template <bool CONJ>
__device__ __forceinline__ void mma_block(float (&acc)[4][4], const u16* xh, const BFrag& f, int lane) {
  BFrag unused;
  mma_block_side<CONJ, false>(acc, xh, f, lane, acc, unused);
}

// One site of one pair (warp). rbuf: row-sample C operands; cbuf: column-sample B^T
// operands. E is replaced by diag(acc_0, acc_1). Two schedules of the same MMAs:
//   IL = false: per (t, s) step 1, conversion of G, step 2 (fewest live registers);
//   IL = true:  per t both step-1 products (s = 0, 1) back to back, and every conversion that
//               has an independent MMA block beside it spread over that block's MMAs (E_1
//               over the first step-1 block, G_0 over the second, G_1 over the first step-2
//               block); only E_0's conversion runs on its own.
// Every accumulator receives its MMAs in the same order in both (acc_s: t = 0, then t = 1)
// and every conversion is the same split2, so the result does not depend on the schedule.
template <bool IL>
__device__ __forceinline__ void pair_site(Frag& E, const u16* rbuf, const u16* cbuf, int lane) {
  float acc[2][4][4];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[s][nt][c] = 0.0f;
  if (!IL) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      BFrag fe;
      to_bfrag(E.v[t], fe);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        float g[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
          for (int c = 0; c < 4; ++c) g[nt][c] = 0.0f;
        mma_block<false>(g, cbuf + (s * 2 + t) * 2 * COP, fe, lane);
        BFrag fg;
        to_bfrag(g, fg);
        mma_block<true>(acc[s], rbuf + (s * 2 + t) * 2 * COP, fg, lane);
      }
    }
  } else {
    BFrag fe[2];
    to_bfrag(E.v[0], fe[0]);  // B operands of E_0^T; E_1's are formed during the first block
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      // step 1: G_s^T = B_{s,t}^T . E_t^T for s = 0, 1
      float g[2][4][4];
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
          for (int c = 0; c < 4; ++c) g[s][nt][c] = 0.0f;
      BFrag fg[2];
      if (t == 0) mma_block_side<false, true>(g[0], cbuf + (0 * 2 + t) * 2 * COP, fe[t], lane, E.v[1], fe[1]);
      else mma_block<false>(g[0], cbuf + (0 * 2 + t) * 2 * COP, fe[t], lane);
      mma_block_side<false, true>(g[1], cbuf + (1 * 2 + t) * 2 * COP, fe[t], lane, g[0], fg[0]);
      // step 2: acc_s += C_{s,t} . G_s (B operand of G_s from G_s^T's accumulators)
      mma_block_side<true, true>(acc[0], rbuf + (0 * 2 + t) * 2 * COP, fg[0], lane, g[1], fg[1]);
      mma_block<true>(acc[1], rbuf + (1 * 2 + t) * 2 * COP, fg[1], lane);
    }
  }
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int c = 0; c < 4; ++c) E.v[s][nt][c] = acc[s][nt][c];
}

__device__ __forceinline__ void init_e(Frag& E, int lane) {
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int c = 0; c < 4; ++c) E.v[t][nt][c] = 0.0f;
  if (lane == 0) E.v[0][0][0] = 1.0f;
}

__device__ __forceinline__ int renorm(Frag& E) {
  float mx = 0.0f;
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int c = 0; c < 4; ++c) mx = fmaxf(mx, fabsf(E.v[t][nt][c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const int e = RealBits<float>::exponent(mx);
  const float sc = RealBits<float>::pow2_neg(e);
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int c = 0; c < 4; ++c) E.v[t][nt][c] *= sc;
  return e;
}

// ln|a|, a = E_0[0][0] + E_1[0][0]: row 0, column 0 of the real (n-tile 0) and imaginary
// (n-tile 2) parts, held by lane 0 (valid in lane 0 only).
__device__ __forceinline__ float half_log_mod(const Frag& E, int e2) {
  const float re = E.v[0][0][0] + E.v[1][0][0];
  const float im = E.v[0][2][0] + E.v[1][2][0];
  const float mod2 = fmaf(re, re, im * im);
  return fmaf(0.5f, logf(mod2), float(e2) * 0.69314718055994530942f);
}

// CTA of TR x TC pair warps (one pair each) and the staging warps (four, or one copy warp
// for split operands) over a ring of NSTG stages; a stage holds one site of the operands of
// the tile's TR row samples and TC column samples.
template <int TR, int TC, int NSTG, bool IL_, bool PRESPLIT_>
struct CfgTc {
  static constexpr int TR_ = TR, TC_ = TC, NSTG_ = NSTG;
  static constexpr bool PRESPLIT = PRESPLIT_;      // operands from dk_mps_split32: copied, not split
  static constexpr int NW = TR * TC;               // pair warps
  static constexpr int PT = (PRESPLIT ? 1 : 4) * 32;  // staging threads (presplit: one copy warp)
  static constexpr int NT = NW * 32 + PT;
  static constexpr int STAGE = (TR + TC) * SBUF;   // u16 per stage
  static constexpr int CH = (TR + TC) * CHUNKS;    // 16-byte chunks of a stage's site tensors
  static_assert(PRESPLIT || CH % PT == 0, "whole chunks per staging thread");
  static constexpr int PER_THREAD = CH / PT;
  static constexpr bool IL = IL_;                  // pair_site schedule
  static constexpr u32 OPS_BYTES = SBUF * sizeof(u16);  // one sample-site of dk_mps_split32 operands
  static constexpr size_t BAR_OFF = size_t(NSTG) * STAGE * sizeof(u16);
  static constexpr size_t SMEM = BAR_OFF + 2 * NSTG * sizeof(uint64_t) + 16;
};

// Warp roles. Staging warps (complex64 input): for every (tile, site) of the CTA, in order,
// wait until the ring slot is free (empty barrier: one arrival per pair warp), read the site
// tensors of the tile's samples from HBM (16-byte chunks, one site ahead in registers), split
// them into BF16 hi / lo operands in shared memory and arrive on the slot's full barrier (one
// arrival per staging thread, which releases its stores). Copy warp (PRESPLIT, operands from
// dk_mps_split32): one thread waits for the slot and fills it with one 10 KB bulk copy per
// sample, the slot's full barrier counting the bytes. Pair warps: wait for the slot, run one
// site of their pair, release the slot. Every wait is bounded; on a timeout the CTA records
// DEV_TIMEOUT in the status word, raises its abort flag and every role leaves its loop, the
// copy thread after waiting for its copies in flight.
template <class C>
__global__ void __launch_bounds__(C::NT, 1)
    gram32_tc_kernel(const float* __restrict__ mps_r, int m_r, const float* __restrict__ mps_c, int m_c,
                     const GramArgs p) {
  constexpr int TR = C::TR_, TC = C::TC_, NSTG = C::NSTG_;
  extern __shared__ __align__(16) u16 smu[];
  uint64_t* full = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(smu) + C::BAR_OFF);
  uint64_t* empty = full + NSTG;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + NSTG);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTG; ++s) {
      mbar_init(&full[s], C::PRESPLIT ? 1 : C::PT);
      mbar_init(&empty[s], C::NW);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  const int my_tiles = (p.ntiles > int(blockIdx.x)) ? (p.ntiles - 1 - int(blockIdx.x)) / int(gridDim.x) + 1 : 0;
  auto tile_origin = [&](int lt, int& r0, int& c0) {
    int ti, tj;
    decode_tile(p, TR, TC, int(blockIdx.x) + lt * int(gridDim.x), ti, tj);
    r0 = p.row0 + ti * TR;
    c0 = p.col0 + tj * TC;
  };
  auto give_up = [&]() {
    record_status(p.status, DEV_TIMEOUT);
    *abort_flag = 1;
  };

  if (warp >= C::NW && C::PRESPLIT) {
    // ---- copy warp: one thread moves each sample's split operands with one bulk copy ----
    if (lane == 0) {
      const uint8_t* ops_r = reinterpret_cast<const uint8_t*>(mps_r);
      const uint8_t* ops_c = reinterpret_cast<const uint8_t*>(mps_c);
      const long long total = (long long)my_tiles * p.n;
      long long g = 0;  // stage fills issued
      int lt = 0, k = 0, r0 = 0, c0 = 0;
      if (total > 0) tile_origin(0, r0, c0);
      for (; g < total; ++g) {
        const int s = int(g % NSTG);
        const long long use = g / NSTG;
        if (*abort_flag || (use > 0 && !mbar_wait_bounded(&empty[s], u32((use - 1) & 1)))) {
          give_up();
          break;
        }
        u16* st = smu + s * C::STAGE;
        mbar_arrive_expect_tx(&full[s], u32(TR + TC) * C::OPS_BYTES);
#pragma unroll 1
        for (int smp = 0; smp < TR + TC; ++smp) {
          const uint8_t* src = smp < TR ? ops_r + (size_t(k) * m_r + min(r0 + smp, m_r - 1)) * C::OPS_BYTES
                                        : ops_c + (size_t(k) * m_c + min(c0 + smp - TR, m_c - 1)) * C::OPS_BYTES;
          bulk_load(st + smp * SBUF, src, C::OPS_BYTES, &full[s]);
        }
        if (++k == p.n) {
          k = 0;
          ++lt;
          if (g + 1 < total) tile_origin(lt, r0, c0);
        }
      }
      // the copies of the last fills of every slot land before the CTA exits (each is the
      // slot's newest phase, so its parity cannot alias)
      for (long long q = g - 1; q >= 0 && q >= g - NSTG; --q)
        if (!mbar_wait_bounded(&full[int(q % NSTG)], u32((q / NSTG) & 1))) record_status(p.status, DEV_TIMEOUT);
    }
  } else if (warp >= C::NW) {
    // ---- staging ----
    // Each thread owns chunks pt + q * PT (q < PER_THREAD) of every stage and keeps the next
    // site's copies of them in registers: while it converts chunk q of site g it loads chunk q
    // of site g + 1 into the register just freed, so every load has a whole conversion pass to
    // arrive.
    const int pt = threadIdx.x - C::NW * 32;
    const long long total = (long long)my_tiles * p.n;
    // chunk pt + q PT of a stage is chunk w[q % QS] of sample q / QS (QS = CHUNKS / PT)
    constexpr int QS = CHUNKS / C::PT;
    static_assert(CHUNKS % C::PT == 0, "a staging thread's chunks of a sample are the same for every sample");
    int w4[QS];
#pragma unroll
    for (int u = 0; u < QS; ++u) w4[u] = 4 * chunk_of(pt + u * C::PT);
    const float* base[TR + TC];  // the samples of the site being loaded
    auto bases = [&](int k, int r0, int c0) {
#pragma unroll
      for (int smp = 0; smp < TR + TC; ++smp)
        base[smp] = smp < TR ? mps_r + (size_t(k) * m_r + min(r0 + smp, m_r - 1)) * SAMPLE_FLOATS
                             : mps_c + (size_t(k) * m_c + min(c0 + smp - TR, m_c - 1)) * SAMPLE_FLOATS;
    };
    auto load = [&](int q) { return __ldg(reinterpret_cast<const float4*>(base[q / QS] + w4[q % QS])); };
    float4 v[C::PER_THREAD];
    int lt = 0, k = 0, r0 = 0, c0 = 0;  // the site whose chunks v holds
    if (total > 0) {
      tile_origin(0, r0, c0);
      bases(0, r0, c0);
#pragma unroll
      for (int q = 0; q < C::PER_THREAD; ++q) v[q] = load(q);
    }
    for (long long g = 0; g < total; ++g) {
      int nlt = lt, nk = k + 1, nr0 = r0, nc0 = c0;
      const bool more = g + 1 < total;
      if (nk == p.n) {
        nk = 0;
        ++nlt;
        if (more) tile_origin(nlt, nr0, nc0);
      }
      const int s = int(g % NSTG);
      const long long use = g / NSTG;
      if (*abort_flag || (use > 0 && !mbar_wait_bounded(&empty[s], u32((use - 1) & 1)))) {
        give_up();
        break;
      }
      u16* st = smu + s * C::STAGE;
      if (more) bases(nk, nr0, nc0);
#pragma unroll
      for (int q = 0; q < C::PER_THREAD; ++q) {
        const float4 x = v[q];
        if (more) v[q] = load(q);
        const int smp = q / QS, w = w4[q % QS] >> 2;
        put_chunk(st + smp * SBUF, w, x);
      }
      mbar_arrive(&full[s]);
      lt = nlt;
      k = nk;
      r0 = nr0;
      c0 = nc0;
    }
  } else {
    // ---- pair warps ----
    const int wr = warp / TC, wc = warp % TC;
    long long g = 0;  // stages consumed
    bool stop = false;
    for (int lt = 0; lt < my_tiles && !stop; ++lt) {
      int r0, c0;
      tile_origin(lt, r0, c0);
      Frag E;
      init_e(E, lane);
      int e2 = 0;
      for (int k = 0; k < p.n; ++k, ++g) {
        const int s = int(g % NSTG);
        // one decision per warp: the MMAs below are warp-collective
        if (!__all_sync(0xffffffffu, !*abort_flag && mbar_wait_bounded(&full[s], u32((g / NSTG) & 1)))) {
          if (lane == 0) give_up();
          stop = true;
          break;
        }
        const u16* cur = smu + s * C::STAGE;
        pair_site<C::IL>(E, cur + wr * SBUF, cur + (TR + wc) * SBUF, lane);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (k == p.n - 1 || ((k & (RENORM_EVERY - 1)) == RENORM_EVERY - 1)) e2 += renorm(E);
      }
      if (stop) break;
      if (lane == 0) {
        const int i = r0 + wr, j = c0 + wc;
        float d2 = 0.0f, comp = 0.0f;
        if (p.need_kc && i < p.row0 + p.nrows && j < p.col0 + p.ncols) {
          const float* xa = p.x_r + size_t(i) * p.n;
          const float* xb = p.x_c + size_t(j) * p.n;
          for (int f = 0; f < p.n; ++f) kahan_add_sq(d2, comp, __ldg(xa + f) - __ldg(xb + f));
        }
        write_pair(p, half_log_mod(E, e2), d2, i, j);
      }
      __syncwarp();
    }
  }
  __syncthreads();
}

// ln|<psi~_i|psi~_i>| with the same split-BF16 arithmetic (one warp per sample).
__global__ void __launch_bounds__(32) self_overlap32_tc_kernel(const float* __restrict__ mps, int m, int n,
                                                               float* __restrict__ log_norm) {
  extern __shared__ __align__(16) u16 smu[];  // the sample's operands, row and column side alike
  const int lane = threadIdx.x;
  const int i = blockIdx.x;
  Frag E;
  init_e(E, lane);
  int e2 = 0;
  for (int k = 0; k < n; ++k) {
    const float* src = mps + (size_t(k) * m + i) * SAMPLE_FLOATS;
    for (int w = lane; w < CHUNKS; w += 32) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(src) + w);
      put_chunk(smu, w, v);
    }
    __syncwarp();
    pair_site<false>(E, smu, smu, lane);
    if (k == n - 1 || ((k & (RENORM_EVERY - 1)) == RENORM_EVERY - 1)) e2 += renorm(E);
    __syncwarp();
  }
  if (lane == 0) log_norm[i] = half_log_mod(E, e2);
}

// dk_mps_split32: the operands of sample-site u = k m + i (u < m n), one CTA of 128 threads
// per sample-site at a time (grid-stride): the 512 chunks split into a shared-memory copy
// of the operand layout with zeroed row padding, then written out in 16-byte pieces.
__global__ void __launch_bounds__(128) split32_kernel(const float* __restrict__ mps, long long units,
                                                      uint4* __restrict__ ops) {
  __shared__ __align__(16) u16 buf[SBUF];
  constexpr int PIECES = SBUF * int(sizeof(u16)) / 16;
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    for (int r = threadIdx.x; r < SBUF / ROW; r += blockDim.x)  // padding of every operand row
      *reinterpret_cast<uint4*>(buf + r * ROW + 32) = make_uint4(0u, 0u, 0u, 0u);
    const float4* src = reinterpret_cast<const float4*>(mps + size_t(u) * SAMPLE_FLOATS);
    for (int w = threadIdx.x; w < CHUNKS; w += blockDim.x) put_chunk(buf, w, __ldg(src + w));
    __syncthreads();
    const uint4* b4 = reinterpret_cast<const uint4*>(buf);
    for (int q = threadIdx.x; q < PIECES; q += blockDim.x) ops[size_t(u) * PIECES + q] = b4[q];
    __syncthreads();
  }
}

}  // namespace tc32

template <class C>
static dk_status gram32_tc_run(dk_ctx* ctx, const void* mps_r, int m_r, const void* mps_c, int m_c, GramArgs a,
                               cudaStream_t st) {
  a.ntiles = count_tiles(a, C::TR_, C::TC_);
  auto kern = tc32::gram32_tc_kernel<C>;
  // set before every launch: the attribute is per device and cheap to set
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM)) !=
      cudaSuccess)
    return DK_ERR_CUDA;
  long long grid = ctx->sm_count;
  if (grid > a.ntiles) grid = a.ntiles;
  if (grid < 1) return DK_OK;
  kern<<<int(grid), C::NT, C::SMEM, st>>>(static_cast<const float*>(mps_r), m_r, static_cast<const float*>(mps_c),
                                          m_c, a);
  return launch_status();
}

dk_status gram32_tc_launch(dk_ctx* ctx, const void* mps_r, int m_r, const void* mps_c, int m_c, GramArgs a,
                           bool presplit, cudaStream_t st) {
  // Measured fastest of the shapes and schedules that fit the registers (512 samples, d = 256):
  // split operands: 4 x 4 pairs, two stages, IL = false (16 pair warps at 96 registers;
  // 56.6 ms against 58.4 for 4 x 2); complex64 input: 4 x 2 pairs, three stages, IL = true
  // (the staging warps leave 168 registers for 8 pair warps; 4 x 3 tiles spill at 128).
  if (presplit) return gram32_tc_run<tc32::CfgTc<4, 4, 2, false, true>>(ctx, mps_r, m_r, mps_c, m_c, a, st);
  return gram32_tc_run<tc32::CfgTc<4, 2, 3, true, false>>(ctx, mps_r, m_r, mps_c, m_c, a, st);
}

dk_status self_overlap32_tc_launch(const void* mps, int m, int n, float* log_norm, cudaStream_t st) {
  const int smem = tc32::SBUF * 2;
  // set before every launch: the attribute is per device and cheap to set
  if (cudaFuncSetAttribute(tc32::self_overlap32_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
      cudaSuccess)
    return DK_ERR_CUDA;
  tc32::self_overlap32_tc_kernel<<<m, 32, smem, st>>>(static_cast<const float*>(mps), m, n, log_norm);
  return launch_status();
}

}  // namespace dk

DK_API dk_status dk_mps_split32(dk_ctx* ctx, const void* mps, int m, int n, void* ops, size_t ops_bytes,
                                void* stream) {
  using namespace dk;
  if (!ctx || !mps || !ops || m < 1 || n < 1) return DK_ERR_ARG;
  if (!aligned16(mps) || !aligned16(ops)) return DK_ERR_ARG;
  if (ops_bytes < size_t(m) * size_t(n) * site_bytes(32, DK_SPLIT_BF16)) return DK_ERR_WORKSPACE;
  const long long units = (long long)m * n;
  long long grid = (long long)ctx->sm_count * 16;
  if (grid > units) grid = units;
  tc32::split32_kernel<<<int(grid), 128, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<const float*>(mps),
                                                                                   units, static_cast<uint4*>(ops));
  return launch_status();
}
