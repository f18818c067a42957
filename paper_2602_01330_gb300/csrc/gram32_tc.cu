// Bond-32 transfer-chain Gram on tensor cores with split-BF16 operands (bf16x3).
//
// Same contraction as gram32.cu (§II-C, Eqs. 8-10, block-structured, h = 16): per site,
// pair and (s, t), G = E_t B with B = A_s[t](x_j), then E'_s += C G with C = A_s[t](x_i)^dagger.
// Each complex 16 x 16 x 16 product is one real GEMM of the block form
//     [Xr | Xi] (16 x 32) . [[Yr, Yi], [-Yi, Yr]] (32 x 32) = [Zr | Zi] (16 x 32),
// run as m16n8k16 BF16 MMAs with FP32 accumulation. Every FP32 operand v is split into
// v = hi + lo (both BF16) and each product is hi.hi + hi.lo + lo.hi (bf16x3), which keeps
// about 16 significant bits per product; the lo.lo term is dropped.
//
// Dataflow: one warp per pair. E (two 16 x 16 blocks) stays in MMA accumulator fragments
// across sites; an accumulator tile converts directly into the A fragment of the next
// product (the fragment layouts coincide), so step 1 needs no memory traffic for E. The
// step-1 result G is the B operand of step 2 and goes through a per-warp shared buffer
// (transposed by ldmatrix). The CTA stages, per site and double buffered, its row samples
// as C operands and its column samples as B operands, both split into BF16 hi / lo.
#include <cuda_bf16.h>
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
constexpr int COP = 16 * ROW;                // one C operand (16 x 32) in u16
constexpr int BOP = 32 * ROW;                // one B operand (32 x 32) in u16
// Row sample: C operands hi and lo for the 4 (s, t) blocks; column sample: B operands.
constexpr int RBUF = 4 * 2 * COP;            // u16 per row sample
constexpr int CBUF = 4 * 2 * BOP;            // u16 per column sample
constexpr int GBUF = 2 * BOP;                // per-warp G operand, hi and lo

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

__device__ __forceinline__ void ldsm_x4_t(u32 (&r)[4], const u16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}

// (x, y) -> packed BF16 pairs hi and lo with x ~ hi + lo (low half = x).
__device__ __forceinline__ void split2(float x, float y, u32& hi, u32& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x - hf.x, y - hf.y);
  hi = *reinterpret_cast<const u32*>(&h);
  lo = *reinterpret_cast<const u32*>(&l);
}
__device__ __forceinline__ void split1(float x, u16& hi, u16& lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
  hi = *reinterpret_cast<const u16*>(&h);
  lo = *reinterpret_cast<const u16*>(&l);
}
constexpr u32 NEG2 = 0x80008000u;  // flips the sign of both BF16 halves

// Row sample, block (s, t): C[p][k] = Re A[k][p] (k < 16), -Im A[k-16][p] (k >= 16), where
// A[a][p] is compact element (s, j = p, l = 16 t + a). A 16-byte chunk holds elements
// l, l+1 of compact row r = 16 s + p.
__device__ __forceinline__ void put_row_chunk(u16* rbuf, int chunk, float4 v) {
  const int r = chunk >> 4, q = chunk & 15;
  const int s = r >> 4, p = r & 15;
  const int l = 2 * q, t = l >> 4, a = l & 15;
  u16* hi = rbuf + (s * 2 + t) * 2 * COP;
  u16* lo = hi + COP;
  u32 h, w;
  split2(v.x, v.z, h, w);  // Re at a, a+1
  *reinterpret_cast<u32*>(hi + p * ROW + a) = h;
  *reinterpret_cast<u32*>(lo + p * ROW + a) = w;
  split2(v.y, v.w, h, w);  // Im at a, a+1 -> -Im
  *reinterpret_cast<u32*>(hi + p * ROW + 16 + a) = h ^ NEG2;
  *reinterpret_cast<u32*>(lo + p * ROW + 16 + a) = w ^ NEG2;
}

// Column sample, block (s, t): B[b][c] = compact (s, j = c, l = 16 t + b); the operand is
// [[Br, Bi], [-Bi, Br]] (32 x 32). A chunk holds b, b+1 of compact row r = 16 s + c.
// Work item w of a column sample handles chunk col_chunk(w): consecutive items walk the 32
// compact rows (consecutive columns c of the operand) first, so a warp's 16-bit stores
// land in consecutive banks.
__device__ __forceinline__ int col_chunk(int w) { return (w & 31) * 16 + (w >> 5); }
__device__ __forceinline__ void put_col_chunk(u16* cbuf, int chunk, float4 v) {
  const int r = chunk >> 4, q = chunk & 15;
  const int s = r >> 4, c = r & 15;
  const int l = 2 * q, t = l >> 4, b = l & 15;
  u16* hi = cbuf + (s * 2 + t) * 2 * BOP;
  u16* lo = hi + BOP;
  const float re[2] = {v.x, v.z}, im[2] = {v.y, v.w};
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    u16 rh, rl, ih, il;
    split1(re[e], rh, rl);
    split1(im[e], ih, il);
    const int k = b + e;
    hi[k * ROW + c] = rh;
    lo[k * ROW + c] = rl;
    hi[k * ROW + 16 + c] = ih;
    lo[k * ROW + 16 + c] = il;
    hi[(16 + k) * ROW + c] = ih ^ 0x8000u;
    lo[(16 + k) * ROW + c] = il ^ 0x8000u;
    hi[(16 + k) * ROW + 16 + c] = rh;
    lo[(16 + k) * ROW + 16 + c] = rl;
  }
}

// Fragment state of one pair: e[t][nt][4], nt 0..1 = real part columns 0-7 / 8-15,
// nt 2..3 = imaginary part (m16n8 accumulator layout).
struct Frag {
  float v[2][4][4];
};

// acc += X . Yop with X given as 16 x 32 A fragments (hi/lo per k-step) and Yop a 32 x 32
// row-major BF16 operand in shared memory (hi, lo), for the 4 n-tiles. The MMAs are issued
// term-major over the four independent n-tile accumulators, so consecutive MMAs never wait
// on each other.
__device__ __forceinline__ void gemm_16x32x32(float (&acc)[4][4], const u32 (&ahi)[2][4], const u32 (&alo)[2][4],
                                              const u16* yhi, const u16* ylo, int lane) {
  // ldmatrix.trans lane address: tile (k half, n tile) rows = 16 kk + 8 (sel & 1) + (lane & 7)
  const int lr = lane & 7, sel = lane >> 3;  // sel: 0 (k 0-7, nt), 1 (k 8-15, nt), 2 (k 0-7, nt+1), 3
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    u32 bh[2][4], bl[2][4];
#pragma unroll
    for (int np = 0; np < 2; ++np) {  // pairs of n-tiles (2np, 2np+1)
      const int krow = 16 * kk + 8 * (sel & 1) + lr;
      const int ncol = 16 * np + 8 * (sel >> 1);
      ldsm_x4_t(bh[np], yhi + krow * ROW + ncol);
      ldsm_x4_t(bl[np], ylo + krow * ROW + ncol);
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) mma16816(acc[nt], alo[kk], bh[nt >> 1][2 * (nt & 1)], bh[nt >> 1][2 * (nt & 1) + 1]);
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) mma16816(acc[nt], ahi[kk], bl[nt >> 1][2 * (nt & 1)], bl[nt >> 1][2 * (nt & 1) + 1]);
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) mma16816(acc[nt], ahi[kk], bh[nt >> 1][2 * (nt & 1)], bh[nt >> 1][2 * (nt & 1) + 1]);
  }
}

// One site of one pair (warp). rbuf: row-sample C operands; cbuf: column-sample B
// operands; gbuf: this warp's G operand buffer. E is replaced by diag(acc_0, acc_1).
__device__ __forceinline__ void pair_site(Frag& E, const u16* rbuf, const u16* cbuf, u16* gbuf, int lane) {
  const int g = lane >> 2, tq = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[s][nt][c] = 0.0f;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    // A fragments of [Er | Ei] for E_t: k-step 0 = Er (n-tiles 0, 1), k-step 1 = Ei (2, 3)
    u32 ahi[2][4], alo[2][4];
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      const float(&x0)[4] = E.v[t][2 * kk];
      const float(&x1)[4] = E.v[t][2 * kk + 1];
      split2(x0[0], x0[1], ahi[kk][0], alo[kk][0]);
      split2(x0[2], x0[3], ahi[kk][1], alo[kk][1]);
      split2(x1[0], x1[1], ahi[kk][2], alo[kk][2]);
      split2(x1[2], x1[3], ahi[kk][3], alo[kk][3]);
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      // step 1: G = [Er | Ei] . [[Br, Bi], [-Bi, Br]]
      float gacc[4][4];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int c = 0; c < 4; ++c) gacc[nt][c] = 0.0f;
      const u16* bh = cbuf + (s * 2 + t) * 2 * BOP;
      gemm_16x32x32(gacc, ahi, alo, bh, bh + BOP, lane);
      // G operand [[Gr, Gi], [-Gi, Gr]] into the warp buffer (hi, lo)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int col = 8 * nt + 2 * tq;
        u32 h0, l0, h1, l1;
        split2(gacc[nt][0], gacc[nt][1], h0, l0);  // row g
        split2(gacc[nt][2], gacc[nt][3], h1, l1);  // row g + 8
        *reinterpret_cast<u32*>(gbuf + g * ROW + col) = h0;
        *reinterpret_cast<u32*>(gbuf + BOP + g * ROW + col) = l0;
        *reinterpret_cast<u32*>(gbuf + (g + 8) * ROW + col) = h1;
        *reinterpret_cast<u32*>(gbuf + BOP + (g + 8) * ROW + col) = l1;
        // lower half: Gr block (nt 0,1) moves right, Gi block (nt 2,3) moves left negated
        const int col2 = nt < 2 ? col + 16 : col - 16;
        const u32 sg = nt < 2 ? 0u : NEG2;
        *reinterpret_cast<u32*>(gbuf + (16 + g) * ROW + col2) = h0 ^ sg;
        *reinterpret_cast<u32*>(gbuf + BOP + (16 + g) * ROW + col2) = l0 ^ sg;
        *reinterpret_cast<u32*>(gbuf + (24 + g) * ROW + col2) = h1 ^ sg;
        *reinterpret_cast<u32*>(gbuf + BOP + (24 + g) * ROW + col2) = l1 ^ sg;
      }
      __syncwarp();
      // step 2: acc_s += [Cr | Ci] . [[Gr, Gi], [-Gi, Gr]]
      u32 chi[2][4], clo[2][4];
      const u16* ch = rbuf + (s * 2 + t) * 2 * COP;
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const u16* rowp = ch + (lane & 15) * ROW + 16 * kk + 8 * (lane >> 4);
        ldsm_x4(chi[kk], rowp);
        ldsm_x4(clo[kk], rowp + COP);
      }
      gemm_16x32x32(acc[s], chi, clo, gbuf, gbuf + BOP, lane);
      __syncwarp();
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

template <int TR, int TC>
struct CfgTc {
  static constexpr int NW = TR * TC, NT = NW * 32;
  static constexpr int STAGE = TR * RBUF + TC * CBUF;  // u16 per stage
  static constexpr int CH = (TR + TC) * CHUNKS;
  static constexpr int PER_THREAD = (CH + NT - 1) / NT;
  static constexpr int SMEM = (2 * STAGE + NW * GBUF) * 2;
};

template <int TR, int TC>
__global__ void __launch_bounds__(TR * TC * 32, 1)
    gram32_tc_kernel(const float* __restrict__ mps_r, int m_r, const float* __restrict__ mps_c, int m_c,
                     const GramArgs p) {
  using C = CfgTc<TR, TC>;
  extern __shared__ __align__(16) u16 smu[];
  u16* stage[2] = {smu, smu + C::STAGE};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  u16* gbuf = smu + 2 * C::STAGE + warp * GBUF;
  const int wr = warp / TC, wc = warp % TC;

  float4 pre[C::PER_THREAD];
  auto fetch = [&](int r0, int c0, int k) {
#pragma unroll
    for (int q = 0; q < C::PER_THREAD; ++q) {
      const int ch = threadIdx.x + q * C::NT;
      if (ch < C::CH) {
        const int smp = ch / CHUNKS, w = ch % CHUNKS;
        const bool is_row = smp < TR;
        const int part = is_row ? w : col_chunk(w);
        const int idx = is_row ? min(r0 + smp, m_r - 1) : min(c0 + smp - TR, m_c - 1);
        const float* src = (is_row ? mps_r + (size_t(k) * m_r + idx) * SAMPLE_FLOATS
                                   : mps_c + (size_t(k) * m_c + idx) * SAMPLE_FLOATS) + part * 4;
        pre[q] = __ldg(reinterpret_cast<const float4*>(src));
      }
    }
  };
  auto commit = [&](u16* st) {
#pragma unroll
    for (int q = 0; q < C::PER_THREAD; ++q) {
      const int ch = threadIdx.x + q * C::NT;
      if (ch < C::CH) {
        const int smp = ch / CHUNKS, w = ch % CHUNKS;
        if (smp < TR) put_row_chunk(st + smp * RBUF, w, pre[q]);
        else put_col_chunk(st + TR * RBUF + (smp - TR) * CBUF, col_chunk(w), pre[q]);
      }
    }
  };

  const int my_tiles = (p.ntiles > int(blockIdx.x)) ? (p.ntiles - 1 - int(blockIdx.x)) / int(gridDim.x) + 1 : 0;
  for (int lt = 0; lt < my_tiles; ++lt) {
    int ti, tj;
    decode_tile(p, TR, TC, int(blockIdx.x) + lt * int(gridDim.x), ti, tj);
    const int r0 = p.row0 + ti * TR, c0 = p.col0 + tj * TC;
    Frag E;
    init_e(E, lane);
    int e2 = 0;
    fetch(r0, c0, 0);
    __syncthreads();
    commit(stage[0]);
    __syncthreads();
    for (int k = 0; k < p.n; ++k) {
      u16* cur = stage[k & 1];
      if (k + 1 < p.n) fetch(r0, c0, k + 1);
      pair_site(E, cur + wr * RBUF, cur + TR * RBUF + wc * CBUF, gbuf, lane);
      if (k == p.n - 1 || ((k & (RENORM_EVERY - 1)) == RENORM_EVERY - 1)) e2 += renorm(E);
      if (k + 1 < p.n) commit(stage[(k + 1) & 1]);
      __syncthreads();
    }
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

// ln|<psi~_i|psi~_i>| with the same split-BF16 arithmetic (one warp per sample).
__global__ void __launch_bounds__(32) self_overlap32_tc_kernel(const float* __restrict__ mps, int m, int n,
                                                               float* __restrict__ log_norm) {
  extern __shared__ __align__(16) u16 smu[];
  u16* rbuf = smu;
  u16* cbuf = rbuf + RBUF;
  u16* gbuf = cbuf + CBUF;
  const int lane = threadIdx.x;
  const int i = blockIdx.x;
  Frag E;
  init_e(E, lane);
  int e2 = 0;
  for (int k = 0; k < n; ++k) {
    const float* src = mps + (size_t(k) * m + i) * SAMPLE_FLOATS;
    for (int w = lane; w < CHUNKS; w += 32) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(src) + w);
      put_row_chunk(rbuf, w, v);
      const int cw = col_chunk(w);
      put_col_chunk(cbuf, cw, __ldg(reinterpret_cast<const float4*>(src) + cw));
    }
    __syncwarp();
    pair_site(E, rbuf, cbuf, gbuf, lane);
    if (k == n - 1 || ((k & (RENORM_EVERY - 1)) == RENORM_EVERY - 1)) e2 += renorm(E);
    __syncwarp();
  }
  if (lane == 0) log_norm[i] = half_log_mod(E, e2);
}

}  // namespace tc32

dk_status gram32_tc_launch(dk_ctx* ctx, const void* mps_r, int m_r, const void* mps_c, int m_c, GramArgs a,
                           cudaStream_t st) {
  constexpr int TR = 4, TC = 2;
  using C = tc32::CfgTc<TR, TC>;
  a.ntiles = count_tiles(a, TR, TC);
  auto kern = tc32::gram32_tc_kernel<TR, TC>;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) != cudaSuccess)
      return DK_ERR_CUDA;
    attr = true;
  }
  long long grid = ctx->sm_count;
  if (grid > a.ntiles) grid = a.ntiles;
  if (grid < 1) return DK_OK;
  kern<<<int(grid), C::NT, C::SMEM, st>>>(static_cast<const float*>(mps_r), m_r, static_cast<const float*>(mps_c),
                                          m_c, a);
  return launch_status();
}

dk_status self_overlap32_tc_launch(const void* mps, int m, int n, float* log_norm, cudaStream_t st) {
  const int smem = (tc32::RBUF + tc32::CBUF + tc32::GBUF) * 2;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(tc32::self_overlap32_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
      return DK_ERR_CUDA;
    attr = true;
  }
  tc32::self_overlap32_tc_kernel<<<m, 32, smem, st>>>(static_cast<const float*>(mps), m, n, log_norm);
  return launch_status();
}

}  // namespace dk
