// Transfer-chain Gram at bond 32 (reps = 5) on FP32 CUDA cores, one warp per pair.
//
// Same contraction as transfer.cuh (§II-C, Eqs. 8-10, block-structured): per site and
// pair, E'_s = sum_t A_s[t](x_i)^dagger E_t A_s[t](x_j) with h = 16, i.e. for each of the
// four (s, t) terms two complex 16 x 16 x 16 products
//     F = E_t B,  B = A_s[t](x_j);      E'_s += A_s[t](x_i)^dagger F.
// E (two 16 x 16 blocks) and F (one per s) live in shared memory per warp; the warp works on
// both s at once, each lane on a 4 x 4 complex tile of one block, so that every float read
// from shared memory feeds four FMAs (see pair_site). Per site the CTA stages the site tensors of its TR row samples
// (compact layout, rows padded to 272 B) and TC column samples (each 16 x 16 block
// transposed to row-major, rows padded to 144 B) into shared memory, double buffered: the
// next site's tensors are loaded into registers while the current site is contracted.
// Every 4 sites E is rescaled by a power of two (warp-wide max), as in transfer.cuh.
#include <math.h>

#include "common.cuh"
#include "gram_common.cuh"
#include "internal.h"
#include "transfer.cuh"

namespace dk {
namespace c32 {

constexpr int CHI = 32;
constexpr int SAMPLE_FLOATS = CHI * CHI * 2;        // compact site tensor, complex64
// Row-sample buffer: compact rows r = s*16 + j (32 of them), each 32 complex = 256 B, padded
// to 272 B (68 floats): consecutive rows start 4 banks apart, so the 8 rows a warp reads at
// once fall in 8 different 16-byte bank groups.
constexpr int AROW = 68;                             // floats per padded row
constexpr int ABUF = 32 * AROW;                      // floats per row sample
// Column-sample buffer: per (s, t) block a row-major 16 x 16 complex matrix B[b][c], rows
// padded to 144 B (36 floats).
constexpr int BROW = 36;
constexpr int BBLK = 16 * BROW;
constexpr int BBUF = 4 * BBLK;                       // floats per column sample
// Per-warp E (two blocks) and F, row-major, rows padded to 144 B.
constexpr int EBLK = 16 * BROW;

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// Stage one sample's compact site tensor (global, 1024 complex) as a row sample.
__device__ __forceinline__ void put_row_chunk(float* abuf, int chunk, float4 v) {
  // chunk c = 16-byte piece c of the 8 KB tensor: row r = c / 16, position (c % 16) * 4 floats
  const int r = chunk >> 4, q = chunk & 15;
  *reinterpret_cast<float4*>(abuf + r * AROW + q * 4) = v;
}
// ... and as a column sample: element (s, j=c, l = t*16 + b) goes to block (s, t), B[b][c].
__device__ __forceinline__ void put_col_chunk(float* bbuf, int chunk, float4 v) {
  const int r = chunk >> 4, q = chunk & 15;  // r = s*16 + c, elements l = 2q, 2q+1
  const int s = r >> 4, c = r & 15;
  const int l0 = 2 * q;
  const int t = l0 >> 4, b0 = l0 & 15;
  float* blk = bbuf + (s * 2 + t) * BBLK;
  *reinterpret_cast<float2*>(blk + b0 * BROW + 2 * c) = make_float2(v.x, v.y);
  *reinterpret_cast<float2*>(blk + (b0 + 1) * BROW + 2 * c) = make_float2(v.z, v.w);
}

// One site of one pair by one warp. ebuf: 2 blocks E_t (row-major, padded); fbuf: F_0, F_1.
// abuf: row sample (compact, padded rows); bbuf: column sample (transposed blocks).
// Lane L works on block s = L / 16 (both s at once: they read the same E_t) and owns rows
// rg, rg + 4, rg + 8, rg + 12 (the 16 lanes of a half read 4 consecutive rows at a time, in
// different banks), columns 4 cg .. 4 cg + 3 of it (rg = (L % 16) / 4, cg = L % 4): per k-step
// it reads 4 complex of E_t (or of the row sample) and 4 of B (or of F) for 16 complex
// multiply-adds, four FMAs per float read from shared memory, the rate at which the shared-
// memory pipe keeps the FMA pipe busy. acc receives E'_s = block s of the result; every
// entry sees the same additions in the same order as with any other split of the outputs.
__device__ __forceinline__ void pair_site(const float* ebuf, float* fbuf, const float* abuf, const float* bbuf,
                                          int lane, float (&accr)[4][4], float (&acci)[4][4]) {
  const int s = lane >> 4, rg = (lane >> 2) & 3, cg = lane & 3;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      accr[u][v] = 0.0f;
      acci[u][v] = 0.0f;
    }
  float* fs = fbuf + s * EBLK;
#pragma unroll 1
  for (int t = 0; t < 2; ++t) {
    const float* et = ebuf + t * EBLK;
    const float* bb = bbuf + (s * 2 + t) * BBLK;
    // F_s[a][c] = sum_b E_t[a][b] B[b][c], a = rg + 4u, c in 4cg .. 4cg+3
    float fr[4][4], fi[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        fr[u][v] = 0.0f;
        fi[u][v] = 0.0f;
      }
#pragma unroll 2
    for (int b2 = 0; b2 < 8; ++b2) {  // two b per step
      float4 e[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) e[u] = ld4(et + (rg + 4 * u) * BROW + 4 * b2);
#pragma unroll
      for (int bb_ = 0; bb_ < 2; ++bb_) {
        const int b = 2 * b2 + bb_;
        const float4 x0 = ld4(bb + b * BROW + 8 * cg);
        const float4 x1 = ld4(bb + b * BROW + 8 * cg + 4);
        const float br[4] = {x0.x, x0.z, x1.x, x1.z};
        const float bi[4] = {x0.y, x0.w, x1.y, x1.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float er = bb_ == 0 ? e[u].x : e[u].z;
          const float ei = bb_ == 0 ? e[u].y : e[u].w;
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            fr[u][v] = fmaf(er, br[v], fr[u][v]);
            fi[u][v] = fmaf(er, bi[v], fi[u][v]);
            fr[u][v] = fmaf(-ei, bi[v], fr[u][v]);
            fi[u][v] = fmaf(ei, br[v], fi[u][v]);
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      float* fp = fs + (rg + 4 * u) * BROW + 8 * cg;
      *reinterpret_cast<float4*>(fp) = make_float4(fr[u][0], fi[u][0], fr[u][1], fi[u][1]);
      *reinterpret_cast<float4*>(fp + 4) = make_float4(fr[u][2], fi[u][2], fr[u][3], fi[u][3]);
    }
    __syncwarp();
    // E'_s[p][c] += sum_a conj(A_s[t][a][p]) F_s[a][c], p = rg + 4u: row p of the
    // compact tensor at block s, positions t*16 + a.
    const float* ar = abuf + (s * 16 + rg) * AROW + t * 32;
#pragma unroll 2
    for (int a2 = 0; a2 < 8; ++a2) {
      float4 y[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) y[u] = ld4(ar + 4 * u * AROW + 4 * a2);
#pragma unroll
      for (int aa = 0; aa < 2; ++aa) {
        const int a = 2 * a2 + aa;
        const float4 f0 = ld4(fs + a * BROW + 8 * cg);
        const float4 f1 = ld4(fs + a * BROW + 8 * cg + 4);
        const float gr[4] = {f0.x, f0.z, f1.x, f1.z};
        const float gi[4] = {f0.y, f0.w, f1.y, f1.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float cr = aa == 0 ? y[u].x : y[u].z;
          const float ci = aa == 0 ? y[u].y : y[u].w;
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            accr[u][v] = fmaf(cr, gr[v], accr[u][v]);
            acci[u][v] = fmaf(cr, gi[v], acci[u][v]);
            accr[u][v] = fmaf(ci, gi[v], accr[u][v]);
            acci[u][v] = fmaf(-ci, gr[v], acci[u][v]);
          }
        }
      }
    }
    __syncwarp();
  }
}

// Write E := diag(acc_0, acc_1) (block s from the lanes of half s), rescaling by a power of
// two when asked; returns the exponent taken out (warp-uniform).
__device__ __forceinline__ int store_e(float* ebuf, int lane, float (&accr)[4][4], float (&acci)[4][4],
                                       bool renorm) {
  const int s = lane >> 4, rg = (lane >> 2) & 3, cg = lane & 3;
  int e = 0;
  if (renorm) {
    float mx = 0.0f;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) mx = fmaxf(mx, fmaxf(fabsf(accr[u][v]), fabsf(acci[u][v])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    e = RealBits<float>::exponent(mx);
    const float sc = RealBits<float>::pow2_neg(e);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        accr[u][v] *= sc;
        acci[u][v] *= sc;
      }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    float* ep = ebuf + s * EBLK + (rg + 4 * u) * BROW + 8 * cg;
    *reinterpret_cast<float4*>(ep) = make_float4(accr[u][0], acci[u][0], accr[u][1], acci[u][1]);
    *reinterpret_cast<float4*>(ep + 4) = make_float4(accr[u][2], acci[u][2], accr[u][3], acci[u][3]);
  }
  __syncwarp();
  return e;
}

__device__ __forceinline__ void init_e(float* ebuf, int lane) {
  for (int i = lane; i < 2 * EBLK; i += 32) ebuf[i] = 0.0f;
  __syncwarp();
  if (lane == 0) ebuf[0] = 1.0f;
  __syncwarp();
}

// ln|a|, a = E_0[0][0] + E_1[0][0] (after the last site), as in transfer.cuh.
__device__ __forceinline__ float half_log_mod(const float* ebuf, int e2) {
  const float re = ebuf[0] + ebuf[EBLK];
  const float im = ebuf[1] + ebuf[EBLK + 1];
  const float mod2 = fmaf(re, re, im * im);
  return fmaf(0.5f, logf(mod2), float(e2) * 0.69314718055994530942f);
}

template <int TR, int TC>
struct Cfg32 {
  static constexpr int NW = TR * TC, NT = NW * 32;
  static constexpr int STAGE = TR * ABUF + TC * BBUF;                 // floats per stage
  static constexpr int CHUNKS = (TR + TC) * (SAMPLE_FLOATS / 4);        // 16-byte chunks per stage
  static constexpr int PER_THREAD = (CHUNKS + NT - 1) / NT;
  static constexpr int SMEM = (2 * STAGE + NW * 4 * EBLK) * 4;  // + per warp E (2 blocks), F (2 blocks)
};

template <int TR, int TC>
__global__ void __launch_bounds__(TR * TC * 32, 1)
    gram32_f32_kernel(const float* __restrict__ mps_r, int m_r, const float* __restrict__ mps_c, int m_c,
                      const GramArgs p) {
  using C = Cfg32<TR, TC>;
  extern __shared__ __align__(16) float sm[];
  float* stage[2] = {sm, sm + C::STAGE};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* ebuf = sm + 2 * C::STAGE + warp * 4 * EBLK;
  float* fbuf = ebuf + 2 * EBLK;
  const int wr = warp / TC, wc = warp % TC;

  float4 pre[C::PER_THREAD];
  auto fetch = [&](int r0, int c0, int k) {  // site k of the tile at (r0, c0) into registers
#pragma unroll
    for (int q = 0; q < C::PER_THREAD; ++q) {
      const int ch = threadIdx.x + q * C::NT;
      if (ch < C::CHUNKS) {
        const int smp = ch / (SAMPLE_FLOATS / 4), part = ch % (SAMPLE_FLOATS / 4);
        const bool is_row = smp < TR;
        const int idx = is_row ? min(r0 + smp, m_r - 1) : min(c0 + smp - TR, m_c - 1);
        const float* src = (is_row ? mps_r + (size_t(k) * m_r + idx) * SAMPLE_FLOATS
                                   : mps_c + (size_t(k) * m_c + idx) * SAMPLE_FLOATS) + part * 4;
        pre[q] = __ldg(reinterpret_cast<const float4*>(src));
      }
    }
  };
  auto commit = [&](float* st) {
#pragma unroll
    for (int q = 0; q < C::PER_THREAD; ++q) {
      const int ch = threadIdx.x + q * C::NT;
      if (ch < C::CHUNKS) {
        const int smp = ch / (SAMPLE_FLOATS / 4), part = ch % (SAMPLE_FLOATS / 4);
        if (smp < TR) put_row_chunk(st + smp * ABUF, part, pre[q]);
        else put_col_chunk(st + TR * ABUF + (smp - TR) * BBUF, part, pre[q]);
      }
    }
  };

  const int my_tiles = (p.ntiles > int(blockIdx.x)) ? (p.ntiles - 1 - int(blockIdx.x)) / int(gridDim.x) + 1 : 0;
  for (int lt = 0; lt < my_tiles; ++lt) {
    int ti, tj;
    decode_tile(p, TR, TC, int(blockIdx.x) + lt * int(gridDim.x), ti, tj);
    const int r0 = p.row0 + ti * TR, c0 = p.col0 + tj * TC;
    init_e(ebuf, lane);
    int e2 = 0;
    fetch(r0, c0, 0);
    __syncthreads();
    commit(stage[0]);
    __syncthreads();
    for (int k = 0; k < p.n; ++k) {
      float* cur = stage[k & 1];
      if (k + 1 < p.n) fetch(r0, c0, k + 1);
      float accr[4][4], acci[4][4];
      pair_site(ebuf, fbuf, cur + wr * ABUF, cur + TR * ABUF + wc * BBUF, lane, accr, acci);
      const bool rn = (k == p.n - 1) || ((k & (RENORM_EVERY - 1)) == RENORM_EVERY - 1);
      e2 += store_e(ebuf, lane, accr, acci, rn);
      if (k + 1 < p.n) commit(stage[(k + 1) & 1]);
      __syncthreads();
    }
    if (lane == 0) {
      const int i = r0 + wr, j = c0 + wc;
      // K_c: ||x_i - x_j||^2 by one lane with the shared epilogue's compensated sum
      float d2 = 0.0f, comp = 0.0f;
      if (p.need_kc && i < p.row0 + p.nrows && j < p.col0 + p.ncols) {
        const float* xa = p.x_r + size_t(i) * p.n;
        const float* xb = p.x_c + size_t(j) * p.n;
        for (int f = 0; f < p.n; ++f) kahan_add_sq(d2, comp, __ldg(xa + f) - __ldg(xb + f));
      }
      write_pair(p, half_log_mod(ebuf, e2), d2, i, j);
    }
    __syncwarp();
  }
}

// ln|<psi~_i|psi~_i>| with exactly the pair arithmetic above (one warp per sample).
__global__ void __launch_bounds__(32) self_overlap32_kernel(const float* __restrict__ mps, int m, int n,
                                                            float* __restrict__ log_norm) {
  extern __shared__ __align__(16) float sm[];
  float* abuf = sm;
  float* bbuf = abuf + ABUF;
  float* ebuf = bbuf + BBUF;
  float* fbuf = ebuf + 2 * EBLK;
  const int lane = threadIdx.x;
  const int i = blockIdx.x;
  init_e(ebuf, lane);
  int e2 = 0;
  for (int k = 0; k < n; ++k) {
    const float* src = mps + (size_t(k) * m + i) * SAMPLE_FLOATS;
    for (int ch = lane; ch < SAMPLE_FLOATS / 4; ch += 32) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(src) + ch);
      put_row_chunk(abuf, ch, v);
      put_col_chunk(bbuf, ch, v);
    }
    __syncwarp();
    float accr[4][4], acci[4][4];
    pair_site(ebuf, fbuf, abuf, bbuf, lane, accr, acci);
    const bool rn = (k == n - 1) || ((k & (RENORM_EVERY - 1)) == RENORM_EVERY - 1);
    e2 += store_e(ebuf, lane, accr, acci, rn);
  }
  if (lane == 0) log_norm[i] = half_log_mod(ebuf, e2);
}

}  // namespace c32

dk_status gram32_launch(dk_ctx* ctx, const void* mps_r, int m_r, const void* mps_c, int m_c, GramArgs a,
                        cudaStream_t st) {
  constexpr int TR = 2, TC = 4;
  using C = c32::Cfg32<TR, TC>;
  a.ntiles = count_tiles(a, TR, TC);
  auto kern = c32::gram32_f32_kernel<TR, TC>;
  // set before every launch: the attribute is per device and cheap to set
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) !=
      cudaSuccess)
    return DK_ERR_CUDA;
  long long grid = ctx->sm_count;
  if (grid > a.ntiles) grid = a.ntiles;
  if (grid < 1) return DK_OK;
  kern<<<int(grid), C::NT, C::SMEM, st>>>(static_cast<const float*>(mps_r), m_r, static_cast<const float*>(mps_c),
                                          m_c, a);
  return launch_status();
}

dk_status self_overlap32_launch(const void* mps, int m, int n, float* log_norm, cudaStream_t st) {
  const int smem = (c32::ABUF + c32::BBUF + 4 * c32::EBLK) * 4;
  // set before every launch: the attribute is per device and cheap to set
  if (cudaFuncSetAttribute(c32::self_overlap32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
      cudaSuccess)
    return DK_ERR_CUDA;
  c32::self_overlap32_kernel<<<m, 32, smem, st>>>(static_cast<const float*>(mps), m, n, log_norm);
  return launch_status();
}

}  // namespace dk
