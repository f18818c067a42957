// Block-statevector Gram (see gram_blocks.cu) on tensor cores with split-BF16 operands.
//
// For a block product state the overlap factorises over the blocks, and each factor
// G_B(i, j) = sum_k conj(a_i[k]) b_j[k] over the 2^b amplitudes is one element of a dense
// complex matrix product: over a tile of row and column samples, a GEMM with K = 2^b. Here
//   Re G = sum ar br + ai bi,   Im G = sum ar bi - ai br
// run as mma.sync m16n8k16 BF16 products with FP32 accumulation, every FP32 amplitude v
// split as v ~ hi + lo (both BF16, |v - hi - lo| <= 2^-18 |v|) and each product taken as
// lo.hi + hi.lo + hi.hi (bf16x3; the lo.lo term is dropped), so a product keeps about 17
// significant bits.
//
// Layout: dk_block_states in this precision stores, per (block, sample) and chunk of 16
// amplitudes, one 128-byte row of four BF16 planes [hi_re | hi_im | lo_re | lo_im] (8 bytes
// per amplitude, as complex64).
// A CTA computes a 128 x 64 pair tile with 8 warps (4 x 2, 32 x 32 pairs each); per
// 16-amplitude step the operand rows of its 192 samples (4 planes x 32 bytes each) are
// copied with cp.async into a double-buffered stage, padded to 144 bytes per row so the
// ldmatrix reads of 8 rows hit 8 different 16-byte bank groups. After the last step of a
// block each pair adds log2 |G_B|^2 to its running sum in shared memory; the epilogue is the
// common one (write_pair). The self-norms come from a small kernel that issues, element by
// element, the same MMA sequence (block_selfnorm_tc_kernel), so K_q(x, x) = 1 exactly.
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"
#include "gram_common.cuh"
#include "internal.h"

namespace dk {
namespace gbtc {

using u16 = uint16_t;
using u32 = uint32_t;

constexpr int KC = 16;                 // complex amplitudes per step (one k16 per plane)
constexpr int TC = 64;                 // pair tile: (32 WM) rows x 64 columns
constexpr int ROWB = 144;              // staged sample row: 4 planes x 32 B + 16 B pad
constexpr int NSLOT = 32;              // pairs per thread
// WM warps along the rows (4: 128 x 64 tiles, 8 warps; 2: 64 x 64 tiles, 4 warps), 2 along
// the columns, each warp 32 x 32 pairs
template <int WM>
struct TileCfg {
  static constexpr int TR = 32 * WM, NT = 64 * WM;
  static constexpr int STAGE_A = TR * ROWB, STAGE = (TR + TC) * ROWB;
  static constexpr int COPIES = (TR + TC) * 8 / NT;  // 16-byte copies per thread per stage
  static constexpr size_t SMEM = 2 * STAGE + size_t(NSLOT) * NT * sizeof(float);
};
// self-norm kernel: 16 samples per warp
constexpr int STAGE_N = 16 * ROWB;
constexpr u32 NEG2 = 0x80008000u;      // flips the sign of both BF16 halves

__device__ __forceinline__ void mma16816(float (&d)[4], const u32 (&a)[4], u32 b0, u32 b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(u32 (&r)[4], u32 addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

__device__ __forceinline__ void cp_async16(u32 dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void lg_add(float& lg, float re, float im) { lg += log2f(fmaf(re, re, im * im)); }
__device__ __forceinline__ float half_log_lg(float lg) { return lg * (0.5f * 0.69314718055994530942f); }

// The Gram block of p (symmetric or rectangular), p.ntiles tiles of TR x 64 pairs.
template <int WM>
__global__ void __launch_bounds__(64 * WM, 8 / WM)
    gram_blocks_tc_kernel(const unsigned char* __restrict__ sr, int m_r, const unsigned char* __restrict__ sc,
                          int m_c, int nb, int dp, const GramArgs p) {
  using T = TileCfg<WM>;
  constexpr int TR = T::TR, NT = T::NT, STAGE = T::STAGE, STAGE_A = T::STAGE_A;
  extern __shared__ __align__(128) unsigned char smem[];
  float* s_lg = reinterpret_cast<float*>(smem + 2 * STAGE);
  const u32 sbase = smem_u32(smem);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;
  const int g = lane >> 2, t4 = lane & 3;
  const int cpb = dp / KC, total = nb * cpb;
  const size_t sample_bytes = size_t(dp) * 8;  // four BF16 planes of dp values
  // ldmatrix lane offsets inside a stage (bytes): A (rows x k) and B (columns x k)
  const int a_row = (lane & 7) + 8 * ((lane >> 3) & 1), a_k = 8 * (lane >> 4);
  const int b_row = (lane & 7) + 8 * (lane >> 4), b_k = 8 * ((lane >> 3) & 1);
  for (int t = blockIdx.x; t < p.ntiles; t += gridDim.x) {
    int ti, tj;
    decode_tile(p, TR, TC, t, ti, tj);
    const int r0 = p.row0 + ti * TR, c0 = p.col0 + tj * TC;
    // stage loader: (TR + 64) rows x 8 pieces of 16 B
    auto issue = [&](int c, int buf) {
      const int blk = c / cpb, k0 = (c - blk * cpb) * KC;
#pragma unroll
      for (int h = 0; h < T::COPIES; ++h) {
        const int q = tid + NT * h;
        const int row = q >> 3, piece = q & 7;
        const bool is_a = row < TR;
        const int smp = is_a ? min(r0 + row, m_r - 1) : min(c0 + row - TR, m_c - 1);
        const unsigned char* src = (is_a ? sr + (size_t(blk) * m_r + smp) * sample_bytes
                                         : sc + (size_t(blk) * m_c + smp) * sample_bytes) +
                                   size_t(k0) * 8 + piece * 16;
        cp_async16(sbase + buf * STAGE + row * ROWB + piece * 16, src);
      }
      cp_async_commit();
    };
    float re[2][4][4], im[2][4][4];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v)
#pragma unroll
        for (int e = 0; e < 4; ++e) re[u][v][e] = im[u][v][e] = 0.0f;
    for (int s = 0; s < NSLOT; ++s) s_lg[s * NT + tid] = 0.0f;
    issue(0, 0);
    for (int c = 0; c < total; ++c) {
      const int buf = c & 1;
      if (c + 1 < total) {
        issue(c + 1, buf ^ 1);
        cp_async_wait_1();
      } else {
        cp_async_wait_0();
      }
      __syncthreads();
      const u32 sa = sbase + buf * STAGE, sb = sa + STAGE_A;
      // B fragments of the warp's 4 column tiles for the 4 planes: bf[plane][tile][2]
      u32 bf[4][4][2];
#pragma unroll
      for (int pl = 0; pl < 4; ++pl)
#pragma unroll
        for (int np = 0; np < 2; ++np) {
          u32 r[4];
          ldsm_x4(r, sb + (wn * 32 + np * 16 + b_row) * ROWB + pl * 32 + b_k * 2);
          bf[pl][2 * np][0] = r[0];
          bf[pl][2 * np][1] = r[1];
          bf[pl][2 * np + 1][0] = r[2];
          bf[pl][2 * np + 1][1] = r[3];
        }
      // real parts of the row amplitudes (planes 0 hi, 2 lo), then imaginary (1 hi, 3 lo)
#pragma unroll
      for (int part = 0; part < 2; ++part) {
        u32 ahi[2][4], alo[2][4];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const u32 addr = sa + (wm * 32 + u * 16 + a_row) * ROWB + a_k * 2;
          ldsm_x4(ahi[u], addr + part * 32);
          ldsm_x4(alo[u], addr + (2 + part) * 32);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            // part 0 (ar): re += ar br, im += ar bi;  part 1 (ai): re += ai bi, im -= ai br
            const int pr_hi = part ? 1 : 0, pr_lo = part ? 3 : 2;  // plane feeding re
            const int pi_hi = part ? 0 : 1, pi_lo = part ? 2 : 3;  // plane feeding im
            const u32 sg = part ? NEG2 : 0u;                        // - ai br
            mma16816(re[u][v], alo[u], bf[pr_hi][v][0], bf[pr_hi][v][1]);
            mma16816(re[u][v], ahi[u], bf[pr_lo][v][0], bf[pr_lo][v][1]);
            mma16816(re[u][v], ahi[u], bf[pr_hi][v][0], bf[pr_hi][v][1]);
            mma16816(im[u][v], alo[u], bf[pi_hi][v][0] ^ sg, bf[pi_hi][v][1] ^ sg);
            mma16816(im[u][v], ahi[u], bf[pi_lo][v][0] ^ sg, bf[pi_lo][v][1] ^ sg);
            mma16816(im[u][v], ahi[u], bf[pi_hi][v][0] ^ sg, bf[pi_hi][v][1] ^ sg);
          }
      }
      if ((c + 1) % cpb == 0) {
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              float& lg = s_lg[((u * 4 + v) * 4 + e) * NT + tid];
              lg_add(lg, re[u][v][e], im[u][v][e]);
              re[u][v][e] = im[u][v][e] = 0.0f;
            }
      }
      __syncthreads();  // the stage is overwritten by the copy issued next
    }
#pragma unroll 1
    for (int u = 0; u < 2; ++u)
#pragma unroll 1
      for (int v = 0; v < 4; ++v)
#pragma unroll 1
        for (int e = 0; e < 4; ++e) {
          const int i = r0 + wm * 32 + u * 16 + g + 8 * (e >> 1);
          const int j = c0 + wn * 32 + v * 8 + 2 * t4 + (e & 1);
          const float hl = half_log_lg(s_lg[((u * 4 + v) * 4 + e) * NT + tid]);
          float d2 = 0.0f, comp = 0.0f;
          if (p.need_kc && i < p.row0 + p.nrows && j < p.col0 + p.ncols && !(p.symmetric && j < i)) {
            const float* xa = p.x_r + size_t(i) * p.n;
            const float* xb = p.x_c + size_t(j) * p.n;
            for (int f = 0; f < p.n; ++f) kahan_add_sq(d2, comp, __ldg(xa + f) - __ldg(xb + f));
          }
          write_pair(p, hl, d2, i, j);
        }
  }
}

// ln N_i for the states of m samples: a CTA per 16 samples, its warps taking the blocks in
// turn (blk = warp, warp + NORM_WARPS, ...). A warp computes the 16 x 16 diagonal block of the
// block's Gram with exactly the per-element MMA sequence of gram_blocks_tc_kernel (same
// planes, same three products in the same order into re and im, same steps) and keeps
// |G_B(i, i)|^2 in shared memory; then one thread per sample adds the log2 terms in block
// order, as the Gram kernel does. Every element of an m16n8k16 product is a function of its
// own row and column only, and the diagonal element (i, i) sits at the same fragment
// position (row i mod 16, column i mod 8) in both kernels, so the diagonal is bit-identical
// to the Gram's and K_q(x, x) = 1 exactly.
constexpr int NORM_WARPS = 8;
__global__ void __launch_bounds__(NORM_WARPS * 32)
    block_selfnorm_tc_kernel(const unsigned char* __restrict__ s, int m, int nb, int dp, float* __restrict__ log_norm) {
  extern __shared__ __align__(128) unsigned char nsm[];
  float* g2 = reinterpret_cast<float*>(nsm + NORM_WARPS * 2 * STAGE_N);  // [block][16 samples]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.x * 16;
  const int cpb = dp / KC;
  const size_t sample_bytes = size_t(dp) * 8;
  const int a_row = (lane & 7) + 8 * ((lane >> 3) & 1), a_k = 8 * (lane >> 4);
  const int b_row = (lane & 7) + 8 * (lane >> 4), b_k = 8 * ((lane >> 3) & 1);
  const u32 sw = smem_u32(nsm + warp * 2 * STAGE_N);
  auto issue = [&](int blk, int k0, int buf) {
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int q = lane + 32 * h;
      const int row = q >> 3, piece = q & 7;
      const int smp = min(i0 + row, m - 1);
      const unsigned char* src = s + (size_t(blk) * m + smp) * sample_bytes + size_t(k0) * 8 + piece * 16;
      cp_async16(sw + buf * STAGE_N + row * ROWB + piece * 16, src);
    }
    cp_async_commit();
  };
  // this lane's diagonal elements: rows g and g + 8 of column tiles 0 and 1 when column
  // 2 t4 or 2 t4 + 1 equals g
  const int g = lane >> 2, t4 = lane & 3;
  const bool holds = (g >> 1) == t4;
  const int e_lo = g & 1;  // accumulator index of (g, g) in tile 0; (g + 8, g + 8) is 2 + e_lo in tile 1
  for (int blk = warp; blk < nb; blk += NORM_WARPS) {
    float re[2][4], im[2][4];
#pragma unroll
    for (int v = 0; v < 2; ++v)
#pragma unroll
      for (int e = 0; e < 4; ++e) re[v][e] = im[v][e] = 0.0f;
    issue(blk, 0, 0);
    for (int c = 0; c < cpb; ++c) {
      const int buf = c & 1;
      if (c + 1 < cpb) {
        issue(blk, (c + 1) * KC, buf ^ 1);
        cp_async_wait_1();
      } else {
        cp_async_wait_0();
      }
      __syncwarp();
      const u32 sa = sw + buf * STAGE_N;
      u32 bf[4][2][2];
#pragma unroll
      for (int pl = 0; pl < 4; ++pl) {
        u32 r[4];
        ldsm_x4(r, sa + b_row * ROWB + pl * 32 + b_k * 2);
        bf[pl][0][0] = r[0];
        bf[pl][0][1] = r[1];
        bf[pl][1][0] = r[2];
        bf[pl][1][1] = r[3];
      }
#pragma unroll
      for (int part = 0; part < 2; ++part) {
        u32 ahi[4], alo[4];
        const u32 addr = sa + a_row * ROWB + a_k * 2;
        ldsm_x4(ahi, addr + part * 32);
        ldsm_x4(alo, addr + (2 + part) * 32);
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          const int pr_hi = part ? 1 : 0, pr_lo = part ? 3 : 2;
          const int pi_hi = part ? 0 : 1, pi_lo = part ? 2 : 3;
          const u32 sg = part ? NEG2 : 0u;
          mma16816(re[v], alo, bf[pr_hi][v][0], bf[pr_hi][v][1]);
          mma16816(re[v], ahi, bf[pr_lo][v][0], bf[pr_lo][v][1]);
          mma16816(re[v], ahi, bf[pr_hi][v][0], bf[pr_hi][v][1]);
          mma16816(im[v], alo, bf[pi_hi][v][0] ^ sg, bf[pi_hi][v][1] ^ sg);
          mma16816(im[v], ahi, bf[pi_lo][v][0] ^ sg, bf[pi_lo][v][1] ^ sg);
          mma16816(im[v], ahi, bf[pi_hi][v][0] ^ sg, bf[pi_hi][v][1] ^ sg);
        }
      }
      __syncwarp();  // the stage is overwritten by the copy issued next
    }
    if (holds) {
      // (selects, not a run-time index, keep the accumulators in registers)
      const float r0 = e_lo ? re[0][1] : re[0][0], q0 = e_lo ? im[0][1] : im[0][0];
      const float r1 = e_lo ? re[1][3] : re[1][2], q1 = e_lo ? im[1][3] : im[1][2];
      g2[blk * 16 + g] = fmaf(r0, r0, q0 * q0);
      g2[blk * 16 + g + 8] = fmaf(r1, r1, q1 * q1);
    }
  }
  __syncthreads();
  if (threadIdx.x < 16 && i0 + int(threadIdx.x) < m) {
    float lg = 0.0f;
    for (int blk = 0; blk < nb; ++blk) lg += log2f(g2[blk * 16 + threadIdx.x]);  // lg_add's order
    log_norm[i0 + threadIdx.x] = half_log_lg(lg);
  }
}

}  // namespace gbtc

dk_status block_selfnorm_tc_launch(const void* states, int m, int nb, int dp, float* log_norm, cudaStream_t st) {
  const size_t smem = size_t(gbtc::NORM_WARPS) * 2 * gbtc::STAGE_N + size_t(nb) * 16 * sizeof(float);
  if (smem > 227 * 1024) return DK_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(gbtc::block_selfnorm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
      cudaSuccess)
    return DK_ERR_CUDA;
  gbtc::block_selfnorm_tc_kernel<<<(m + 15) / 16, gbtc::NORM_WARPS * 32, smem, st>>>(
      static_cast<const unsigned char*>(states), m, nb, dp, log_norm);
  return launch_status();
}

template <int WM>
static dk_status launch_tc(dk_ctx* ctx, const void* sr, int m_r, const void* sc, int m_c, int nb, int dp, GramArgs a,
                           int ntiles, cudaStream_t st) {
  using T = gbtc::TileCfg<WM>;
  auto kern = gbtc::gram_blocks_tc_kernel<WM>;
  // set before every launch: the attribute is per device and cheap to set
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(T::SMEM)) !=
      cudaSuccess)
    return DK_ERR_CUDA;
  a.ntiles = ntiles;
  long long grid = (long long)(8 / WM) * ctx->sm_count;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) return DK_OK;
  kern<<<int(grid), T::NT, T::SMEM, st>>>(static_cast<const unsigned char*>(sr), m_r,
                                          static_cast<const unsigned char*>(sc), m_c, nb, dp, a);
  return launch_status();
}

dk_status gram_blocks_tc_launch(dk_ctx* ctx, const void* sr, int m_r, const void* sc, int m_c, int nb, int dp,
                                GramArgs a, cudaStream_t st) {
  // tile rows 128 (2 CTAs of 8 warps per SM) or 64 (4 CTAs of 4 warps): the fewer waves x tile
  // area, the larger tile on ties (its stages serve more pairs)
  GramArgs a4 = a, a2 = a;
  const int t4 = count_tiles(a4, gbtc::TileCfg<4>::TR, gbtc::TC);
  const int t2 = count_tiles(a2, gbtc::TileCfg<2>::TR, gbtc::TC);
  const long long s4 = 2LL * ctx->sm_count, s2 = 4LL * ctx->sm_count;
  const long long cost4 = 2 * ((t4 + s4 - 1) / s4), cost2 = (t2 + s2 - 1) / s2;
  if (cost4 <= cost2) return launch_tc<4>(ctx, sr, m_r, sc, m_c, nb, dp, a4, t4, st);
  return launch_tc<2>(ctx, sr, m_r, sc, m_c, nb, dp, a2, t2, st);
}

}  // namespace dk
