// Gram matrix of a block-structured feature map from its block statevectors (§II-C).
//
// With entanglers only inside blocks of b consecutive qubits, |psi(x)> is the Kronecker
// product of the blocks' states |psi_B(x_B)>, so the overlap of Eq. 9 factorises,
//     a(x_i, x_j) = prod_B <psi_B(x_i)|psi_B(x_j)>,    log K_q = sum_B ln |G_B(i, j)|^2,
// and each G_B is a dense complex matrix product over the 2^b amplitudes of block B: the
// exact tensor-network contraction of a block product state, with no bond truncation.
//
//   * block_states_kernel: one CTA per (block, sample) builds the block's statevector in
//     FP64 (block_state.cuh) and stores it rounded to complex64, layout
//     states[B][i][k], k < dpad = max(2^b, KC) (a short last block is zero-padded, which
//     leaves every overlap unchanged).
//   * gram_blocks_kernel<RU>: (16 RU) x 64 pair tiles (RU = 8: 128 x 64, or 4: 64 x 64 when
//     that fills the GPU better), 256 threads with RU x 4 pairs each; per block the K = dpad
//     contraction runs in 16-amplitude chunks staged through shared memory (register prefetch
//     of the next chunk, double buffer, rows swizzled so a warp's operand reads are
//     conflict-free), FP32 FMAs on CUDA cores. After a block each pair adds log2 |G_B|^2 to
//     a running sum kept in shared memory (no underflow however many blocks). The epilogue is
//     the one of every Gram kernel: log K_q = 2 ln|a| - ln N_i - ln N_j, the RBF kernel
//     (Kahan FP32 distance) and the mix.
//   * block_selfnorm_kernel: ln N_i = ln|a(x_i, x_i)| with exactly the per-pair arithmetic of
//     gram_blocks_kernel (same chunk order, same FMA sequence), so K_q(x, x) = 1 exactly.
#include <cuda_bf16.h>
#include <math.h>

#include "block_state.cuh"
#include "common.cuh"
#include "gram_common.cuh"
#include "internal.h"

namespace dk {
namespace gblk {

constexpr int KC = 16;           // amplitudes per chunk
constexpr int TC = 64;           // pair tile: (16 RU) rows x TC columns, RU = 4 or 8 rows per thread
constexpr int NT = 256;          // threads: 16 x 16
// Shared operand rows: column c of a tile sits at swz(c) = c + 2 (c / 16), i.e. 16 bytes of
// padding after every 16 complex values, so the 8 column groups a warp reads at one k (each
// 4 consecutive complex values, 32 B) fall in distinct banks; row stride 74 (= 72 + 2) also
// spreads the transposed stores of the loader.
constexpr int SROW = 74;     // column tile row stride (64 + 2 x 4 pad + 2)
template <int RU>
struct RowTile {
  static constexpr int TR = 16 * RU;
  static constexpr int SROW_A = TR + 2 * (TR / 16) + 2;
  static constexpr size_t SMEM = 2 * KC * (SROW_A + SROW) * sizeof(float2) + RU * 4 * NT * sizeof(float);
};
__device__ __forceinline__ int swz(int c) { return c + 2 * (c >> 4); }
constexpr int BUILD_NT = 128;

__host__ __device__ inline int dpad_of(int b) { return (1 << b) > KC ? (1 << b) : KC; }

// acc += conj(a) b, the one complex multiply-accumulate of every overlap here
__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}

// running sum of log2 |G_B|^2 over the blocks (one float per pair; never underflows)
__device__ __forceinline__ void lg_add(float& lg, float2 g) { lg += log2f(fmaf(g.x, g.x, g.y * g.y)); }

// ln|a| from the log2 sum of |a|^2
__device__ __forceinline__ float half_log_lg(float lg) { return lg * (0.5f * 0.69314718055994530942f); }

// The operand form of the tensor-core Grams, same 8 bytes per amplitude as complex64: per
// chunk of 16 amplitudes one 128-byte row of four BF16 planes [hi_re | hi_im | lo_re | lo_im]
// of 16 values each, v ~ hi + lo; zeros past the dim amplitudes of the state.
__device__ inline void store_split(float2* out, const float2* psf, int dim, int dp) {
  __nv_bfloat16* pl = reinterpret_cast<__nv_bfloat16*>(out);
  for (int k = threadIdx.x; k < dp; k += BUILD_NT) {
    const float vr = k < dim ? psf[k].x : 0.0f, vi = k < dim ? psf[k].y : 0.0f;
    const __nv_bfloat16 hr = __float2bfloat16_rn(vr), hi = __float2bfloat16_rn(vi);
    __nv_bfloat16* row = pl + (k >> 4) * 64 + (k & 15);
    row[0] = hr;
    row[16] = hi;
    row[32] = __float2bfloat16_rn(vr - __bfloat162float(hr));
    row[48] = __float2bfloat16_rn(vi - __bfloat162float(hi));
  }
}

// split = 0: complex64 [dpad]; split = 1: the split-BF16 operand form (store_split)
__global__ void __launch_bounds__(BUILD_NT) block_states_kernel(const float* __restrict__ x, int m, int n, int b,
                                                                int reps, double angle_scale, int pairs_kind,
                                                                int split, float2* __restrict__ states) {
  extern __shared__ __align__(16) unsigned char raw[];
  blockstate::Coeffs& C = *reinterpret_cast<blockstate::Coeffs*>(raw);
  double2* psi = reinterpret_cast<double2*>(raw + ((sizeof(blockstate::Coeffs) + 15) & ~size_t(15)));
  double2* ph = psi + (1 << b);
  const int blk = blockIdx.x, i = blockIdx.y;
  const int start = blk * b;
  const int bl = min(b, n - start);
  const int dp = dpad_of(b);
  float2* out = states + (size_t(blk) * m + i) * dp;
  const int dim = 1 << bl;
  if (!split) {
    blockstate::build(psi, ph, C, x + size_t(i) * n + start, bl, reps, angle_scale, pairs_kind, threadIdx.x,
                      BUILD_NT);
    for (int k = threadIdx.x; k < dp; k += BUILD_NT)
      out[k] = k < dim ? make_float2(float(psi[k].x), float(psi[k].y)) : make_float2(0.0f, 0.0f);
    return;
  }
  // split-BF16 operands: the state in FP32 (see blockstate::build_f32), in the same buffer
  float2* psf = reinterpret_cast<float2*>(psi);
  float2* phf = psf + (1 << b);
  blockstate::build_f32(psf, phf, C, x + size_t(i) * n + start, bl, reps, angle_scale, pairs_kind, threadIdx.x,
                        BUILD_NT);
  store_split(out, psf, dim, dp);
}

// The split-BF16 states of blocks of b = 7 + log2(R) qubits, built with the amplitudes in
// registers (blockstate::build_f32_regs); a shorter last block takes the shared-memory form.
template <int R>
__global__ void __launch_bounds__(BUILD_NT) block_states_split_kernel(const float* __restrict__ x, int m, int n,
                                                                      int b, int reps, double angle_scale,
                                                                      int pairs_kind, float2* __restrict__ states) {
  extern __shared__ __align__(16) unsigned char raw[];
  blockstate::Coeffs& C = *reinterpret_cast<blockstate::Coeffs*>(raw);
  float2* psf = reinterpret_cast<float2*>(raw + ((sizeof(blockstate::Coeffs) + 15) & ~size_t(15)));
  float2* phf = psf + (1 << b);
  const int blk = blockIdx.x, i = blockIdx.y;
  const int start = blk * b;
  const int bl = min(b, n - start);
  const int dp = dpad_of(b);
  float2* out = states + (size_t(blk) * m + i) * dp;
  if (bl == b)
    blockstate::build_f32_regs<R>(psf, phf, C, x + size_t(i) * n + start, reps, angle_scale, pairs_kind,
                                  threadIdx.x);
  else
    blockstate::build_f32(psf, phf, C, x + size_t(i) * n + start, bl, reps, angle_scale, pairs_kind, threadIdx.x,
                          BUILD_NT);
  store_split(out, psf, 1 << bl, dp);
}

// One CTA per sample: thread B forms <psi_B|psi_B> with the Gram kernel's sequential
// per-pair FMA order, then thread 0 multiplies the blocks in order as the Gram kernel does.
constexpr int NORM_NT = 128;
__global__ void __launch_bounds__(NORM_NT) block_selfnorm_kernel(const float2* __restrict__ states, int m, int nb,
                                                                 int dp, float* __restrict__ log_norm) {
  extern __shared__ float2 s_g[];  // nb overlaps
  const int i = blockIdx.x;
  for (int blk = threadIdx.x; blk < nb; blk += NORM_NT) {
    const float4* a = reinterpret_cast<const float4*>(states + (size_t(blk) * m + i) * dp);
    float2 acc = make_float2(0.0f, 0.0f);
    for (int k = 0; k < dp / 2; ++k) {
      const float4 v = __ldg(a + k);
      cmac(acc, make_float2(v.x, v.y), make_float2(v.x, v.y));
      cmac(acc, make_float2(v.z, v.w), make_float2(v.z, v.w));
    }
    s_g[blk] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float lg = 0.0f;
    for (int blk = 0; blk < nb; ++blk) lg_add(lg, s_g[blk]);
    log_norm[i] = half_log_lg(lg);
  }
}

template <int RU>
__global__ void __launch_bounds__(NT, 2) gram_blocks_kernel(const float2* __restrict__ sr, int m_r,
                                                            const float2* __restrict__ sc, int m_c, int nb, int dp,
                                                            const GramArgs p) {
  // dynamic shared memory: the double-buffered operand tiles (rows: TR x KC, columns: TC x KC,
  // stored k-major), then the running log2 sums of each thread's pairs (touched once per
  // block: kept here, not in registers, which go to the accumulators and the operand loads)
  constexpr int TR = RowTile<RU>::TR, SROW_A = RowTile<RU>::SROW_A;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto As = reinterpret_cast<float2(*)[KC][SROW_A]>(smem_raw);
  auto Bs = reinterpret_cast<float2(*)[KC][SROW]>(smem_raw + 2 * KC * SROW_A * sizeof(float2));
  auto s_lg = reinterpret_cast<float(*)[NT]>(smem_raw + 2 * KC * (SROW_A + SROW) * sizeof(float2));
  // a warp covers 4 x 8 threads (32 x 32 pairs): lane -> (ty % 4, tx % 8), warp -> (ty / 4, tx / 8)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ty = (warp >> 1) * 4 + (lane >> 3), tx = (warp & 1) * 8 + (lane & 7);
  // loader: thread -> (rows lr and, for RU = 8, lr + 64; float4 lq and lq + 4 of each row's chunk)
  const int lr = tid >> 2, lq = tid & 3;
  const int cpb = dp / KC;  // chunks per block
  const int total = nb * cpb;
  const int my_tiles = (p.ntiles > int(blockIdx.x)) ? (p.ntiles - 1 - int(blockIdx.x)) / int(gridDim.x) + 1 : 0;
  for (int lt = 0; lt < my_tiles; ++lt) {
    int ti, tj;
    decode_tile(p, TR, TC, int(blockIdx.x) + lt * int(gridDim.x), ti, tj);
    const int r0 = p.row0 + ti * TR, c0 = p.col0 + tj * TC;
    const int ar0 = min(r0 + lr, m_r - 1), ar1 = min(r0 + 64 + lr, m_r - 1), bc = min(c0 + lr, m_c - 1);
    float4 pa[RU / 2], pb[2];
    auto fetch = [&](int c) {
      const int blk = c / cpb, k0 = (c - blk * cpb) * KC;
      const float4* a0 = reinterpret_cast<const float4*>(sr + (size_t(blk) * m_r + ar0) * dp + k0);
      const float4* a1 = reinterpret_cast<const float4*>(sr + (size_t(blk) * m_r + ar1) * dp + k0);
      const float4* bb = reinterpret_cast<const float4*>(sc + (size_t(blk) * m_c + bc) * dp + k0);
      pa[0] = __ldg(a0 + lq);
      pa[1] = __ldg(a0 + lq + 4);
      if constexpr (RU == 8) {
        pa[2] = __ldg(a1 + lq);
        pa[3] = __ldg(a1 + lq + 4);
      }
      pb[0] = __ldg(bb + lq);
      pb[1] = __ldg(bb + lq + 4);
    };
    auto commit = [&](int buf) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = 2 * (lq + 4 * h);
        As[buf][k][swz(lr)] = make_float2(pa[h].x, pa[h].y);
        As[buf][k + 1][swz(lr)] = make_float2(pa[h].z, pa[h].w);
        if constexpr (RU == 8) {
          As[buf][k][swz(lr + 64)] = make_float2(pa[2 + h].x, pa[2 + h].y);
          As[buf][k + 1][swz(lr + 64)] = make_float2(pa[2 + h].z, pa[2 + h].w);
        }
        Bs[buf][k][swz(lr)] = make_float2(pb[h].x, pb[h].y);
        Bs[buf][k + 1][swz(lr)] = make_float2(pb[h].z, pb[h].w);
      }
    };
    float2 acc[RU][4];
#pragma unroll
    for (int u = 0; u < RU; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        acc[u][v] = make_float2(0.0f, 0.0f);
        s_lg[u * 4 + v][tid] = 0.0f;
      }
    fetch(0);
    commit(0);
    __syncthreads();
    for (int c = 0; c < total; ++c) {
      const int buf = c & 1;
      if (c + 1 < total) fetch(c + 1);
#pragma unroll
      for (int kk = 0; kk < KC; ++kk) {
        float2 av[RU], bv[4];
#pragma unroll
        for (int h = 0; h < RU / 2; ++h) {
          const float4 a = *reinterpret_cast<const float4*>(&As[buf][kk][swz(ty * RU) + 2 * h]);
          av[2 * h] = make_float2(a.x, a.y);
          av[2 * h + 1] = make_float2(a.z, a.w);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float4 b = *reinterpret_cast<const float4*>(&Bs[buf][kk][swz(tx * 4) + 2 * h]);
          bv[2 * h] = make_float2(b.x, b.y);
          bv[2 * h + 1] = make_float2(b.z, b.w);
        }
#pragma unroll
        for (int u = 0; u < RU; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) cmac(acc[u][v], av[u], bv[v]);
      }
      if ((c + 1) % cpb == 0) {
#pragma unroll
        for (int u = 0; u < RU; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            float lg = s_lg[u * 4 + v][tid];
            lg_add(lg, acc[u][v]);
            s_lg[u * 4 + v][tid] = lg;
            acc[u][v] = make_float2(0.0f, 0.0f);
          }
      }
      if (c + 1 < total) commit(buf ^ 1);
      __syncthreads();
    }
#pragma unroll 1
    for (int u = 0; u < RU; ++u)
#pragma unroll 1
      for (int v = 0; v < 4; ++v) {
        const int i = r0 + ty * RU + u, j = c0 + tx * 4 + v;
        float d2 = 0.0f, comp = 0.0f;
        if (p.need_kc && i < p.row0 + p.nrows && j < p.col0 + p.ncols && !(p.symmetric && j < i)) {
          const float* xa = p.x_r + size_t(i) * p.n;
          const float* xb = p.x_c + size_t(j) * p.n;
          for (int f = 0; f < p.n; ++f) kahan_add_sq(d2, comp, __ldg(xa + f) - __ldg(xb + f));
        }
        write_pair(p, half_log_lg(s_lg[u * 4 + v][tid]), d2, i, j);
      }
    __syncthreads();  // s_lg is reset by the next tile
  }
}

}  // namespace gblk
}  // namespace dk

DK_API size_t dk_block_states_bytes(int m, int n, int block) {
  if (m < 1 || n < 1 || block < 0 || block > dk::blockstate::MAXB) return 0;
  const int b = block > 0 ? block : n;
  if (b > dk::blockstate::MAXB) return 0;
  const int nb = (n + b - 1) / b;
  return size_t(nb) * m * dk::gblk::dpad_of(b) * sizeof(float2);
}

DK_API size_t dk_block_states_workspace_bytes(dk_ctx* ctx, int m, int n, int block, dk_precision prec) {
  using namespace dk;
  if (!ctx || m < 1 || n < 1 || dk_block_states_bytes(m, n, block) == 0) return 0;
  if (prec != DK_PREC_BF16X3 || ctx->block_form == DK_BLOCK_MMA_SYNC) return 0;
  const int b = block > 0 ? block : n;
  return block_selfnorm_umma_ws_bytes(m, (n + b - 1) / b);
}

DK_API dk_status dk_block_states(dk_ctx* ctx, const float* x, int m, int n, const dk_fmap* fm, int entangler,
                                 dk_precision prec, void* states, float* log_norm, void* ws, size_t ws_bytes,
                                 void* stream) {
  using namespace dk;
  if (!ctx || !x || !fm || !states || m < 1 || n < 1) return DK_ERR_ARG;
  if (prec != DK_PREC_F32 && prec != DK_PREC_BF16X3) return DK_ERR_UNSUPPORTED;
  if (fm->reps < 1 || fm->reps > 5) return DK_ERR_ARG;
  if (entangler != DK_ENT_CHAIN && entangler != DK_ENT_FULL) return DK_ERR_ARG;
  if (!aligned16(states)) return DK_ERR_ARG;
  if (dk_block_states_bytes(m, n, fm->block) == 0) return DK_ERR_UNSUPPORTED;
  if (m > 65535) return DK_ERR_UNSUPPORTED;  // grid y
  const int b = fm->block > 0 ? fm->block : n;
  const int nb = (n + b - 1) / b;
  if (size_t(nb) * sizeof(float2) > 48 * 1024) return DK_ERR_UNSUPPORTED;  // self-norm staging
  const int kind = fm->entangle ? entangler : -1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int split = prec == DK_PREC_BF16X3 ? 1 : 0;
  dk_status s = DK_OK;
  if (split && b >= 7) {
    // the FP32 build of the split form needs half the state storage: twice the CTAs per SM
    const size_t smem = blockstate::smem_bytes_f32(b);
    auto launch = [&](auto kern) {
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
        return DK_ERR_CUDA;
      kern<<<dim3(nb, m), gblk::BUILD_NT, smem, st>>>(x, m, n, b, fm->reps, double(fm->angle_scale), kind,
                                                      static_cast<float2*>(states));
      return launch_status();
    };
    switch (b) {
      case 7: s = launch(gblk::block_states_split_kernel<1>); break;
      case 8: s = launch(gblk::block_states_split_kernel<2>); break;
      case 9: s = launch(gblk::block_states_split_kernel<4>); break;
      case 10: s = launch(gblk::block_states_split_kernel<8>); break;
      case 11: s = launch(gblk::block_states_split_kernel<16>); break;
      default: s = launch(gblk::block_states_split_kernel<32>); break;
    }
  } else {
    if (cudaFuncSetAttribute(gblk::block_states_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(blockstate::smem_bytes(b))) != cudaSuccess)
      return DK_ERR_CUDA;
    const size_t smem = split ? blockstate::smem_bytes_f32(b) : blockstate::smem_bytes(b);
    gblk::block_states_kernel<<<dim3(nb, m), gblk::BUILD_NT, smem, st>>>(x, m, n, b, fm->reps,
                                                                        double(fm->angle_scale), kind, split,
                                                                        static_cast<float2*>(states));
    s = launch_status();
  }
  if (s != DK_OK || !log_norm) return s;
  if (split)
    return ctx->block_form == DK_BLOCK_MMA_SYNC
               ? block_selfnorm_tc_launch(states, m, nb, gblk::dpad_of(b), log_norm, st)
               : block_selfnorm_umma_launch(ctx, states, m, nb, gblk::dpad_of(b), log_norm, ws, ws_bytes, st);
  gblk::block_selfnorm_kernel<<<m, gblk::NORM_NT, nb * sizeof(float2), st>>>(static_cast<const float2*>(states), m,
                                                                           nb, gblk::dpad_of(b), log_norm);
  return launch_status();
}

DK_API size_t dk_gram_blocks_workspace_bytes(dk_ctx* ctx, int n, int block, int nrows, int ncols, dk_precision prec,
                                            int symmetric, int with_kc) {
  using namespace dk;
  if (!ctx || n < 1 || nrows < 1 || ncols < 1 || dk_block_states_bytes(1, n, block) == 0) return 0;
  if (prec != DK_PREC_BF16X3 || ctx->block_form == DK_BLOCK_MMA_SYNC) return 0;
  const int b = block > 0 ? block : n;
  GramArgs a{};
  a.n = n;
  a.nrows = nrows;
  a.ncols = ncols;
  a.symmetric = symmetric ? 1 : 0;
  a.need_kc = with_kc ? 1 : 0;
  return gram_blocks_umma_ws_bytes(ctx, a, (n + b - 1) / b);
}

DK_API dk_status dk_gram_blocks(dk_ctx* ctx, const void* states_rows, int m_rows, const void* states_cols, int m_cols,
                                int n, int block, int row0, int nrows, int col0, int ncols, const float* lnorm_rows,
                                const float* lnorm_cols, const float* x_rows, const float* x_cols, float gamma,
                                float w, dk_precision prec, float* k_out, float* kq_out, float* kc_out,
                                float* logkq_out, long long ld, int symmetric, void* ws, size_t ws_bytes,
                                void* stream) {
  using namespace dk;
  if (prec != DK_PREC_F32 && prec != DK_PREC_BF16X3) return DK_ERR_UNSUPPORTED;
  if (!ctx || !states_rows || !states_cols || !lnorm_rows || !lnorm_cols) return DK_ERR_ARG;
  if (m_rows < 1 || m_cols < 1 || n < 1 || nrows < 0 || ncols < 0 || row0 < 0 || col0 < 0) return DK_ERR_ARG;
  if (row0 + nrows > m_rows || col0 + ncols > m_cols) return DK_ERR_ARG;
  if (dk_block_states_bytes(1, n, block) == 0) return DK_ERR_UNSUPPORTED;
  if (!aligned16(states_rows) || !aligned16(states_cols)) return DK_ERR_ARG;
  if (!k_out && !kq_out && !kc_out && !logkq_out) return DK_ERR_ARG;
  if (ld < ncols) return DK_ERR_ARG;
  if (symmetric && (row0 != col0 || nrows != ncols || states_rows != states_cols)) return DK_ERR_ARG;
  const bool need_kc = kc_out || (k_out && w != 1.0f);
  if (need_kc && (!x_rows || !x_cols)) return DK_ERR_ARG;
  if (nrows == 0 || ncols == 0) return DK_OK;
  const int b = block > 0 ? block : n;
  GramArgs a{};
  a.n = n;
  a.row0 = row0;
  a.nrows = nrows;
  a.col0 = col0;
  a.ncols = ncols;
  a.symmetric = symmetric ? 1 : 0;
  a.lnorm_r = lnorm_rows;
  a.lnorm_c = lnorm_cols;
  a.x_r = x_rows;
  a.x_c = x_cols;
  a.gamma = gamma;
  a.w = w;
  a.k = k_out;
  a.kq = kq_out;
  a.kc = kc_out;
  a.lkq = logkq_out;
  a.ld = ld;
  a.status = ctx->status;
  a.need_kc = need_kc ? 1 : 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (prec == DK_PREC_BF16X3) {
    if (ctx->block_form == DK_BLOCK_MMA_SYNC)
      return gram_blocks_tc_launch(ctx, states_rows, m_rows, states_cols, m_cols, (n + b - 1) / b, gblk::dpad_of(b),
                                   a, st);
    return gram_blocks_umma_launch(ctx, states_rows, m_rows, states_cols, m_cols, (n + b - 1) / b, gblk::dpad_of(b),
                                   a, ws, ws_bytes, st);
  }
  // tile shape: estimated time = waves x tile area / per-pair efficiency (the 128 x 64 tile
  // runs about 15 % more pairs per second than 64 x 64, which fills the GPU better when
  // there are few tiles, e.g. a batch of decision rows)
  const long long slots = 2LL * ctx->sm_count;
  GramArgs a8 = a, a4 = a;
  a8.ntiles = count_tiles(a8, gblk::RowTile<8>::TR, gblk::TC);
  a4.ntiles = count_tiles(a4, gblk::RowTile<4>::TR, gblk::TC);
  const double cost8 = double((a8.ntiles + slots - 1) / slots) * 2.0 / 1.15;
  const double cost4 = double((a4.ntiles + slots - 1) / slots);
  const int nbk = (n + b - 1) / b, dp = gblk::dpad_of(b);
  const float2* srp = static_cast<const float2*>(states_rows);
  const float2* scp = static_cast<const float2*>(states_cols);
  if (cost8 <= cost4) {
    auto kern = gblk::gram_blocks_kernel<8>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(gblk::RowTile<8>::SMEM)) !=
        cudaSuccess)
      return DK_ERR_CUDA;
    const int grid = int(a8.ntiles < slots ? a8.ntiles : slots);
    kern<<<grid, gblk::NT, gblk::RowTile<8>::SMEM, st>>>(srp, m_rows, scp, m_cols, nbk, dp, a8);
  } else {
    auto kern = gblk::gram_blocks_kernel<4>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(gblk::RowTile<4>::SMEM)) !=
        cudaSuccess)
      return DK_ERR_CUDA;
    const int grid = int(a4.ntiles < slots ? a4.ntiles : slots);
    kern<<<grid, gblk::NT, gblk::RowTile<4>::SMEM, st>>>(srp, m_rows, scp, m_cols, nbk, dp, a4);
  }
  return launch_status();
}

DK_API dk_status dk_set_block_gram_form(dk_ctx* ctx, int form) {
  if (!ctx || (form != DK_BLOCK_TCGEN05 && form != DK_BLOCK_MMA_SYNC)) return DK_ERR_ARG;
  ctx->block_form = form;
  return DK_OK;
}
