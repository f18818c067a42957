// Tiled quantum-kernel Gram with the RBF kernel and the dual-kernel mix fused in.
//
// Paper: §II-C (Eqs. 7-10: K_q = |<psi(x_i)|psi(x_j)>|^2 by exact tensor-network
// contraction), §II-B (Eq. 3: RBF), §II-D (Eq. 11: K = w K_q + (1 - w) K_c; blocks of
// (row, column) pairs contracted by a worker).
//
// Design (one GPU, persistent CTAs):
//  * A CTA owns a TR x TC tile of pairs; each thread owns one pair and keeps its chi x chi
//    transfer matrix E in registers for all n sites (transfer.cuh).
//  * Per site the tile needs the site tensors of TR row samples and TC column samples.
//    With the site-major MPS layout these are two contiguous runs of samples, fetched by
//    TMA (cp.async.bulk.tensor, 128-byte swizzle) into a STAGES-deep shared-memory ring
//    guarded by full/empty mbarriers. Thread 0 refills the stage released one site
//    earlier, so the copy of site k+STAGES-1 overlaps the arithmetic of site k.
//  * The swizzle puts the 16-byte chunk c of sample t's 128-byte row at c XOR (t & 7):
//    the 8 distinct samples that a quarter-warp reads land in 8 different bank groups.
//  * Tiles are handed out round-robin to a grid of (SMs x resident CTAs); the symmetric
//    Gram enumerates only the upper-triangular tiles and writes each pair twice.
//  * Epilogue per pair: log K_q from the rescaled amplitude and the per-sample
//    log-norms, K_q = exp(log K_q), K_c = exp(-gamma ||x_i - x_j||^2) with a compensated
//    FP32 sum over the features, K = w K_q + (1 - w) K_c.
#include <math.h>

#include <atomic>

#include "common.cuh"
#include "internal.h"
#include "gram_common.cuh"
#include "transfer.cuh"

namespace dk {

template <typename real_, int CHI_, int WTR_, int WTC_, int PR_, int PC_, int WR_, int WC_, int STAGES_, int MINB_,
          int SPS_ = 1>
struct GramCfg {
  using real = real_;
  static constexpr int CHI = CHI_, H = CHI_ / 2;
  static constexpr int WTR = WTR_, WTC = WTC_, PR = PR_, PC = PC_, WR = WR_, WC = WC_;
  static constexpr int STAGES = STAGES_, MINB = MINB_;
  static constexpr int SPS = SPS_;  // sites per pipeline stage (one barrier wait per stage)
  static constexpr int NWARPS = WR * WC;
  static constexpr int NTHREADS = NWARPS * 32;
  static constexpr int TR = WR * WTR * PR;   // row samples per tile
  static constexpr int TC = WC * WTC * PC;   // column samples per tile
  static constexpr int CPLX = 2 * int(sizeof(real));
  static constexpr int SITE_BYTES = CHI * CHI * CPLX;      // compact site tensor of one sample
  static constexpr int NROW = SITE_BYTES / 128;            // 128-byte rows per sample-site
  // Per side and stage: [128-byte row r][site u][sample slot][128 B]; one (r, u) plane of
  // T samples is T * 128 bytes and starts on a 1024-byte boundary (the swizzle period).
  static constexpr int PLANE_R = ((TR * 128 + 1023) / 1024) * 1024;
  static constexpr int PLANE_C = ((TC * 128 + 1023) / 1024) * 1024;
  static constexpr int HBUF_R = SPS * PLANE_R;  // one 128-byte row of TR samples, SPS sites
  static constexpr int HBUF_C = SPS * PLANE_C;
  static constexpr int ROW_BOX = NROW * HBUF_R;
  static constexpr int COL_BOX = NROW * HBUF_C;
  static constexpr int STAGE_BYTES = ROW_BOX + COL_BOX;
  static constexpr int TX_BYTES = SPS * (TR + TC) * SITE_BYTES;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + STAGES * 8 + 2 * STAGES * 4 + 16 + 1024;
  static_assert(SITE_BYTES % 128 == 0, "site tensor must be a whole number of 128-byte rows");
  static_assert(WTR * WTC == 32, "a warp is WTR x WTC threads");
  static_assert(H * CPLX >= 16 && (H * CPLX) % 16 == 0, "a sub-block column must be whole 16-byte chunks");
  static_assert(SPS == 1 || (TR % 8 == 0 && TC % 8 == 0), "multi-site stages need 1024-byte planes");
};

// Fills the h x h sub-block A_s[t] (rows: left bond l = t*h + a, columns j) of one sample
// from a swizzled stage buffer. In the compact layout element (s, j, l) of a sample-site
// sits at complex index (s*h + j)*chi + l, so each sub-block column is h consecutive
// complex numbers; the TMA 128-byte swizzle stores chunk c of sample slot u at c ^ (u & 7).
template <class Cfg>
struct SubLoad {
  using real = typename Cfg::real;
  static constexpr int H = Cfg::H;
  const uint8_t* buf;  // row-0 buffer of this side at the current site (shared memory)
  int hbuf;            // bytes between the 128-byte-row buffers of this side
  int slot0;           // sample slot of this thread's first row/column
  int stride;          // slot distance between this thread's rows/columns
  __device__ __forceinline__ void operator()(int p, int s, int t, Blk<real, H>& blk) const {
    constexpr int CPLX = Cfg::CPLX;
    constexpr int NCH = H * CPLX / 16;  // chunks per sub-block column
    const int slot = slot0 + p * stride;
    const uint8_t* row0 = buf + slot * 128;
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const int off = ((s * H + j) * Cfg::CHI + t * H) * CPLX;
      const int r = off >> 7;
      const int c0 = (off & 127) >> 4;
#pragma unroll
      for (int q = 0; q < NCH; ++q) {
        const uint8_t* a = row0 + r * hbuf + (((c0 + q) ^ (slot & 7)) << 4);
        if constexpr (sizeof(real) == 4) {
          const float4 v = *reinterpret_cast<const float4*>(a);
          blk.r[2 * q][j] = v.x;
          blk.i[2 * q][j] = v.y;
          blk.r[2 * q + 1][j] = v.z;
          blk.i[2 * q + 1][j] = v.w;
        } else {
          const double2 v = *reinterpret_cast<const double2*>(a);
          blk.r[q][j] = v.x;
          blk.i[q][j] = v.y;
        }
      }
    }
  }
};

template <class Cfg>
__global__ void __launch_bounds__(Cfg::NTHREADS, Cfg::MINB)
    gram_kernel(const __grid_constant__ CUtensorMap tm_r, const __grid_constant__ CUtensorMap tm_c,
                const GramArgs p) {
  using real = typename Cfg::real;
  constexpr int H = Cfg::H, STAGES = Cfg::STAGES, PR = Cfg::PR, PC = Cfg::PC, SPS = Cfg::SPS;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  // 1024-byte aligned base for the 128-byte swizzle, kept as shared-memory pointer arithmetic
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * Cfg::STAGE_BYTES);
  int* released = reinterpret_cast<int*>(full + STAGES);  // warps done with each stage
  int* inflight = released + STAGES;                       // parity + 1 of the last load per stage
  volatile int* abort_flag = inflight + STAGES;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  // Thread (lr, lc) of warp (wr, wc) owns rows slot_r + pr*WTR and columns slot_c + pc*WTC:
  // the 8 lanes of a quarter-warp read 8 consecutive column samples and one row sample.
  const int slot_r = (warp / Cfg::WC) * (Cfg::WTR * PR) + lane / Cfg::WTC;
  const int slot_c = (warp % Cfg::WC) * (Cfg::WTC * PC) + lane % Cfg::WTC;

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      released[s] = 0;
      inflight[s] = 0;
    }
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tensormap(&tm_r);
    prefetch_tensormap(&tm_c);
  }
  __syncthreads();

  const int steps = (p.n + SPS - 1) / SPS;  // pipeline stages per tile
  const int my_tiles = (p.ntiles > int(blockIdx.x)) ? (p.ntiles - 1 - int(blockIdx.x)) / int(gridDim.x) + 1 : 0;
  const long long total = (long long)my_tiles * steps;

  auto tile_origin = [&](int local, int& r0, int& c0) {
    int ti, tj;
    decode_tile(p, Cfg::TR, Cfg::TC, int(blockIdx.x) + local * int(gridDim.x), ti, tj);
    r0 = p.row0 + ti * Cfg::TR;
    c0 = p.col0 + tj * Cfg::TC;
  };
  // Load sites js*SPS .. js*SPS+SPS-1 of the tile at (r0, c0) into stage `st` (one thread);
  // sites past n arrive as zeros and are skipped.
  auto issue = [&](int st, uint32_t parity, int r0, int c0, int js) {
    uint8_t* base = smem + st * Cfg::STAGE_BYTES;
    inflight[st] = int(parity) + 1;
    mbar_arrive_expect_tx(&full[st], Cfg::TX_BYTES);
#pragma unroll
    for (int h = 0; h < Cfg::NROW; ++h) {
      tma_load_3d(base + h * Cfg::HBUF_R, &tm_r, &full[st], h * 32, r0, js * SPS);
      tma_load_3d(base + Cfg::ROW_BOX + h * Cfg::HBUF_C, &tm_c, &full[st], h * 32, c0, js * SPS);
    }
  };

  if (tid == 0) {
    int tile = 0, js = 0, r0 = 0, c0 = 0;
    for (int q = 0; q < STAGES && q < total; ++q) {
      if (js == 0) tile_origin(tile, r0, c0);
      issue(q, 0u, r0, c0, js);
      if (++js == steps) {
        js = 0;
        ++tile;
      }
    }
  }

  PairE<real, H> st[PR][PC];
  int r0 = 0, c0 = 0;
  int sidx = 0, js = 0, tile = 0;
  uint32_t ph = 0;
  long long q = 0;
  for (; q < total; ++q) {
    if (js == 0) {
#pragma unroll
      for (int pr = 0; pr < PR; ++pr)
#pragma unroll
        for (int pc = 0; pc < PC; ++pc) st[pr][pc].init();
      tile_origin(tile, r0, c0);
    }
    if (!mbar_wait_bounded(&full[sidx], ph)) {
      record_status(p.status, DEV_TIMEOUT);
      *abort_flag = 1;
      break;
    }
    const uint8_t* base = smem + sidx * Cfg::STAGE_BYTES;
    // Not unrolled: one site's code (~1200 instructions) is reused for every site of the
    // stage; unrolled stages of 4 or 8 sites overflow the instruction cache.
#pragma unroll 1
    for (int u = 0; u < SPS; ++u) {
      const int k = js * SPS + u;
      if (SPS > 1 && k >= p.n) break;
      const SubLoad<Cfg> ldi{base + u * Cfg::PLANE_R, Cfg::HBUF_R, slot_r, Cfg::WTR};
      const SubLoad<Cfg> ldj{base + Cfg::ROW_BOX + u * Cfg::PLANE_C, Cfg::HBUF_C, slot_c, Cfg::WTC};
      site_step<real, H, PR, PC>(st, ldi, ldj, k == p.n - 1 || ((k & (RENORM_EVERY - 1)) == RENORM_EVERY - 1));
    }
    // Release the stage; the last warp to do so refills it with the stage STAGES ahead, so
    // no thread ever waits for the others to free a buffer.
    __syncwarp();
    if (lane == 0) {
      __threadfence_block();
      if (atomicAdd(&released[sidx], 1) == Cfg::NWARPS - 1) {
        released[sidx] = 0;
        __threadfence_block();
        if (q + STAGES < total) {
          int jj = js + STAGES, tt = tile;
          while (jj >= steps) {
            jj -= steps;
            ++tt;
          }
          int rr = r0, cc = c0;
          if (tt != tile) tile_origin(tt, rr, cc);  // once per tile, not per stage
          fence_proxy_async_smem();
          issue(sidx, ph ^ 1u, rr, cc, jj);
        }
      }
    }
    if (js == steps - 1) {
      // ||x_i - x_j||^2 of this thread's pairs, Kahan sums over the features, all pairs
      // interleaved; rows / columns past the block read the last valid sample and are dropped.
      float d2s[PR][PC], d2c[PR][PC];
#pragma unroll
      for (int pr = 0; pr < PR; ++pr)
#pragma unroll
        for (int pc = 0; pc < PC; ++pc) {
          d2s[pr][pc] = 0.0f;
          d2c[pr][pc] = 0.0f;
        }
      if (p.need_kc) {
        const float* xr[PR];
        const float* xc[PC];
#pragma unroll
        for (int pr = 0; pr < PR; ++pr)
          xr[pr] = p.x_r + size_t(min(r0 + slot_r + pr * Cfg::WTR, p.row0 + p.nrows - 1)) * p.n;
#pragma unroll
        for (int pc = 0; pc < PC; ++pc)
          xc[pc] = p.x_c + size_t(min(c0 + slot_c + pc * Cfg::WTC, p.col0 + p.ncols - 1)) * p.n;
        // Features 8 at a time as float4 pairs when every row is 16-byte aligned (n a multiple
        // of 8), two groups in flight: the loads of a tile's epilogue then take a sixteenth of
        // the L2 round trips of the scalar loop. Same additions in the same order.
        const bool vec8 = (p.n & 7) == 0 && ((reinterpret_cast<uintptr_t>(p.x_r) | reinterpret_cast<uintptr_t>(p.x_c)) & 15) == 0;
        if (vec8) {
#pragma unroll 2
          for (int f = 0; f < p.n; f += 8) {
            float4 a[PR][2], b[PC][2];
#pragma unroll
            for (int pr = 0; pr < PR; ++pr) {
              a[pr][0] = __ldg(reinterpret_cast<const float4*>(xr[pr] + f));
              a[pr][1] = __ldg(reinterpret_cast<const float4*>(xr[pr] + f + 4));
            }
#pragma unroll
            for (int pc = 0; pc < PC; ++pc) {
              b[pc][0] = __ldg(reinterpret_cast<const float4*>(xc[pc] + f));
              b[pc][1] = __ldg(reinterpret_cast<const float4*>(xc[pc] + f + 4));
            }
#pragma unroll
            for (int e = 0; e < 8; ++e)
#pragma unroll
              for (int pr = 0; pr < PR; ++pr)
#pragma unroll
                for (int pc = 0; pc < PC; ++pc)
                  kahan_add_sq(d2s[pr][pc], d2c[pr][pc], f4_get(a[pr][e >> 2], e & 3) - f4_get(b[pc][e >> 2], e & 3));
          }
        } else {
#pragma unroll 4
          for (int f = 0; f < p.n; ++f) {
            float a[PR], b[PC];
#pragma unroll
            for (int pr = 0; pr < PR; ++pr) a[pr] = __ldg(xr[pr] + f);
#pragma unroll
            for (int pc = 0; pc < PC; ++pc) b[pc] = __ldg(xc[pc] + f);
#pragma unroll
            for (int pr = 0; pr < PR; ++pr)
#pragma unroll
              for (int pc = 0; pc < PC; ++pc) kahan_add_sq(d2s[pr][pc], d2c[pr][pc], a[pr] - b[pc]);
          }
        }
      }
#pragma unroll
      for (int pr = 0; pr < PR; ++pr)
#pragma unroll
        for (int pc = 0; pc < PC; ++pc)
          write_pair(p, st[pr][pc].half_log_mod(), d2s[pr][pc], r0 + slot_r + pr * Cfg::WTR,
                          c0 + slot_c + pc * Cfg::WTC);
    }
    if (*abort_flag) break;
    if (++sidx == STAGES) {
      sidx = 0;
      ph ^= 1u;
    }
    if (++js == steps) {
      js = 0;
      ++tile;
    }
  }
  // After a timeout, let the copies still in flight land before the CTA leaves.
  __syncthreads();
  if (tid == 0 && *abort_flag) {
    for (int s = 0; s < STAGES; ++s)
      if (inflight[s] > 0 && !mbar_wait_bounded(&full[s], uint32_t(inflight[s] - 1))) break;
  }
}

template <class Cfg>
struct GramLauncher {
  static dk_status run(dk_ctx* ctx, const void* mps_r, int m_r, const void* mps_c, int m_c, const GramArgs& a,
                       cudaStream_t st) {
    CUtensorMap tmr, tmc;
    dk_status s = encode_mps_map(ctx, &tmr, mps_r, m_r, a.n, Cfg::SITE_BYTES, Cfg::TR, Cfg::SPS);
    if (s != DK_OK) return s;
    s = encode_mps_map(ctx, &tmc, mps_c, m_c, a.n, Cfg::SITE_BYTES, Cfg::TC, Cfg::SPS);
    if (s != DK_OK) return s;
    auto kern = gram_kernel<Cfg>;
    // The shared-memory opt-in is per device: set before every launch (a cheap host call).
    // Resident CTAs per SM depend only on the kernel and the architecture, so the first
    // query's answer serves every device and thread (a relaxed atomic, computed at most a
    // few times in a race).
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM_BYTES) != cudaSuccess)
      return DK_ERR_CUDA;
    static std::atomic<int> occ_cache{-1};
    int occ = occ_cache.load(std::memory_order_relaxed);
    if (occ < 0) {
      int o = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, Cfg::NTHREADS, Cfg::SMEM_BYTES) != cudaSuccess)
        return DK_ERR_CUDA;
      occ = o > 0 ? o : 1;
      occ_cache.store(occ, std::memory_order_relaxed);
    }
    long long grid = (long long)ctx->sm_count * occ;
    if (grid > a.ntiles) grid = a.ntiles;
    if (grid < 1) return DK_OK;
    kern<<<int(grid), Cfg::NTHREADS, Cfg::SMEM_BYTES, st>>>(tmr, tmc, a);
    return launch_status();
  }
};

// Tile shapes: GramCfg<real, chi, warp WTR x WTC threads, PR x PC pairs per thread,
// WR x WC warps, stages, min CTAs per SM>.
using F32_P11 = GramCfg<float, 4, 4, 8, 1, 1, 4, 2, 4, 2>;     // 16 x 16 pairs, 256 threads
using F32_P21 = GramCfg<float, 4, 4, 8, 2, 1, 4, 4, 4, 1>;     // 32 x 32 pairs, 512 threads
using F32_P22 = GramCfg<float, 4, 4, 8, 2, 2, 4, 2, 4, 1>;     // 32 x 32 pairs, 256 threads
using F32_P12 = GramCfg<float, 4, 8, 4, 1, 2, 4, 4, 4, 1>;     // 32 x 32 pairs, 512 threads
using F32_P22w = GramCfg<float, 4, 4, 8, 2, 2, 6, 2, 4, 1>;    // 48 x 32 pairs, 384 threads
using F32_P21w = GramCfg<float, 4, 4, 8, 2, 1, 4, 3, 4, 1>;    // 32 x 24 pairs, 384 threads
using F32_P14 = GramCfg<float, 4, 8, 4, 1, 4, 4, 2, 4, 1>;     // 32 x 32 pairs, 256 threads
using F32_P22wS2 = GramCfg<float, 4, 4, 8, 2, 2, 6, 2, 3, 1, 2>;  // 48 x 32 pairs, 384 threads, 2 sites/stage
using F32_P22S2 = GramCfg<float, 4, 4, 8, 2, 2, 4, 2, 3, 1, 2>;   // 32 x 32 pairs, 256 threads, 2 sites/stage
using F32_P22wS4 = GramCfg<float, 4, 4, 8, 2, 2, 6, 2, 2, 1, 4>;  // 48 x 32 pairs, 384 threads, 4 sites/stage
using F32_P22wS8 = GramCfg<float, 4, 4, 8, 2, 2, 6, 2, 2, 1, 8>;  // 48 x 32 pairs, 384 threads, 8 sites/stage
using F32_P22S8 = GramCfg<float, 4, 4, 8, 2, 2, 4, 2, 2, 1, 8>;   // 32 x 32 pairs, 256 threads, 8 sites/stage
using F32_P22hS8 = GramCfg<float, 4, 4, 8, 2, 2, 2, 2, 2, 2, 8>;  // 16 x 32 pairs, 128 threads, 2 CTAs per SM
using F32_P22vS8 = GramCfg<float, 4, 4, 8, 2, 2, 4, 1, 2, 2, 8>;  // 32 x 16 pairs, 128 threads, 2 CTAs per SM
using F32_P22qS4 = GramCfg<float, 4, 4, 8, 2, 2, 2, 1, 2, 4, 4>;  // 16 x 16 pairs, 64 threads, 4 CTAs per SM
using F32_P22tS4 = GramCfg<float, 4, 4, 8, 2, 2, 4, 1, 2, 3, 4>;  // 32 x 16 pairs, 128 threads, 3 CTAs per SM
using F32_P22qS6 = GramCfg<float, 4, 4, 8, 2, 2, 2, 1, 2, 4, 6>;  // 16 x 16 pairs, 4 CTAs per SM, 6 sites/stage
using F32_P22vS5 = GramCfg<float, 4, 4, 8, 2, 2, 4, 1, 3, 2, 5>;  // 32 x 16 pairs, 2 CTAs per SM, 3 stages of 5
using F32_P22oS4 = GramCfg<float, 4, 4, 8, 2, 2, 1, 1, 2, 8, 4>;  // 8 x 16 pairs, one warp, 8 CTAs per SM
using F64_P11 = GramCfg<double, 4, 4, 8, 1, 1, 4, 2, 4, 1>;    // 16 x 16 pairs, 256 threads
using F32X8_P11 = GramCfg<float, 8, 4, 8, 1, 1, 4, 2, 4, 1>;   // chi = 8: 16 x 16 pairs, 256 threads
using F32X8_S4 = GramCfg<float, 8, 4, 8, 1, 1, 4, 2, 2, 1, 4>;    // chi = 8: 16 x 16, 2 stages of 4 sites
using F32X8_S2 = GramCfg<float, 8, 4, 8, 1, 1, 4, 2, 3, 1, 2>;    // chi = 8: 16 x 16, 3 stages of 2 sites
using F32X8_h = GramCfg<float, 8, 4, 8, 1, 1, 2, 2, 2, 2, 4>;     // chi = 8: 8 x 16, 128 threads, 2 CTAs per SM
using F32X8_q = GramCfg<float, 8, 4, 8, 1, 1, 2, 1, 2, 4, 2>;     // chi = 8: 8 x 8, 64 threads, 4 CTAs per SM

template <class Cfg>
static dk_status launch_gram(dk_ctx* ctx, const void* mps_r, int m_r, const void* mps_c, int m_c, GramArgs a,
                             cudaStream_t st) {
  a.ntiles = count_tiles(a, Cfg::TR, Cfg::TC);
  return GramLauncher<Cfg>::run(ctx, mps_r, m_r, mps_c, m_c, a, st);
}

struct CfgInfo {
  int tile_rows, tile_cols, threads;
};
template <class Cfg>
constexpr CfgInfo info_of() {
  return CfgInfo{Cfg::TR, Cfg::TC, Cfg::NTHREADS};
}
// Shapes selectable for complex64 / chi 4, in id order 1..19; the built-in choice is kF32Chi4Default.
static const CfgInfo kF32Chi4[] = {info_of<F32_P11>(),  info_of<F32_P21>(),  info_of<F32_P22>(), info_of<F32_P12>(),
                                   info_of<F32_P22w>(), info_of<F32_P21w>(), info_of<F32_P14>(),
                                   info_of<F32_P22wS2>(), info_of<F32_P22S2>(), info_of<F32_P22wS4>(),
                                   info_of<F32_P22wS8>(), info_of<F32_P22S8>(),
                                   info_of<F32_P22hS8>(), info_of<F32_P22vS8>(), info_of<F32_P22qS4>(),
                                   info_of<F32_P22tS4>(), info_of<F32_P22qS6>(), info_of<F32_P22vS5>(),
                                   info_of<F32_P22oS4>()};
constexpr int kF32Chi4Default = 17;  // 16 x 16 pairs, 4 CTAs per SM, 6-site stages: fastest on the n = 784 Gram and rows
static const CfgInfo kF64Chi4[] = {info_of<F64_P11>()};
constexpr int kF32Chi8Default = 2;  // 16 x 16 pairs, 2 stages of 4 sites: fastest at d = 256
static const CfgInfo kF32Chi8[] = {info_of<F32X8_P11>(), info_of<F32X8_S4>(), info_of<F32X8_S2>(),
                                   info_of<F32X8_h>(), info_of<F32X8_q>()};

static dk_status gram_dispatch(dk_ctx* ctx, const void* mps_r, int m_r, const void* mps_c, int m_c, int chi,
                               dk_dtype dtype, dk_precision prec, const GramArgs& a, cudaStream_t st) {
  if (dtype == DK_C64 && prec == DK_PREC_F32 && chi == 4) {
    const int id = ctx->gram_config > 0 ? ctx->gram_config : kF32Chi4Default;
    switch (id) {
      case 1: return launch_gram<F32_P11>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 2: return launch_gram<F32_P21>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 4: return launch_gram<F32_P12>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 5: return launch_gram<F32_P22w>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 6: return launch_gram<F32_P21w>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 7: return launch_gram<F32_P14>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 8: return launch_gram<F32_P22wS2>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 9: return launch_gram<F32_P22S2>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 10: return launch_gram<F32_P22wS4>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 11: return launch_gram<F32_P22wS8>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 12: return launch_gram<F32_P22S8>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 13: return launch_gram<F32_P22hS8>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 14: return launch_gram<F32_P22vS8>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 15: return launch_gram<F32_P22qS4>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 16: return launch_gram<F32_P22tS4>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 17: return launch_gram<F32_P22qS6>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 18: return launch_gram<F32_P22vS5>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 19: return launch_gram<F32_P22oS4>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 3: return launch_gram<F32_P22>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      default: return launch_gram<F32_P22qS6>(ctx, mps_r, m_r, mps_c, m_c, a, st);
    }
  }
  if (dtype == DK_C128 && prec == DK_PREC_F64 && chi == 4)
    return launch_gram<F64_P11>(ctx, mps_r, m_r, mps_c, m_c, a, st);
  if (dtype == DK_C64 && prec == DK_PREC_F32 && chi == 8) {
    // shape ids index the bond-8 table; an id beyond it (e.g. one chosen for bond 4) gives
    // the default
    switch (ctx->gram_config) {
      case 1: return launch_gram<F32X8_P11>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 3: return launch_gram<F32X8_S2>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 4: return launch_gram<F32X8_h>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      case 5: return launch_gram<F32X8_q>(ctx, mps_r, m_r, mps_c, m_c, a, st);
      default: return launch_gram<F32X8_S4>(ctx, mps_r, m_r, mps_c, m_c, a, st);  // kF32Chi8Default
    }
  }
  if (dtype == DK_C64 && prec == DK_PREC_F32 && chi == 32) return gram32_launch(ctx, mps_r, m_r, mps_c, m_c, a, st);
  if (dtype == DK_C64 && prec == DK_PREC_BF16X3 && chi == 32)
    return gram32_tc_launch(ctx, mps_r, m_r, mps_c, m_c, a, false, st);
  if (dtype == DK_SPLIT_BF16 && prec == DK_PREC_BF16X3 && chi == 32)
    return gram32_tc_launch(ctx, mps_r, m_r, mps_c, m_c, a, true, st);
  return DK_ERR_UNSUPPORTED;
}

}  // namespace dk

DK_API dk_status dk_gram_tile(dk_ctx* ctx, const void* mps_rows, int m_rows, const void* mps_cols, int m_cols,
                              int n, int chi_max, dk_dtype dtype, int row0, int nrows, int col0, int ncols,
                              const float* log_norm_rows, const float* log_norm_cols, const float* x_rows,
                              const float* x_cols, float gamma, float w, dk_precision prec, float* k_out,
                              float* kq_out, float* kc_out, float* logkq_out, int64_t ld, int symmetric,
                              void* stream) {
  using namespace dk;
  if (!ctx || !mps_rows || !mps_cols || n < 1 || m_rows < 1 || m_cols < 1) return DK_ERR_ARG;
  if (row0 < 0 || nrows < 0 || col0 < 0 || ncols < 0) return DK_ERR_ARG;
  if ((long long)row0 + nrows > m_rows || (long long)col0 + ncols > m_cols) return DK_ERR_ARG;
  if (!aligned16(mps_rows) || !aligned16(mps_cols)) return DK_ERR_ARG;
  const bool any_out = k_out || kq_out || kc_out || logkq_out;
  if (any_out && ld < ncols) return DK_ERR_ARG;
  if (symmetric) {
    if (mps_rows != mps_cols || row0 != col0 || nrows != ncols || m_rows != m_cols) return DK_ERR_ARG;
    if (x_rows != x_cols || log_norm_rows != log_norm_cols) return DK_ERR_ARG;
    if (any_out && ld < nrows) return DK_ERR_ARG;
  }
  const bool need_x = kc_out != nullptr || (k_out != nullptr && w != 1.0f);
  if (need_x && (!x_rows || !x_cols)) return DK_ERR_ARG;
  if (!(w >= 0.0f && w <= 1.0f)) return DK_ERR_ARG;
  if (nrows == 0 || ncols == 0 || !any_out) return DK_OK;

  GramArgs a{};
  a.n = n;
  a.row0 = row0;
  a.nrows = nrows;
  a.col0 = col0;
  a.ncols = ncols;
  a.symmetric = symmetric ? 1 : 0;
  a.lnorm_r = log_norm_rows;
  a.lnorm_c = log_norm_cols;
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
  a.need_kc = need_x ? 1 : 0;
  return gram_dispatch(ctx, mps_rows, m_rows, mps_cols, m_cols, chi_max, dtype, prec, a,
                       static_cast<cudaStream_t>(stream));
}

DK_API int dk_gram_config_count(dk_dtype dtype, int chi_max) {
  if (dtype == DK_C64 && chi_max == 4) return int(sizeof(dk::kF32Chi4) / sizeof(dk::kF32Chi4[0]));
  if (dtype == DK_C128 && chi_max == 4) return int(sizeof(dk::kF64Chi4) / sizeof(dk::kF64Chi4[0]));
  if (dtype == DK_C64 && chi_max == 8) return int(sizeof(dk::kF32Chi8) / sizeof(dk::kF32Chi8[0]));
  return 0;
}

DK_API dk_status dk_gram_config_info(dk_dtype dtype, int chi_max, int id, int* tile_rows, int* tile_cols,
                                     int* threads) {
  const int count = dk_gram_config_count(dtype, chi_max);
  if (id < 0 || id > count || count == 0) return DK_ERR_ARG;
  const dk::CfgInfo* tab = dtype == DK_C64 ? (chi_max == 4 ? dk::kF32Chi4 : dk::kF32Chi8) : dk::kF64Chi4;
  const int dflt = dtype == DK_C64 ? (chi_max == 4 ? dk::kF32Chi4Default : dk::kF32Chi8Default) : 1;
  const int idx = (id == 0 ? dflt : id) - 1;
  if (tile_rows) *tile_rows = tab[idx].tile_rows;
  if (tile_cols) *tile_cols = tab[idx].tile_cols;
  if (threads) *threads = tab[idx].threads;
  return DK_OK;
}

DK_API dk_status dk_set_gram_config(dk_ctx* ctx, int id) {
  if (!ctx || id < 0 || id > dk_gram_config_count(DK_C64, 4)) return DK_ERR_ARG;
  ctx->gram_config = id;
  return DK_OK;
}

DK_API dk_status dk_dual_kernel_rows(dk_ctx* ctx, const void* mps_test, const float* x_test,
                                     const float* log_norm_test, int b, const void* mps_train, const float* x_train,
                                     const float* log_norm_train, int m, int n, int chi_max, dk_dtype dtype,
                                     float gamma, float w, dk_precision prec, float* k_out, float* kq_out,
                                     float* kc_out, float* logkq_out, void* stream) {
  if (b == 0) return ctx ? DK_OK : DK_ERR_ARG;
  return dk_gram_tile(ctx, mps_test, b, mps_train, m, n, chi_max, dtype, 0, b, 0, m, log_norm_test, log_norm_train,
                      x_test, x_train, gamma, w, prec, k_out, kq_out, kc_out, logkq_out, m, 0, stream);
}
