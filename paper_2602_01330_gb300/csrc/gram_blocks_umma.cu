// Block-statevector Gram (see gram_blocks.cu) on the fifth-generation tensor cores:
// tcgen05.mma with both operands in shared memory and FP32 accumulators in tensor memory.
//
// For block B and a tile of 128 row samples x BN column samples the factor of the overlap
// is the complex GEMM G_B = A^H B over K = 2^b amplitudes, taken with split-BF16 operands
// (v ~ hi + lo) and FP32 accumulation as lo.hi + hi.lo + hi.hi (bf16x3, the precision of
// gram_blocks_tc.cu). Two instruction forms (Cfg):
//   wide (128 x 128 tiles): per 16 amplitudes six 128 x 256 x 16 MMAs, D1 = a_re [b_re; b_im]
//             and D2 = a_im [b_re; b_im], the 256 B rows being the tile's column rows and a
//             second copy of them one plane further on; Re = D1_re + D2_im, Im = D1_im - D2_re;
//   narrow (128 x 64 tiles): twelve 128 x 64 x 16 MMAs, six into Re G (ar br + ai bi) and six
//             into Im G (ar bi - ai br, the minus through the instruction's negate-B bit).
//
// Warp roles of a CTA (one CTA per SM, persistent over its work items):
//   warp 0    one thread issues the TMA loads: per (item, block, 16-amplitude chunk) one
//             128-byte row per sample (the chunk's four BF16 planes, which dk_block_states
//             interleaves in HBM) for the 128 row and BN column samples (twice for the wide
//             form), 128-byte swizzle, into a ring of stages (full / empty mbarriers);
//   warp 1    allocates the tensor memory (512 columns wide, 256 narrow) and one thread
//             issues the MMAs; tcgen05.commit releases each stage to the loader and hands a
//             finished block's accumulator to the epilogue;
//   warps 2-9 the epilogue: thread (TMEM lane r, column half h) reads BN/2 columns of Re and
//             Im of row r, adds log2 |G_B|^2 to its running sums and frees the accumulator
//             (narrow: two accumulators, so block B's epilogue runs under the MMAs of block
//             B + 1); after an item's last block it writes the tile through the common
//             epilogue (write_pair) with the squared distances of the RBF kernel, which
//             rbf_d2_kernel computed beforehand (feature rows staged through shared memory,
//             the per-pair Kahan FP32 sum of every Gram kernel), or, when a rectangular
//             tile's blocks are split over several items, its partial log2 sums.
//
// Self-norms (diagonal mode): a unit is one (diagonal tile, block) pair with A = B in shared
// memory. The diagonal tile of the symmetric Gram issues the same instructions on the same
// shared-memory contents, so |G_B(i, i)|^2 is bit-identical in both; the epilogue stores it
// per (block, sample) and a second kernel adds the log2 terms in block order, as the Gram
// epilogue does, so K_q(x, x) = 1 exactly.
#include <math.h>

#include "common.cuh"
#include "gram_common.cuh"
#include "internal.h"

namespace dk {
namespace gbum {

using u32 = uint32_t;
using u64 = uint64_t;

constexpr int BM = 128;     // tile rows = MMA M = TMEM lanes
constexpr int ROWB = 128;   // one 16-amplitude chunk of a sample: 4 planes x 16 BF16
constexpr int NEPI = 8;     // epilogue warps
constexpr int NTHREADS = (2 + NEPI) * 32;

// BN columns per tile. Narrow form (WIDE = false): N = BN instructions into [Re | Im]
// accumulators, two of them (double-buffered). Wide form (BN = 128): the column rows are
// staged twice, the second copy shifted by one plane (16 BF16), so at byte offset 0 / 64 of
// a row the 256 rows [copy 1; copy 2] hold [b_re; b_im] of the hi / lo planes; the N = 256
// instructions D1 = a_re [b_re; b_im]^T and D2 = a_im [b_re; b_im]^T fill one accumulator of
// 512 columns, and Re = D1[:, re] + D2[:, im], Im = D1[:, im] - D2[:, re] in the epilogue.
template <int BN, bool WIDE>
struct Cfg {
  static_assert(BN % 16 == 0 && BN >= 32 && BN <= 128, "MMA N for M = 128");
  static_assert(!WIDE || BN == 128, "the wide form pairs 128 real and 128 imaginary rows");
  static constexpr int A_BYTES = BM * ROWB;
  static constexpr int B_BYTES = BN * ROWB;                   // one copy of the column rows
  static constexpr int STAGE = A_BYTES + (WIDE ? 2 : 1) * B_BYTES;  // multiples of 1024 (swizzle atoms)
  static constexpr int NST = WIDE ? 4 : 6;                    // stages in the ring
  static constexpr int NACC = WIDE ? 1 : 2;                   // accumulators
  static constexpr int ACC = WIDE ? 4 * BN : 2 * BN;          // TMEM columns of one accumulator
  static constexpr u32 TMEM_COLS = NACC * ACC;                // a power of two, >= 32
  static constexpr int CPT = BN / 2;                          // columns per epilogue thread
  static constexpr size_t SMEM = 1024 + size_t(NST) * STAGE + 256;
};

// Instruction descriptor of kind::f16: F32 accumulator, BF16 A and B, both K-major,
// M = 128, N = the template argument; neg_b negates B.
template <int N>
__host__ __device__ constexpr u32 idesc(bool neg_b) {
  static_assert(N % 16 == 0 && N >= 16 && N <= 256, "MMA N for M = 128");
  return (1u << 4) | (1u << 7) | (1u << 10) | (neg_b ? (1u << 14) : 0u) | (u32(N >> 3) << 17) | (u32(BM >> 4) << 24);
}

// Shared-memory descriptor of a K-major operand in the 128-byte swizzle layout written by
// TMA: rows of 128 bytes, 8-row atoms 1024 bytes apart; `saddr` may sit 32 p bytes into a
// row (plane p), the swizzle being applied to the final address.
__device__ __forceinline__ u64 sw128_desc(u32 saddr) {
  return u64((saddr & 0x3FFFFu) >> 4) | (u64(1) << 16) | (u64(1024 >> 4) << 32) | (u64(1) << 46) | (u64(2) << 61);
}

__device__ __forceinline__ void tc_alloc(u32 dst, u32 ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(u32 taddr, u32 ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// `bar` receives one arrival once every MMA this thread issued so far has completed
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// D (+)= A B^T, D in tensor memory; accumulate = 0 overwrites D
__device__ __forceinline__ void tc_mma(u32 d, u64 a, u64 b, u32 id, u32 accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(accumulate)
      : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane from two column offsets, waited for
__device__ __forceinline__ void tc_ld16x2(u32 ta, u32 tb, float (&va)[16], float (&vb)[16]) {
  u32 a[16], b[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, "
      "[%33];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]), "=r"(a[8]),
        "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15]), "=r"(b[0]),
        "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]), "=r"(b[5]), "=r"(b[6]), "=r"(b[7]), "=r"(b[8]), "=r"(b[9]),
        "=r"(b[10]), "=r"(b[11]), "=r"(b[12]), "=r"(b[13]), "=r"(b[14]), "=r"(b[15])
      : "r"(ta), "r"(tb)
      : "memory");
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    va[e] = __uint_as_float(a[e]);
    vb[e] = __uint_as_float(b[e]);
  }
}

__device__ __forceinline__ float half_log_lg(float lg) { return lg * (0.5f * 0.69314718055994530942f); }
__device__ __forceinline__ float abs2(float re, float im) { return fmaf(re, re, __fmul_rn(im, im)); }

// Gram mode (diag = 0): tiles of p (symmetric or rectangular); with ksplit > 1 (rectangular
// only) each tile's blocks are split into ksplit ranges, each range a work item whose partial
// log2 sums go to part[split][i - row0][j - col0] for split_finish_kernel. Diagonal mode
// (diag = 1): n_units = ceil(m_diag / 128) * nb items (diagonal tile, block) over the states
// of tm_r, |G_B(i, i)|^2 written to g2_out[blk][i].
template <int BN, bool WIDE>
__global__ void __launch_bounds__(NTHREADS, 1)
    gram_blocks_umma_kernel(const __grid_constant__ CUtensorMap tm_r, const __grid_constant__ CUtensorMap tm_c,
                            const GramArgs p, int nb, int cpb, int diag, int n_units, float* __restrict__ g2_out,
                            int m_diag, int ksplit, float* __restrict__ part) {
  using C = Cfg<BN, WIDE>;
  constexpr int NSTAGES = C::NST;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NSTAGES * C::STAGE);
  uint64_t* empty = full + NSTAGES;
  uint64_t* acc_full = empty + NSTAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* done = acc_empty + 2;
  u32* tmem_slot = reinterpret_cast<u32*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < NSTAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], NEPI);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tensormap(&tm_r);
    if (!diag) prefetch_tensormap(&tm_c);
  }
  if (warp == 1) {
    tc_alloc(smem_u32(tmem_slot), C::TMEM_COLS);
    tc_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const u32 tmem = *tmem_slot;

  const int grid = int(gridDim.x), bid = int(blockIdx.x);
  // Work items of this CTA: w = bid, bid + grid, ... < n_items. Gram mode: tile w / ksplit,
  // blocks [b0, b1) of its split w % ksplit; diagonal mode: diagonal tile w / nb, block w % nb.
  // An item is a sequence of units (one per block); every role walks the same sequence.
  const int n_items = diag ? n_units : p.ntiles * ksplit;
  auto item = [&](int w, int& r0, int& c0, int& b0, int& b1, int& split) {
    if (diag) {
      const int ti = w / nb;
      b0 = w - ti * nb;
      b1 = b0 + 1;
      r0 = c0 = ti * BM;
      split = 0;
    } else {
      const int t = w / ksplit;
      split = w - t * ksplit;
      b0 = int((long long)split * nb / ksplit);
      b1 = int((long long)(split + 1) * nb / ksplit);
      int ti, tj;
      decode_tile(p, BM, BN, t, ti, tj);
      r0 = p.row0 + ti * BM;
      c0 = p.col0 + tj * BN;
    }
  };
  auto give_up = [&]() {
    record_status(p.status, DEV_TIMEOUT);
    *abort_flag = 1;
  };

  if (warp == 0) {
    // ---- TMA loader ----
    if (lane == 0) {
      const u32 tx = WIDE ? (diag ? u32(2 * C::A_BYTES) : u32(C::STAGE)) : (diag ? u32(C::A_BYTES) : u32(C::STAGE));
      long long it = 0;  // stage fills issued
      bool stop = false;
      for (int w = bid; w < n_items && !stop && !*abort_flag; w += grid) {
        int r0, c0, b0, b1, split;
        item(w, r0, c0, b0, b1, split);
        for (int blk = b0; blk < b1 && !stop; ++blk) {
          for (int c = 0; c < cpb; ++c) {
            const int s = int(it % NSTAGES);
            const long long round = it / NSTAGES;
            if (round > 0 && !mbar_wait_bounded(&empty[s], u32((round - 1) & 1))) {
              give_up();
              stop = true;
              break;
            }
            uint8_t* sa = smem + s * C::STAGE;
            mbar_arrive_expect_tx(&full[s], tx);
            tma_load_3d(sa, &tm_r, &full[s], c * 64, r0, blk);
            if (!diag) tma_load_3d(sa + C::A_BYTES, &tm_c, &full[s], c * 64, c0, blk);
            if (WIDE)  // the column rows again, one plane on (x + 16: 32 bytes, a 16-byte multiple)
              tma_load_3d(sa + (diag ? C::A_BYTES : C::A_BYTES + C::B_BYTES), diag ? &tm_r : &tm_c, &full[s],
                          c * 64 + 16, diag ? r0 : c0, blk);
            ++it;
          }
        }
      }
      // every issued copy has landed before the CTA may exit
      for (int s = 0; s < NSTAGES; ++s)
        if (it > s && !mbar_wait_bounded(&full[s], u32(((it - 1 - s) / NSTAGES) & 1))) record_status(p.status, DEV_TIMEOUT);
    }
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      constexpr u32 ID_POS = idesc<BN>(false), ID_NEG = idesc<BN>(true), ID_W = idesc<2 * BN>(false);
      long long it = 0, k = 0;  // stages consumed, units issued
      bool stop = false;
      for (int w = bid; w < n_items && !stop && !*abort_flag; w += grid) {
        int r0, c0, b0, b1, split;
        item(w, r0, c0, b0, b1, split);
        for (int blk = b0; blk < b1 && !stop; ++blk, ++k) {
          const int a = C::NACC == 2 ? int(k & 1) : 0;
          const long long use = C::NACC == 2 ? (k >> 1) : k;
          if (use > 0 && !mbar_wait_bounded(&acc_empty[a], u32((use - 1) & 1))) {
            give_up();
            stop = true;
            break;
          }
          tc_fence_after();
          const u32 d_re = tmem + u32(a * C::ACC), d_im = d_re + BN;
          for (int c = 0; c < cpb; ++c, ++it) {
            const int s = int(it % NSTAGES);
            if (!mbar_wait_bounded(&full[s], u32((it / NSTAGES) & 1))) {
              give_up();
              stop = true;
              break;
            }
            tc_fence_after();
            const u32 sa = smem_u32(smem + s * C::STAGE);
            const u32 sb = diag ? sa : sa + C::A_BYTES;
            // planes: 0 hi(re), 1 hi(im), 2 lo(re), 3 lo(im), 32 bytes apart in a row
            const u64 a0 = sw128_desc(sa), a1 = sw128_desc(sa + 32), a2 = sw128_desc(sa + 64),
                      a3 = sw128_desc(sa + 96);
            const u32 acc = c > 0 ? 1u : 0u;
            if (WIDE) {
              // B = [column rows; the copy one plane on]: [b_re; b_im] at offset 0 (hi), 64 (lo)
              const u64 bh = sw128_desc(sb), bl = sw128_desc(sb + 64);
              const u32 d1 = d_re, d2 = d_re + 2 * BN;
              tc_mma(d1, a2, bh, ID_W, acc);  // D1 += a_re [b_re; b_im]
              tc_mma(d1, a0, bl, ID_W, 1u);
              tc_mma(d1, a0, bh, ID_W, 1u);
              tc_mma(d2, a3, bh, ID_W, acc);  // D2 += a_im [b_re; b_im]
              tc_mma(d2, a1, bl, ID_W, 1u);
              tc_mma(d2, a1, bh, ID_W, 1u);
              tc_commit(&empty[s]);
              continue;
            }
            const u64 b0d = sw128_desc(sb), b1d = sw128_desc(sb + 32), b2d = sw128_desc(sb + 64),
                      b3d = sw128_desc(sb + 96);
            tc_mma(d_re, a2, b0d, ID_POS, acc);  // Re += ar br
            tc_mma(d_re, a0, b2d, ID_POS, 1u);
            tc_mma(d_re, a0, b0d, ID_POS, 1u);
            tc_mma(d_re, a3, b1d, ID_POS, 1u);   // Re += ai bi
            tc_mma(d_re, a1, b3d, ID_POS, 1u);
            tc_mma(d_re, a1, b1d, ID_POS, 1u);
            tc_mma(d_im, a2, b1d, ID_POS, acc);  // Im += ar bi
            tc_mma(d_im, a0, b3d, ID_POS, 1u);
            tc_mma(d_im, a0, b1d, ID_POS, 1u);
            tc_mma(d_im, a3, b0d, ID_NEG, 1u);   // Im -= ai br
            tc_mma(d_im, a1, b2d, ID_NEG, 1u);
            tc_mma(d_im, a1, b0d, ID_NEG, 1u);
            tc_commit(&empty[s]);
          }
          if (!stop) tc_commit(&acc_full[a]);
        }
      }
      tc_commit(done);
      if (!mbar_wait_bounded(done, 0u)) record_status(p.status, DEV_TIMEOUT);
    }
  } else {
    // ---- epilogue ----
    const int q = warp & 3;           // the TMEM lane quarter this warp may access
    const int h = (warp - 2) >> 2;    // column half
    const int r = 32 * q + lane;      // tile row = TMEM lane
    const u32 t_row = tmem + (u32(32 * q) << 16) + u32(h * C::CPT);
    float lg[C::CPT];
#pragma unroll
    for (int u = 0; u < C::CPT; ++u) lg[u] = 0.0f;
    long long k = 0;
    bool stop = false;
    for (int w = bid; w < n_items && !stop; w += grid) {
      int r0, c0, b0, b1, split;
      item(w, r0, c0, b0, b1, split);
      const int i = r0 + r;
      for (int blk = b0; blk < b1; ++blk, ++k) {
        const int a = C::NACC == 2 ? int(k & 1) : 0;
        const u32 par = C::NACC == 2 ? u32((k >> 1) & 1) : u32(k & 1);
        // one decision per warp: the loads below are warp-collective
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&acc_full[a], par))) {
          if (lane == 0) give_up();
          stop = true;
          break;
        }
        tc_fence_after();
        float dg = 0.0f;
#pragma unroll
        for (int cc = 0; cc < C::CPT / 16; ++cc) {
          float re[16], im[16];
          tc_ld16x2(t_row + u32(a * C::ACC + 16 * cc), t_row + u32(a * C::ACC + BN + 16 * cc), re, im);
          if (WIDE) {  // re, im hold ar br, ar bi; D2 holds ai br, ai bi
            float x2[16], y2[16];
            tc_ld16x2(t_row + u32(2 * BN + 16 * cc), t_row + u32(3 * BN + 16 * cc), x2, y2);
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              re[e] = re[e] + y2[e];
              im[e] = im[e] - x2[e];
            }
          }
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const float g2 = abs2(re[e], im[e]);
            if (diag) {
              if (h * C::CPT + 16 * cc + e == r) dg = g2;
            } else {
              lg[16 * cc + e] += log2f(g2);
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[a]);
        if (diag) {
          if (r / C::CPT == h && i < m_diag) g2_out[size_t(blk) * m_diag + i] = dg;
        }
      }
      if (diag || stop) continue;
      // end of the item: the tile's outputs, or (split over the blocks) its partial log sums
#pragma unroll
      for (int u = 0; u < C::CPT; ++u) {
        const int j = c0 + h * C::CPT + u;
        const bool valid = i < p.row0 + p.nrows && j < p.col0 + p.ncols && !(p.symmetric && j < i);
        const size_t at = size_t(i - p.row0) * size_t(p.ncols) + size_t(j - p.col0);
        if (ksplit > 1) {
          if (valid) part[size_t(split) * size_t(p.nrows) * size_t(p.ncols) + at] = lg[u];
        } else {
          write_pair(p, half_log_lg(lg[u]), (valid && p.need_kc) ? p.d2[at] : 0.0f, i, j);
        }
        lg[u] = 0.0f;
      }
    }
  }

  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tc_dealloc(tmem, C::TMEM_COLS);
  }
}

// Squared feature distances of the pairs of a Gram block (RBF kernel, Eq. 3): 64 x 64 pairs
// per tile, 256 threads with 4 x 4 pairs each, feature rows staged through shared memory 32
// features at a time; per pair the Kahan FP32 sum of (x_i[f] - x_j[f])^2 over f = 0 .. n-1 in
// order, the additions of every Gram kernel's epilogue. d2[(i - row0) ld2 + (j - col0)];
// symmetric blocks get the pairs with j >= i.
constexpr int RT = 64, RF = 32;
__global__ void __launch_bounds__(256) rbf_d2_kernel(const GramArgs p, float* __restrict__ d2, int ld2) {
  __shared__ float xr[RF][RT + 1], xc[RF][RT + 1];  // [feature][sample]
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int t = blockIdx.x; t < p.ntiles; t += gridDim.x) {
    int ti, tj;
    decode_tile(p, RT, RT, t, ti, tj);
    const int r0 = p.row0 + ti * RT, c0 = p.col0 + tj * RT;
    float s[4][4], cmp[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) s[a][b] = cmp[a][b] = 0.0f;
    for (int f0 = 0; f0 < p.n; f0 += RF) {
      const int nf = min(RF, p.n - f0);
      __syncthreads();  // the previous chunk has been read
      for (int e = threadIdx.x; e < RF * RT; e += 256) {
        const int f = e & (RF - 1), r = e >> 5;
        const int ir = min(r0 + r, p.row0 + p.nrows - 1), jc = min(c0 + r, p.col0 + p.ncols - 1);
        xr[f][r] = f < nf ? __ldg(p.x_r + size_t(ir) * p.n + f0 + f) : 0.0f;
        xc[f][r] = f < nf ? __ldg(p.x_c + size_t(jc) * p.n + f0 + f) : 0.0f;
      }
      __syncthreads();
      for (int f = 0; f < nf; ++f) {
        float va[4], vb[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) va[a] = xr[f][ty + 16 * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) vb[b] = xc[f][tx + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) kahan_add_sq(s[a][b], cmp[a][b], va[a] - vb[b]);
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int i = r0 + ty + 16 * a, j = c0 + tx + 16 * b;
        if (i < p.row0 + p.nrows && j < p.col0 + p.ncols && !(p.symmetric && j < i))
          d2[size_t(i - p.row0) * size_t(ld2) + size_t(j - p.col0)] = s[a][b];
      }
  }
}

// Outputs of a rectangular block computed with its blocks split over ksplit work items: the
// partial log2 sums added in split order, then the common epilogue.
__global__ void split_finish_kernel(const GramArgs p, const float* __restrict__ part, int ksplit) {
  const long long np = (long long)p.nrows * p.ncols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < np; e += (long long)gridDim.x * blockDim.x) {
    float lg = 0.0f;
    for (int s = 0; s < ksplit; ++s) lg += part[size_t(s) * size_t(np) + size_t(e)];
    const int i = p.row0 + int(e / p.ncols), j = p.col0 + int(e % p.ncols);
    write_pair(p, half_log_lg(lg), p.need_kc ? p.d2[e] : 0.0f, i, j);
  }
}

// ln N_i from the per-block diagonal |G_B(i, i)|^2: log2 terms added in block order, as the
// Gram epilogue adds them.
__global__ void selfnorm_sum_kernel(const float* __restrict__ g2, int m, int nb, float* __restrict__ log_norm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  float lg = 0.0f;
  for (int b = 0; b < nb; ++b) lg += log2f(g2[size_t(b) * m + i]);
  log_norm[i] = half_log_lg(lg);
}

// Tensor map over split-BF16 block states [block][sample][dp/16 chunks x 64 BF16]: box of
// one 128-byte chunk row x box_rows samples x 1 block, 128-byte swizzle, zeros past m.
dk_status encode_states_map(dk_ctx* ctx, CUtensorMap* map, const void* states, int m, int nb, int dp, int box_rows) {
  cuuint64_t dims[3] = {cuuint64_t(4) * cuuint64_t(dp), cuuint64_t(m), cuuint64_t(nb)};
  cuuint64_t strides[2] = {cuuint64_t(8) * cuuint64_t(dp), cuuint64_t(8) * cuuint64_t(dp) * cuuint64_t(m)};
  cuuint32_t box[3] = {64u, cuuint32_t(box_rows), 1u};
  cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult r = ctx->encode_tiled(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(states), dims, strides,
                                 box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? DK_OK : DK_ERR_CUDA;
}

// The shared-memory opt-in is a per-device, per-function attribute: it is set before every
// launch (a cheap host call), so no process-wide flag has to track devices or threads.
template <int BN, bool WIDE>
dk_status set_smem() {
  if (cudaFuncSetAttribute(gram_blocks_umma_kernel<BN, WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(Cfg<BN, WIDE>::SMEM)) != cudaSuccess)
    return DK_ERR_CUDA;
  return DK_OK;
}

// Caller-provided scratch of one Gram launch: the RBF distances (nrows x ncols floats, when
// K_c is needed) and, for a rectangular block split over ksplit items, the partial log2 sums
// (ksplit x nrows x ncols floats), each starting on a 256-byte boundary of `ws`.
struct Scratch {
  size_t d2_bytes, part_bytes;
  size_t total() const { return d2_bytes + part_bytes; }
};

inline size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

inline Scratch scratch_of(const GramArgs& a, int ksplit) {
  const size_t np = size_t(a.nrows) * size_t(a.ncols);
  return {a.need_kc ? round256(np * sizeof(float)) : 0, ksplit > 1 ? round256(size_t(ksplit) * np * sizeof(float)) : 0};
}

template <int BN, bool WIDE>
dk_status launch_gram(dk_ctx* ctx, const void* sr, int m_r, const void* sc, int m_c, int nb, int dp, GramArgs a,
                      int ntiles, int ksplit, void* ws, size_t ws_bytes, cudaStream_t st) {
  const Scratch need = scratch_of(a, ksplit);
  if (need.total() > 0 && (!ws || ws_bytes < need.total() || !aligned16(ws))) return DK_ERR_WORKSPACE;
  CUtensorMap tr, tc;
  dk_status s = encode_states_map(ctx, &tr, sr, m_r, nb, dp, BM);
  if (s == DK_OK) s = encode_states_map(ctx, &tc, sc, m_c, nb, dp, BN);
  if (s == DK_OK) s = set_smem<BN, WIDE>();
  if (s != DK_OK) return s;
  a.ntiles = count_tiles(a, BM, BN);  // also sets the tile grid (tiles_r, tiles_c) the kernel decodes
  if (a.ntiles != ntiles) return DK_ERR_ARG;
  const long long items = (long long)ntiles * ksplit;
  const int grid = int(items < ctx->sm_count ? items : ctx->sm_count);
  if (grid < 1) return DK_OK;
  // squared distances of the RBF kernel first, into the caller's scratch
  float* d2 = need.d2_bytes ? static_cast<float*>(ws) : nullptr;
  if (a.need_kc) {
    GramArgs ar = a;
    ar.ntiles = count_tiles(ar, RT, RT);
    const int rgrid = ar.ntiles < 8 * ctx->sm_count ? ar.ntiles : 8 * ctx->sm_count;
    rbf_d2_kernel<<<rgrid, 256, 0, st>>>(ar, d2, a.ncols);
    s = launch_status();
    a.d2 = d2;
  }
  float* part = need.part_bytes ? reinterpret_cast<float*>(static_cast<uint8_t*>(ws) + need.d2_bytes) : nullptr;
  const size_t np = size_t(a.nrows) * size_t(a.ncols);
  if (s == DK_OK) {
    gram_blocks_umma_kernel<BN, WIDE><<<grid, NTHREADS, Cfg<BN, WIDE>::SMEM, st>>>(tr, tc, a, nb, dp / 16, 0, 0,
                                                                                   nullptr, 0, ksplit, part);
    s = launch_status();
  }
  if (s == DK_OK && part) {
    const long long fgrid = (long long)(np + 255) / 256;
    split_finish_kernel<<<int(fgrid < 16LL * ctx->sm_count ? fgrid : 16LL * ctx->sm_count), 256, 0, st>>>(a, part,
                                                                                                       ksplit);
    s = launch_status();
  }
  return s;
}

// The launch plan of a block Gram: symmetric: 128 x 128 tiles, all blocks in one item (the
// diagonal tiles are then the self-norm units, bit for bit). Rectangular: 128 x 128 tiles
// with the blocks split over up to 8 items per tile when there are fewer tiles than SMs, or
// 128 x 64 tiles, whichever takes less time by waves x blocks per item (a 128 x 64
// tile-block costs about 0.92 of a 128 x 128 one: its N = 64 MMAs are bound by shared-memory
// reads).
struct Plan {
  bool wide;
  int ntiles, ksplit;
};

inline Plan plan_gram(const dk_ctx* ctx, GramArgs a, int nb) {
  const int t128 = count_tiles(a, BM, 128);
  if (a.symmetric) return {true, t128, 1};
  const int t64 = count_tiles(a, BM, 64);
  const long long sms = ctx->sm_count;
  long long ks = t128 < sms ? sms / t128 : 1;
  if (ks > nb) ks = nb;
  if (ks > 8) ks = 8;
  if (ks < 1) ks = 1;
  const double cost128 = double((t128 * ks + sms - 1) / sms) * double((nb + ks - 1) / ks);
  const double cost64 = double((t64 + sms - 1) / sms) * double(nb) * 0.92;
  if (cost128 <= cost64) return {true, t128, int(ks)};
  return {false, t64, 1};
}

}  // namespace gbum

size_t gram_blocks_umma_ws_bytes(const dk_ctx* ctx, GramArgs a, int nb) {
  const gbum::Plan pl = gbum::plan_gram(ctx, a, nb);
  return gbum::scratch_of(a, pl.ksplit).total();
}

dk_status gram_blocks_umma_launch(dk_ctx* ctx, const void* sr, int m_r, const void* sc, int m_c, int nb, int dp,
                                  GramArgs a, void* ws, size_t ws_bytes, cudaStream_t st) {
  const gbum::Plan pl = gbum::plan_gram(ctx, a, nb);
  if (pl.wide)
    return gbum::launch_gram<128, true>(ctx, sr, m_r, sc, m_c, nb, dp, a, pl.ntiles, pl.ksplit, ws, ws_bytes, st);
  return gbum::launch_gram<64, false>(ctx, sr, m_r, sc, m_c, nb, dp, a, pl.ntiles, 1, ws, ws_bytes, st);
}

size_t block_selfnorm_umma_ws_bytes(int m, int nb) { return gbum::round256(size_t(nb) * size_t(m) * sizeof(float)); }

dk_status block_selfnorm_umma_launch(dk_ctx* ctx, const void* states, int m, int nb, int dp, float* log_norm,
                                     void* ws, size_t ws_bytes, cudaStream_t st) {
  using namespace gbum;
  const long long units = (long long)((m + BM - 1) / BM) * nb;
  if (units > 0x7fffffffLL) return DK_ERR_UNSUPPORTED;
  if (!ws || ws_bytes < block_selfnorm_umma_ws_bytes(m, nb) || !aligned16(ws)) return DK_ERR_WORKSPACE;
  CUtensorMap t;
  dk_status s = encode_states_map(ctx, &t, states, m, nb, dp, BM);
  if (s == DK_OK) s = set_smem<128, true>();
  if (s != DK_OK) return s;
  float* g2 = static_cast<float*>(ws);
  GramArgs a{};
  a.status = ctx->status;
  const int grid = int(units < ctx->sm_count ? units : ctx->sm_count);
  gram_blocks_umma_kernel<128, true><<<grid, NTHREADS, Cfg<128, true>::SMEM, st>>>(t, t, a, nb, dp / 16, 1, int(units),
                                                                                  g2, m, 1, nullptr);
  s = launch_status();
  if (s == DK_OK) {
    selfnorm_sum_kernel<<<(m + 255) / 256, 256, 0, st>>>(g2, m, nb, log_norm);
    s = launch_status();
  }
  return s;
}

}  // namespace dk
