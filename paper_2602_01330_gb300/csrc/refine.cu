// Refinement of the large kernel values of a Gram block in double-word FP32 arithmetic.
//
// The transfer chain (§II-C, Eqs. 8-10) rounds E at every site. In FP32 the rounding of
// the chain's dominant direction performs a random walk over the n sites, so a kernel value
// K_q of order one carries a relative error of about sqrt(n) * 6 u (7e-6 at n = 784 for the
// bond-4 FP32 kernels; 1e-3 for split-BF16 products at bond 32 and n = 256), while a small
// K_q has the same relative error and hence a tiny absolute one. This pass scans a block
// that a Gram call has written and recomputes every entry with K_q > tau: the amplitude
// a_ij and both self-overlaps N_i, N_j by the same chain with E held as unevaluated sums
// hi + lo of two floats (double-word numbers, about 44 significant bits). The site tensors
// are the stored complex64 ones, exact as FP32 inputs, so only the arithmetic changes:
//   products    x (double-word) * y (float): p = hi y rounded, its exact error
//               fma(hi, y, -p), plus lo y;
//   dot products Dot2 accumulation: the rounded sum of the p's with TwoSum's exact error of
//               every addition and the product errors in a second float; normalised with
//               Fast2Sum into hi + lo once per output element (Ogita, Rump and Oishi, 2005);
//   rescaling   hi and lo multiplied by the same power of two (exact).
// __fadd_rn / __fmul_rn keep the error-free transforms from being contracted into FMAs.
// log K_q = 2 ln|a_ij| - ln N_i - ln N_j is then formed in FP64 and K_q, K = w K_q +
// (1 - w) K_c and log K_q are written back (K_c is read from the block, or recomputed with
// the Gram kernels' compensated feature sum). Entries with K_q <= tau keep their values.
//
// Bond 4 and 8: one thread per pair, E in registers, hits queued per warp so that the
// chains run 32 at a time. Bond 32: one warp per pair, E, the intermediate F and the two
// samples' site blocks in shared memory; each warp tests 32 entries at once and works
// through the hits among them.
#include <math.h>

#include "common.cuh"
#include "gram_common.cuh"
#include "internal.h"

namespace dk {
namespace rf {

struct DW {
  float hi, lo;
};

// Dot2 accumulator: s holds the rounded running sum, c the running sum of the errors.
struct Acc {
  float s, c;
};

__device__ __forceinline__ void acc_add(Acc& A, DW x, float y) {
  const float p = __fmul_rn(x.hi, y);
  float q = fmaf(x.hi, y, -p);
  q = fmaf(x.lo, y, q);
  const float s = __fadd_rn(A.s, p);
  const float bp = __fsub_rn(s, A.s);
  const float e = __fadd_rn(__fsub_rn(A.s, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  A.s = s;
  A.c = __fadd_rn(A.c, __fadd_rn(e, q));
}

__device__ __forceinline__ DW acc_get(const Acc& A) {
  const float s = __fadd_rn(A.s, A.c);
  return {s, __fsub_rn(A.c, __fsub_rn(s, A.s))};
}

__device__ __forceinline__ int exponent_of(float v) { return int((__float_as_uint(v) >> 23) & 0xffu) - 127; }
__device__ __forceinline__ float pow2_neg(int e) { return __uint_as_float(uint32_t(127 - e) << 23); }

// ln|a| for a = (re + i im) 2^e2, with explicitly rounded operations so that every call site
// gives the same bits for the same amplitude (a pair and a self-overlap of one sample agree).
__device__ __forceinline__ double half_log_of(double re, double im, int e2) {
  const double mod2 = __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im));
  return __dadd_rn(__dmul_rn(0.5, log(mod2)), __dmul_rn(double(e2), 0.69314718055994530942));
}

// Complex element (s, jc, l) of a sample's compact site tensor (chi x chi complex64).
__device__ __forceinline__ float2 site_elem(const float2* a, int chi, int h, int s, int jc, int l) {
  return __ldg(a + (s * h + jc) * chi + l);
}

// ---------------- bond 4 / 8: one thread per chain ----------------

template <int H>
struct ChainE {
  DW r[2][H][H], i[2][H][H];
};

// ln|<psi~_i|psi~_j>| by the double-word chain (FP64 result). mi / mj: the two MPS, with
// sample counts m_i / m_j (site-major layout).
template <int H>
__device__ double chain_half_log(const float2* __restrict__ mi, int m_i, int i, const float2* __restrict__ mj, int m_j,
                                 int j, int n) {
  constexpr int CHI = 2 * H;
  ChainE<H> E;
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int a = 0; a < H; ++a)
#pragma unroll
      for (int c = 0; c < H; ++c) E.r[t][a][c] = E.i[t][a][c] = DW{0.0f, 0.0f};
  E.r[0][0][0] = DW{1.0f, 0.0f};
  int e2 = 0;
  for (int k = 0; k < n; ++k) {
    const float2* ai = mi + (size_t(k) * m_i + i) * (CHI * CHI);
    const float2* aj = mj + (size_t(k) * m_j + j) * (CHI * CHI);
    Acc nr[2][H][H], ni[2][H][H];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int c = 0; c < H; ++c) nr[s][p][c] = ni[s][p][c] = Acc{0.0f, 0.0f};
#pragma unroll
    for (int t = 0; t < 2; ++t) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        // F = E_t B with B[b][c] = A_s[t](x_j)[b][c] = element (s, c, t H + b) of sample j
        DW fr[H][H], fi[H][H];
#pragma unroll
        for (int c = 0; c < H; ++c) {
          float br[H], bi[H];
#pragma unroll
          for (int b = 0; b < H; ++b) {
            const float2 v = site_elem(aj, CHI, H, s, c, t * H + b);
            br[b] = v.x;
            bi[b] = v.y;
          }
#pragma unroll
          for (int a = 0; a < H; ++a) {
            Acc xr{0.0f, 0.0f}, xi{0.0f, 0.0f};
#pragma unroll
            for (int b = 0; b < H; ++b) {
              acc_add(xr, E.r[t][a][b], br[b]);
              acc_add(xr, E.i[t][a][b], -bi[b]);
              acc_add(xi, E.r[t][a][b], bi[b]);
              acc_add(xi, E.i[t][a][b], br[b]);
            }
            fr[a][c] = acc_get(xr);
            fi[a][c] = acc_get(xi);
          }
        }
        // E'_s[p][c] += sum_a conj(C[a][p]) F[a][c], C[a][p] = element (s, p, t H + a) of sample i
#pragma unroll
        for (int p = 0; p < H; ++p) {
          float cr[H], ci[H];
#pragma unroll
          for (int a = 0; a < H; ++a) {
            const float2 v = site_elem(ai, CHI, H, s, p, t * H + a);
            cr[a] = v.x;
            ci[a] = v.y;
          }
#pragma unroll
          for (int c = 0; c < H; ++c)
#pragma unroll
            for (int a = 0; a < H; ++a) {
              acc_add(nr[s][p][c], fr[a][c], cr[a]);
              acc_add(nr[s][p][c], fi[a][c], ci[a]);
              acc_add(ni[s][p][c], fi[a][c], cr[a]);
              acc_add(ni[s][p][c], fr[a][c], -ci[a]);
            }
        }
      }
    }
    float mx = 0.0f;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int c = 0; c < H; ++c) {
          E.r[s][p][c] = acc_get(nr[s][p][c]);
          E.i[s][p][c] = acc_get(ni[s][p][c]);
          mx = fmaxf(mx, fmaxf(fabsf(E.r[s][p][c].hi), fabsf(E.i[s][p][c].hi)));
        }
    if (mx > 0.0f && ((k & 3) == 3 || k == n - 1)) {
      const int e = exponent_of(mx);
      const float sc = pow2_neg(e);
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int p = 0; p < H; ++p)
#pragma unroll
          for (int c = 0; c < H; ++c) {
            E.r[s][p][c] = DW{E.r[s][p][c].hi * sc, E.r[s][p][c].lo * sc};
            E.i[s][p][c] = DW{E.i[s][p][c].hi * sc, E.i[s][p][c].lo * sc};
          }
      e2 += e;
    }
  }
  const double re =
      (double(E.r[0][0][0].hi) + double(E.r[0][0][0].lo)) + (double(E.r[1][0][0].hi) + double(E.r[1][0][0].lo));
  const double im =
      (double(E.i[0][0][0].hi) + double(E.i[0][0][0].lo)) + (double(E.i[1][0][0].hi) + double(E.i[1][0][0].lo));
  return half_log_of(re, im, e2);
}

struct RefineArgs {
  GramArgs g;            // block, outputs, x, gamma, w (lnorm unused)
  const float2* mps_r;
  const float2* mps_c;
  int m_r, m_c;
  float tau, log_tau;
  // With a caller workspace: flags of the samples that some entry above tau needs, and their
  // double-word ln-norms, computed once per sample (rows [0, m_r), columns after them; the
  // column arrays alias the row arrays for a symmetric block). NULL: each refined entry
  // computes both of its norms itself.
  int* flag_r;
  int* flag_c;
  double* norm_r;
  double* norm_c;
};

__device__ __forceinline__ bool is_hit(const RefineArgs& a, long long at) {
  if (a.g.kq) return a.g.kq[at] > a.tau;
  return a.g.lkq[at] > a.log_tau;
}

// K_c of pair (i, j) as the Gram kernels form it: the compensated FP32 sum of squared
// feature differences in feature order.
__device__ __forceinline__ float kc_of(const GramArgs& g, long long at, int i, int j) {
  if (g.kc) return g.kc[at];
  if (!g.need_kc) return 0.0f;
  float d2 = 0.0f, comp = 0.0f;
  const float* xa = g.x_r + size_t(i) * g.n;
  const float* xb = g.x_c + size_t(j) * g.n;
  for (int f = 0; f < g.n; ++f) kahan_add_sq(d2, comp, __ldg(xa + f) - __ldg(xb + f));
  return expf(-g.gamma * d2);
}

__device__ __forceinline__ void write_refined(const GramArgs& g, long long at, int i, int j, double lkq_d) {
  const float kq = float(exp(lkq_d));
  const float lkq = float(lkq_d);
  const float kc = kc_of(g, at, i, j);
  const float k = g.w * kq + (1.0f - g.w) * kc;
  if (g.k) g.k[at] = k;
  if (g.kq) g.kq[at] = kq;
  if (g.lkq) g.lkq[at] = lkq;
  if (g.symmetric && i != j) {
    const long long b = (long long)(j - g.row0) * g.ld + (i - g.col0);
    if (g.k) g.k[b] = k;
    if (g.kq) g.kq[b] = kq;
    if (g.kc) g.kc[b] = kc;
    if (g.lkq) g.lkq[b] = lkq;
  }
}

// Each warp tests 32 entries at a time and queues the hits in shared memory; whenever 32
// are queued every lane takes one, so the chains run with full warps even when the hits
// are sparse (a lone hit per warp would otherwise cost the warp its whole chain time).
constexpr int SMALL_WARPS = 4;

template <int H>
__device__ __forceinline__ void refine_one(const RefineArgs& a, int i, int j, long long at) {
  const double lij = chain_half_log<H>(a.mps_r, a.m_r, i, a.mps_c, a.m_c, j, a.g.n);
  const double lii = a.norm_r ? a.norm_r[i] : chain_half_log<H>(a.mps_r, a.m_r, i, a.mps_r, a.m_r, i, a.g.n);
  const double ljj = a.norm_c ? a.norm_c[j] : chain_half_log<H>(a.mps_c, a.m_c, j, a.mps_c, a.m_c, j, a.g.n);
  write_refined(a.g, at, i, j, 2.0 * lij - lii - ljj);
}

// Marks the samples whose ln-norm some entry above tau needs (all entries of the block,
// same test as the refinement pass). Several threads may store the same 1: benign.
__global__ void __launch_bounds__(256) mark_kernel(const RefineArgs a) {
  const GramArgs& g = a.g;
  const long long total = (long long)g.nrows * g.ncols;
  for (long long e = blockIdx.x * 256LL + threadIdx.x; e < total; e += (long long)gridDim.x * 256) {
    const int r = int(e / g.ncols), c = int(e - (long long)r * g.ncols);
    const int i = g.row0 + r, j = g.col0 + c;
    if (g.symmetric && j <= i) continue;
    if (is_hit(a, (long long)r * g.ld + c)) {
      a.flag_r[i] = 1;
      a.flag_c[j] = 1;
    }
  }
}

// ln-norms of the marked samples: entries u < m_r are row samples, the rest column samples
// (none for a symmetric block). Marked samples are queued per warp as in the pass itself.
template <int H>
__device__ __forceinline__ void norm_one(const RefineArgs& a, int u) {
  if (u < a.m_r) a.norm_r[u] = chain_half_log<H>(a.mps_r, a.m_r, u, a.mps_r, a.m_r, u, a.g.n);
  else a.norm_c[u - a.m_r] = chain_half_log<H>(a.mps_c, a.m_c, u - a.m_r, a.mps_c, a.m_c, u - a.m_r, a.g.n);
}

template <int H>
__global__ void __launch_bounds__(128) norms_small_kernel(const RefineArgs a, int n_units) {
  __shared__ int q[4][64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  int count = 0;
  for (int base = (blockIdx.x * 4 + warp) * 32; base < n_units; base += gridDim.x * 4 * 32) {
    const int u = base + lane;
    const bool hit = u < n_units && (u < a.m_r ? a.flag_r[u] : a.flag_c[u - a.m_r]) != 0;
    const unsigned mask = __ballot_sync(0xffffffffu, hit);
    if (hit) q[warp][count + __popc(mask & below)] = u;
    count += __popc(mask);
    __syncwarp();
    if (count >= 32) {
      norm_one<H>(a, q[warp][lane]);
      __syncwarp();
      const int rest = count - 32;
      const int t = lane < rest ? q[warp][32 + lane] : 0;
      __syncwarp();
      if (lane < rest) q[warp][lane] = t;
      count = rest;
      __syncwarp();
    }
  }
  if (lane < count) norm_one<H>(a, q[warp][lane]);
}

template <int H>
__global__ void __launch_bounds__(SMALL_WARPS * 32) refine_small_kernel(const RefineArgs a) {
  __shared__ int qi[SMALL_WARPS][64], qj[SMALL_WARPS][64];
  __shared__ long long qa[SMALL_WARPS][64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const GramArgs& g = a.g;
  const long long total = (long long)g.nrows * g.ncols;
  const long long nwarps = (long long)gridDim.x * SMALL_WARPS;
  const unsigned below = (1u << lane) - 1u;
  int count = 0;
  for (long long base = (blockIdx.x * (long long)SMALL_WARPS + warp) * 32; base < total; base += nwarps * 32) {
    const long long e = base + lane;
    bool hit = false;
    long long at = 0;
    int i = 0, j = 0;
    if (e < total) {
      const int r = int(e / g.ncols), c = int(e - (long long)r * g.ncols);
      i = g.row0 + r;
      j = g.col0 + c;
      at = (long long)r * g.ld + c;
      hit = !(g.symmetric && j <= i) && is_hit(a, at);
    }
    const unsigned mask = __ballot_sync(0xffffffffu, hit);
    if (hit) {
      const int pos = count + __popc(mask & below);
      qi[warp][pos] = i;
      qj[warp][pos] = j;
      qa[warp][pos] = at;
    }
    count += __popc(mask);
    __syncwarp();
    if (count >= 32) {
      refine_one<H>(a, qi[warp][lane], qj[warp][lane], qa[warp][lane]);
      __syncwarp();
      const int rest = count - 32;
      int ti = 0, tj = 0;
      long long ta = 0;
      if (lane < rest) {
        ti = qi[warp][32 + lane];
        tj = qj[warp][32 + lane];
        ta = qa[warp][32 + lane];
      }
      __syncwarp();
      if (lane < rest) {
        qi[warp][lane] = ti;
        qj[warp][lane] = tj;
        qa[warp][lane] = ta;
      }
      count = rest;
      __syncwarp();
    }
  }
  if (lane < count) refine_one<H>(a, qi[warp][lane], qj[warp][lane], qa[warp][lane]);
}

// ---------------- bond 32: one warp per chain ----------------

constexpr int H32 = 16, CHI32 = 32;
constexpr int WARPS32 = 4;
// per warp: E (2 blocks) and F as double-word 16 x 16 complex: [blk][re/im][hi/lo][16][16]
constexpr int EW = 2 * 2 * 2 * 256;  // floats of E
constexpr int FW = 2 * 2 * 256;      // floats of F
constexpr int BW = 2 * 256;          // floats of one 16 x 16 complex float block [re/im][16][16]
constexpr int WARP_FLOATS = EW + FW + 2 * BW;

__device__ __forceinline__ float& dw_ref(float* base, int blk, int ri, int hl, int r, int c) {
  return base[(((blk * 2 + ri) * 2 + hl) * 16 + r) * 16 + c];
}

// ln|<psi~_i|psi~_j>| at bond 32 by one warp (result valid in every lane).
__device__ double chain32_half_log(const float2* __restrict__ mi, int m_i, int i, const float2* __restrict__ mj,
                                   int m_j, int j, int n, float* wbuf, int lane) {
  float* E = wbuf;
  float* F = E + EW;
  float* B = F + FW;  // column-sample block B[b][c]
  float* C = B + BW;  // row-sample block C[a][p]
  for (int q = lane; q < EW; q += 32) E[q] = 0.0f;
  __syncwarp();
  if (lane == 0) dw_ref(E, 0, 0, 0, 0, 0) = 1.0f;
  __syncwarp();
  int e2 = 0;
  for (int k = 0; k < n; ++k) {
    const float2* ai = mi + (size_t(k) * m_i + i) * (CHI32 * CHI32);
    const float2* aj = mj + (size_t(k) * m_j + j) * (CHI32 * CHI32);
    // lane owns outputs o = lane + 32 q (q < 8): row o / 16, column o % 16
    Acc nr[2][8], ni[2][8];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int q = 0; q < 8; ++q) nr[s][q] = ni[s][q] = Acc{0.0f, 0.0f};
    for (int t = 0; t < 2; ++t) {
      for (int s = 0; s < 2; ++s) {
        __syncwarp();
        for (int q = lane; q < 256; q += 32) {
          const int rr = q >> 4, cc = q & 15;
          const float2 vb = site_elem(aj, CHI32, H32, s, cc, t * H32 + rr);  // B[rr][cc]
          B[rr * 16 + cc] = vb.x;
          B[256 + rr * 16 + cc] = vb.y;
          const float2 vc = site_elem(ai, CHI32, H32, s, cc, t * H32 + rr);  // C[a = rr][p = cc]
          C[rr * 16 + cc] = vc.x;
          C[256 + rr * 16 + cc] = vc.y;
        }
        __syncwarp();
        // F[a][c] = sum_b E_t[a][b] B[b][c]
#pragma unroll 1
        for (int q = 0; q < 8; ++q) {
          const int o = lane + 32 * q, a = o >> 4, c = o & 15;
          Acc xr{0.0f, 0.0f}, xi{0.0f, 0.0f};
          for (int b = 0; b < 16; ++b) {
            const DW er{dw_ref(E, t, 0, 0, a, b), dw_ref(E, t, 0, 1, a, b)};
            const DW ei{dw_ref(E, t, 1, 0, a, b), dw_ref(E, t, 1, 1, a, b)};
            const float br = B[b * 16 + c], bi = B[256 + b * 16 + c];
            acc_add(xr, er, br);
            acc_add(xr, ei, -bi);
            acc_add(xi, er, bi);
            acc_add(xi, ei, br);
          }
          const DW fr = acc_get(xr), fi = acc_get(xi);
          dw_ref(F, 0, 0, 0, a, c) = fr.hi;
          dw_ref(F, 0, 0, 1, a, c) = fr.lo;
          dw_ref(F, 0, 1, 0, a, c) = fi.hi;
          dw_ref(F, 0, 1, 1, a, c) = fi.lo;
        }
        __syncwarp();
        // E'_s[p][c] += sum_a conj(C[a][p]) F[a][c]
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int o = lane + 32 * q, p = o >> 4, c = o & 15;
          for (int a2 = 0; a2 < 16; ++a2) {
            const DW fr{dw_ref(F, 0, 0, 0, a2, c), dw_ref(F, 0, 0, 1, a2, c)};
            const DW fi{dw_ref(F, 0, 1, 0, a2, c), dw_ref(F, 0, 1, 1, a2, c)};
            const float cr = C[a2 * 16 + p], ci = C[256 + a2 * 16 + p];
            acc_add(nr[s][q], fr, cr);
            acc_add(nr[s][q], fi, ci);
            acc_add(ni[s][q], fi, cr);
            acc_add(ni[s][q], fr, -ci);
          }
        }
      }
    }
    __syncwarp();
    float mx = 0.0f;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int o = lane + 32 * q, p = o >> 4, c = o & 15;
        const DW vr = acc_get(nr[s][q]), vi = acc_get(ni[s][q]);
        dw_ref(E, s, 0, 0, p, c) = vr.hi;
        dw_ref(E, s, 0, 1, p, c) = vr.lo;
        dw_ref(E, s, 1, 0, p, c) = vi.hi;
        dw_ref(E, s, 1, 1, p, c) = vi.lo;
        mx = fmaxf(mx, fmaxf(fabsf(vr.hi), fabsf(vi.hi)));
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncwarp();
    if (mx > 0.0f && ((k & 3) == 3 || k == n - 1)) {
      const int e = exponent_of(mx);
      const float sc = pow2_neg(e);
      for (int q = lane; q < EW; q += 32) E[q] *= sc;
      e2 += e;
    }
    __syncwarp();
  }
  const double re = (double(dw_ref(E, 0, 0, 0, 0, 0)) + double(dw_ref(E, 0, 0, 1, 0, 0))) +
                    (double(dw_ref(E, 1, 0, 0, 0, 0)) + double(dw_ref(E, 1, 0, 1, 0, 0)));
  const double im = (double(dw_ref(E, 0, 1, 0, 0, 0)) + double(dw_ref(E, 0, 1, 1, 0, 0))) +
                    (double(dw_ref(E, 1, 1, 0, 0, 0)) + double(dw_ref(E, 1, 1, 1, 0, 0)));
  __syncwarp();
  return half_log_of(re, im, e2);
}

__global__ void __launch_bounds__(WARPS32 * 32) refine32_kernel(const RefineArgs a) {
  extern __shared__ __align__(16) float smf[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* wbuf = smf + warp * WARP_FLOATS;
  const GramArgs& g = a.g;
  const long long total = (long long)g.nrows * g.ncols;
  const long long nwarps = (long long)gridDim.x * WARPS32;
  for (long long base = (blockIdx.x * (long long)WARPS32 + warp) * 32; base < total; base += nwarps * 32) {
    const long long e = base + lane;
    bool hit = false;
    long long at = 0;
    int i = 0, j = 0;
    if (e < total) {
      const int r = int(e / g.ncols), c = int(e - (long long)r * g.ncols);
      i = g.row0 + r;
      j = g.col0 + c;
      at = (long long)r * g.ld + c;
      hit = !(g.symmetric && j <= i) && is_hit(a, at);
    }
    unsigned mask = __ballot_sync(0xffffffffu, hit);
    while (mask) {
      const int src = __ffs(mask) - 1;
      mask &= mask - 1;
      const int hi_ = __shfl_sync(0xffffffffu, i, src), hj = __shfl_sync(0xffffffffu, j, src);
      const double lij = chain32_half_log(a.mps_r, a.m_r, hi_, a.mps_c, a.m_c, hj, g.n, wbuf, lane);
      const double lii = a.norm_r ? a.norm_r[hi_]
                                  : chain32_half_log(a.mps_r, a.m_r, hi_, a.mps_r, a.m_r, hi_, g.n, wbuf, lane);
      const double ljj = a.norm_c ? a.norm_c[hj]
                                  : chain32_half_log(a.mps_c, a.m_c, hj, a.mps_c, a.m_c, hj, g.n, wbuf, lane);
      if (lane == src) write_refined(g, at, i, j, 2.0 * lij - lii - ljj);
      __syncwarp();
    }
  }
}

// ln-norms of the marked samples at bond 32: one warp per sample (marked samples often sit
// next to each other, so each warp takes a single sample and the chains run side by side).
__global__ void __launch_bounds__(WARPS32 * 32) norms32_kernel(const RefineArgs a, int n_units) {
  extern __shared__ __align__(16) float smf[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* wbuf = smf + warp * WARP_FLOATS;
  for (int v = blockIdx.x * WARPS32 + warp; v < n_units; v += gridDim.x * WARPS32) {
    if ((v < a.m_r ? a.flag_r[v] : a.flag_c[v - a.m_r]) == 0) continue;  // warp-uniform
    double l;
    if (v < a.m_r) l = chain32_half_log(a.mps_r, a.m_r, v, a.mps_r, a.m_r, v, a.g.n, wbuf, lane);
    else l = chain32_half_log(a.mps_c, a.m_c, v - a.m_r, a.mps_c, a.m_c, v - a.m_r, a.g.n, wbuf, lane);
    if (lane == 0) {
      if (v < a.m_r) a.norm_r[v] = l;
      else a.norm_c[v - a.m_r] = l;
    }
    __syncwarp();
  }
}

inline size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

// ---------------- block-statevector Gram: one warp per refined entry ----------------
//
// A block product state's overlap factorises over the blocks (§II-C, block-structured
// entanglers): log K_q = sum_B [log |<a_B|b_B>|^2 - log <a_B|a_B> - log <b_B|b_B>], each
// factor a complex dot product of the block's 2^b stored amplitudes. The Gram kernels form
// these dot products in FP32 (or split BF16) and sum their logs; over 79 blocks of 1024
// amplitudes the relative error of K_q reaches 5e-5 (FP32) and 4e-4 (split BF16) on values
// of order one. The refinement forms all three dot products of every block exactly as
// products of the stored values (TwoProd residuals) with Dot2 accumulation per lane,
// reduces the lanes in FP64 and sums the logs in FP64.
struct BlockRefineArgs {
  GramArgs g;
  const void* sr;
  const void* sc;
  int m_r, m_c, nb, dp, split;  // split: states in the split-BF16 layout
  float tau, log_tau;
};

// Amplitude k of (block B, sample i) of a block-state buffer: complex64 values, or per 16
// amplitudes one 128-byte row of BF16 planes [hi re | hi im | lo re | lo im], value = hi + lo.
__device__ __forceinline__ float2 block_amp(const void* st, int m, int dp, int split, int B, int i, int k) {
  const size_t base = (size_t(B) * m + i) * size_t(dp);
  if (!split) return __ldg(static_cast<const float2*>(st) + base + k);
  const uint16_t* row = static_cast<const uint16_t*>(st) + (base + size_t(k & ~15)) * 4;
  const int q = k & 15;
  const float hr = __uint_as_float(uint32_t(__ldg(row + q)) << 16);
  const float hi = __uint_as_float(uint32_t(__ldg(row + 16 + q)) << 16);
  const float lr = __uint_as_float(uint32_t(__ldg(row + 32 + q)) << 16);
  const float li = __uint_as_float(uint32_t(__ldg(row + 48 + q)) << 16);
  return make_float2(hr + lr, hi + li);  // exact: hi + lo holds at most 16 significant bits
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double acc_value(const Acc& A) { return double(A.s) + double(A.c); }

// log K_q of pair (i, j) from all blocks, by one warp (valid in every lane).
__device__ double block_pair_logk(const BlockRefineArgs& a, int i, int j, int lane) {
  double lk = 0.0;
  for (int B = 0; B < a.nb; ++B) {
    Acc re{0.0f, 0.0f}, im{0.0f, 0.0f}, na{0.0f, 0.0f}, nb_{0.0f, 0.0f};
    for (int k = lane; k < a.dp; k += 32) {
      const float2 u = block_amp(a.sr, a.m_r, a.dp, a.split, B, i, k);
      const float2 v = block_amp(a.sc, a.m_c, a.dp, a.split, B, j, k);
      // <u|v> = sum conj(u) v
      acc_add(re, DW{u.x, 0.0f}, v.x);
      acc_add(re, DW{u.y, 0.0f}, v.y);
      acc_add(im, DW{u.x, 0.0f}, v.y);
      acc_add(im, DW{u.y, 0.0f}, -v.x);
      acc_add(na, DW{u.x, 0.0f}, u.x);
      acc_add(na, DW{u.y, 0.0f}, u.y);
      acc_add(nb_, DW{v.x, 0.0f}, v.x);
      acc_add(nb_, DW{v.y, 0.0f}, v.y);
    }
    const double dr = warp_sum(acc_value(re)), di = warp_sum(acc_value(im));
    const double da = warp_sum(acc_value(na)), db = warp_sum(acc_value(nb_));
    const double mod2 = __dadd_rn(__dmul_rn(dr, dr), __dmul_rn(di, di));
    lk += log(mod2) - log(da) - log(db);
  }
  return lk;
}

__global__ void __launch_bounds__(128) blocks_refine_kernel(const BlockRefineArgs a) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const GramArgs& g = a.g;
  const long long total = (long long)g.nrows * g.ncols;
  const long long nwarps = (long long)gridDim.x * 4;
  for (long long base = (blockIdx.x * 4LL + warp) * 32; base < total; base += nwarps * 32) {
    const long long e = base + lane;
    bool hit = false;
    long long at = 0;
    int i = 0, j = 0;
    if (e < total) {
      const int r = int(e / g.ncols), c = int(e - (long long)r * g.ncols);
      i = g.row0 + r;
      j = g.col0 + c;
      at = (long long)r * g.ld + c;
      hit = !(g.symmetric && j <= i) && (g.kq ? g.kq[at] > a.tau : g.lkq[at] > a.log_tau);
    }
    unsigned mask = __ballot_sync(0xffffffffu, hit);
    while (mask) {
      const int src = __ffs(mask) - 1;
      mask &= mask - 1;
      const int hi_ = __shfl_sync(0xffffffffu, i, src), hj = __shfl_sync(0xffffffffu, j, src);
      const double lk = block_pair_logk(a, hi_, hj, lane);
      if (lane == src) write_refined(g, at, i, j, lk);
      __syncwarp();
    }
  }
}

}  // namespace rf
}  // namespace dk

using namespace dk;

DK_API size_t dk_gram_refine_workspace_bytes(int m_rows, int m_cols) {
  if (m_rows < 1 || m_cols < 1) return 0;
  const size_t u = size_t(m_rows) + size_t(m_cols);
  return rf::round256(u * sizeof(int)) + rf::round256(u * sizeof(double));
}

DK_API dk_status dk_gram_refine(dk_ctx* ctx, const void* mps_rows, int m_rows, const void* mps_cols, int m_cols, int n,
                                int chi_max, dk_dtype dtype, int row0, int nrows, int col0, int ncols,
                                const float* x_rows, const float* x_cols, float gamma, float w, float tau,
                                float* k_out, float* kq_out, float* kc_out, float* logkq_out, long long ld,
                                int symmetric, void* ws, size_t ws_bytes, void* stream) {
  if (!ctx || !mps_rows || !mps_cols || m_rows < 1 || m_cols < 1 || n < 1) return DK_ERR_ARG;
  if (dtype != DK_C64) return DK_ERR_UNSUPPORTED;
  if (chi_max != 4 && chi_max != 8 && chi_max != 32) return DK_ERR_UNSUPPORTED;
  if (nrows < 0 || ncols < 0 || row0 < 0 || col0 < 0 || row0 + nrows > m_rows || col0 + ncols > m_cols)
    return DK_ERR_ARG;
  if (!kq_out && !logkq_out) return DK_ERR_ARG;
  if (ld < ncols) return DK_ERR_ARG;
  if (!(tau > 0.0f) || !(tau < 1.0f)) return DK_ERR_ARG;
  if (symmetric && (row0 != col0 || nrows != ncols || mps_rows != mps_cols)) return DK_ERR_ARG;
  const bool need_kc = k_out && w != 1.0f && !kc_out;
  if (need_kc && (!x_rows || !x_cols)) return DK_ERR_ARG;
  if (!aligned16(mps_rows) || !aligned16(mps_cols)) return DK_ERR_ARG;
  if (ws && (ws_bytes < dk_gram_refine_workspace_bytes(m_rows, m_cols) || !aligned16(ws))) return DK_ERR_WORKSPACE;
  if (nrows == 0 || ncols == 0) return DK_OK;
  rf::RefineArgs a{};
  a.g.n = n;
  a.g.row0 = row0;
  a.g.nrows = nrows;
  a.g.col0 = col0;
  a.g.ncols = ncols;
  a.g.symmetric = symmetric ? 1 : 0;
  a.g.x_r = x_rows;
  a.g.x_c = x_cols;
  a.g.gamma = gamma;
  a.g.w = w;
  a.g.k = k_out;
  a.g.kq = kq_out;
  a.g.kc = kc_out;
  a.g.lkq = logkq_out;
  a.g.ld = ld;
  a.g.status = ctx->status;
  a.g.need_kc = need_kc ? 1 : 0;
  a.mps_r = static_cast<const float2*>(mps_rows);
  a.mps_c = static_cast<const float2*>(mps_cols);
  a.m_r = m_rows;
  a.m_c = m_cols;
  a.tau = tau;
  a.log_tau = logf(tau);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long total = (long long)nrows * ncols;
  const int smem32 = rf::WARPS32 * rf::WARP_FLOATS * int(sizeof(float));
  if (chi_max == 32 &&
      (cudaFuncSetAttribute(rf::refine32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem32) != cudaSuccess ||
       cudaFuncSetAttribute(rf::norms32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem32) != cudaSuccess))
    return DK_ERR_CUDA;
  if (ws) {
    // the ln-norms of every sample an entry above tau needs, once per sample
    const size_t u = size_t(m_rows) + size_t(m_cols);
    uint8_t* b = static_cast<uint8_t*>(ws);
    a.flag_r = reinterpret_cast<int*>(b);
    a.norm_r = reinterpret_cast<double*>(b + rf::round256(u * sizeof(int)));
    a.flag_c = symmetric ? a.flag_r : a.flag_r + m_rows;
    a.norm_c = symmetric ? a.norm_r : a.norm_r + m_rows;
    const int n_units = symmetric ? m_rows : m_rows + m_cols;
    if (cudaMemsetAsync(a.flag_r, 0, u * sizeof(int), st) != cudaSuccess) return DK_ERR_CUDA;
    long long mg = (total + 255) / 256;
    if (mg > 8LL * ctx->sm_count) mg = 8LL * ctx->sm_count;
    rf::mark_kernel<<<int(mg), 256, 0, st>>>(a);
    dk_status s = launch_status();
    if (s != DK_OK) return s;
    if (chi_max == 32) {
      long long ng = (n_units + rf::WARPS32 - 1) / rf::WARPS32;  // a warp per sample
      if (ng > 64LL * ctx->sm_count) ng = 64LL * ctx->sm_count;
      rf::norms32_kernel<<<int(ng), rf::WARPS32 * 32, smem32, st>>>(a, n_units);
    } else {
      long long ng = (n_units + 127) / 128;
      if (ng > 16LL * ctx->sm_count) ng = 16LL * ctx->sm_count;
      if (chi_max == 4) rf::norms_small_kernel<2><<<int(ng), 128, 0, st>>>(a, n_units);
      else rf::norms_small_kernel<4><<<int(ng), 128, 0, st>>>(a, n_units);
    }
    s = launch_status();
    if (s != DK_OK) return s;
  }
  if (chi_max == 32) {
    const int smem = smem32;
    long long grid = (total + rf::WARPS32 * 32 * 32 - 1) / (rf::WARPS32 * 32 * 32);
    const long long cap = 8LL * ctx->sm_count;
    if (grid > cap) grid = cap;
    rf::refine32_kernel<<<int(grid), rf::WARPS32 * 32, smem, st>>>(a);
    return launch_status();
  }
  long long grid = (total + rf::SMALL_WARPS * 32 * 8 - 1) / (rf::SMALL_WARPS * 32 * 8);
  const long long cap = 16LL * ctx->sm_count;
  if (grid > cap) grid = cap;
  if (chi_max == 4) rf::refine_small_kernel<2><<<int(grid), rf::SMALL_WARPS * 32, 0, st>>>(a);
  else rf::refine_small_kernel<4><<<int(grid), rf::SMALL_WARPS * 32, 0, st>>>(a);
  return launch_status();
}

DK_API dk_status dk_gram_blocks_refine(dk_ctx* ctx, const void* states_rows, int m_rows, const void* states_cols,
                                       int m_cols, int n, int block, dk_precision prec, int row0, int nrows, int col0,
                                       int ncols, const float* x_rows, const float* x_cols, float gamma, float w,
                                       float tau, float* k_out, float* kq_out, float* kc_out, float* logkq_out,
                                       long long ld, int symmetric, void* stream) {
  if (!ctx || !states_rows || !states_cols || m_rows < 1 || m_cols < 1 || n < 1) return DK_ERR_ARG;
  if (prec != DK_PREC_F32 && prec != DK_PREC_BF16X3) return DK_ERR_UNSUPPORTED;
  if (dk_block_states_bytes(1, n, block) == 0) return DK_ERR_UNSUPPORTED;
  if (nrows < 0 || ncols < 0 || row0 < 0 || col0 < 0 || row0 + nrows > m_rows || col0 + ncols > m_cols)
    return DK_ERR_ARG;
  if (!kq_out && !logkq_out) return DK_ERR_ARG;
  if (ld < ncols) return DK_ERR_ARG;
  if (!(tau > 0.0f) || !(tau < 1.0f)) return DK_ERR_ARG;
  if (symmetric && (row0 != col0 || nrows != ncols || states_rows != states_cols)) return DK_ERR_ARG;
  const bool need_kc = k_out && w != 1.0f && !kc_out;
  if (need_kc && (!x_rows || !x_cols)) return DK_ERR_ARG;
  if (!aligned16(states_rows) || !aligned16(states_cols)) return DK_ERR_ARG;
  if (nrows == 0 || ncols == 0) return DK_OK;
  const int b = block > 0 ? block : n;
  rf::BlockRefineArgs a{};
  a.g.n = n;
  a.g.row0 = row0;
  a.g.nrows = nrows;
  a.g.col0 = col0;
  a.g.ncols = ncols;
  a.g.symmetric = symmetric ? 1 : 0;
  a.g.x_r = x_rows;
  a.g.x_c = x_cols;
  a.g.gamma = gamma;
  a.g.w = w;
  a.g.k = k_out;
  a.g.kq = kq_out;
  a.g.kc = kc_out;
  a.g.lkq = logkq_out;
  a.g.ld = ld;
  a.g.status = ctx->status;
  a.g.need_kc = need_kc ? 1 : 0;
  a.sr = states_rows;
  a.sc = states_cols;
  a.m_r = m_rows;
  a.m_c = m_cols;
  a.nb = (n + b - 1) / b;
  a.dp = (1 << b) > 16 ? (1 << b) : 16;
  a.split = prec == DK_PREC_BF16X3 ? 1 : 0;
  a.tau = tau;
  a.log_tau = logf(tau);
  const long long total = (long long)nrows * ncols;
  long long grid = (total + 4 * 32 - 1) / (4 * 32);
  if (grid > 16LL * ctx->sm_count) grid = 16LL * ctx->sm_count;
  rf::blocks_refine_kernel<<<int(grid), 128, 0, static_cast<cudaStream_t>(stream)>>>(a);
  return launch_status();
}
