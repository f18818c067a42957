// MPS of the feature-map state (§II-C, Eq. 6) and its self-overlap normalisation.
//
// Construction (exact, no truncation). Write qubit k's computational-basis value after the
// single-qubit layer of repetition rho as z_k^(rho) (z^(0) = 0). The RZZ layers are
// diagonal, so the amplitude of |z^(r)> is a sum over the intermediate values z^(1..r-1)
// of a product of
//   * per-qubit factors  G_k[z^(rho)][z^(rho-1)],  G_k = RZ(angle_scale x_k) H,
//   * per-bond phases    exp(-i theta_k/2 (-1)^(z_k^(rho) XOR z_{k+1}^(rho))),
//                        theta_k = 2 (pi - x_k)(pi - x_{k+1}).
// Grouping (z_k^(1), ..., z_k^(r)) into one bond index c (bit rho-1 = z^(rho)) of size
// 2^r turns this sum into an MPS with closed-form site tensors
//   A^(k)_s[c'][c] = [top bit of c == s] * L_k(c) * exp(-i theta_{k-1}/2 (r - 2 popc(c' XOR c))),
//   L_k(c) = 2^(-r/2) (-1)^popc(c AND c>>1) exp(-i angle_scale x_k / 2 (r - 2 popc(c))),
// (left bond of site 0 of size 1 without phase; right bond of site n-1 summed over).
//
// The top bit of every bond is a copy of the physical value s of the site to its left,
// so A_s only has columns in block s of the bond. A left-to-right sweep in FP64 then
// canonicalises block by block: for each site and each s, M_s = R A_s[:, block s] (rows:
// the stored left bond, columns: the h_a = 2^(r-1) closed-form columns of block s),
// Householder QR M_s = Q_s R_s, Q_s stored as block s of the left-canonical tensor, and
// R = diag(R_0, R_1) carried to the next site. The last site's column vector is
// normalised (its norm is the state's norm), so the stored state has unit norm before
// rounding to complex64 / complex128.
//
// Stored layout (compact, see include/dualk.h): A[k][i][s][j][l], j < h = chi/2 the
// column inside block s (bond position s*h + j), l < chi the left bond position.
//
// Block-structured entanglers (dk_fmap.block = b): the RZZ of the pair (k-1, k) is applied
// only when k is not a multiple of b, i.e. both qubits lie in one block; elsewhere theta = 0
// and the bond phase is 1, so the same closed form holds with the chain cut at the block
// boundaries (the stored bond there keeps its size; QR leaves rounding-level columns).
//
// The self-overlap kernel then runs the Gram transfer arithmetic (transfer.cuh) on each
// sample's own rounded tensors and stores ln|<psi~|psi~>|, the normaliser that makes the
// Gram diagonal exactly 1.
#include <math.h>

#include "common.cuh"
#include "internal.h"
#include "transfer.cuh"

namespace dk {

template <typename T>
struct cx {
  T x, y;
};
using cd = cx<double>;
__device__ __forceinline__ float fmx(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmx(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ cd mk(double x, double y) { return cd{x, y}; }
template <typename T>
__device__ __forceinline__ cx<T> mkc(T x, T y) { return cx<T>{x, y}; }
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) { return mkc(fmx(a.x, b.x, -a.y * b.y), fmx(a.x, b.y, a.y * b.x)); }
template <typename T>
__device__ __forceinline__ cx<T> cconjmul(cx<T> a, cx<T> b) { return mkc(fmx(a.x, b.x, a.y * b.y), fmx(a.x, b.y, -a.y * b.x)); }
template <typename T>
__device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return mkc(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return mkc(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return mkc(a.x * s, a.y * s); }
template <typename T>
__device__ __forceinline__ cx<T> cconj(cx<T> a) { return mkc(a.x, -a.y); }
template <typename T>
__device__ __forceinline__ T cabs2(cx<T> a) { return fmx(a.x, a.x, a.y * a.y); }

constexpr double PI_D = 3.14159265358979323846;

// RZZ on the pair (k-1, k)? ent_block = 0: no entanglers; b >= 1: only inside blocks of b
// (the open chain is b = n).
__host__ __device__ __forceinline__ bool entangled(int ent_block, int k) {
  return ent_block > 0 && k % ent_block != 0;
}

// Closed-form factors of one site for RP repetitions: u^e and w^e for e in [-RP, RP],
// u = exp(-i phi/2), w = exp(-i theta/2) (unit modulus, so u^-e = conj(u^e)).
template <int RP, typename T = double>
struct SiteFactors {
  using C = cx<T>;
  C up[RP + 1];
  C wp[RP + 1];
  __device__ __forceinline__ void make(double phi, double theta) {
    double sn, cs;
    sincos(-0.5 * phi, &sn, &cs);
    const cd u = mk(cs, sn);
    sincos(-0.5 * theta, &sn, &cs);
    make_from(u, mk(cs, sn));
  }
  __device__ __forceinline__ void make_from(C u, C w) {
    up[0] = mkc(T(1), T(0));
    wp[0] = mkc(T(1), T(0));
#pragma unroll
    for (int q = 1; q <= RP; ++q) {
      up[q] = cmul(up[q - 1], u);
      wp[q] = cmul(wp[q - 1], w);
    }
  }
  // powers by exponent in -RP..RP, picked with selects so that a run-time exponent does
  // not send the tables to local memory
  __device__ __forceinline__ static C pick(const C (&tab)[RP + 1], int e) {
    const int a = e >= 0 ? e : -e;
    C r = tab[0];
#pragma unroll
    for (int q = 1; q <= RP; ++q) r = a == q ? tab[q] : r;
    return e >= 0 ? r : cconj(r);
  }
  __device__ __forceinline__ C upow(int e) const { return pick(up, e); }
  __device__ __forceinline__ C wpow(int e) const { return pick(wp, e); }
  // L_k(c) = 2^(-r/2) (-1)^popc(c & c>>1) u^(r - 2 popc(c))
  __device__ __forceinline__ C local(int c) const {
    constexpr double amp = RP == 1 ? 0.70710678118654752440 : RP == 2 ? 0.5 : RP == 3 ? 0.35355339059327376220
                         : RP == 4 ? 0.25 : 0.17677669529663688110;
    const T sign = (__popc(c & (c >> 1)) & 1) ? T(-amp) : T(amp);
    return cscale(upow(RP - 2 * __popc(c)), sign);
  }
  // bond phase between closed-form left index cp and right index c
  __device__ __forceinline__ C bond(int cp, int c) const { return wpow(RP - 2 * __popc(cp ^ c)); }
};

__device__ __forceinline__ void store_cplx(void* out, size_t idx, cd v, int c128) {
  if (c128) reinterpret_cast<double2*>(out)[idx] = make_double2(v.x, v.y);
  else reinterpret_cast<float2*>(out)[idx] = make_float2(float(v.x), float(v.y));
}

// QR of a P x C complex matrix (C <= 2) by classical Gram-Schmidt with one
// re-orthogonalisation pass, in registers. nref <= C columns are orthonormalised; R is
// nref x C (rows >= nref zero), Q's columns >= nref are zero. A column whose residual
// vanishes gets a zero Q column and a zero R diagonal (the product Q R is still M).
template <int P, int C>
__device__ __forceinline__ void qr_cgs2(const cd (&M)[P][C], int nref, cd (&Q)[P][C], cd (&R)[C][C]) {
#pragma unroll
  for (int r = 0; r < C; ++r)
#pragma unroll
    for (int c = 0; c < C; ++c) R[r][c] = mk(0.0, 0.0);
#pragma unroll
  for (int c = 0; c < C; ++c) {
    cd v[P];
#pragma unroll
    for (int i = 0; i < P; ++i) v[i] = M[i][c];
    if (c < nref) {
#pragma unroll
      for (int pass = 0; pass < 2; ++pass)
#pragma unroll
        for (int q = 0; q < c; ++q) {
          cd r = mk(0.0, 0.0);
#pragma unroll
          for (int i = 0; i < P; ++i) r = cadd(r, cconjmul(Q[i][q], v[i]));
          R[q][c] = cadd(R[q][c], r);
#pragma unroll
          for (int i = 0; i < P; ++i) v[i] = csub(v[i], cmul(Q[i][q], r));
        }
      double n2 = 0.0;
#pragma unroll
      for (int i = 0; i < P; ++i) n2 += cabs2(v[i]);
      const double inv = n2 > 1e-300 ? rsqrt(n2) : 0.0;
      R[c][c] = mk(n2 * inv, 0.0);
#pragma unroll
      for (int i = 0; i < P; ++i) Q[i][c] = cscale(v[i], inv);
    } else {
#pragma unroll
      for (int q = 0; q < C; ++q) {
        if (q < nref) {
          cd r = mk(0.0, 0.0);
#pragma unroll
          for (int i = 0; i < P; ++i) r = cadd(r, cconjmul(Q[i][q], v[i]));
          R[q][c] = r;
        }
      }
#pragma unroll
      for (int i = 0; i < P; ++i) Q[i][c] = mk(0.0, 0.0);
    }
  }
}

__device__ __forceinline__ cd shfl_cd(unsigned mask, cd v, int lane_mask) {
  return mk(__shfl_xor_sync(mask, v.x, lane_mask), __shfl_xor_sync(mask, v.y, lane_mask));
}

// Two threads per sample, one per bond block s; HS = stored block size chi/2, HA =
// closed-form block size 2^(r-1) <= 2. A CTA is one (possibly partial) warp holding
// blockDim.x / 2 samples; the launch picks the width so that the FP64 work spreads over
// all SMs. The exponentials of site k+1 are evaluated while site k is factorised, so they
// stay off the chain's dependency path. With log_norm set, the kernel also runs the Gram's
// transfer arithmetic (transfer.cuh, in `real`, on the FMA pipes) on each sample's own
// rounded tensors as they are produced, giving ln|<psi~|psi~>| bit-identical to the Gram
// diagonal without a second pass.
template <int HS, int HA, int RP, typename real>
__global__ void __launch_bounds__(32) mps_build_pair_kernel(const float* __restrict__ x, int m, int n,
                                                            double angle_scale, int ent_block,
                                                            void* __restrict__ out, int32_t* __restrict__ bond,
                                                            float* __restrict__ log_norm) {
  constexpr int P = 2 * HS;  // stored left-bond positions
  constexpr int CHI = 2 * HS;
  constexpr int c128 = sizeof(real) == 8 ? 1 : 0;
  const int s = threadIdx.x & 1;
  const int i0 = blockIdx.x * (blockDim.x >> 1) + (threadIdx.x >> 1);
  const unsigned mask = blockDim.x >= 32 ? 0xffffffffu : ((1u << blockDim.x) - 1u);
  const bool live = i0 < m;
  const int i = live ? i0 : m - 1;  // dead lanes shadow the last sample and store nothing
  const float* xs = x + size_t(i) * n;
  cd R[2][HS][HA];
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int j = 0; j < HS; ++j)
#pragma unroll
      for (int c = 0; c < HA; ++c) R[t][j][c] = mk(0.0, 0.0);
  R[0][0][0] = mk(1.0, 0.0);
  int act = 1;  // active left-bond positions (pk_0 + pk_1 of the previous site)
  const size_t per = size_t(CHI) * CHI;  // complex entries per sample-site
  // this thread's exponential for site k: s = 0 -> exp(-i angle_scale x_k / 2),
  // s = 1 -> exp(-i theta_{k-1} / 2), theta_{k-1} = 2 (pi - x_{k-1})(pi - x_k)
  auto expo = [&](int k) {
    const double xk = double(xs[k]);
    const double xp = k > 0 ? double(xs[k - 1]) : 0.0;
    const double arg = s == 0 ? -0.5 * angle_scale * xk : (entangled(ent_block, k) ? -(PI_D - xp) * (PI_D - xk) : 0.0);
    double sn, cs;
    sincos(arg, &sn, &cs);
    return mk(cs, sn);
  };
  PairE<real, HS> chain[1][1];
  chain[0][0].init();
  cd e_cur = expo(0);
  for (int k = 0; k < n; ++k) {
    const cd e_next = (k + 1 < n) ? expo(k + 1) : mk(1.0, 0.0);  // independent of this site's chain
    SiteFactors<RP> f;
    {
      const cd other = shfl_cd(mask, e_cur, 1);
      f.make_from(s == 0 ? e_cur : other, s == 0 ? other : e_cur);
    }
    const size_t base = (size_t(k) * m + i) * per + size_t(s) * HS * CHI;
    if (bond && i0 == 0 && s == 0) bond[k] = act;
    cd Qs[P][HS];  // this thread's block of the stored tensor, columns j >= the active ones zero
    if (k < n - 1) {
      cd M[P][HA];
#pragma unroll
      for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int j = 0; j < HS; ++j)
#pragma unroll
          for (int cc = 0; cc < HA; ++cc) {
            const int c = s * HA + cc;
            cd acc = mk(0.0, 0.0);
#pragma unroll
            for (int cp = 0; cp < HA; ++cp) acc = cadd(acc, cmul(R[t][j][cp], f.bond(t * HA + cp, c)));
            M[t * HS + j][cc] = cmul(f.local(c), acc);
          }
      const int nref = act < HA ? act : HA;
      cd Q[P][HA], Rr[HA][HA];
      qr_cgs2<P, HA>(M, nref, Q, Rr);
#pragma unroll
      for (int j = 0; j < HS; ++j)
#pragma unroll
        for (int l = 0; l < P; ++l) Qs[l][j] = j < HA ? Q[l][j] : mk(0.0, 0.0);
      // R <- diag(R_0, R_1): keep this block, take the other from the partner lane
#pragma unroll
      for (int j = 0; j < HS; ++j)
#pragma unroll
        for (int cc = 0; cc < HA; ++cc) {
          const cd mine = j < HA ? Rr[j][cc] : mk(0.0, 0.0);
          const cd other = shfl_cd(mask, mine, 1);
          R[0][j][cc] = s == 0 ? mine : other;  // selects keep R in registers
          R[1][j][cc] = s == 0 ? other : mine;
        }
      act = 2 * nref;
    } else {
      cd v[P];
      double nrm2 = 0.0;
#pragma unroll
      for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int j = 0; j < HS; ++j) {
          cd acc = mk(0.0, 0.0);
#pragma unroll
          for (int cc = 0; cc < HA; ++cc) {
            const int c = s * HA + cc;
            cd inner = mk(0.0, 0.0);
#pragma unroll
            for (int cp = 0; cp < HA; ++cp) inner = cadd(inner, cmul(R[t][j][cp], f.bond(t * HA + cp, c)));
            acc = cadd(acc, cmul(f.local(c), inner));
          }
          v[t * HS + j] = acc;
          nrm2 += cabs2(acc);
        }
      nrm2 += __shfl_xor_sync(mask, nrm2, 1);
      const double inv = nrm2 > 0.0 ? rsqrt(nrm2) : 0.0;
#pragma unroll
      for (int j = 0; j < HS; ++j)
#pragma unroll
        for (int l = 0; l < P; ++l) Qs[l][j] = j == 0 ? cscale(v[l], inv) : mk(0.0, 0.0);
      if (bond && i0 == 0 && s == 0) bond[n] = 1;
    }
    // the stored values, rounded once: to memory and, for the self-overlap, to registers
    real qr[HS][P], qi[HS][P];
#pragma unroll
    for (int j = 0; j < HS; ++j)
#pragma unroll
      for (int l = 0; l < P; ++l) {
        qr[j][l] = real(Qs[l][j].x);
        qi[j][l] = real(Qs[l][j].y);
      }
    if (live) {
#pragma unroll
      for (int j = 0; j < HS; ++j)
#pragma unroll
        for (int l = 0; l < P; ++l) store_cplx(out, base + j * CHI + l, Qs[l][j], c128);
    }
    if (log_norm) {
      // both threads of the sample hold the full site tensor after the swap
      real ar[2][HS][P], ai[2][HS][P];
#pragma unroll
      for (int j = 0; j < HS; ++j)
#pragma unroll
        for (int l = 0; l < P; ++l) {
          const real orr = __shfl_xor_sync(mask, qr[j][l], 1);
          const real oi = __shfl_xor_sync(mask, qi[j][l], 1);
          ar[0][j][l] = s == 0 ? qr[j][l] : orr;
          ai[0][j][l] = s == 0 ? qi[j][l] : oi;
          ar[1][j][l] = s == 0 ? orr : qr[j][l];
          ai[1][j][l] = s == 0 ? oi : qi[j][l];
        }
      // sub-block A_s[t]: rows l = t*HS + a, columns j (as in the Gram kernels' loaders)
      auto ld = [&](int, int ss, int t, Blk<real, HS>& blk) {
#pragma unroll
        for (int j = 0; j < HS; ++j)
#pragma unroll
          for (int a = 0; a < HS; ++a) {
            blk.r[a][j] = ar[ss][j][t * HS + a];
            blk.i[a][j] = ai[ss][j][t * HS + a];
          }
      };
      site_step<real, HS, 1, 1>(chain, ld, ld, k == n - 1 || ((k & (RENORM_EVERY - 1)) == RENORM_EVERY - 1));
    }
    e_cur = e_next;
  }
  if (log_norm && live && s == 0) log_norm[i] = chain[0][0].half_log_mod();
}

// Phase exp(i a) for an angle given as an unevaluated sum a = hi + lo, |lo| <= 2^-22 |hi|:
// sincosf of hi, then the first-order correction by lo (the neglected term is lo^2 / 2).
__device__ __forceinline__ cx<float> expi_split(float hi, float lo) {
  float sn, cs;
  sincosf(hi, &sn, &cs);
  return mkc(fmaf(-lo, sn, cs), fmaf(lo, cs, sn));
}

// pi - v as hi + lo for a float v in [0, pi] (Fast2Sum of the float pi against v, plus the
// float pi's own error); the pair carries pi - v to about 2^-48 relative
__device__ __forceinline__ void pi_minus(float v, float& hi, float& lo) {
  constexpr float PI_HI = 3.14159274101257324219f;   // pi rounded to float
  constexpr float PI_LO = -8.74227800037248e-8f;     // pi - PI_HI
  hi = PI_HI - v;
  lo = ((PI_HI - hi) - v) + PI_LO;
}

// Eight threads per sample for the bond-4 tensors (chi_max = 4, reps <= 2): thread q of a
// sample's group handles block s = q >> 2 and row (t, j) = ((q >> 1) & 1, q & 1) of that
// block's 4 x HA matrix M_s, and the Gram-Schmidt sums over the 4 rows are shuffle
// reductions inside the group. The arithmetic runs in `creal`: FP64 for complex128
// output, and for complex64 output FP32 by default or FP64 on request (dk_fmap.qr_prec).
// FP64 issues at a small fraction of the FP32 rate on GB300, and the gauge QR of the exact
// bond-4 chain truncates nothing, so the FP32 sweep only adds rounding of the size of the
// complex64 storage's own. In FP32 the rotation angles are formed exactly enough by
// error-free transforms (pi - x and the products as float pairs), so the only FP32 error
// in a phase is sincosf's. The exponentials of site k+1 are evaluated while site k is factorised;
// with log_norm set, every thread also runs the Gram's transfer arithmetic on the
// sample's stored tensors (gathered by shuffles) so that ln|<psi~|psi~>| is bit-identical
// to the Gram diagonal.
template <int HA, int RP, typename real, typename creal>
__global__ void __launch_bounds__(32) mps_build_oct_kernel(const float* __restrict__ x, int m, int n,
                                                           double angle_scale, int ent_block,
                                                           void* __restrict__ out, int32_t* __restrict__ bond,
                                                           float* __restrict__ log_norm) {
  using C = cx<creal>;
  constexpr int HS = 2, CHI = 4;
  constexpr bool c128 = sizeof(real) == 8;   // stored precision
  constexpr bool f64 = sizeof(creal) == 8;   // arithmetic precision
  const int q = threadIdx.x & 7;
  const int s = q >> 2, t = (q >> 1) & 1, j = q & 1;
  const int row = t * HS + j;  // this thread's left-bond position
  const int i0 = blockIdx.x * (blockDim.x >> 3) + (threadIdx.x >> 3);
  const unsigned mask = blockDim.x >= 32 ? 0xffffffffu : ((1u << blockDim.x) - 1u);
  const bool live = i0 < m;
  const int i = live ? i0 : m - 1;
  const int base_lane = threadIdx.x & ~7;
  const float* xs = x + size_t(i) * n;
  const C zero = mkc(creal(0), creal(0));
  // Rrow[cp] = R_t[j][cp]: row j of the previous site's block-t factor (HA columns)
  C Rrow[HA];
#pragma unroll
  for (int c = 0; c < HA; ++c) Rrow[c] = zero;
  if (t == 0 && j == 0) Rrow[0] = mkc(creal(1), creal(0));
  int act = 1;
  // -angle_scale / 2 as a float pair (FP32 form)
  const float g_hi = float(-0.5 * angle_scale);
  const float g_lo = float(-0.5 * angle_scale - double(g_hi));
  // thread q & 1 == 0: u_k = exp(-i angle_scale x_k / 2); q & 1 == 1: w_k =
  // exp(-i (pi - x_{k-1})(pi - x_k)) (one factor of the RZZ phase, see mps_build_pair_kernel)
  auto expo = [&](int k) -> C {
    const float xk = xs[k];
    const float xp = k > 0 ? xs[k - 1] : 0.0f;
    const bool ent = entangled(ent_block, k);
    if constexpr (f64) {
      const double arg = (q & 1) == 0 ? -0.5 * angle_scale * double(xk)
                                      : (ent ? -(PI_D - double(xp)) * (PI_D - double(xk)) : 0.0);
      double sn, cs;
      sincos(arg, &sn, &cs);
      return mkc(cs, sn);
    } else {
      float hi, lo;
      if ((q & 1) == 0) {
        hi = g_hi * xk;
        lo = fmaf(g_hi, xk, -hi) + g_lo * xk;
      } else if (ent) {
        float ah, al, bh, bl;
        pi_minus(xp, ah, al);
        pi_minus(xk, bh, bl);
        const float ph = ah * bh;
        const float pl = fmaf(ah, bh, -ph) + fmaf(ah, bl, al * bh);
        hi = -ph;
        lo = -pl;
      } else {
        hi = 0.0f;
        lo = 0.0f;
      }
      return expi_split(hi, lo);
    }
  };
  auto gsum = [&](creal v) {  // sum over the 4 threads of this block
    v += __shfl_xor_sync(mask, v, 1);
    v += __shfl_xor_sync(mask, v, 2);
    return v;
  };
  auto gsumc = [&](C v) { return mkc(gsum(v.x), gsum(v.y)); };
  auto inv_sqrt = [](creal v) -> creal {
    if constexpr (f64) return rsqrt(v);
    else return __frsqrt_rn(v);
  };
  constexpr creal TINY = f64 ? creal(1e-300) : creal(1e-30);
  PairE<real, HS> chain[1][1];
  chain[0][0].init();
  C e_cur = expo(0);
  for (int k = 0; k < n; ++k) {
    const C e_next = (k + 1 < n) ? expo(k + 1) : mkc(creal(1), creal(0));
    SiteFactors<RP, creal> f;
    {
      const C u = mkc(__shfl_sync(mask, e_cur.x, base_lane), __shfl_sync(mask, e_cur.y, base_lane));
      const C w = mkc(__shfl_sync(mask, e_cur.x, base_lane + 1), __shfl_sync(mask, e_cur.y, base_lane + 1));
      f.make_from(u, w);
    }
    if (bond && i0 == 0 && q == 0) bond[k] = act;
    C qv[HS];  // this thread's row of Q_s: stored element (s, jc, l = row) for jc < HS
    if (k < n - 1) {
      C mrow[HA];
#pragma unroll
      for (int cc = 0; cc < HA; ++cc) {
        const int c = s * HA + cc;
        C acc = zero;
#pragma unroll
        for (int cp = 0; cp < HA; ++cp) acc = cadd(acc, cmul(Rrow[cp], f.bond(t * HA + cp, c)));
        mrow[cc] = cmul(f.local(c), acc);
      }
      const int nref = act < HA ? act : HA;
      // classical Gram-Schmidt with one re-orthogonalisation pass over the 4 rows
      C qrow[HA], rcol[HA][HA];
#pragma unroll
      for (int a = 0; a < HA; ++a)
#pragma unroll
        for (int b = 0; b < HA; ++b) rcol[a][b] = zero;
#pragma unroll
      for (int c = 0; c < HA; ++c) {
        C v = mrow[c];
        if (c < nref) {
#pragma unroll
          for (int pass = 0; pass < 2; ++pass)
#pragma unroll
            for (int pq = 0; pq < c; ++pq) {
              const C r = gsumc(cconjmul(qrow[pq], v));
              rcol[pq][c] = cadd(rcol[pq][c], r);
              v = csub(v, cmul(qrow[pq], r));
            }
          const creal n2 = gsum(cabs2(v));
          const creal inv = n2 > TINY ? inv_sqrt(n2) : creal(0);
          rcol[c][c] = mkc(n2 * inv, creal(0));
          qrow[c] = cscale(v, inv);
        } else {
#pragma unroll
          for (int pq = 0; pq < HA; ++pq)
            if (pq < nref) rcol[pq][c] = gsumc(cconjmul(qrow[pq], v));
          qrow[c] = zero;
        }
      }
#pragma unroll
      for (int jc = 0; jc < HS; ++jc) qv[jc] = jc < HA ? qrow[jc < HA ? jc : 0] : zero;
      // next R row for this thread: row j of block t's factor, which every thread of block t
      // holds after the reductions (thread 4 t + j holds block t and the same j, so its
      // row-j pick is the one wanted)
      const int src = base_lane + 4 * t + j;
#pragma unroll
      for (int cp = 0; cp < HA; ++cp) {
        C mine = rcol[0][cp];
        if constexpr (HA > 1) mine = j == 1 ? rcol[1][cp] : mine;
        else mine = j == 1 ? zero : mine;
        Rrow[cp] = mkc(__shfl_sync(mask, mine.x, src), __shfl_sync(mask, mine.y, src));
      }
      act = 2 * nref;
    } else {
      C acc = zero;
#pragma unroll
      for (int cc = 0; cc < HA; ++cc) {
        const int c = s * HA + cc;
        C inner = zero;
#pragma unroll
        for (int cp = 0; cp < HA; ++cp) inner = cadd(inner, cmul(Rrow[cp], f.bond(t * HA + cp, c)));
        acc = cadd(acc, cmul(f.local(c), inner));
      }
      creal n2 = cabs2(acc);
      n2 += __shfl_xor_sync(mask, n2, 1);
      n2 += __shfl_xor_sync(mask, n2, 2);
      n2 += __shfl_xor_sync(mask, n2, 4);
      const creal inv = n2 > creal(0) ? inv_sqrt(n2) : creal(0);
      qv[0] = cscale(acc, inv);
      qv[1] = zero;
      if (bond && i0 == 0 && q == 0) bond[n] = 1;
    }
    // the stored values, rounded once: to memory and, for the self-overlap, to registers
    real vr[HS], vi[HS];
#pragma unroll
    for (int jc = 0; jc < HS; ++jc) {
      vr[jc] = real(qv[jc].x);
      vi[jc] = real(qv[jc].y);
    }
    if (live) {
      const size_t base = (size_t(k) * m + i) * (CHI * CHI);
#pragma unroll
      for (int jc = 0; jc < HS; ++jc) {
        const size_t idx = base + (s * HS + jc) * CHI + row;
        if constexpr (c128) reinterpret_cast<double2*>(out)[idx] = make_double2(vr[jc], vi[jc]);
        else reinterpret_cast<float2*>(out)[idx] = make_float2(vr[jc], vi[jc]);
      }
    }
    if (log_norm) {
      // gather the sample's 16 stored values: element (s', jc, l) from thread 4 s' + l
      real ar[2][HS][CHI], ai[2][HS][CHI];
#pragma unroll
      for (int ss = 0; ss < 2; ++ss)
#pragma unroll
        for (int l = 0; l < CHI; ++l)
#pragma unroll
          for (int jc = 0; jc < HS; ++jc) {
            ar[ss][jc][l] = __shfl_sync(mask, vr[jc], base_lane + 4 * ss + l);
            ai[ss][jc][l] = __shfl_sync(mask, vi[jc], base_lane + 4 * ss + l);
          }
      auto ld = [&](int, int ss, int tt, Blk<real, HS>& blk) {
#pragma unroll
        for (int jc = 0; jc < HS; ++jc)
#pragma unroll
          for (int a = 0; a < HS; ++a) {
            blk.r[a][jc] = ar[ss][jc][tt * HS + a];
            blk.i[a][jc] = ai[ss][jc][tt * HS + a];
          }
      };
      site_step<real, HS, 1, 1>(chain, ld, ld, k == n - 1 || ((k & (RENORM_EVERY - 1)) == RENORM_EVERY - 1));
    }
    e_cur = e_next;
  }
  if (log_norm && live && q == 0) log_norm[i] = chain[0][0].half_log_mod();
}

// One warp per sample for wide bonds (closed-form block HA >= 4): the same sweep with the
// matrices in shared memory, lanes parallel over columns and rows.
template <int HS, int HA>
struct WarpQr {
  cd R[2][HS][HA];
  cd Rn[2][HS][HA];
  cd M[2 * HS][HA];
  cd Q[2 * HS][HA];
  cd L[2 * HA];
  double beta[HA];
  cd alpha[HA];
  double part[32];
};

template <int HS, int HA, int RP>
__global__ void __launch_bounds__(32) mps_build_warp_kernel(const float* __restrict__ x, int m, int n,
                                                            double angle_scale, int ent_block, int out_c128,
                                                            void* __restrict__ out, int32_t* __restrict__ bond) {
  constexpr int P = 2 * HS;
  constexpr int CHI = 2 * HS;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  WarpQr<HS, HA>& S = *reinterpret_cast<WarpQr<HS, HA>*>(smem_raw);
  const int lane = threadIdx.x;
  const int i = blockIdx.x;
  if (i >= m) return;
  const float* xs = x + size_t(i) * n;
  for (int e = lane; e < 2 * HS * HA; e += 32) (&S.R[0][0][0])[e] = mk(0.0, 0.0);
  __syncwarp();
  if (lane == 0) S.R[0][0][0] = mk(1.0, 0.0);
  int act = 1;
  double xprev = 0.0;
  const size_t per = size_t(CHI) * CHI;
  SiteFactors<RP> f;
  for (int k = 0; k < n; ++k) {
    const double xk = double(xs[k]);
    f.make(angle_scale * xk, entangled(ent_block, k) ? 2.0 * (PI_D - xprev) * (PI_D - xk) : 0.0);
    for (int c = lane; c < 2 * HA; c += 32) S.L[c] = f.local(c);
    __syncwarp();
    const size_t base = (size_t(k) * m + i) * per;
    if (bond && i == 0 && lane == 0) bond[k] = act;
    if (k < n - 1) {
      int pk = 0;
      for (int s = 0; s < 2; ++s) {
        // M_s = R A_s[:, block s]
        for (int e = lane; e < P * HA; e += 32) {
          const int row = e / HA, cc = e - row * HA;
          const int t = row / HS, j = row - t * HS;
          const int c = s * HA + cc;
          cd acc = mk(0.0, 0.0);
          for (int cp = 0; cp < HA; ++cp) acc = cadd(acc, cmul(S.R[t][j][cp], f.bond(t * HA + cp, c)));
          S.M[row][cc] = cmul(S.L[c], acc);
        }
        __syncwarp();
        const int nref = act < HA ? act : HA;
        for (int j = 0; j < nref; ++j) {
          // column norm below the diagonal, rows split over lanes
          double part = 0.0;
          for (int r = j + lane; r < P; r += 32) part += cabs2(S.M[r][j]);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
          if (lane == 0) {
            const cd x0 = S.M[j][j];
            const double ax0 = sqrt(cabs2(x0));
            const double sigma = sqrt(part);
            if (sigma > 0.0) {
              const cd u = ax0 > 0.0 ? cscale(x0, 1.0 / ax0) : mk(1.0, 0.0);
              S.alpha[j] = cscale(u, -sigma);
              S.M[j][j] = cscale(u, ax0 + sigma);
              S.beta[j] = 1.0 / (sigma * (sigma + ax0));
            } else {
              S.alpha[j] = mk(0.0, 0.0);
              S.beta[j] = 0.0;
            }
          }
          __syncwarp();
          const int c = lane;
          if (c > j && c < HA && S.beta[j] != 0.0) {
            cd w = mk(0.0, 0.0);
            for (int r = j; r < P; ++r) w = cadd(w, cconjmul(S.M[r][j], S.M[r][c]));
            w = cscale(w, S.beta[j]);
            for (int r = j; r < P; ++r) S.M[r][c] = csub(S.M[r][c], cmul(S.M[r][j], w));
          }
          __syncwarp();
        }
        // explicit Q, lane per column
        if (lane < HA) {
          const int c = lane;
          for (int r = 0; r < P; ++r) S.Q[r][c] = mk((r == c && c < nref) ? 1.0 : 0.0, 0.0);
          if (c < nref) {
            for (int j = nref - 1; j >= 0; --j) {
              if (S.beta[j] == 0.0) continue;
              cd w = mk(0.0, 0.0);
              for (int r = j; r < P; ++r) w = cadd(w, cconjmul(S.M[r][j], S.Q[r][c]));
              w = cscale(w, S.beta[j]);
              for (int r = j; r < P; ++r) S.Q[r][c] = csub(S.Q[r][c], cmul(S.M[r][j], w));
            }
          }
        }
        __syncwarp();
        for (int e = lane; e < HS * HA; e += 32) {
          const int j = e / HA, cc = e - j * HA;
          cd v = mk(0.0, 0.0);
          if (j < nref) {
            if (cc == j) v = S.alpha[j];
            else if (cc > j) v = S.M[j][cc];
          }
          S.Rn[s][j][cc] = v;
        }
        for (int e = lane; e < HS * P; e += 32) {
          const int j = e / P, l = e - j * P;
          store_cplx(out, base + (s * HS + j) * CHI + l, (j < nref) ? S.Q[l][j] : mk(0.0, 0.0), out_c128);
        }
        pk += nref;
        __syncwarp();
      }
      for (int e = lane; e < 2 * HS * HA; e += 32) (&S.R[0][0][0])[e] = (&S.Rn[0][0][0])[e];
      act = pk;
      __syncwarp();
    } else {
      // last site: v_s[row] = sum_{c in block s} L(c) sum_cp R[t][j][cp] bond(cp, c), normalised jointly
      double part = 0.0;
      for (int e = lane; e < 2 * P; e += 32) {
        const int s = e / P, row = e - s * P;
        const int t = row / HS, j = row - t * HS;
        cd acc = mk(0.0, 0.0);
        for (int cc = 0; cc < HA; ++cc) {
          const int c = s * HA + cc;
          cd inner = mk(0.0, 0.0);
          for (int cp = 0; cp < HA; ++cp) inner = cadd(inner, cmul(S.R[t][j][cp], f.bond(t * HA + cp, c)));
          acc = cadd(acc, cmul(S.L[c], inner));
        }
        S.M[row][s] = acc;  // reuse M as the 2 column vectors (HA >= 2)
        part += cabs2(acc);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      __syncwarp();
      const double inv = part > 0.0 ? 1.0 / sqrt(part) : 0.0;
      for (int e = lane; e < 2 * HS * P; e += 32) {
        const int s = e / (HS * P), rem = e - s * HS * P;
        const int j = rem / P, l = rem - j * P;
        store_cplx(out, base + (s * HS + j) * CHI + l, j == 0 ? cscale(S.M[l][s], inv) : mk(0.0, 0.0), out_c128);
      }
      if (bond && i == 0 && lane == 0) bond[n] = 1;
    }
    xprev = xk;
    __syncwarp();
  }
}

// ln|<psi~_i|psi~_i>| of the stored tensors, one thread per sample, by the Gram arithmetic.
template <typename real, int H>
struct GlobalSub {
  const real* site;  // this sample's compact tensor at the current site
  __device__ __forceinline__ void operator()(int, int s, int t, Blk<real, H>& blk) const {
    constexpr int CHI = 2 * H;
#pragma unroll
    for (int j = 0; j < H; ++j)
#pragma unroll
      for (int a = 0; a < H; ++a) {
        const int idx = 2 * ((s * H + j) * CHI + t * H + a);
        blk.r[a][j] = site[idx];
        blk.i[a][j] = site[idx + 1];
      }
  }
};

template <typename real, int H>
__global__ void __launch_bounds__(32) self_overlap_kernel(const real* __restrict__ mps, int m, int n,
                                                           float* __restrict__ log_norm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  constexpr size_t PER = size_t(2 * H) * (2 * H) * 2;  // reals per sample-site
  PairE<real, H> st[1][1];
  st[0][0].init();
  for (int k = 0; k < n; ++k) {
    const GlobalSub<real, H> ld{mps + (size_t(k) * m + i) * PER};
    const bool last = (k == n - 1);
    site_step<real, H, 1, 1>(st, ld, ld, last || ((k % RENORM_EVERY) == RENORM_EVERY - 1));
  }
  log_norm[i] = st[0][0].half_log_mod();
}

// Threads per CTA of the pair kernel: full warps while there are enough samples to give
// every SM one, narrower CTAs (fewer samples each) otherwise, so that more SMs share the
// FP64 work.
static int pair_kernel_lanes(int m, int sm_count) {
  int lanes = 32;
  while (lanes > 8 && (2 * m + lanes - 1) / lanes < sm_count) lanes >>= 1;
  return lanes;
}

template <int HS, int HA>
static dk_status launch_build(const float* x, int m, int n, const dk_fmap* fm, int c128, void* mps, int32_t* bond,
                              float* log_norm, int sm_count, cudaStream_t st, bool* fused_norm) {
  const bool fp64_qr = c128 || fm->qr_prec == DK_PREC_F64;
  const int eb = !fm->entangle ? 0 : ((fm->block >= 1 && fm->block < n) ? fm->block : n);
  *fused_norm = false;
  if constexpr (HA <= 2) {
    constexpr int RP = HA == 1 ? 1 : 2;
    // the fused self-overlap covers the bond-4 tensors (the Gram kernels' HS = 2)
    float* ln = HS == 2 ? log_norm : nullptr;
    // Bond 4: 8 threads per sample. FP32 arithmetic (complex64 output, qr_prec F32) at
    // every size; FP64 arithmetic while the set is small enough that the per-sample chain
    // latency, not the FP64 issue rate, sets the time (up to about 2.5 warps per SM
    // sub-partition), and two threads per sample beyond that, where the 8-thread form's
    // extra reduction instructions cost more than its shorter chain saves.
    const bool small = (m + 3) / 4 <= 10 * sm_count;
    if (HS == 2 && (!fp64_qr || small)) {
      // 4 samples per warp-sized CTA; fewer per CTA when that would leave SMs idle
      const int spc = (m + 3) / 4 >= sm_count ? 4 : ((m + 1) / 2 >= sm_count ? 2 : 1);
      const int grid = (m + spc - 1) / spc;
      const double as = double(fm->angle_scale);
      if (c128) {
        mps_build_oct_kernel<HA, RP, double, double><<<grid, 8 * spc, 0, st>>>(x, m, n, as, eb, mps, bond, ln);
      } else if (fp64_qr) {
        mps_build_oct_kernel<HA, RP, float, double><<<grid, 8 * spc, 0, st>>>(x, m, n, as, eb, mps, bond, ln);
      } else {
        mps_build_oct_kernel<HA, RP, float, float><<<grid, 8 * spc, 0, st>>>(x, m, n, as, eb, mps, bond, ln);
      }
      *fused_norm = ln != nullptr;
      return launch_status();
    }
    const int lanes = pair_kernel_lanes(m, sm_count);
    const int grid = (2 * m + lanes - 1) / lanes;
    if (c128) {
      mps_build_pair_kernel<HS, HA, RP, double><<<grid, lanes, 0, st>>>(x, m, n, double(fm->angle_scale),
                                                                       eb, mps, bond, ln);
    } else {
      mps_build_pair_kernel<HS, HA, RP, float><<<grid, lanes, 0, st>>>(x, m, n, double(fm->angle_scale),
                                                                      eb, mps, bond, ln);
    }
    *fused_norm = ln != nullptr;
  } else {
    const size_t smem = sizeof(WarpQr<HS, HA>);
    constexpr int RP = HA == 4 ? 3 : HA == 8 ? 4 : 5;
    auto kern = mps_build_warp_kernel<HS, HA, RP>;
    if (smem > 48 * 1024) {
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
        return DK_ERR_CUDA;
    }
    kern<<<m, 32, smem, st>>>(x, m, n, double(fm->angle_scale), eb, c128, mps, bond);
  }
  return launch_status();
}

DK_API dk_status dk_self_overlap(dk_ctx* ctx, const void* mps, int m, int n, int chi_max, dk_dtype dtype,
                                 dk_precision prec, float* log_norm, void* stream) {
  using namespace dk;
  if (!ctx || !mps || !log_norm || m < 1 || n < 1) return DK_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (prec == DK_PREC_BF16X3) {
    if (dtype != DK_C64 || chi_max != 32) return DK_ERR_UNSUPPORTED;
    return self_overlap32_tc_launch(mps, m, n, log_norm, st);
  }
  if ((prec == DK_PREC_F32 && dtype != DK_C64) || (prec == DK_PREC_F64 && dtype != DK_C128)) return DK_ERR_UNSUPPORTED;
  if (prec != DK_PREC_F32 && prec != DK_PREC_F64) return DK_ERR_UNSUPPORTED;
  return self_overlap_launch(mps, m, n, chi_max, dtype, log_norm, st);
}

}  // namespace dk

DK_API dk_status dk_mps_build(dk_ctx* ctx, const float* x, int m, int n, const dk_fmap* fm, dk_dtype dtype,
                              void* mps, int32_t* bond_dims, float* log_norm, void* stream) {
  using namespace dk;
  if (!ctx || !x || !fm || !mps || m < 1 || n < 1) return DK_ERR_ARG;
  if (fm->reps < 1 || fm->reps > 5) return DK_ERR_ARG;
  if (fm->qr_prec != DK_PREC_F32 && fm->qr_prec != DK_PREC_F64) return DK_ERR_ARG;
  if (fm->block < 0) return DK_ERR_ARG;
  if (dtype != DK_C64 && dtype != DK_C128) return DK_ERR_ARG;
  const int chi = fm->chi_max;
  if (chi != 4 && chi != 8 && chi != 16 && chi != 32) return DK_ERR_UNSUPPORTED;
  if (chi < (1 << fm->reps)) return DK_ERR_UNSUPPORTED;
  if (!aligned16(mps)) return DK_ERR_ARG;
  if (log_norm && !(chi == 4 || (dtype == DK_C64 && (chi == 8 || chi == 32)))) return DK_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int c128 = dtype == DK_C128 ? 1 : 0;
  dk_status s = DK_ERR_UNSUPPORTED;
  bool fused = false;
  // (stored block HS = chi/2, closed-form block HA = 2^(reps-1))
  if (chi == 4 && fm->reps == 1) s = launch_build<2, 1>(x, m, n, fm, c128, mps, bond_dims, log_norm, ctx->sm_count, st, &fused);
  else if (chi == 4 && fm->reps == 2) s = launch_build<2, 2>(x, m, n, fm, c128, mps, bond_dims, log_norm, ctx->sm_count, st, &fused);
  else if (chi == 8 && fm->reps == 1) s = launch_build<4, 1>(x, m, n, fm, c128, mps, bond_dims, log_norm, ctx->sm_count, st, &fused);
  else if (chi == 8 && fm->reps == 2) s = launch_build<4, 2>(x, m, n, fm, c128, mps, bond_dims, log_norm, ctx->sm_count, st, &fused);
  else if (chi == 8 && fm->reps == 3) s = launch_build<4, 4>(x, m, n, fm, c128, mps, bond_dims, log_norm, ctx->sm_count, st, &fused);
  else if (chi == 16 && fm->reps == 4) s = launch_build<8, 8>(x, m, n, fm, c128, mps, bond_dims, log_norm, ctx->sm_count, st, &fused);
  else if (chi == 32 && fm->reps == 5) s = launch_build<16, 16>(x, m, n, fm, c128, mps, bond_dims, log_norm, ctx->sm_count, st, &fused);
  if (s != DK_OK || !log_norm || fused) return s;
  return self_overlap_launch(mps, m, n, chi, dtype, log_norm, st);
}

dk_status dk::self_overlap_launch(const void* mps, int m, int n, int chi, dk_dtype dtype, float* log_norm,
                                  cudaStream_t st) {
  using namespace dk;
  // one warp per CTA: each thread runs a whole n-site chain, so spread the chains over SMs
  const int grid = (m + 31) / 32;
  if (dtype == DK_C64 && chi == 32) return self_overlap32_launch(mps, m, n, log_norm, st);
  if (dtype == DK_C64 && chi == 8) {
    self_overlap_kernel<float, 4><<<grid, 32, 0, st>>>(static_cast<const float*>(mps), m, n, log_norm);
  } else if (dtype == DK_C64 && chi == 4) {
    self_overlap_kernel<float, 2><<<grid, 32, 0, st>>>(static_cast<const float*>(mps), m, n, log_norm);
  } else if (dtype == DK_C128 && chi == 4) {
    self_overlap_kernel<double, 2><<<grid, 32, 0, st>>>(static_cast<const double*>(mps), m, n, log_norm);
  } else {
    return DK_ERR_UNSUPPORTED;
  }
  return launch_status();
}
