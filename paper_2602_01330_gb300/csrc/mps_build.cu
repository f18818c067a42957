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
// The self-overlap kernel then runs the Gram transfer arithmetic (transfer.cuh) on each
// sample's own rounded tensors and stores ln|<psi~|psi~>|, the normaliser that makes the
// Gram diagonal exactly 1.
#include <math.h>

#include "common.cuh"
#include "internal.h"
#include "transfer.cuh"

namespace dk {

struct cd {
  double x, y;
};
__device__ __forceinline__ cd mk(double x, double y) { return cd{x, y}; }
__device__ __forceinline__ cd cmul(cd a, cd b) { return mk(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x)); }
__device__ __forceinline__ cd cconjmul(cd a, cd b) { return mk(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x)); }
__device__ __forceinline__ cd cadd(cd a, cd b) { return mk(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cd csub(cd a, cd b) { return mk(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cd cscale(cd a, double s) { return mk(a.x * s, a.y * s); }
__device__ __forceinline__ cd cconj(cd a) { return mk(a.x, -a.y); }
__device__ __forceinline__ double cabs2(cd a) { return fma(a.x, a.x, a.y * a.y); }

constexpr double PI_D = 3.14159265358979323846;

// Closed-form factors of one site: u^e and w^e for e in [-r, r], u = exp(-i phi/2),
// w = exp(-i theta/2) (both unit modulus, so u^-e = conj(u^e)).
struct SiteFactors {
  cd up[6];
  cd wp[6];
  double amp;
  int reps;
  __device__ __forceinline__ void make(double phi, double theta, int r) {
    reps = r;
    amp = exp2(-0.5 * r);
    double sn, cs;
    sincos(-0.5 * phi, &sn, &cs);
    const cd u = mk(cs, sn);
    sincos(-0.5 * theta, &sn, &cs);
    const cd w = mk(cs, sn);
    up[0] = mk(1.0, 0.0);
    wp[0] = mk(1.0, 0.0);
#pragma unroll
    for (int q = 1; q < 6; ++q) {
      up[q] = cmul(up[q - 1], u);
      wp[q] = cmul(wp[q - 1], w);
    }
  }
  __device__ __forceinline__ cd upow(int e) const { return e >= 0 ? up[e] : cconj(up[-e]); }
  __device__ __forceinline__ cd wpow(int e) const { return e >= 0 ? wp[e] : cconj(wp[-e]); }
  // L_k(c)
  __device__ __forceinline__ cd local(int c) const {
    const double sign = (__popc(c & (c >> 1)) & 1) ? -amp : amp;
    return cscale(upow(reps - 2 * __popc(c)), sign);
  }
  // bond phase between closed-form left index cp and right index c
  __device__ __forceinline__ cd bond(int cp, int c) const { return wpow(reps - 2 * __popc(cp ^ c)); }
};

// Householder QR of a P x C complex matrix (static sizes, registers), nref <= C reflectors.
// On return Q holds the first nref columns of Q (others zero) and R the nref x C upper
// trapezoidal factor (rows >= nref zero).
template <int P, int C>
__device__ __forceinline__ void householder_qr(cd (&M)[P][C], int nref, cd (&Q)[P][C], cd (&R)[C][C]) {
  double beta[C];
  cd alpha[C];
#pragma unroll
  for (int j = 0; j < C; ++j) {
    beta[j] = 0.0;
    alpha[j] = mk(0.0, 0.0);
    if (j < nref && j < P) {
      double sigma2 = 0.0;
#pragma unroll
      for (int i = j; i < P; ++i) sigma2 += cabs2(M[i][j]);
      const cd x0 = M[j][j];
      const double ax0 = sqrt(cabs2(x0));
      const double sigma = sqrt(sigma2);
      if (sigma > 0.0) {
        const cd u = ax0 > 0.0 ? cscale(x0, 1.0 / ax0) : mk(1.0, 0.0);
        alpha[j] = cscale(u, -sigma);
        M[j][j] = cscale(u, ax0 + sigma);  // v_0; v_i = M[i][j] below
        beta[j] = 1.0 / (sigma * (sigma + ax0));
#pragma unroll
        for (int c = j + 1; c < C; ++c) {
          cd w = mk(0.0, 0.0);
#pragma unroll
          for (int i = j; i < P; ++i) w = cadd(w, cconjmul(M[i][j], M[i][c]));
          w = cscale(w, beta[j]);
#pragma unroll
          for (int i = j; i < P; ++i) M[i][c] = csub(M[i][c], cmul(M[i][j], w));
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < C; ++r)
#pragma unroll
    for (int c = 0; c < C; ++c) {
      cd v = mk(0.0, 0.0);
      if (r < nref) {
        if (c == r) v = alpha[r];
        else if (c > r) v = M[r][c];
      }
      R[r][c] = v;
    }
#pragma unroll
  for (int c = 0; c < C; ++c) {
    cd col[P];
#pragma unroll
    for (int i = 0; i < P; ++i) col[i] = mk((i == c && c < nref) ? 1.0 : 0.0, 0.0);
#pragma unroll
    for (int j = C - 1; j >= 0; --j) {
      if (j < nref && j < P && beta[j] != 0.0 && c < nref) {
        cd w = mk(0.0, 0.0);
#pragma unroll
        for (int i = j; i < P; ++i) w = cadd(w, cconjmul(M[i][j], col[i]));
        w = cscale(w, beta[j]);
#pragma unroll
        for (int i = j; i < P; ++i) col[i] = csub(col[i], cmul(M[i][j], w));
      }
    }
#pragma unroll
    for (int i = 0; i < P; ++i) Q[i][c] = col[i];
  }
}

__device__ __forceinline__ void store_cplx(void* out, size_t idx, cd v, int c128) {
  if (c128) reinterpret_cast<double2*>(out)[idx] = make_double2(v.x, v.y);
  else reinterpret_cast<float2*>(out)[idx] = make_float2(float(v.x), float(v.y));
}

// One thread per sample; HS = stored block size chi/2, HA = closed-form block size 2^(r-1).
template <int HS, int HA>
__global__ void __launch_bounds__(128) mps_build_thread_kernel(const float* __restrict__ x, int m, int n, int reps,
                                                               double angle_scale, int entangle, int out_c128,
                                                               void* __restrict__ out, int32_t* __restrict__ bond) {
  constexpr int P = 2 * HS;   // stored left-bond positions
  constexpr int CHI = 2 * HS;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
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
  double xprev = 0.0;
  const size_t per = size_t(CHI) * CHI;  // complex entries per sample-site
  SiteFactors f;
  for (int k = 0; k < n; ++k) {
    const double xk = double(xs[k]);
    f.make(angle_scale * xk, (entangle && k > 0) ? 2.0 * (PI_D - xprev) * (PI_D - xk) : 0.0, reps);
    const size_t base = (size_t(k) * m + i) * per;
    if (bond && i == 0) bond[k] = act;
    if (k < n - 1) {
      cd Rn[2][HS][HA];
      int pk = 0;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
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
        householder_qr<P, HA>(M, nref, Q, Rr);
#pragma unroll
        for (int j = 0; j < HS; ++j)
#pragma unroll
          for (int l = 0; l < P; ++l) store_cplx(out, base + (s * HS + j) * CHI + l, j < HA ? Q[l][j] : mk(0.0, 0.0), out_c128);
#pragma unroll
        for (int j = 0; j < HS; ++j)
#pragma unroll
          for (int cc = 0; cc < HA; ++cc) Rn[s][j][cc] = j < HA ? Rr[j][cc] : mk(0.0, 0.0);
        pk += nref;
      }
#pragma unroll
      for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int j = 0; j < HS; ++j)
#pragma unroll
          for (int c = 0; c < HA; ++c) R[t][j][c] = Rn[t][j][c];
      act = pk;
    } else {
      cd v[2][P];
      double nrm2 = 0.0;
#pragma unroll
      for (int s = 0; s < 2; ++s)
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
            v[s][t * HS + j] = acc;
            nrm2 += cabs2(acc);
          }
      const double inv = nrm2 > 0.0 ? 1.0 / sqrt(nrm2) : 0.0;
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int j = 0; j < HS; ++j)
#pragma unroll
          for (int l = 0; l < P; ++l)
            store_cplx(out, base + (s * HS + j) * CHI + l, j == 0 ? cscale(v[s][l], inv) : mk(0.0, 0.0), out_c128);
      if (bond && i == 0) bond[n] = 1;
    }
    xprev = xk;
  }
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

template <int HS, int HA>
__global__ void __launch_bounds__(32) mps_build_warp_kernel(const float* __restrict__ x, int m, int n, int reps,
                                                            double angle_scale, int entangle, int out_c128,
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
  SiteFactors f;
  for (int k = 0; k < n; ++k) {
    const double xk = double(xs[k]);
    f.make(angle_scale * xk, (entangle && k > 0) ? 2.0 * (PI_D - xprev) * (PI_D - xk) : 0.0, reps);
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
__global__ void __launch_bounds__(128) self_overlap_kernel(const real* __restrict__ mps, int m, int n,
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

template <int HS, int HA>
static dk_status launch_build(const float* x, int m, int n, const dk_fmap* fm, int c128, void* mps, int32_t* bond,
                              cudaStream_t st) {
  if constexpr (HA <= 2) {
    mps_build_thread_kernel<HS, HA><<<(m + 127) / 128, 128, 0, st>>>(x, m, n, fm->reps, double(fm->angle_scale),
                                                                    fm->entangle, c128, mps, bond);
  } else {
    const size_t smem = sizeof(WarpQr<HS, HA>);
    auto kern = mps_build_warp_kernel<HS, HA>;
    if (smem > 48 * 1024) {
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
        return DK_ERR_CUDA;
    }
    kern<<<m, 32, smem, st>>>(x, m, n, fm->reps, double(fm->angle_scale), fm->entangle, c128, mps, bond);
  }
  return launch_status();
}

}  // namespace dk

DK_API dk_status dk_mps_build(dk_ctx* ctx, const float* x, int m, int n, const dk_fmap* fm, dk_dtype dtype,
                              void* mps, int32_t* bond_dims, float* log_norm, void* stream) {
  using namespace dk;
  if (!ctx || !x || !fm || !mps || m < 1 || n < 1) return DK_ERR_ARG;
  if (fm->reps < 1 || fm->reps > 5) return DK_ERR_ARG;
  if (dtype != DK_C64 && dtype != DK_C128) return DK_ERR_ARG;
  const int chi = fm->chi_max;
  if (chi != 4 && chi != 8 && chi != 16 && chi != 32) return DK_ERR_UNSUPPORTED;
  if (chi < (1 << fm->reps)) return DK_ERR_UNSUPPORTED;
  if (!aligned16(mps)) return DK_ERR_ARG;
  if (log_norm && chi != 4) return DK_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int c128 = dtype == DK_C128 ? 1 : 0;
  dk_status s = DK_ERR_UNSUPPORTED;
  // (stored block HS = chi/2, closed-form block HA = 2^(reps-1))
  if (chi == 4 && fm->reps == 1) s = launch_build<2, 1>(x, m, n, fm, c128, mps, bond_dims, st);
  else if (chi == 4 && fm->reps == 2) s = launch_build<2, 2>(x, m, n, fm, c128, mps, bond_dims, st);
  else if (chi == 8 && fm->reps == 1) s = launch_build<4, 1>(x, m, n, fm, c128, mps, bond_dims, st);
  else if (chi == 8 && fm->reps == 2) s = launch_build<4, 2>(x, m, n, fm, c128, mps, bond_dims, st);
  else if (chi == 8 && fm->reps == 3) s = launch_build<4, 4>(x, m, n, fm, c128, mps, bond_dims, st);
  else if (chi == 16 && fm->reps == 4) s = launch_build<8, 8>(x, m, n, fm, c128, mps, bond_dims, st);
  else if (chi == 32 && fm->reps == 5) s = launch_build<16, 16>(x, m, n, fm, c128, mps, bond_dims, st);
  if (s != DK_OK || !log_norm) return s;
  const int grid = (m + 127) / 128;
  if (dtype == DK_C64) {
    self_overlap_kernel<float, 2><<<grid, 128, 0, st>>>(static_cast<const float*>(mps), m, n, log_norm);
  } else {
    self_overlap_kernel<double, 2><<<grid, 128, 0, st>>>(static_cast<const double*>(mps), m, n, log_norm);
  }
  return launch_status();
}
