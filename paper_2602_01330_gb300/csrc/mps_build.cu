// MPS of the feature-map state (§II-C, Eq. 6) and its self-overlap normalisation.
//
// Construction (exact, no truncation). Write qubit k's computational-basis value
// after the single-qubit layer of repetition rho as z_k^(rho) (z^(0) = 0). Each RZZ
// layer is diagonal, so the amplitude of |z^(r)> is a sum over the intermediate
// values z^(1..r-1) of a product of
//   * per-qubit factors  G_k[z^(rho)][z^(rho-1)],  G_k = RZ(angle_scale x_k) H,
//   * per-bond phases    exp(-i theta_k/2 (-1)^(z_k^(rho) XOR z_{k+1}^(rho))),
//                        theta_k = 2 (pi - x_k)(pi - x_{k+1}).
// Grouping the values (z_k^(1), ..., z_k^(r)) into one bond index of size 2^r turns
// this sum into an MPS whose site tensor has a closed form:
//   A^(k)[s][l][c] = [top bit of c == s] * L_k(c) * exp(-i theta_{k-1}/2 (r - 2 popc(l XOR c))),
//   L_k(c) = 2^(-r/2) (-1)^popc(c AND c>>1) exp(-i angle_scale x_k / 2 (r - 2 popc(c))),
// with the left bond of site 0 of size 1 (no phase) and the right bond of site n-1
// summed over. One warp per sample then sweeps left to right in FP64: M = R A^(k)
// (rows (s, l'), columns c), Householder QR M = Q R, store Q as the left-canonical
// tensor of site k, carry R to the next site. The final 1 x 1 R is the norm, which is
// dropped, so the stored state has unit norm before rounding to complex64/128.
//
// The self-overlap kernel then runs the Gram transfer arithmetic (transfer.cuh) on each
// sample's own rounded tensors and stores ln|<psi~|psi~>|, the normaliser that makes
// the Gram diagonal exactly 1.
#include <math.h>

#include "common.cuh"
#include "internal.h"
#include "transfer.cuh"

namespace dk {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {  // conj(a) * b
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cexpi(double t) {
  double s, c;
  sincos(t, &s, &c);
  return make_double2(c, s);
}

template <int CHIA>
struct QrSmem {
  double2 R[CHIA][CHIA];        // carried left factor, D x Dl
  double2 M[2 * CHIA][CHIA];    // site matrix, then Householder vectors (lower) and R' (upper)
  double2 Qb[2 * CHIA][CHIA];   // explicit Q, P x p
  double2 L[CHIA];              // per-qubit path factors L_k(c)
  double2 ph[8];                // bond phase per popcount, index 0..r
  double2 alpha[CHIA];          // diagonal of R'
  double beta[CHIA];            // 2 / |v|^2 of each reflector
};

template <int CHIA, int WPB>
__global__ void __launch_bounds__(WPB * 32) mps_build_kernel(const float* __restrict__ x, int m, int n, int reps,
                                                             double angle_scale, int entangle, int chi_out,
                                                             int out_c128, void* __restrict__ out,
                                                             int32_t* __restrict__ bond_out) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  QrSmem<CHIA>& W = reinterpret_cast<QrSmem<CHIA>*>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int sample = blockIdx.x * WPB + (threadIdx.x >> 5);
  if (sample >= m) return;  // the whole warp leaves together
  const float* xs = x + size_t(sample) * n;
  const double PI = 3.14159265358979323846;
  const double amp = pow(0.5, 0.5 * reps);

  int D = 1;   // rows of R (stored left bond of the current site)
  int Dl = 1;  // columns of R (closed-form left bond of the current site)
  if (lane == 0) W.R[0][0] = make_double2(1.0, 0.0);
  double xprev = 0.0;
  const size_t site_stride = size_t(m) * 2 * chi_out * chi_out;  // complex entries per site

  for (int k = 0; k < n; ++k) {
    const bool last = (k == n - 1);
    const int Q = last ? 1 : CHIA;
    const int P = 2 * D;
    const int pk = P < Q ? P : Q;
    const double xk = double(xs[k]);
    const double phi = angle_scale * xk;
    const double theta = (entangle && k > 0) ? 2.0 * (PI - xprev) * (PI - xk) : 0.0;
    if (lane < CHIA) {
      const int c = lane;
      const int pc = __popc(c);
      const double sign = (__popc(c & (c >> 1)) & 1) ? -1.0 : 1.0;
      const double2 e = cexpi(-0.5 * phi * double(reps - 2 * pc));
      W.L[c] = make_double2(sign * amp * e.x, sign * amp * e.y);
    }
    if (lane <= reps) W.ph[lane] = cexpi(-0.5 * theta * double(reps - 2 * lane));
    __syncwarp();

    // M = R A^(k): rows (s, l') with row = s * D + l', columns c.
    if (!last) {
      for (int c = lane; c < Q; c += 32) {
        const int top = (c >> (reps - 1)) & 1;
        const double2 lc = W.L[c];
        for (int row = 0; row < P; ++row) {
          const int s = row / D, lp = row - s * D;
          double2 acc = make_double2(0.0, 0.0);
          if (s == top) {
            for (int l = 0; l < Dl; ++l) acc = cadd(acc, cmul(W.R[lp][l], W.ph[__popc(l ^ c)]));
            acc = cmul(lc, acc);
          }
          W.M[row][c] = acc;
        }
      }
    } else {
      for (int row = lane; row < P; row += 32) {
        const int s = row / D, lp = row - s * D;
        double2 acc = make_double2(0.0, 0.0);
        for (int c = 0; c < CHIA; ++c) {
          if (((c >> (reps - 1)) & 1) != s) continue;
          double2 inner = make_double2(0.0, 0.0);
          for (int l = 0; l < Dl; ++l) inner = cadd(inner, cmul(W.R[lp][l], W.ph[__popc(l ^ c)]));
          acc = cadd(acc, cmul(W.L[c], inner));
        }
        W.M[row][0] = acc;
      }
    }
    __syncwarp();

    // Householder QR of M (P x Q), pk reflectors; lane c owns column c.
    for (int j = 0; j < pk; ++j) {
      if (lane == j) {
        double sigma2 = 0.0;
        for (int i = j; i < P; ++i) sigma2 = fma(W.M[i][j].x, W.M[i][j].x, fma(W.M[i][j].y, W.M[i][j].y, sigma2));
        const double2 x0 = W.M[j][j];
        const double ax0 = hypot(x0.x, x0.y);
        const double sigma = sqrt(sigma2);
        if (sigma == 0.0) {
          W.beta[j] = 0.0;
          W.alpha[j] = make_double2(0.0, 0.0);
        } else {
          const double2 u = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
          W.alpha[j] = make_double2(-u.x * sigma, -u.y * sigma);
          W.M[j][j] = make_double2(u.x * (ax0 + sigma), u.y * (ax0 + sigma));
          W.beta[j] = 1.0 / (sigma * (sigma + ax0));
        }
      }
      __syncwarp();
      const int c = lane;
      if (c > j && c < Q && W.beta[j] != 0.0) {
        double2 w = make_double2(0.0, 0.0);
        for (int i = j; i < P; ++i) w = cadd(w, cconjmul(W.M[i][j], W.M[i][c]));
        const double2 f = make_double2(W.beta[j] * w.x, W.beta[j] * w.y);
        for (int i = j; i < P; ++i) {
          const double2 t = cmul(W.M[i][j], f);
          W.M[i][c] = make_double2(W.M[i][c].x - t.x, W.M[i][c].y - t.y);
        }
      }
      __syncwarp();
    }

    // Q = H_0 ... H_{pk-1} [I; 0]; lane c < pk forms column c.
    if (lane < pk) {
      const int c = lane;
      for (int i = 0; i < P; ++i) W.Qb[i][c] = make_double2(i == c ? 1.0 : 0.0, 0.0);
      for (int j = pk - 1; j >= 0; --j) {
        if (W.beta[j] == 0.0) continue;
        double2 w = make_double2(0.0, 0.0);
        for (int i = j; i < P; ++i) w = cadd(w, cconjmul(W.M[i][j], W.Qb[i][c]));
        const double2 f = make_double2(W.beta[j] * w.x, W.beta[j] * w.y);
        for (int i = j; i < P; ++i) {
          const double2 t = cmul(W.M[i][j], f);
          W.Qb[i][c] = make_double2(W.Qb[i][c].x - t.x, W.Qb[i][c].y - t.y);
        }
      }
    }
    __syncwarp();

    // R' (pk x Q) becomes the carried factor; lane c owns column c.
    for (int c = lane; c < Q; c += 32) {
      for (int r = 0; r < pk; ++r) {
        double2 v = make_double2(0.0, 0.0);
        if (c == r) v = W.alpha[r];
        else if (c > r) v = W.M[r][c];
        W.R[r][c] = v;
      }
    }

    // Store Q as A[k][sample][s][r][l] = Q[s*D + l][r], zero-padded to chi_out.
    const int per = 2 * chi_out * chi_out;
    const size_t base = size_t(k) * site_stride + size_t(sample) * per;
    for (int e = lane; e < per; e += 32) {
      const int l = e % chi_out;
      const int r = (e / chi_out) % chi_out;
      const int s = e / (chi_out * chi_out);
      double2 v = make_double2(0.0, 0.0);
      if (r < pk && l < D) v = W.Qb[s * D + l][r];
      if (out_c128) {
        reinterpret_cast<double2*>(out)[base + e] = v;
      } else {
        reinterpret_cast<float2*>(out)[base + e] = make_float2(float(v.x), float(v.y));
      }
    }
    if (bond_out && sample == 0 && lane == 0) {
      bond_out[k] = D;
      if (last) bond_out[n] = 1;
    }
    D = pk;
    Dl = Q;
    xprev = xk;
    __syncwarp();
  }
}

// ln|<psi~_i|psi~_i>| of the stored tensors, one thread per sample, by the Gram arithmetic.
template <typename real, int CHI>
struct GlobalCol {
  const uint8_t* base;  // this sample's tensor at the current site
  __device__ __forceinline__ void operator()(int s, int col, real (&re)[CHI], real (&im)[CHI]) const {
    const real* p = reinterpret_cast<const real*>(base) + 2 * ((s * CHI + col) * CHI);
#pragma unroll
    for (int l = 0; l < CHI; ++l) {
      re[l] = p[2 * l];
      im[l] = p[2 * l + 1];
    }
  }
};

template <typename real, int CHI>
__global__ void __launch_bounds__(128) self_overlap_kernel(const uint8_t* __restrict__ mps, int m, int n,
                                                           float* __restrict__ log_norm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  constexpr size_t SB = size_t(2) * CHI * CHI * 2 * sizeof(real);
  Chain<real, CHI> ch;
  ch.init();
  for (int k = 0; k < n; ++k) {
    GlobalCol<real, CHI> ld{mps + (size_t(k) * m + i) * SB};
    ch.step(ld, ld);
  }
  log_norm[i] = ch.half_log_mod();
}

template <int CHIA>
static dk_status launch_build(const float* x, int m, int n, const dk_fmap* fm, int out_c128, void* mps,
                              int32_t* bond, cudaStream_t st) {
  constexpr int WPB = CHIA <= 8 ? 4 : 1;
  const size_t smem = WPB * sizeof(QrSmem<CHIA>);
  auto kern = mps_build_kernel<CHIA, WPB>;
  if (smem > 48 * 1024) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
      return DK_ERR_CUDA;
  }
  const int grid = (m + WPB - 1) / WPB;
  kern<<<grid, WPB * 32, smem, st>>>(x, m, n, fm->reps, double(fm->angle_scale), fm->entangle, fm->chi_max,
                                     out_c128, mps, bond);
  return launch_status();
}

}  // namespace dk

// Largest stored bond of the left-canonical sweep: D_0 = 1, D_{k+1} = min(2 D_k, 2^reps),
// and 1 to the right of the last site.
static int max_stored_bond(int n, int reps) {
  const int chia = 1 << reps;
  int d = 1, mx = 1;
  for (int k = 0; k < n; ++k) {
    const int q = (k == n - 1) ? 1 : chia;
    const int p = (2 * d < q) ? 2 * d : q;
    if (p > mx) mx = p;
    if (d > mx) mx = d;
    d = p;
  }
  return mx;
}

DK_API dk_status dk_mps_build(dk_ctx* ctx, const float* x, int m, int n, const dk_fmap* fm, dk_dtype dtype,
                              void* mps, int32_t* bond_dims, float* log_norm, void* stream) {
  using namespace dk;
  if (!ctx || !x || !fm || !mps || m < 1 || n < 1) return DK_ERR_ARG;
  if (fm->reps < 1 || fm->reps > 5) return DK_ERR_ARG;
  if (dtype != DK_C64 && dtype != DK_C128) return DK_ERR_ARG;
  const int chi = fm->chi_max;
  if (chi != 2 && chi != 4 && chi != 8 && chi != 16 && chi != 32) return DK_ERR_UNSUPPORTED;
  if (chi < max_stored_bond(n, fm->reps)) return DK_ERR_UNSUPPORTED;
  if (!aligned16(mps)) return DK_ERR_ARG;
  if (log_norm && !((dtype == DK_C64 && chi == 4) || (dtype == DK_C128 && (chi == 2 || chi == 4))))
    return DK_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int c128 = dtype == DK_C128 ? 1 : 0;
  dk_status s;
  switch (fm->reps) {
    case 1: s = launch_build<2>(x, m, n, fm, c128, mps, bond_dims, st); break;
    case 2: s = launch_build<4>(x, m, n, fm, c128, mps, bond_dims, st); break;
    case 3: s = launch_build<8>(x, m, n, fm, c128, mps, bond_dims, st); break;
    case 4: s = launch_build<16>(x, m, n, fm, c128, mps, bond_dims, st); break;
    default: s = launch_build<32>(x, m, n, fm, c128, mps, bond_dims, st); break;
  }
  if (s != DK_OK || !log_norm) return s;
  const int grid = (m + 127) / 128;
  const uint8_t* p = static_cast<const uint8_t*>(mps);
  if (dtype == DK_C64) {
    self_overlap_kernel<float, 4><<<grid, 128, 0, st>>>(p, m, n, log_norm);
  } else if (chi == 2) {
    self_overlap_kernel<double, 2><<<grid, 128, 0, st>>>(p, m, n, log_norm);
  } else {
    self_overlap_kernel<double, 4><<<grid, 128, 0, st>>>(p, m, n, log_norm);
  }
  return launch_status();
}
