// Data pre-processing of §II-A on the GPU: standardisation (zero mean, unit variance per
// pixel), PCA (the leading eigenvectors of the covariance of the standardised training rows)
// and min-max scaling of the projected features to [0, range_max].
//
// * Column statistics: two passes per column in FP64 (a constant column gets scale 1).
// * Covariance C = Z^T Z / (m - 1): 32 x 32 output tiles, the standardised rows staged in
//   shared memory 32 at a time, FP32 accumulation.
// * Eigenvectors: parallel cyclic Jacobi (round-robin pairing: every round rotates p/2
//   disjoint index pairs, a sweep is p - 1 rounds). A round is two launches: the rotation
//   angles of all pairs from the current matrix, then one thread per 2 x 2 block (i1, j1) x
//   (i2, j2) applying both rotations at once, J1^T B J2, so rows and columns move together;
//   the eigenvector matrix is kept transposed (row i = eigenvector i), so its update is a
//   row update. A fixed number of sweeps runs without host synchronisation; the remaining
//   relative off-diagonal norm is returned.
// * Selection: eigenvalues ranked in decreasing order (the smaller index first on ties), the
//   leading k rows written with the sign that makes the entry of largest magnitude positive.
// * Transform: y = ((x - mean) / scale) C_k^T by 32 x 32 tiles; min-max scaling fitted on
//   the training rows (or given) and applied with clipping.
//
// Working memory (A and V^T, 2 p^2 floats, plus the rotation table) is a caller-provided
// workspace of dk_pca_workspace_bytes(p) bytes.
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace dk {
namespace pca {

constexpr int T32 = 32;

__global__ void __launch_bounds__(256) col_stats_kernel(const float* __restrict__ x, int m, int p,
                                                        float* __restrict__ mean, float* __restrict__ scale) {
  const int c = blockIdx.x * 32 + (threadIdx.x & 31), rg = threadIdx.x >> 5;
  __shared__ double red[8][32];
  __shared__ double s_mean[32];
  double s = 0.0;
  if (c < p)
    for (int r = rg; r < m; r += 8) s += double(x[(long long)r * p + c]);
  red[rg][threadIdx.x & 31] = s;
  __syncthreads();
  if (rg == 0) {
    double t = 0.0;
    for (int g = 0; g < 8; ++g) t += red[g][threadIdx.x];
    s_mean[threadIdx.x] = t / m;
  }
  __syncthreads();
  const double mu = s_mean[threadIdx.x & 31];
  double q = 0.0;
  if (c < p)
    for (int r = rg; r < m; r += 8) {
      const double d = double(x[(long long)r * p + c]) - mu;
      q += d * d;
    }
  __syncthreads();
  red[rg][threadIdx.x & 31] = q;
  __syncthreads();
  if (rg == 0 && c < p) {
    double t = 0.0;
    for (int g = 0; g < 8; ++g) t += red[g][threadIdx.x];
    const double var = t / m;
    mean[c] = float(mu);
    scale[c] = var > 0.0 ? float(sqrt(var)) : 1.0f;
  }
}

// C[i][j] = sum_r z_ri z_rj / (m - 1), z_rc = (x_rc - mean_c) / scale_c; 32 x 32 tiles
__global__ void __launch_bounds__(256) cov_kernel(const float* __restrict__ x, int m, int p,
                                                  const float* __restrict__ mean, const float* __restrict__ scale,
                                                  float* __restrict__ A) {
  __shared__ float zi[T32][T32 + 1], zj[T32][T32 + 1];
  const int i0 = blockIdx.y * T32, j0 = blockIdx.x * T32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of 4 outputs per thread
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int r0 = 0; r0 < m; r0 += T32) {
    for (int e = threadIdx.x; e < T32 * T32; e += 256) {
      const int rr = e / T32, cc = e % T32, r = r0 + rr;
      const int ci = i0 + cc, cj = j0 + cc;
      zi[rr][cc] = (r < m && ci < p) ? (x[(long long)r * p + ci] - mean[ci]) / scale[ci] : 0.0f;
      zj[rr][cc] = (r < m && cj < p) ? (x[(long long)r * p + cj] - mean[cj]) / scale[cj] : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < T32; ++rr) {
      const float b = zj[rr][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(zi[rr][ty * 4 + q], b, acc[q]);
    }
    __syncthreads();
  }
  const float inv = 1.0f / float(m - 1);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + ty * 4 + q, j = j0 + tx;
    if (i < p && j < p) A[(long long)i * p + j] = acc[q] * inv;
  }
}

// Vt = identity
__global__ void eye_kernel(float* __restrict__ Vt, int p) {
  const long long n = (long long)p * p;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    Vt[e] = (e / p == e % p) ? 1.0f : 0.0f;
}

// index of round-robin position t in round r (positions 0..pe-1, pe even; 0 stays put)
__device__ __forceinline__ int rr_pos(int t, int r, int pe) { return t == 0 ? 0 : 1 + (t - 1 + r) % (pe - 1); }

// rotation angles of pair k of round r: (i, j, c, s) with i < j; a pair holding the
// padding index p (odd p) is the identity
__device__ __forceinline__ void jacobi_pair_params(const float* A, int p, int pe, int r, int k, int2* ij,
                                                   float4* cs) {
  int i = rr_pos(k, r, pe), j = rr_pos(pe - 1 - k, r, pe);
  if (i > j) {
    const int t = i;
    i = j;
    j = t;
  }
  float c = 1.0f, s = 0.0f, t = 0.0f;
  if (j < p) {
    const float aii = A[(long long)i * p + i], ajj = A[(long long)j * p + j], aij = A[(long long)i * p + j];
    if (fabsf(aij) > 1e-30f) {
      // angle that zeroes a_ij: tau = (a_jj - a_ii) / (2 a_ij), t the smaller root
      const float tau = (ajj - aii) / (2.0f * aij);
      t = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
      c = __frsqrt_rn(1.0f + t * t);  // correctly rounded: c^2 + s^2 - 1 stays unbiased
      s = t * c;
    }
  }
  ij[k] = make_int2(i, j);
  cs[k] = make_float4(c, s, t, 0.0f);
}

// the rotation angles of round r (the first round of a fit)
__global__ void jacobi_params_kernel(const float* __restrict__ A, int p, int pe, int r, int2* __restrict__ ij,
                                     float4* __restrict__ cs) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < pe / 2) jacobi_pair_params(A, p, pe, r, k, ij, cs);
}

// one round: block (k1) handles the rows of pair k1; thread k2 the 2 x 2 block with the
// columns of pair k2: B' = J1^T B J2 (J = [[c, s], [-s, c]]); the block's pair also rotates
// rows i1, j1 of V^T
//
// One launch per round: the CTA that finishes the round last (a counter each CTA bumps after
// a fence) computes the next round's angles from the finished matrix, so no launch of its
// own and no CTA waits for another; it also resets the counter. r_next < 0: last round.
__global__ void __launch_bounds__(256) jacobi_rotate_kernel(float* __restrict__ A, float* __restrict__ Vt, int p,
                                                            int npairs, int2* __restrict__ ij,
                                                            float4* __restrict__ cs, unsigned* __restrict__ done,
                                                            int pe, int r_next) {
  const int k1 = blockIdx.x;
  const int2 a = ij[k1];
  const float4 r1 = cs[k1];
  const int i1 = a.x, j1 = a.y;
  const bool has_j1 = j1 < p;
  for (int k2 = threadIdx.x; k2 < npairs; k2 += blockDim.x) {
    const int2 b = ij[k2];
    const float4 r2 = cs[k2];
    const int i2 = b.x, j2 = b.y;
    const bool has_j2 = j2 < p;
    const float b00 = A[(long long)i1 * p + i2];
    const float b01 = has_j2 ? A[(long long)i1 * p + j2] : 0.0f;
    const float b10 = has_j1 ? A[(long long)j1 * p + i2] : 0.0f;
    const float b11 = (has_j1 && has_j2) ? A[(long long)j1 * p + j2] : 0.0f;
    // rows: R0 = c1 B0 - s1 B1, R1 = s1 B0 + c1 B1
    const float q00 = r1.x * b00 - r1.y * b10, q01 = r1.x * b01 - r1.y * b11;
    const float q10 = r1.y * b00 + r1.x * b10, q11 = r1.y * b01 + r1.x * b11;
    // columns: C0 = c2 R.0 - s2 R.1, C1 = s2 R.0 + c2 R.1
    float n00 = r2.x * q00 - r2.y * q01, n01 = r2.y * q00 + r2.x * q01;
    float n10 = r2.x * q10 - r2.y * q11, n11 = r2.y * q10 + r2.x * q11;
    if (k1 == k2 && has_j1) {
      // the pair's own block: the rotation zeroes its off-diagonal, and the diagonal moves
      // by -/+ t a_ij, which keeps the trace to one rounding
      n00 = b00 - r1.z * b01;
      n11 = b11 + r1.z * b01;
      n01 = 0.0f;
      n10 = 0.0f;
    }
    A[(long long)i1 * p + i2] = n00;
    if (has_j2) A[(long long)i1 * p + j2] = n01;
    if (has_j1) A[(long long)j1 * p + i2] = n10;
    if (has_j1 && has_j2) A[(long long)j1 * p + j2] = n11;
  }
  if (has_j1) {
    for (int col = threadIdx.x; col < p; col += blockDim.x) {
      const float u = Vt[(long long)i1 * p + col], v = Vt[(long long)j1 * p + col];
      Vt[(long long)i1 * p + col] = r1.x * u - r1.y * v;
      Vt[(long long)j1 * p + col] = r1.y * u + r1.x * v;
    }
  }
  if (r_next < 0) return;
  __shared__ bool last;
  __threadfence();  // this CTA's writes of A are visible before it counts itself done
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(done, 1u) == unsigned(npairs - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();  // every other CTA's writes are visible to this one
  for (int k = threadIdx.x; k < npairs; k += blockDim.x) jacobi_pair_params(A, p, pe, r_next, k, ij, cs);
  if (threadIdx.x == 0) *done = 0u;
}

// sqrt(off-diagonal sum of squares / total sum of squares) of A
__global__ void __launch_bounds__(256) off_norm_kernel(const float* __restrict__ A, int p, float* __restrict__ out) {
  double off = 0.0, all = 0.0;
  const long long n = (long long)p * p;
  for (long long e = threadIdx.x; e < n; e += 256) {
    const double v = A[e];
    all += v * v;
    if (e / p != e % p) off += v * v;
  }
  __shared__ double s_off[256], s_all[256];
  s_off[threadIdx.x] = off;
  s_all[threadIdx.x] = all;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      s_off[threadIdx.x] += s_off[threadIdx.x + h];
      s_all[threadIdx.x] += s_all[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s_all[0] > 0.0 ? float(sqrt(s_off[0] / s_all[0])) : 0.0f;
}

// block i: the rank of eigenvalue A_ii among all (decreasing, smaller index first on ties);
// if below k, row rank of the output is row i of V^T with the sign of its largest entry
__global__ void __launch_bounds__(256) select_kernel(const float* __restrict__ A, const float* __restrict__ Vt, int p,
                                                     int k, float* __restrict__ comps, float* __restrict__ eig) {
  const int i = blockIdx.x;
  const float li = A[(long long)i * p + i];
  __shared__ int s_rank[256];
  __shared__ float s_best[256];
  __shared__ int s_bi[256];
  int cnt = 0;
  for (int j = threadIdx.x; j < p; j += 256) {
    const float lj = A[(long long)j * p + j];
    if (lj > li || (lj == li && j < i)) ++cnt;
  }
  s_rank[threadIdx.x] = cnt;
  float best = -1.0f;
  int bi = p;
  for (int c = threadIdx.x; c < p; c += 256) {
    const float v = fabsf(Vt[(long long)i * p + c]);
    if (v > best) {
      best = v;
      bi = c;
    }
  }
  s_best[threadIdx.x] = best;
  s_bi[threadIdx.x] = bi;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      s_rank[threadIdx.x] += s_rank[threadIdx.x + h];
      const float ob = s_best[threadIdx.x + h];
      const int oi = s_bi[threadIdx.x + h];
      if (ob > s_best[threadIdx.x] || (ob == s_best[threadIdx.x] && oi < s_bi[threadIdx.x])) {
        s_best[threadIdx.x] = ob;
        s_bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const int rank = s_rank[0];
  if (rank >= k) return;
  const float sign = Vt[(long long)i * p + s_bi[0]] < 0.0f ? -1.0f : 1.0f;
  for (int c = threadIdx.x; c < p; c += 256) comps[(long long)rank * p + c] = sign * Vt[(long long)i * p + c];
  if (threadIdx.x == 0) eig[rank] = li;
}

// out[r][q] = sum_c ((x_rc - mean_c) / scale_c) comps[q][c]; 32 x 32 tiles (rows x components)
__global__ void __launch_bounds__(256) transform_kernel(const float* __restrict__ x, int m, int p,
                                                        const float* __restrict__ mean, const float* __restrict__ scale,
                                                        const float* __restrict__ comps, int k, float* __restrict__ out) {
  __shared__ float zs[T32][T32 + 1], cs_[T32][T32 + 1];
  const int r0 = blockIdx.y * T32, q0 = blockIdx.x * T32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int c0 = 0; c0 < p; c0 += T32) {
    for (int e = threadIdx.x; e < T32 * T32; e += 256) {
      const int a = e / T32, b = e % T32;
      const int r = r0 + a, c = c0 + b, q = q0 + a;
      zs[a][b] = (r < m && c < p) ? (x[(long long)r * p + c] - mean[c]) / scale[c] : 0.0f;
      cs_[a][b] = (q < k && c < p) ? comps[(long long)q * p + c] : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int b = 0; b < T32; ++b) {
      const float w = cs_[tx][b];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fmaf(zs[ty * 4 + u][b], w, acc[u]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int r = r0 + ty * 4 + u, q = q0 + tx;
    if (r < m && q < k) out[(long long)r * k + q] = acc[u];
  }
}

__global__ void __launch_bounds__(256) minmax_fit_kernel(const float* __restrict__ y, int m, int k,
                                                         float* __restrict__ lo, float* __restrict__ hi) {
  const int c = blockIdx.x * 32 + (threadIdx.x & 31), rg = threadIdx.x >> 5;
  float mn = INFINITY, mx = -INFINITY;
  if (c < k)
    for (int r = rg; r < m; r += 8) {
      const float v = y[(long long)r * k + c];
      mn = fminf(mn, v);
      mx = fmaxf(mx, v);
    }
  __shared__ float smn[8][32], smx[8][32];
  smn[rg][threadIdx.x & 31] = mn;
  smx[rg][threadIdx.x & 31] = mx;
  __syncthreads();
  if (rg == 0 && c < k) {
    for (int g = 1; g < 8; ++g) {
      mn = fminf(mn, smn[g][threadIdx.x]);
      mx = fmaxf(mx, smx[g][threadIdx.x]);
    }
    lo[c] = mn;
    hi[c] = mx;
  }
}

__global__ void minmax_apply_kernel(float* __restrict__ y, long long n, int k, const float* __restrict__ lo,
                                    const float* __restrict__ hi, float range_max) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int c = int(e % k);
    const float span = hi[c] - lo[c];
    float v = span > 0.0f ? (y[e] - lo[c]) / span * range_max : 0.0f;
    y[e] = fminf(fmaxf(v, 0.0f), range_max);
  }
}

struct Workspace {
  float* A;
  float* Vt;
  int2* ij;
  float4* cs;
  unsigned* done;  // CTAs finished in the current Jacobi round
};

inline size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

inline size_t workspace_bytes(int p) {
  const size_t pe = size_t(p + (p & 1));
  return 2 * round256(size_t(p) * p * sizeof(float)) + round256(pe / 2 * sizeof(int2)) +
         round256(pe / 2 * sizeof(float4)) + 256;
}

inline Workspace carve(void* ws, int p) {
  uint8_t* b = static_cast<uint8_t*>(ws);
  const size_t pe = size_t(p + (p & 1));
  Workspace w;
  w.A = reinterpret_cast<float*>(b);
  b += round256(size_t(p) * p * sizeof(float));
  w.Vt = reinterpret_cast<float*>(b);
  b += round256(size_t(p) * p * sizeof(float));
  w.ij = reinterpret_cast<int2*>(b);
  b += round256(pe / 2 * sizeof(int2));
  w.cs = reinterpret_cast<float4*>(b);
  b += round256(pe / 2 * sizeof(float4));
  w.done = reinterpret_cast<unsigned*>(b);
  return w;
}

// the fit on a carved workspace (shared by the entry points)
dk_status fit(dk_ctx* ctx, const float* x, int m, int p, int k, int sweeps, const Workspace& w, float* mean,
              float* scale, float* comps, float* eig, float* off_norm, cudaStream_t st) {
  col_stats_kernel<<<(p + 31) / 32, 256, 0, st>>>(x, m, p, mean, scale);
  cov_kernel<<<dim3((p + T32 - 1) / T32, (p + T32 - 1) / T32), 256, 0, st>>>(x, m, p, mean, scale, w.A);
  const int fill_blocks = int(((long long)p * p + 255) / 256 < 4096 ? ((long long)p * p + 255) / 256 : 4096);
  eye_kernel<<<fill_blocks, 256, 0, st>>>(w.Vt, p);
  const int pe = p + (p & 1), np = pe / 2;
  if (cudaMemsetAsync(w.done, 0, sizeof(unsigned), st) != cudaSuccess) return DK_ERR_CUDA;
  jacobi_params_kernel<<<(np + 255) / 256, 256, 0, st>>>(w.A, p, pe, 0, w.ij, w.cs);
  const int rounds = sweeps * (pe - 1);
  for (int q = 0; q < rounds; ++q) {
    const int r_next = q + 1 < rounds ? (q + 1) % (pe - 1) : -1;
    jacobi_rotate_kernel<<<np, 256, 0, st>>>(w.A, w.Vt, p, np, w.ij, w.cs, w.done, pe, r_next);
  }
  if (off_norm) off_norm_kernel<<<1, 256, 0, st>>>(w.A, p, off_norm);
  select_kernel<<<p, 256, 0, st>>>(w.A, w.Vt, p, k, comps, eig);
  return launch_status();
}

}  // namespace pca
}  // namespace dk

using namespace dk;

DK_API size_t dk_pca_workspace_bytes(int p) { return p < 2 || p > DK_PCA_MAX_FEATURES ? 0 : pca::workspace_bytes(p); }

DK_API dk_status dk_pca_fit(dk_ctx* ctx, const float* x, int m, int p, int k, int sweeps, void* workspace,
                            size_t workspace_bytes, float* mean, float* scale, float* components,
                            float* eigenvalues, float* off_norm, void* stream) {
  if (!ctx || !x || !workspace || !mean || !scale || !components || !eigenvalues) return DK_ERR_ARG;
  if (m < 2 || p < 2 || k < 1 || k > p || sweeps < 1 || sweeps > 100) return DK_ERR_ARG;
  if (p > DK_PCA_MAX_FEATURES) return DK_ERR_UNSUPPORTED;
  if (workspace_bytes < pca::workspace_bytes(p) || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
    return DK_ERR_WORKSPACE;
  return pca::fit(ctx, x, m, p, k, sweeps, pca::carve(workspace, p), mean, scale, components, eigenvalues,
                  off_norm, static_cast<cudaStream_t>(stream));
}

DK_API dk_status dk_pca_transform(dk_ctx* ctx, const float* x, int m, int p, const float* mean, const float* scale,
                                  const float* components, int k, int fit_range, float range_max, float* lo,
                                  float* hi, float* out, void* stream) {
  if (!ctx || !x || !mean || !scale || !components || !lo || !hi || !out) return DK_ERR_ARG;
  if (m < 1 || p < 1 || k < 1 || k > p || !(range_max > 0.0f)) return DK_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  pca::transform_kernel<<<dim3((k + pca::T32 - 1) / pca::T32, (m + pca::T32 - 1) / pca::T32), 256, 0, st>>>(
      x, m, p, mean, scale, components, k, out);
  if (fit_range) pca::minmax_fit_kernel<<<(k + 31) / 32, 256, 0, st>>>(out, m, k, lo, hi);
  const long long n = (long long)m * k;
  const int blocks = int((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192);
  pca::minmax_apply_kernel<<<blocks, 256, 0, st>>>(out, n, k, lo, hi, range_max);
  return launch_status();
}

// ---------------------------------------------------------------------------------------
// dk_pca_fit_noalloc: the same fit with its working memory in a fixed device array.
//
// For callers that cannot hand this library device memory of their own: a host program
// whose device memory is owned and capped by another framework, a plug-in that receives
// only its input and output pointers, or a loop that must not stall on or fail in an
// allocation midway. The working memory for up to DK_PCA_NOALLOC_MAX_FEATURES features
// lives in the file-scope array below, which every GPU that loads the library holds until
// the process exits. Host code cannot pass the array's name to a kernel (on the host it
// names a stand-in, not device memory), so the first call on each device looks up the
// array's device address with that device current and keeps it for later calls.

namespace dk {
namespace pca {

constexpr size_t round256_c(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t noalloc_bytes() {
  return 2 * round256_c(size_t(DK_PCA_NOALLOC_MAX_FEATURES) * DK_PCA_NOALLOC_MAX_FEATURES * sizeof(float)) +
         round256_c(DK_PCA_NOALLOC_MAX_FEATURES / 2 * sizeof(int2)) +
         round256_c(DK_PCA_NOALLOC_MAX_FEATURES / 2 * sizeof(float4)) + 256;
}

static __device__ __align__(256) unsigned char g_noalloc_scratch[noalloc_bytes()];

constexpr int MAX_DEVICES = 64;
static void* g_noalloc_ptr[MAX_DEVICES] = {};
static std::mutex g_noalloc_mu;

// device address of g_noalloc_scratch on `device`, looked up once with that device current
static dk_status noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= MAX_DEVICES) return DK_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return DK_ERR_CUDA;
    if (cur != device && cudaSetDevice(device) != cudaSuccess) return DK_ERR_CUDA;
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (cur != device && cudaSetDevice(cur) != cudaSuccess) return DK_ERR_CUDA;
    if (e != cudaSuccess || !ptr) return DK_ERR_CUDA;
    g_noalloc_ptr[device] = ptr;
  }
  *out = g_noalloc_ptr[device];
  return DK_OK;
}

}  // namespace pca
}  // namespace dk

DK_API dk_status dk_pca_fit_noalloc(dk_ctx* ctx, const float* x, int m, int p, int k, int sweeps, float* mean,
                                    float* scale, float* components, float* eigenvalues, float* off_norm,
                                    void* stream) {
  if (!ctx || !x || !mean || !scale || !components || !eigenvalues) return DK_ERR_ARG;
  if (m < 2 || p < 2 || k < 1 || k > p || sweeps < 1 || sweeps > 100) return DK_ERR_ARG;
  if (p > DK_PCA_NOALLOC_MAX_FEATURES) return DK_ERR_UNSUPPORTED;
  void* scratch = nullptr;
  const dk_status s = pca::noalloc_scratch(ctx->device, &scratch);
  if (s != DK_OK) return s;
  // every part of the scratch that the fit reads is written earlier in the same call (the
  // covariance, the identity, each round's rotation table, the round counter, which the fit
  // clears), so nothing else needs clearing
  return pca::fit(ctx, x, m, p, k, sweeps, pca::carve(scratch, p), mean, scale, components, eigenvalues, off_norm,
                  static_cast<cudaStream_t>(stream));
}
