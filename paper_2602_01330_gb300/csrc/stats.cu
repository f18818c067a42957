// Concentration diagnostics of a quantum-kernel Gram: the spread of the off-diagonal
// values. §I of the paper names exponential concentration (similarities of distinct inputs
// collapsing toward a constant as the qubit count grows) as the quantum kernel's
// fundamental limit, and its conclusion asks for kernel diagnostics beside accuracy.
//
// One grid-stride pass over the entries of a block (for a symmetric Gram: the strict upper
// triangle, each unordered pair once): count, sum and sum of squares of K_q and of log K_q
// (finite values only; log K_q stays exact where K_q underflows to 0), accumulated in FP64
// per thread, reduced per CTA and added atomically into the caller's doubles; a one-thread
// kernel then forms the means and variances from the sums.
#include <math.h>
#include <stdint.h>

#include "common.cuh"
#include "internal.h"

namespace dk {
namespace stats {

constexpr int NT = 256;

__global__ void __launch_bounds__(NT) gram_stats_kernel(const float* __restrict__ kq, const float* __restrict__ lkq,
                                                        long long ld, int nrows, int ncols, int symmetric,
                                                        double* __restrict__ out) {
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const long long total = (long long)nrows * ncols;
  for (long long e = (long long)blockIdx.x * NT + threadIdx.x; e < total; e += (long long)gridDim.x * NT) {
    const int i = int(e / ncols), j = int(e - (long long)i * ncols);
    if (symmetric && j <= i) continue;
    const long long o = (long long)i * ld + j;
    if (kq) {
      const double v = kq[o];
      acc[0] += 1.0;
      acc[1] += v;
      acc[2] += v * v;
    }
    if (lkq) {
      const float lf = lkq[o];
      if (isfinite(lf)) {
        const double l = lf;
        acc[3] += 1.0;
        acc[4] += l;
        acc[5] += l * l;
      }
    }
  }
  __shared__ double red[NT / 32][6];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    double v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w][threadIdx.x];
    atomicAdd(out + threadIdx.x, s);
  }
}

// Means and population variances from the sums: out[6..9] = mean K_q, var K_q, mean log K_q,
// var log K_q (NaN when nothing was counted; a variance rounding below 0 is set to 0).
__global__ void gram_stats_finish_kernel(double* __restrict__ out) {
  if (threadIdx.x != 0) return;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const double c = out[3 * q], s1 = out[3 * q + 1], s2 = out[3 * q + 2];
    const double mean = c > 0.0 ? s1 / c : nan("");
    const double var = c > 0.0 ? fmax(s2 / c - mean * mean, 0.0) : nan("");
    out[6 + 2 * q] = mean;
    out[7 + 2 * q] = var;
  }
}

}  // namespace stats
}  // namespace dk

using namespace dk;

DK_API dk_status dk_gram_stats(dk_ctx* ctx, const float* kq, const float* logkq, long long ld, int nrows, int ncols,
                               int symmetric, double* out, void* stream) {
  if (!ctx || (!kq && !logkq) || !out || nrows < 1 || ncols < 1 || ld < ncols) return DK_ERR_ARG;
  if (symmetric && nrows != ncols) return DK_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(out, 0, 10 * sizeof(double), st) != cudaSuccess) return DK_ERR_CUDA;
  const long long total = (long long)nrows * ncols;
  long long blocks = (total + stats::NT * 8 - 1) / (stats::NT * 8);
  const long long cap = (long long)ctx->sm_count * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  stats::gram_stats_kernel<<<int(blocks), stats::NT, 0, st>>>(kq, logkq, ld, nrows, ncols, symmetric, out);
  dk_status s = launch_status();
  if (s != DK_OK) return s;
  stats::gram_stats_finish_kernel<<<1, 32, 0, st>>>(out);
  return launch_status();
}
