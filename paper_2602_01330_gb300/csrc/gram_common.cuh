// Arguments, tile enumeration and the fused epilogue shared by the Gram kernels.
//
// Epilogue (§II-B Eq. 3, §II-C Eq. 10, §II-D Eq. 11): log K_q = 2 ln|a| - ln N_i - ln N_j,
// K_q = exp(log K_q), K_c = exp(-gamma ||x_i - x_j||^2), K = w K_q + (1 - w) K_c.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace dk {

struct GramArgs {
  int n;
  int row0, nrows, col0, ncols;
  int tiles_r, tiles_c, ntiles;
  int symmetric;
  const float* lnorm_r;
  const float* lnorm_c;
  const float* x_r;
  const float* x_c;
  float gamma, w;
  float* k;
  float* kq;
  float* kc;
  float* lkq;
  long long ld;
  unsigned* status;
  int need_kc;  // K_c is needed (k_out with w != 1, or kc_out)
  const float* d2;  // squared distances of the block's pairs, nrows x ncols (kernels that take them precomputed)
};

// First column tile of row tile ti that holds a pair with j >= i (symmetric Gram): the
// tile (ti, tj) covers rows from ti*TR and columns up to (tj+1)*TC - 1.
__host__ __device__ __forceinline__ int first_upper_tile(int ti, int tr, int tc) { return (ti * tr) / tc; }

// Tile index t (row-major over the tiles that are computed) -> (row tile, column tile).
__device__ __forceinline__ void decode_tile(const GramArgs& p, int tr, int tc, int t, int& ti, int& tj) {
  if (p.symmetric) {
    int r = 0;
    while (true) {
      const int first = first_upper_tile(r, tr, tc);
      const int cnt = first < p.tiles_c ? p.tiles_c - first : 0;
      if (t < cnt || r + 1 >= p.tiles_r) {
        ti = r;
        tj = first + t;
        return;
      }
      t -= cnt;
      ++r;
    }
  } else {
    ti = t / p.tiles_c;
    tj = t - ti * p.tiles_c;
  }
}

// Component c (compile-time after unrolling) of a float4.
__device__ __forceinline__ float f4_get(const float4& v, int c) {
  return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w;
}

// Compensated (Kahan) FP32 accumulation of one squared feature difference.
__device__ __forceinline__ void kahan_add_sq(float& sum, float& comp, float d) {
  const float y = fmaf(d, d, -comp);
  const float t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

__device__ __forceinline__ void write_pair(const GramArgs& p, float half_log, float d2, int i, int j) {
  if (i >= p.row0 + p.nrows || j >= p.col0 + p.ncols) return;
  if (p.symmetric && j < i) return;
  const float lr = p.lnorm_r ? p.lnorm_r[i] : 0.0f;
  const float lc = p.lnorm_c ? p.lnorm_c[j] : 0.0f;
  const float lkq = 2.0f * half_log - lr - lc;
  const float kq = expf(lkq);
  const float kc = p.need_kc ? expf(-p.gamma * d2) : 0.0f;
  const float k = p.w * kq + (1.0f - p.w) * kc;
  const long long a = (long long)(i - p.row0) * p.ld + (j - p.col0);
  if (p.k) p.k[a] = k;
  if (p.kq) p.kq[a] = kq;
  if (p.kc) p.kc[a] = kc;
  if (p.lkq) p.lkq[a] = lkq;
  if (p.symmetric && i != j) {
    const long long b = (long long)(j - p.col0) * p.ld + (i - p.row0);
    if (p.k) p.k[b] = k;
    if (p.kq) p.kq[b] = kq;
    if (p.kc) p.kc[b] = kc;
    if (p.lkq) p.lkq[b] = lkq;
  }
}


// Number of tiles a launch covers (host): all TR x TC tiles of the block, or for the
// symmetric Gram only those holding a pair with j >= i.
inline int count_tiles(GramArgs& a, int tr, int tc) {
  a.tiles_r = (a.nrows + tr - 1) / tr;
  a.tiles_c = (a.ncols + tc - 1) / tc;
  if (!a.symmetric) return a.tiles_r * a.tiles_c;
  long long cnt = 0;
  for (int ti = 0; ti < a.tiles_r; ++ti) {
    const int first = first_upper_tile(ti, tr, tc);
    if (first < a.tiles_c) cnt += a.tiles_c - first;
  }
  return int(cnt);
}

}  // namespace dk
