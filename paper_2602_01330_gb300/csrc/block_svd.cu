// MPS of a block-structured feature map from its block statevectors, with SVD truncation.
//
// With entanglers only inside blocks of b consecutive qubits (the block product structure of
// §II-C) the state is the Kronecker product of the blocks' states, so every block can be
// simulated exactly as a dense 2^b statevector (b <= 12) and cut into MPS site tensors by
// a left-to-right sweep of singular value decompositions. This covers entanglers whose bond
// exceeds the 2^reps of the nearest-neighbour closed form (all-to-all ZZ inside a block:
// rank up to 2^(b/2)), where the bond cap and the singular value cutoff truncate.
//
// One warp per (sample, block), up to four warps per CTA that never wait on each other. Per
// block, in FP64 shared memory:
//   1. the statevector: per repetition a Walsh-Hadamard pass per qubit, then the diagonal
//      phase exp(-i Phi(z)), Phi(z) = sum_q (scale x_q / 2) z_q + sum_{(q,r)} (pi - x_q)(pi - x_r) z_q z_r
//      over z in {+1, -1}^b (RZ and RZZ are diagonal and commute);
//   2. for the cut after each qubit: the remainder as an r x c matrix M (rows: left bond and
//      physical value, columns: the qubits to the right), one-sided Jacobi (Hestenes) on the
//      rows until they are mutually orthogonal, M' = J M with J unitary; the row norms are the
//      singular values. Rows are ranked by norm, the kept ones (s > cutoff s_0, at most the
//      bond cap) are rescaled to the norm of the whole spectrum and become the next
//      remainder in place (each kept row splits into its two halves, addressed through a
//      row-offset table, so nothing is copied); the site tensor is J^dagger restricted to the
//      kept rows, its columns orthonormal (left-canonical). The last qubit stores the
//      remaining normalised vector.
//
// Output layout: the compact block layout of the Gram kernels (include/dualk.h), with a
// general site tensor B_s[a][j] "lifted" into it: block s of the right bond holds column j of
// B_s and both copies t = 0, 1 of the left bond hold row a, so the Gram's block transfer
// E'_s = sum_t A_s[t]^dagger E_t A_s[t] equals B_s^dagger (E_0 + E_1) B_s, the plain transfer
// of the general MPS. A kept bond of at most chi_max / 2 therefore runs through the existing
// chi_max Gram kernels unchanged.
#include <math.h>

#include "block_state.cuh"
#include "common.cuh"
#include "internal.h"

namespace dk {
namespace bsvd {

constexpr int MAXB = blockstate::MAXB;
constexpr int MAXR = 32;        // rows of M: 2 x kept bond <= chi_max <= 32
constexpr int MAX_SWEEPS = 40;  // Jacobi sweeps per cut (quadratic convergence needs ~6-10)
constexpr double ORTH_TOL = 1e-14;  // rotate while |<p,q>| > tol sqrt(|p|^2 |q|^2)
// The remainder always has unit Frobenius norm (the left factors are isometries and the kept
// spectrum is rescaled to the whole), so a row with squared norm below FLOOR2 is rounding
// noise of a rank-deficient cut: rotating such rows against each other never converges and
// drives them into underflow, so pairs involving one are left alone. Rows that the cutoff
// can keep (s > 1e-10 s_0, s_0 >= 1/sqrt(32)) are far above it.
constexpr double FLOOR2 = 1e-30;
constexpr int MAX_WARPS = 4;    // warps (blocks) per CTA
constexpr size_t SMEM_CAP = 227 * 1024;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {  // conj(a) b
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// Working memory of one warp (one block of one sample); the state and its phase factors follow.
struct WarpShared {
  double2 J[MAXR][MAXR];  // accumulated row rotations of the current cut
  double nrm[MAXR];       // squared row norms
  int rowbase[MAXR];      // offset of each row of M in the state buffer
  int nextbase[MAXR];
  int perm[MAXR];         // rows by decreasing norm
  blockstate::Coeffs coef;
  double scale;           // renormalisation of the kept rows
  int keep;               // kept bond of the current cut
};

// Bytes per warp for blocks of b qubits, and warps per CTA
inline size_t warp_bytes(int b) {
  return ((sizeof(WarpShared) + 15) & ~size_t(15)) + 2 * (size_t(1) << b) * sizeof(double2);
}
inline int warps_per_cta(int b) {
  const size_t w = SMEM_CAP / warp_bytes(b);
  return int(w < 1 ? 1 : (w > size_t(MAX_WARPS) ? MAX_WARPS : w));
}

// (k, round t) -> row of the round-robin pairing of r rows (r even): row 0 stays, the rest rotate
__device__ __forceinline__ int rr_row(int k, int t, int r) { return k == 0 ? 0 : ((k - 1 + t) % (r - 1)) + 1; }

__device__ __forceinline__ void store(void* out, size_t idx, double2 v, int c128) {
  if (c128) reinterpret_cast<double2*>(out)[idx] = v;
  else reinterpret_cast<float2*>(out)[idx] = make_float2(float(v.x), float(v.y));
}

__global__ void __launch_bounds__(128) bond_init_kernel(int32_t* bond, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= n; k += gridDim.x * blockDim.x) bond[k] = 1;
}

// UW warps per (sample, block) unit: u = sample * nb + block. UW = 1: several units per CTA,
// each one warp with warp-level barriers only (units never wait on each other); UW = 4: one
// unit per CTA (blocks whose state leaves room for one unit per SM).
template <int UW>
__device__ __forceinline__ void unit_sync() {
  if constexpr (UW == 1) __syncwarp();
  else __syncthreads();
}

template <int UW>
__global__ void __launch_bounds__(MAX_WARPS * 32)
    block_svd_kernel(const float* __restrict__ x, int m, int n, int b, int nb, int reps, double angle_scale,
                     int pairs_kind, double cutoff, int cap, int chi, int out_c128, size_t wbytes,
                     void* __restrict__ out, int32_t* __restrict__ bond, float* __restrict__ discarded) {
  constexpr int NTU = 32 * UW;  // threads per unit
  extern __shared__ __align__(16) unsigned char raw[];
  const int slot = threadIdx.x / NTU, tid = threadIdx.x % NTU, lane = threadIdx.x & 31, wu = tid >> 5;
  const long long unit = (long long)blockIdx.x * (blockDim.x / NTU) + slot;
  if (unit >= (long long)m * nb) return;  // the whole unit (UW = 4: the whole CTA)
  unsigned char* mine = raw + slot * wbytes;
  WarpShared& S = *reinterpret_cast<WarpShared*>(mine);
  double2* psi = reinterpret_cast<double2*>(mine + ((sizeof(WarpShared) + 15) & ~size_t(15)));
  double2* ph = psi + (1 << b);
  const int i = int(unit / nb), blk = int(unit % nb);
  const int start = blk * b;
  const int bl = min(b, n - start);
  const int dim = 1 << bl;
  const float* xs = x + size_t(i) * n;
  const int h = chi / 2;
  const size_t per = size_t(chi) * chi;  // complex entries per sample-site
  double disc = 0.0;                     // thread 0: discarded weight over this block's cuts

  // ---- 1. block statevector ----
  if constexpr (UW == 1)
    blockstate::build(psi, ph, S.coef, xs + start, bl, reps, angle_scale, pairs_kind, tid, NTU,
                      blockstate::WarpSync());
  else
    blockstate::build(psi, ph, S.coef, xs + start, bl, reps, angle_scale, pairs_kind, tid, NTU,
                      blockstate::CtaSync());
  // ---- 2. SVD sweep over the block's cuts ----
  int r = 2, c = dim / 2;
  if (tid < 2) S.rowbase[tid] = tid * c;
  unit_sync<UW>();
  for (int q = 0; q < bl; ++q) {
    const int site = start + q;
    const size_t base = (size_t(site) * m + i) * per;
    if (q == bl - 1) {
      // last qubit: the remaining (r x 1) vector, normalised, is column 0 of each block s
      double p = 0.0;
      if (tid < r) {  // r <= 32: warp 0 holds every row
        const double2 v = psi[S.rowbase[tid]];
        p = v.x * v.x + v.y * v.y;
      }
      for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
      if (tid == 0) S.scale = p > 0.0 ? 1.0 / sqrt(p) : 0.0;
      unit_sync<UW>();
      const double inv = S.scale;
      for (size_t e = tid; e < per; e += NTU) {
        const int s = int(e / (size_t(h) * chi)), j = int((e / chi) % h), l = int(e % chi);
        const int a = l % h, row = 2 * a + s;
        double2 v = make_double2(0.0, 0.0);
        if (j == 0 && 2 * a < r) {
          const double2 w = psi[S.rowbase[row]];
          v = make_double2(w.x * inv, w.y * inv);
        }
        store(out, base + e, v, out_c128);
      }
      break;
    }
    for (int e = tid; e < r * r; e += NTU) S.J[e / r][e % r] = make_double2(e / r == e % r ? 1.0 : 0.0, 0.0);
    unit_sync<UW>();
    // one-sided Jacobi on the r rows (length c), r/2 disjoint pairs per round, a lane group each
    const int npairs = r / 2;
    int tpp = NTU / npairs;
    if (tpp > 32) tpp = 32;
    tpp = 1 << (31 - __clz(tpp));  // lanes per pair, a power of two within one warp
    const int g = tid / tpp, gl = tid % tpp;
    for (int sweep = 0; sweep < MAX_SWEEPS; ++sweep) {
      int rotated = 0;
      for (int t = 0; t < r - 1; ++t) {
        const bool act = g < npairs;
        const int rp = act ? rr_row(g, t, r) : 0, rq = act ? rr_row(r - 1 - g, t, r) : 1;
        const double2* P = psi + S.rowbase[rp];
        const double2* Q = psi + S.rowbase[rq];
        double al = 0.0, be = 0.0, gx = 0.0, gy = 0.0;
        if (act)
          for (int col = gl; col < c; col += tpp) {
            const double2 u = P[col], v = Q[col];
            al += u.x * u.x + u.y * u.y;
            be += v.x * v.x + v.y * v.y;
            const double2 w = cconjmul(u, v);
            gx += w.x;
            gy += w.y;
          }
        for (int o = tpp / 2; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          gx += __shfl_xor_sync(0xffffffffu, gx, o);
          gy += __shfl_xor_sync(0xffffffffu, gy, o);
        }
        const double gm = sqrt(gx * gx + gy * gy);
        if (act && fmin(al, be) > FLOOR2 && gm > ORTH_TOL * sqrt(al * be)) {
          // rows p' = c p - s e^{-i phi} q, q' = s p + c e^{-i phi} q with gamma = |gamma| e^{i phi}
          const double zeta = (be - al) / (2.0 * gm);
          const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
          const double2 phs = make_double2(gx / gm, -gy / gm);  // e^{-i phi}
          double2* Pw = psi + S.rowbase[rp];
          double2* Qw = psi + S.rowbase[rq];
          for (int col = gl; col < c; col += tpp) {
            const double2 u = Pw[col], v = cmul(phs, Qw[col]);
            Pw[col] = make_double2(cs * u.x - sn * v.x, cs * u.y - sn * v.y);
            Qw[col] = make_double2(sn * u.x + cs * v.x, sn * u.y + cs * v.y);
          }
          for (int col = gl; col < r; col += tpp) {
            const double2 u = S.J[rp][col], v = cmul(phs, S.J[rq][col]);
            S.J[rp][col] = make_double2(cs * u.x - sn * v.x, cs * u.y - sn * v.y);
            S.J[rq][col] = make_double2(sn * u.x + cs * v.x, sn * u.y + cs * v.y);
          }
          rotated = 1;
        }
        unit_sync<UW>();
      }
      int any;
      if constexpr (UW == 1) any = __any_sync(0xffffffffu, rotated);
      else any = __syncthreads_or(rotated);
      if (!any) break;
    }
    // squared row norms: each warp sums rows in turn
    for (int row = wu; row < r; row += UW) {
      const double2* P = psi + S.rowbase[row];
      double p = 0.0;
      for (int col = lane; col < c; col += 32) p += P[col].x * P[col].x + P[col].y * P[col].y;
      for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
      if (lane == 0) S.nrm[row] = p;
    }
    unit_sync<UW>();
    if (tid < r) {
      int rank = 0;
      for (int j = 0; j < r; ++j) rank += (S.nrm[j] > S.nrm[tid] || (S.nrm[j] == S.nrm[tid] && j < tid)) ? 1 : 0;
      S.perm[rank] = tid;
    }
    unit_sync<UW>();
    if (tid == 0) {
      const double top = S.nrm[S.perm[0]];
      const double floor2 = cutoff * cutoff * top;
      double total = 0.0, kept = 0.0;
      int keep = 0;
      for (int k = 0; k < r; ++k) {
        const double v = S.nrm[S.perm[k]];
        total += v;
        if (keep < cap && v > floor2) {
          ++keep;
          kept += v;
        }
      }
      if (keep == 0) {  // a zero remainder: keep one (zero) row so the chain stays defined
        keep = 1;
        kept = S.nrm[S.perm[0]];
      }
      disc += total > kept ? (total - kept) / total : 0.0;
      S.scale = kept > 0.0 ? sqrt(total / kept) : 1.0;
      S.keep = keep;
      if (bond) atomicMax(bond + site + 1, keep);
    }
    unit_sync<UW>();
    const int keep = S.keep;
    // site tensor: B_s[a][j] = conj(J[perm[j]][2 a + s]) for j < keep, lifted (both t)
    for (size_t e = tid; e < per; e += NTU) {
      const int s = int(e / (size_t(h) * chi)), j = int((e / chi) % h), l = int(e % chi);
      const int a = l % h, row = 2 * a + s;
      double2 v = make_double2(0.0, 0.0);
      if (j < keep && row < r) v = cconj(S.J[S.perm[j]][row]);
      store(out, base + e, v, out_c128);
    }
    // next remainder: kept rows rescaled, each split into its two halves
    for (int k = wu; k < keep; k += UW) {
      double2* P = psi + S.rowbase[S.perm[k]];
      for (int col = lane; col < c; col += 32) P[col] = make_double2(P[col].x * S.scale, P[col].y * S.scale);
    }
    if (tid < 2 * keep) S.nextbase[tid] = S.rowbase[S.perm[tid >> 1]] + (tid & 1) * (c / 2);
    unit_sync<UW>();
    if (tid < 2 * keep) S.rowbase[tid] = S.nextbase[tid];
    r = 2 * keep;
    c /= 2;
    unit_sync<UW>();
  }
  if (tid == 0 && discarded && disc > 0.0) atomicAdd(discarded + i, float(disc));
}

}  // namespace bsvd
}  // namespace dk

DK_API dk_status dk_mps_build_blocks(dk_ctx* ctx, const float* x, int m, int n, const dk_fmap* fm, int entangler,
                                     double cutoff, dk_dtype dtype, void* mps, int32_t* bond_dims, float* log_norm,
                                     float* discarded, void* stream) {
  using namespace dk;
  if (!ctx || !x || !fm || !mps || m < 1 || n < 1) return DK_ERR_ARG;
  if (fm->reps < 1 || fm->reps > 5) return DK_ERR_ARG;
  if (entangler != DK_ENT_CHAIN && entangler != DK_ENT_FULL) return DK_ERR_ARG;
  if (!(cutoff >= 0.0 && cutoff < 1.0)) return DK_ERR_ARG;
  if (dtype != DK_C64 && dtype != DK_C128) return DK_ERR_ARG;
  if (!aligned16(mps)) return DK_ERR_ARG;
  const int b = fm->block > 0 ? fm->block : n;
  if (fm->block < 0 || b > bsvd::MAXB) return DK_ERR_UNSUPPORTED;
  const int chi = fm->chi_max;
  if (chi != 4 && chi != 8 && chi != 16 && chi != 32) return DK_ERR_UNSUPPORTED;
  if (log_norm && !(chi == 4 || (dtype == DK_C64 && (chi == 8 || chi == 32)))) return DK_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int kind = fm->entangle ? entangler : -1;  // -1: no pair is entangled
  const int nb = (n + b - 1) / b;
  const int wpc = bsvd::warps_per_cta(b);  // units that fit in one CTA's shared memory
  const size_t wbytes = bsvd::warp_bytes(b);
  if (bond_dims) bsvd::bond_init_kernel<<<1, 128, 0, st>>>(bond_dims, n);
  if (discarded && cudaMemsetAsync(discarded, 0, size_t(m) * sizeof(float), st) != cudaSuccess) return DK_ERR_CUDA;
  const long long units = (long long)m * nb;
  const int c128 = dtype == DK_C128 ? 1 : 0;
  if (wpc >= 2) {  // a warp per unit, several units per CTA
    const size_t smem = size_t(wpc) * wbytes;
    if (cudaFuncSetAttribute(bsvd::block_svd_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
        cudaSuccess)
      return DK_ERR_CUDA;
    bsvd::block_svd_kernel<1><<<int((units + wpc - 1) / wpc), wpc * 32, smem, st>>>(
        x, m, n, b, nb, fm->reps, double(fm->angle_scale), kind, cutoff, chi / 2, chi, c128, wbytes, mps, bond_dims,
        discarded);
  } else {  // large blocks: four warps per unit, one unit per CTA
    if (cudaFuncSetAttribute(bsvd::block_svd_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(wbytes)) !=
        cudaSuccess)
      return DK_ERR_CUDA;
    bsvd::block_svd_kernel<4><<<int(units), 128, wbytes, st>>>(x, m, n, b, nb, fm->reps, double(fm->angle_scale), kind,
                                                                cutoff, chi / 2, chi, c128, wbytes, mps, bond_dims,
                                                                discarded);
  }
  dk_status s = launch_status();
  if (s != DK_OK || !log_norm) return s;
  return self_overlap_launch(mps, m, n, chi, dtype, log_norm, st);
}
