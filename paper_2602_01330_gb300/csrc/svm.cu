// One-against-one SVM on precomputed kernel values: the consumer of the Gram and of the
// dual-kernel rows (§II-B: dual problem Eqs. 1-2, decision function Eqs. 4-5, one-against-
// one voting; §II-D: the mixed kernel K = w K_q + (1 - w) K_c of Eq. 11 and the 5-fold
// cross-validation over C and w).
//
// Training: one CTA per (job, class pair). A job is one training set (a list of sample
// indices into the kernel matrix) with its C and w, so a whole cross-validation grid (folds x
// C x w) is one launch. The CTA compacts the pair's samples (in list order), then runs
// sequential minimal optimisation with the second-order working-set rule of Fan, Chen and
// Lin (JMLR 6, 2005): per step a block-wide argmax picks i, the kernel row of i is gathered
// from the Gram in global memory (L2-resident), a block-wide argmin of the guaranteed
// decrease picks j, one thread solves the two-variable problem, and the gradient is updated
// with rows i and j. Multipliers and gradient are FP64 in shared memory, the working-set
// choice compares FP32 copies (the kernel values are the FP32 Gram outputs); nothing else is
// written until the end, so no global scratch is used. The loop ends when the largest KKT
// violation is below tol, or after max_iter steps.
//
// Prediction: one CTA per (job, row): the row's kernel values against the job's training
// samples are staged in shared memory, each class pair's decision value is one warp-wide dot
// product with its coefficients, and the votes pick the class.
#include <math.h>
#include <stdint.h>

#include "common.cuh"
#include "internal.h"

namespace dk {
namespace svm {

constexpr int NT = 256;        // threads per CTA
constexpr int NW = NT / 32;
constexpr int MAX_CLASS = 32;

__host__ __device__ inline void pair_of(int p, int n_class, int& c1, int& c2) {
  int c = 0, base = 0;
  while (p >= base + (n_class - 1 - c)) {
    base += n_class - 1 - c;
    ++c;
  }
  c1 = c;
  c2 = c + 1 + (p - base);
}

// kernel value K(r, c) of the mixed matrix
__device__ __forceinline__ float kval(const float* kq, const float* kc, long long ld, float w, int r, int c) {
  const long long o = (long long)r * ld + c;
  float v = 0.0f;
  if (kq) v = w * __ldg(kq + o);
  if (kc) v = fmaf(1.0f - w, __ldg(kc + o), v);
  return v;
}

struct ArgBest {
  double v;
  int i;
};

// block-wide max (want_max) or min of (v, i); ties go to the smaller index; i = -1 for none
__device__ ArgBest block_arg(ArgBest a, bool want_max, ArgBest* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  auto better = [&](const ArgBest& x, const ArgBest& y) {  // is x preferable to y
    if (x.i < 0) return false;
    if (y.i < 0) return true;
    if (x.v != y.v) return want_max ? x.v > y.v : x.v < y.v;
    return x.i < y.i;
  };
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ArgBest b{__shfl_xor_sync(0xffffffffu, a.v, o), __shfl_xor_sync(0xffffffffu, a.i, o)};
    if (better(b, a)) a = b;
  }
  __syncthreads();
  if (lane == 0) red[warp] = a;
  __syncthreads();
  ArgBest r = red[0];
  for (int w2 = 1; w2 < NW; ++w2)
    if (better(red[w2], r)) r = red[w2];
  return r;
}

__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w2 = 0; w2 < NW; ++w2) s += red[w2];
  return s;
}

struct TrainArgs {
  const float* kq;
  const float* kc;
  long long ld;
  int n;           // samples of the kernel matrix (valid indices 0..n-1)
  unsigned* status;
  const float* w;
  const float* C;
  const int32_t* idx;
  const int32_t* count;
  int m_max;
  const int32_t* labels;
  int n_class;
  int n_pairs;
  double tol;
  int max_iter;
  float* coef;
  float* bias;
  int32_t* iters;
};

struct ArgF {
  float v;
  int i;
};

__device__ __forceinline__ bool better_f(const ArgF& x, const ArgF& y, bool want_max) {
  if (x.i < 0) return false;
  if (y.i < 0) return true;
  if (x.v != y.v) return want_max ? x.v > y.v : x.v < y.v;
  return x.i < y.i;
}

__device__ __forceinline__ void warp_arg_f(ArgF& x, bool want_max) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ArgF b{__shfl_xor_sync(0xffffffffu, x.v, o), __shfl_xor_sync(0xffffffffu, x.i, o)};
    if (better_f(b, x, want_max)) x = b;
  }
}

// block-wide (argmax of x, argmin of y) in one pass; ties to the smaller index, i = -1 if empty
__device__ void block_argmax_argmin(ArgF& x, ArgF& y, ArgF* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  warp_arg_f(x, true);
  warp_arg_f(y, false);
  __syncthreads();
  if (lane == 0) {
    red[warp] = x;
    red[NW + warp] = y;
  }
  __syncthreads();
  x = red[0];
  y = red[NW];
  for (int w2 = 1; w2 < NW; ++w2) {
    if (better_f(red[w2], x, true)) x = red[w2];
    if (better_f(red[NW + w2], y, false)) y = red[NW + w2];
  }
}

__device__ ArgF block_argmin(ArgF x, ArgF* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  warp_arg_f(x, false);
  __syncthreads();
  if (lane == 0) red[warp] = x;
  __syncthreads();
  ArgF r = red[0];
  for (int w2 = 1; w2 < NW; ++w2)
    if (better_f(red[w2], r, false)) r = red[w2];
  return r;
}

constexpr unsigned char IN_UP = 1, IN_LOW = 2;

// membership of one multiplier in the upper / lower index sets
__device__ __forceinline__ unsigned char set_flags(double alpha, double C, int y) {
  unsigned char f = 0;
  if ((y > 0 && alpha < C) || (y < 0 && alpha > 0.0)) f |= IN_UP;
  if ((y > 0 && alpha > 0.0) || (y < 0 && alpha < C)) f |= IN_LOW;
  return f;
}

// Shared memory (dynamic), per sample of the pair: alpha, grad (FP64), v = -y grad (FP32
// copy for the working-set choice), kd, krow_i, krow_j (FP32 kernel values), gi (kernel
// index), pos (position in the job's list), y (int8) and the set flags (uint8).
// Arithmetic: the gradient and the multipliers are FP64; the choice of the working pair
// compares FP32 copies (FP64 issues at a small fraction of the FP32 rate on GB300, and the
// choice is a heuristic: any violating pair makes progress); the stopping test re-reads the
// two chosen gradients in FP64.
__global__ void __launch_bounds__(NT) ovo_train_kernel(const TrainArgs a) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int p = blockIdx.x, job = blockIdx.y;
  const int mm = a.m_max;
  double* alpha = reinterpret_cast<double*>(sm_raw);
  double* grad = alpha + mm;
  float* vf = reinterpret_cast<float*>(grad + mm);
  float* kd = vf + mm;
  float* ki = kd + mm;
  float* kj = ki + mm;
  int* gi = reinterpret_cast<int*>(kj + mm);
  int* pos = gi + mm;
  signed char* ys = reinterpret_cast<signed char*>(pos + mm);
  unsigned char* fl = reinterpret_cast<unsigned char*>(ys + mm);
  __shared__ ArgF red_f[2 * NW];
  __shared__ ArgBest red_a[NW];
  __shared__ double red_d[NW];
  __shared__ int s_np, s_n1, s_warp_base[NW + 1];
  __shared__ double s_ci, s_cj;

  int c1, c2;
  pair_of(p, a.n_class, c1, c2);
  const int cnt = min(max(a.count[job], 0), mm);
  const int32_t* idx = a.idx + (long long)job * mm;
  const float w = a.w[job];
  const double C = double(a.C[job]);
  float* coef = a.coef + ((long long)job * a.n_pairs + p) * mm;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // 1. the pair's samples, in list order (warp ballots + a block prefix per chunk of NT)
  if (tid == 0) {
    s_np = 0;
    s_n1 = 0;
  }
  __syncthreads();
  for (int k0 = 0; k0 < cnt; k0 += NT) {
    const int k = k0 + tid;
    int lab = -1, g = 0;
    if (k < cnt) {
      g = idx[k];
      if (g >= 0 && g < a.n) lab = a.labels[g];
      else record_status(a.status, DEV_BAD_INDEX);  // skipped
    }
    const bool in = lab == c1 || lab == c2;
    const unsigned bal = __ballot_sync(0xffffffffu, in);
    if (lane == 0) s_warp_base[warp + 1] = __popc(bal);
    __syncthreads();
    if (tid == 0) {
      s_warp_base[0] = s_np;
      for (int w2 = 1; w2 <= NW; ++w2) s_warp_base[w2] += s_warp_base[w2 - 1];
    }
    __syncthreads();
    if (in) {
      const int dst = s_warp_base[warp] + __popc(bal & ((1u << lane) - 1u));
      gi[dst] = g;
      pos[dst] = k;
      ys[dst] = lab == c1 ? 1 : -1;
      if (lab == c1) atomicAdd(&s_n1, 1);
    }
    __syncthreads();
    if (tid == 0) s_np = s_warp_base[NW];
    __syncthreads();
  }
  const int np = s_np;
  const int n1 = s_n1;
  // positions of the job's list outside the pair (and past count) get coefficient 0
  for (int k = tid; k < mm; k += NT) coef[k] = 0.0f;
  if (np == 0 || n1 == 0 || n1 == np) {  // a class of the pair is absent from this job
    if (tid == 0) {
      a.bias[(long long)job * a.n_pairs + p] = 0.0f;
      if (a.iters) a.iters[(long long)job * a.n_pairs + p] = 0;
    }
    return;
  }
  for (int t = tid; t < np; t += NT) {
    alpha[t] = 0.0;
    grad[t] = -1.0;
    vf[t] = float(ys[t]);  // -y (-1)
    fl[t] = set_flags(0.0, C, ys[t]);
    kd[t] = kval(a.kq, a.kc, a.ld, w, gi[t], gi[t]);
  }
  __syncthreads();

  // 2. SMO with second-order working-set selection
  int it = 0;
  bool converged = false;
  for (; it < a.max_iter; ++it) {
    ArgF up{0.0f, -1}, low{0.0f, -1};
    for (int t = tid; t < np; t += NT) {
      const float v = vf[t];
      const unsigned char f = fl[t];
      if ((f & IN_UP) && (up.i < 0 || v > up.v)) up = ArgF{v, t};
      if ((f & IN_LOW) && (low.i < 0 || v < low.v)) low = ArgF{v, t};
    }
    block_argmax_argmin(up, low, red_f);
    if (up.i < 0 || low.i < 0) {
      converged = true;
      break;
    }
    const int i = up.i;
    const double vmax = -double(ys[i]) * grad[i];
    if (vmax - (-double(ys[low.i]) * grad[low.i]) < a.tol) {
      converged = true;
      break;
    }
    // kernel row of i over the pair's samples
    for (int t = tid; t < np; t += NT) ki[t] = kval(a.kq, a.kc, a.ld, w, gi[i], gi[t]);
    __syncthreads();
    // j: the lower-set index with the largest guaranteed decrease (vmax - v_t)^2 / curvature
    const float vmax_f = up.v, kdi = kd[i];
    ArgF jb{0.0f, -1};
    for (int t = tid; t < np; t += NT) {
      const float v = vf[t];
      if ((fl[t] & IN_LOW) && v < vmax_f) {
        const float gap = vmax_f - v;
        float curv = kdi + kd[t] - 2.0f * ki[t];
        if (!(curv > 0.0f)) curv = 1e-12f;
        const float obj = -(gap * gap) / curv;
        if (jb.i < 0 || obj < jb.v) jb = ArgF{obj, t};
      }
    }
    const ArgF bj = block_argmin(jb, red_f);
    if (bj.i < 0) {
      converged = true;
      break;
    }
    const int j = bj.i;
    if (tid == 0) {
      // exact step t along a_i += y_i t, a_j -= y_j t (keeps sum y a), clipped to the box
      const double yi = ys[i], yj = ys[j];
      const double ai = alpha[i], aj = alpha[j];
      double eta = double(kd[i]) + double(kd[j]) - 2.0 * double(ki[j]);
      if (!(eta > 0.0)) eta = 1e-12;
      const double vj = -yj * grad[j];
      double step = (vmax - vj) / eta;
      double lo = -1e300, hi = 1e300;
      // a_i + y_i t in [0, C]
      if (yi > 0) {
        lo = fmax(lo, -ai);
        hi = fmin(hi, C - ai);
      } else {
        lo = fmax(lo, ai - C);
        hi = fmin(hi, ai);
      }
      // a_j - y_j t in [0, C]
      if (yj < 0) {
        lo = fmax(lo, -aj);
        hi = fmin(hi, C - aj);
      } else {
        lo = fmax(lo, aj - C);
        hi = fmin(hi, aj);
      }
      step = fmin(fmax(step, lo), hi);
      const double da_i = yi * step, da_j = -yj * step;
      alpha[i] = ai + da_i;
      alpha[j] = aj + da_j;
      fl[i] = set_flags(alpha[i], C, ys[i]);
      fl[j] = set_flags(alpha[j], C, ys[j]);
      s_ci = yi * da_i;
      s_cj = yj * da_j;
    }
    for (int t = tid; t < np; t += NT) kj[t] = kval(a.kq, a.kc, a.ld, w, gi[j], gi[t]);
    __syncthreads();
    const double ci = s_ci, cj = s_cj;
    for (int t = tid; t < np; t += NT) {
      const double yt = ys[t];
      const double g = grad[t] + yt * (ci * double(ki[t]) + cj * double(kj[t]));
      grad[t] = g;
      vf[t] = float(-yt * g);
    }
    __syncthreads();
  }

  // 3. bias (Eq. 5): minus the mean of y grad over the free multipliers, or minus the
  // midpoint of the feasible interval when none is free
  double sfree = 0.0, nfree = 0.0, ub = 1e300, lb = -1e300;
  for (int t = tid; t < np; t += NT) {
    const double yt = ys[t];
    const double yg = yt * grad[t];
    const double at = alpha[t];
    if (at > 0.0 && at < C) {
      sfree += yg;
      nfree += 1.0;
    } else if ((at >= C && yt < 0) || (at <= 0.0 && yt > 0)) {
      ub = fmin(ub, yg);
    } else {
      lb = fmax(lb, yg);
    }
  }
  const double tf = block_sum(sfree, red_d);
  const double tn = block_sum(nfree, red_d);
  const ArgBest bu = block_arg(ArgBest{ub, tid}, false, red_a);
  const ArgBest bb = block_arg(ArgBest{lb, tid}, true, red_a);
  // 4. outputs: a_t y_t at the sample's position in the job's list
  for (int t = tid; t < np; t += NT) coef[pos[t]] = float(alpha[t] * double(ys[t]));
  if (tid == 0) {
    double r;
    if (tn > 0.0) r = tf / tn;
    else if (bu.v < 1e299 && bb.v > -1e299) r = 0.5 * (bu.v + bb.v);
    else r = bu.v < 1e299 ? bu.v : bb.v;
    a.bias[(long long)job * a.n_pairs + p] = float(-r);
    if (a.iters) a.iters[(long long)job * a.n_pairs + p] = converged ? it : -1;
  }
}

struct PredictArgs {
  const float* kq;
  const float* kc;
  long long ld;
  int n_rows, n_cols;  // valid row / column indices of the kernel matrix
  unsigned* status;
  const float* w;
  const int32_t* rows;
  const int32_t* row_count;
  int r_max;
  const int32_t* idx;
  const int32_t* count;
  int m_max;
  const float* coef;
  const float* bias;
  int n_class;
  int n_pairs;
  float* decision;
  int32_t* pred;
};

// Shared memory (dynamic): the row's kernel values (m_max floats) and the pair decisions.
__global__ void __launch_bounds__(NT) ovo_predict_kernel(const PredictArgs a) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  float* kr = reinterpret_cast<float*>(sm_raw);
  float* dec = kr + a.m_max;
  const int r = blockIdx.x, job = blockIdx.y;
  const int rc = a.row_count ? min(a.row_count[job], a.r_max) : a.r_max;
  if (r >= rc) return;
  const int cnt = a.count ? min(max(a.count[job], 0), a.m_max) : a.m_max;
  const int row = a.rows ? a.rows[(long long)job * a.r_max + r] : r;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (row < 0 || row >= a.n_rows) {  // not classified
    if (tid == 0) record_status(a.status, DEV_BAD_INDEX);
    return;
  }
  const int32_t* idx = a.idx ? a.idx + (long long)job * a.m_max : nullptr;
  const float w = a.w[job];
  for (int k = tid; k < cnt; k += NT) {
    const int c = idx ? idx[k] : k;
    if (c >= 0 && c < a.n_cols) {
      kr[k] = kval(a.kq, a.kc, a.ld, w, row, c);
    } else {
      kr[k] = 0.0f;  // this training sample does not contribute
      record_status(a.status, DEV_BAD_INDEX);
    }
  }
  __syncthreads();
  for (int p = warp; p < a.n_pairs; p += NW) {
    const float* cf = a.coef + ((long long)job * a.n_pairs + p) * a.m_max;
    float s = 0.0f;
    for (int k = lane; k < cnt; k += 32) s = fmaf(__ldg(cf + k), kr[k], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const float f = s + a.bias[(long long)job * a.n_pairs + p];
      dec[p] = f;
      if (a.decision) a.decision[((long long)job * a.r_max + r) * a.n_pairs + p] = f;
    }
  }
  __syncthreads();
  if (tid == 0 && a.pred) {
    int votes[MAX_CLASS];
    for (int c = 0; c < a.n_class; ++c) votes[c] = 0;
    for (int p = 0; p < a.n_pairs; ++p) {
      int c1, c2;
      pair_of(p, a.n_class, c1, c2);
      ++votes[dec[p] > 0.0f ? c1 : c2];
    }
    int best = 0;
    for (int c = 1; c < a.n_class; ++c)
      if (votes[c] > votes[best]) best = c;
    a.pred[(long long)job * a.r_max + r] = best;
  }
}

size_t train_smem(int m_max) {
  return size_t(m_max) * (2 * sizeof(double) + 4 * sizeof(float) + 2 * sizeof(int) + 2) + 16;
}

}  // namespace svm
}  // namespace dk

using namespace dk;

DK_API dk_status dk_svm_ovo_train(dk_ctx* ctx, const float* kq, const float* kc, long long ld, int n, int n_jobs,
                                  const float* w, const float* C, const int32_t* idx, const int32_t* count,
                                  int m_max, const int32_t* labels, int n_class, float tol, int max_iter,
                                  float* coef, float* bias, int32_t* iters, void* stream) {
  if (!ctx || (!kq && !kc) || !w || !C || !idx || !count || !labels || !coef || !bias) return DK_ERR_ARG;
  if (n_jobs < 1 || n_jobs > 65535 || m_max < 2 || n < 1 || ld < n || !(tol > 0.0f) || max_iter < 1)
    return DK_ERR_ARG;
  if (n_class < 2 || n_class > svm::MAX_CLASS) return DK_ERR_UNSUPPORTED;
  if (m_max > DK_SVM_MAX_SAMPLES) return DK_ERR_UNSUPPORTED;
  svm::TrainArgs a{kq,  kc,     ld,      n,     ctx->status, w, C, idx, count, m_max, labels, n_class,
                   n_class * (n_class - 1) / 2, double(tol), max_iter, coef, bias, iters};
  const size_t smem = svm::train_smem(m_max);
  // the shared-memory opt-in is per device: set before every launch that needs it
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(svm::ovo_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
          cudaSuccess)
    return DK_ERR_CUDA;
  svm::ovo_train_kernel<<<dim3(a.n_pairs, n_jobs), svm::NT, smem, static_cast<cudaStream_t>(stream)>>>(a);
  return launch_status();
}

DK_API dk_status dk_svm_ovo_predict(dk_ctx* ctx, const float* kq, const float* kc, long long ld, int n_rows,
                                    int n_cols, int n_jobs, const float* w, const int32_t* rows,
                                    const int32_t* row_count, int r_max, const int32_t* idx, const int32_t* count,
                                    int m_max, const float* coef, const float* bias, int n_class, float* decision,
                                    int32_t* pred, void* stream) {
  if (!ctx || (!kq && !kc) || !w || !coef || !bias || (!decision && !pred)) return DK_ERR_ARG;
  if (n_jobs < 1 || n_jobs > 65535 || r_max < 1 || m_max < 1 || n_rows < 1 || n_cols < 1 || ld < n_cols)
    return DK_ERR_ARG;
  if ((!rows && r_max > n_rows) || (!idx && m_max > n_cols)) return DK_ERR_ARG;
  if (n_class < 2 || n_class > svm::MAX_CLASS) return DK_ERR_UNSUPPORTED;
  if (m_max > DK_SVM_MAX_SAMPLES) return DK_ERR_UNSUPPORTED;
  const int n_pairs = n_class * (n_class - 1) / 2;
  svm::PredictArgs a{kq,    kc,        ld,    n_rows, n_cols, ctx->status, w,       rows,     row_count,
                     r_max, idx,       count, m_max,  coef,   bias,        n_class, n_pairs, decision, pred};
  const size_t smem = size_t(m_max + n_pairs) * sizeof(float);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(svm::ovo_predict_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
          cudaSuccess)
    return DK_ERR_CUDA;
  svm::ovo_predict_kernel<<<dim3(r_max, n_jobs), svm::NT, smem, static_cast<cudaStream_t>(stream)>>>(a);
  return launch_status();
}
