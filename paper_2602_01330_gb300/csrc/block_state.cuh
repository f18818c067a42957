// Dense statevector of one block of a block-structured feature map (§II-C, Eq. 6 restricted
// to the block's qubits), computed by the threads of a CTA or of one warp in FP64 shared
// memory.
//
// Per repetition: H on every qubit, then the diagonal layer exp(-i Phi(z)) with
//   Phi(z) = sum_q (angle_scale x_q / 2) z_q + sum_{(q,r) entangled} (pi - x_q)(pi - x_r) z_q z_r,
// z_q = +1 / -1 for bit value 0 / 1 (RZ(angle_scale x_q) and RZZ(2 (pi - x_q)(pi - x_r)) are
// diagonal and commute). Qubit 0 of the block is the most significant bit of the index.
//
// Work saved against the plain gate sequence, all in FP64:
//   * the first H layer acts on |0...0> and gives the uniform state, so the first repetition
//     is psi(z) = 2^(-b/2) exp(-i Phi(z)) directly; later ones run one Walsh-Hadamard
//     butterfly pass per qubit;
//   * the phase factors exp(-i Phi(z)) are computed once and reused by every repetition;
//   * Phi is evaluated from split tables: with z = (zH, zL) the high and low halves of the
//     bits, Phi = A(zH) + B(zL) + sum_{q in H} z_q V_q(zL), V_q(zL) = sum_{r in L} J_qr z_r,
//     a handful of additions per amplitude instead of one term per entangled pair.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "../../include/dualk.h"

namespace dk {
namespace blockstate {

constexpr int MAXB = 12;           // qubits per block
constexpr int MAXH = MAXB / 2;     // bits of each half
constexpr double PI_D = 3.14159265358979323846;

struct Coeffs {
  double hq[MAXB];               // angle_scale x_q / 2
  double jq[MAXB][MAXB];         // (pi - x_q)(pi - x_r) for entangled q < r, else 0
  double ta[1 << MAXH];          // A(zH): the terms inside the high half
  double tb[1 << MAXH];          // B(zL): the terms inside the low half
  double tv[1 << MAXH][MAXH];    // V_q(zL) for the high qubits q
};

// Shared memory a block of bl <= b qubits needs: Coeffs, then psi and the phase factors
// (FP64 for build, FP32 for build_f32).
__host__ __device__ inline size_t smem_bytes(int b) {
  return ((sizeof(Coeffs) + 15) & ~size_t(15)) + 2 * (size_t(1) << b) * sizeof(double2);
}
__host__ __device__ inline size_t smem_bytes_f32(int b) {
  return ((sizeof(Coeffs) + 15) & ~size_t(15)) + 2 * (size_t(1) << b) * sizeof(float2);
}

// Barrier of the threads that build one block together: a whole CTA or one warp.
struct CtaSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct WarpSync {
  __device__ __forceinline__ void operator()() const { __syncwarp(); }
};

__device__ __forceinline__ double2 cmul64(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// psi[0 .. 2^bl) of the block whose features are xb[0 .. bl); ph[0 .. 2^bl) receives the
// phase factors. pairs_kind: DK_ENT_CHAIN, DK_ENT_FULL, or anything else for no entanglers.
// Threads tid = 0 .. nt-1 work together and `sync` is their barrier; ends with a sync.
template <class Sync = CtaSync>
__device__ inline void build(double2* psi, double2* ph, Coeffs& C, const float* xb, int bl, int reps,
                             double angle_scale, int pairs_kind, int tid, int nt, Sync sync = Sync()) {
  const int dim = 1 << bl;
  const int hb = bl >> 1, lb = bl - hb;  // high half: qubits 0 .. hb-1
  if (tid < bl) C.hq[tid] = 0.5 * angle_scale * double(xb[tid]);
  for (int e = tid; e < MAXB * MAXB; e += nt) {
    const int q = e / MAXB, r = e % MAXB;
    const bool on = q < bl && r < bl && q < r &&
                    (pairs_kind == DK_ENT_FULL || (pairs_kind == DK_ENT_CHAIN && r == q + 1));
    C.jq[q][r] = on ? (PI_D - double(xb[q])) * (PI_D - double(xb[r])) : 0.0;
  }
  sync();
  // tables: z of qubit q (q < hb) is bit hb-1-q of zH; of qubit hb+t is bit lb-1-t of zL
  for (int e = tid; e < (1 << hb); e += nt) {
    double a = 0.0;
    for (int q = 0; q < hb; ++q) {
      const double zq = ((e >> (hb - 1 - q)) & 1) ? -1.0 : 1.0;
      double s = C.hq[q];
      for (int r = q + 1; r < hb; ++r) s += ((e >> (hb - 1 - r)) & 1) ? -C.jq[q][r] : C.jq[q][r];
      a += zq * s;
    }
    C.ta[e] = a;
  }
  for (int e = tid; e < (1 << lb); e += nt) {
    double bsum = 0.0;
    for (int t = 0; t < lb; ++t) {
      const int q = hb + t;
      const double zq = ((e >> (lb - 1 - t)) & 1) ? -1.0 : 1.0;
      double s = C.hq[q];
      for (int u = t + 1; u < lb; ++u) s += ((e >> (lb - 1 - u)) & 1) ? -C.jq[q][hb + u] : C.jq[q][hb + u];
      bsum += zq * s;
    }
    C.tb[e] = bsum;
    for (int q = 0; q < hb; ++q) {
      double v = 0.0;
      for (int t = 0; t < lb; ++t) v += ((e >> (lb - 1 - t)) & 1) ? -C.jq[q][hb + t] : C.jq[q][hb + t];
      C.tv[e][q] = v;
    }
  }
  sync();
  const double amp = exp2(-0.5 * double(bl));
  for (int e = tid; e < dim; e += nt) {
    const int zh = e >> lb, zl = e & ((1 << lb) - 1);
    double phi = C.ta[zh] + C.tb[zl];
    for (int q = 0; q < hb; ++q) phi += ((zh >> (hb - 1 - q)) & 1) ? -C.tv[zl][q] : C.tv[zl][q];
    double sn, cs;
    sincos(-phi, &sn, &cs);
    ph[e] = make_double2(cs, sn);
    psi[e] = make_double2(amp * cs, amp * sn);  // first repetition: uniform state times the phases
  }
  sync();
  for (int rep = 1; rep < reps; ++rep) {
    for (int q = 0; q < bl; ++q) {
      const int bit = 1 << (bl - 1 - q);
      for (int e = tid; e < dim / 2; e += nt) {
        const int lo = ((e & ~(bit - 1)) << 1) | (e & (bit - 1));
        const int hi = lo | bit;
        const double2 u = psi[lo], v = psi[hi];
        psi[lo] = make_double2((u.x + v.x) * M_SQRT1_2, (u.y + v.y) * M_SQRT1_2);
        psi[hi] = make_double2((u.x - v.x) * M_SQRT1_2, (u.y - v.y) * M_SQRT1_2);
      }
      sync();
    }
    for (int e = tid; e < dim; e += nt) psi[e] = cmul64(psi[e], ph[e]);
    sync();
  }
}

// An angle in FP64 as an unsigned 32-bit count of 2^-32 turns (angle / 2 pi modulo 1): sums
// of such counts with wraparound are sums of angles modulo 2 pi, exact but for the rounding
// of each term (2^-33 turns, 7e-10 rad).
__device__ __forceinline__ uint32_t turns32(double angle) {
  const double t = angle * (1.0 / 6.283185307179586476925);
  return static_cast<uint32_t>(static_cast<long long>(rint((t - floor(t)) * 4294967296.0)));
}

// The same state in FP32 for operands that are rounded to split BF16 afterwards (about 17
// significant bits). GB300's FP64 rate is a small fraction of its FP32 rate, so only the
// b + b(b-1)/2 angles of the block (angle_scale x_q / 2 and (pi - x_q)(pi - x_r)) are formed in
// FP64; each becomes a 32-bit turn count (turns32), the tables are integer sums of counts and
// an amplitude's phase is hb + 2 integer additions, all modulo 2 pi by wraparound (error
// under 1e-8 rad); the count, read as a signed fraction of a half turn, goes to sincospif
// (angle error ~2e-7 rad from its rounding to FP32, the class of an FP64 phase rounded to
// FP32); the butterflies and the phase multiplications run in FP32 (relative error ~1e-7 per
// amplitude, far below the split's 2^-18 ~ 4e-6).
// each turn count sits in the 8-byte slot of the FP64 value it replaces
__device__ __forceinline__ uint32_t& slot32(double* p, int i) { return *reinterpret_cast<uint32_t*>(p + i); }

// The turn-count tables of build_f32 (ends with a barrier).
template <class Sync>
__device__ inline void tables_f32(Coeffs& C, const float* xb, int bl, double angle_scale, int pairs_kind, int tid,
                                  int nt, Sync sync) {
  const int hb = bl >> 1, lb = bl - hb;
  auto slot = [](double* p, int i) -> uint32_t& { return slot32(p, i); };
  double* hq = C.hq;
  double* jq = &C.jq[0][0];
  double* tv = &C.tv[0][0];
  if (tid < bl) slot(hq, tid) = turns32(0.5 * angle_scale * double(xb[tid]));
  for (int e = tid; e < MAXB * MAXB; e += nt) {
    const int q = e / MAXB, r = e % MAXB;
    const bool on = q < bl && r < bl && q < r &&
                    (pairs_kind == DK_ENT_FULL || (pairs_kind == DK_ENT_CHAIN && r == q + 1));
    slot(jq, e) = on ? turns32((PI_D - double(xb[q])) * (PI_D - double(xb[r]))) : 0u;
  }
  sync();
  // tables: z of qubit q (q < hb) is bit hb-1-q of zH; of qubit hb+t is bit lb-1-t of zL
  for (int e = tid; e < (1 << hb); e += nt) {
    uint32_t a = 0u;
    for (int q = 0; q < hb; ++q) {
      uint32_t s = slot(hq, q);
      for (int r = q + 1; r < hb; ++r) {
        const uint32_t j = slot(jq, q * MAXB + r);
        s += ((e >> (hb - 1 - r)) & 1) ? 0u - j : j;
      }
      a += ((e >> (hb - 1 - q)) & 1) ? 0u - s : s;
    }
    slot(C.ta, e) = a;
  }
  for (int e = tid; e < (1 << lb); e += nt) {
    uint32_t bsum = 0u;
    for (int t = 0; t < lb; ++t) {
      const int q = hb + t;
      uint32_t s = slot(hq, q);
      for (int u = t + 1; u < lb; ++u) {
        const uint32_t j = slot(jq, q * MAXB + hb + u);
        s += ((e >> (lb - 1 - u)) & 1) ? 0u - j : j;
      }
      bsum += ((e >> (lb - 1 - t)) & 1) ? 0u - s : s;
    }
    slot(C.tb, e) = bsum;
    for (int q = 0; q < hb; ++q) {
      uint32_t v = 0u;
      for (int t = 0; t < lb; ++t) {
        const uint32_t j = slot(jq, q * MAXB + hb + t);
        v += ((e >> (lb - 1 - t)) & 1) ? 0u - j : j;
      }
      slot(tv, e * MAXH + q) = v;
    }
  }
  sync();
}

// Phase of amplitude e from the tables, as x half turns (x in [-1, 1)): hb + 2 integer
// additions of turn counts.
__device__ __forceinline__ float phase_x(Coeffs& C, int e, int bl) {
  const int hb = bl >> 1, lb = bl - hb;
  const int zh = e >> lb, zl = e & ((1 << lb) - 1);
  uint32_t phi = slot32(C.ta, zh) + slot32(C.tb, zl);
  for (int q = 0; q < hb; ++q) {
    const uint32_t v = slot32(&C.tv[0][0], zl * MAXH + q);
    phi += ((zh >> (hb - 1 - q)) & 1) ? 0u - v : v;
  }
  return float(static_cast<int>(phi)) * 4.656612873077392578125e-10f;
}

template <class Sync = CtaSync>
__device__ inline void build_f32(float2* psi, float2* ph, Coeffs& C, const float* xb, int bl, int reps,
                                 double angle_scale, int pairs_kind, int tid, int nt, Sync sync = Sync()) {
  const int dim = 1 << bl;
  tables_f32(C, xb, bl, angle_scale, pairs_kind, tid, nt, sync);
  const float amp = exp2f(-0.5f * float(bl));
  for (int e = tid; e < dim; e += nt) {
    const float x = phase_x(C, e, bl);
    float sn, cs;
    sincospif(-x, &sn, &cs);
    ph[e] = make_float2(cs, sn);
    psi[e] = make_float2(amp * cs, amp * sn);
  }
  sync();
  constexpr float R2 = 0.70710678118654752440f;
  for (int rep = 1; rep < reps; ++rep) {
    for (int q = 0; q < bl; ++q) {
      const int bit = 1 << (bl - 1 - q);
      for (int e = tid; e < dim / 2; e += nt) {
        const int lo = ((e & ~(bit - 1)) << 1) | (e & (bit - 1));
        const int hi = lo | bit;
        const float2 u = psi[lo], v = psi[hi];
        psi[lo] = make_float2((u.x + v.x) * R2, (u.y + v.y) * R2);
        psi[hi] = make_float2((u.x - v.x) * R2, (u.y - v.y) * R2);
      }
      sync();
    }
    for (int e = tid; e < dim; e += nt) {
      const float2 a = psi[e], w = ph[e];
      psi[e] = make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
    }
    sync();
  }
}

// build_f32 for blocks of bl = 7 + log2(R) qubits by a CTA of 128 threads, the amplitudes in
// registers: thread t holds e = 128 j + t (j < R). A Walsh-Hadamard pass takes bits 0-4 of
// the index by warp shuffles, bits 7 and up inside the thread, and bits 5-6 together as one
// radix-4 pass through shared memory: three shared-memory accesses per amplitude per
// repetition instead of 2 bl. Same state as build_f32 up to rounding; psi receives it.
template <int R>
__device__ inline void build_f32_regs(float2* psi, float2* ph, Coeffs& C, const float* xb, int reps, double angle_scale,
                                      int pairs_kind, int tid) {
  constexpr int NT = 128, DIM = R * NT;
  constexpr int BL = 7 + (R >= 2) + (R >= 4) + (R >= 8) + (R >= 16) + (R >= 32);
  static_assert((1 << BL) == DIM, "R is a power of two up to 32");
  tables_f32(C, xb, BL, angle_scale, pairs_kind, tid, NT, CtaSync());
  const int lane = tid & 31;
  const float amp = exp2f(-0.5f * float(BL));
  float2 v[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int e = j * NT + tid;
    float sn, cs;
    sincospif(-phase_x(C, e, BL), &sn, &cs);
    ph[e] = make_float2(cs, sn);
    v[j] = make_float2(amp * cs, amp * sn);
  }
  constexpr float R2 = 0.70710678118654752440f;
  for (int rep = 1; rep < reps; ++rep) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const bool upper = (lane >> k) & 1;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const float px = __shfl_xor_sync(0xffffffffu, v[j].x, 1 << k);
        const float py = __shfl_xor_sync(0xffffffffu, v[j].y, 1 << k);
        v[j] = upper ? make_float2((px - v[j].x) * R2, (py - v[j].y) * R2)
                     : make_float2((v[j].x + px) * R2, (v[j].y + py) * R2);
      }
    }
#pragma unroll
    for (int s = 1; s < R; s <<= 1)
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (!(j & s)) {
          const float2 a = v[j], b = v[j | s];
          v[j] = make_float2((a.x + b.x) * R2, (a.y + b.y) * R2);
          v[j | s] = make_float2((a.x - b.x) * R2, (a.y - b.y) * R2);
        }
#pragma unroll
    for (int j = 0; j < R; ++j) psi[j * NT + tid] = v[j];
    __syncthreads();
    for (int g = tid; g < DIM / 4; g += NT) {
      const int base = ((g >> 5) << 7) | (g & 31);  // bits 5 and 6 clear
      const float2 a0 = psi[base], a1 = psi[base | 32], a2 = psi[base | 64], a3 = psi[base | 96];
      const float2 b0 = make_float2(a0.x + a1.x, a0.y + a1.y), b1 = make_float2(a0.x - a1.x, a0.y - a1.y);
      const float2 b2 = make_float2(a2.x + a3.x, a2.y + a3.y), b3 = make_float2(a2.x - a3.x, a2.y - a3.y);
      psi[base] = make_float2((b0.x + b2.x) * 0.5f, (b0.y + b2.y) * 0.5f);
      psi[base | 32] = make_float2((b1.x + b3.x) * 0.5f, (b1.y + b3.y) * 0.5f);
      psi[base | 64] = make_float2((b0.x - b2.x) * 0.5f, (b0.y - b2.y) * 0.5f);
      psi[base | 96] = make_float2((b1.x - b3.x) * 0.5f, (b1.y - b3.y) * 0.5f);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int e = j * NT + tid;
      const float2 a = psi[e], w = ph[e];
      v[j] = make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
    }
    __syncthreads();  // psi is written again below or in the next repetition
  }
#pragma unroll
  for (int j = 0; j < R; ++j) psi[j * NT + tid] = v[j];
  __syncthreads();
}

}  // namespace blockstate
}  // namespace dk
