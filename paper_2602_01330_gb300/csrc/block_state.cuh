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
template <class Sync = CtaSync>
__device__ inline void build_f32(float2* psi, float2* ph, Coeffs& C, const float* xb, int bl, int reps,
                                 double angle_scale, int pairs_kind, int tid, int nt, Sync sync = Sync()) {
  const int dim = 1 << bl;
  const int hb = bl >> 1, lb = bl - hb;
  // each count sits in the 8-byte slot of the FP64 value it replaces
  auto slot = [](double* p, int i) -> uint32_t& { return *reinterpret_cast<uint32_t*>(p + i); };
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
  const float amp = exp2f(-0.5f * float(bl));
  for (int e = tid; e < dim; e += nt) {
    const int zh = e >> lb, zl = e & ((1 << lb) - 1);
    uint32_t phi = slot(C.ta, zh) + slot(C.tb, zl);
    for (int q = 0; q < hb; ++q) {
      const uint32_t v = slot(tv, zl * MAXH + q);
      phi += ((zh >> (hb - 1 - q)) & 1) ? 0u - v : v;
    }
    // phi / 2^32 turns = x half turns, x in [-1, 1)
    const float x = float(static_cast<int>(phi)) * 4.656612873077392578125e-10f;
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

}  // namespace blockstate
}  // namespace dk
