// Dense statevector of one block of a block-structured feature map (§II-C, Eq. 6 restricted
// to the block's qubits), computed by a whole CTA in FP64 shared memory.
//
// Per repetition: H on every qubit (one Walsh-Hadamard butterfly pass per qubit), then the
// diagonal layer exp(-i Phi(z)) with
//   Phi(z) = sum_q (angle_scale x_q / 2) z_q + sum_{(q,r) entangled} (pi - x_q)(pi - x_r) z_q z_r,
// z_q = +1 / -1 for bit value 0 / 1 (RZ(angle_scale x_q) and RZZ(2 (pi - x_q)(pi - x_r)) are
// diagonal and commute). Qubit 0 of the block is the most significant bit of the index.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "../../include/dualk.h"

namespace dk {
namespace blockstate {

constexpr int MAXB = 12;  // qubits per block
constexpr double PI_D = 3.14159265358979323846;

struct Coeffs {
  double hq[MAXB];        // angle_scale x_q / 2
  double jq[MAXB][MAXB];  // (pi - x_q)(pi - x_r) for entangled q < r, else 0
};

__device__ __forceinline__ double2 cmul64(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// psi[0 .. 2^bl) of the block whose features are xb[0 .. bl); pairs_kind DK_ENT_CHAIN,
// DK_ENT_FULL, or anything else for no entanglers. Ends with __syncthreads().
__device__ inline void build(double2* psi, Coeffs& C, const float* xb, int bl, int reps, double angle_scale,
                             int pairs_kind, int tid, int nt) {
  const int dim = 1 << bl;
  if (tid < bl) C.hq[tid] = 0.5 * angle_scale * double(xb[tid]);
  for (int e = tid; e < MAXB * MAXB; e += nt) {
    const int q = e / MAXB, r = e % MAXB;
    const bool on = q < bl && r < bl && q < r &&
                    (pairs_kind == DK_ENT_FULL || (pairs_kind == DK_ENT_CHAIN && r == q + 1));
    C.jq[q][r] = on ? (PI_D - double(xb[q])) * (PI_D - double(xb[r])) : 0.0;
  }
  for (int e = tid; e < dim; e += nt) psi[e] = make_double2(e == 0 ? 1.0 : 0.0, 0.0);
  __syncthreads();
  for (int rep = 0; rep < reps; ++rep) {
    for (int q = 0; q < bl; ++q) {
      const int bit = 1 << (bl - 1 - q);
      for (int e = tid; e < dim / 2; e += nt) {
        const int lo = ((e & ~(bit - 1)) << 1) | (e & (bit - 1));
        const int hi = lo | bit;
        const double2 u = psi[lo], v = psi[hi];
        psi[lo] = make_double2((u.x + v.x) * M_SQRT1_2, (u.y + v.y) * M_SQRT1_2);
        psi[hi] = make_double2((u.x - v.x) * M_SQRT1_2, (u.y - v.y) * M_SQRT1_2);
      }
      __syncthreads();
    }
    for (int e = tid; e < dim; e += nt) {
      double phi = 0.0;
      for (int q = 0; q < bl; ++q) {
        const double zq = ((e >> (bl - 1 - q)) & 1) ? -1.0 : 1.0;
        double pair = 0.0;
        for (int r = q + 1; r < bl; ++r) pair += ((e >> (bl - 1 - r)) & 1) ? -C.jq[q][r] : C.jq[q][r];
        phi += zq * (C.hq[q] + pair);
      }
      double sn, cs;
      sincos(-phi, &sn, &cs);
      psi[e] = cmul64(psi[e], make_double2(cs, sn));
    }
    __syncthreads();
  }
}

}  // namespace blockstate
}  // namespace dk
