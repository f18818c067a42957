// One pair's left-to-right transfer contraction (§II-C, Eqs. 8-10), held in registers.
//
// For a pair (x_i, x_j) the amplitude a = <psi(x_i)|psi(x_j)> of two MPS is
//     E_0 = [1],   E_k = sum_{s in {0,1}} A_s^(k)(x_i)^dagger E_{k-1} A_s^(k)(x_j),   a = E_n,
// with E a chi x chi complex matrix (rows: bond of the conjugated row sample i,
// columns: bond of the column sample j). After each site E is scaled by an exact
// power of two so that max(|Re|, |Im|) lies in [1, 2); the exponents are summed in
// `e2`, so a = E_n[0][0] * 2^e2 never underflows.
//
// Per site the work is F_s = E A_s(x_j) followed by E' = sum_s A_s(x_i)^dagger F_s:
// 4 chi^3 complex multiply-adds = 16 chi^3 FP FMAs, all written as explicit fma() so
// the rounding sequence is fixed: the Gram kernel and the self-overlap kernel use this
// code on the same tensors and get bit-identical diagonal amplitudes.
//
// Operand columns come through a loader: ld(s, col, re[], im[]) yields the chi complex
// entries A_s[l][col], l = 0..chi-1 (one right-bond column of the site tensor).
#pragma once

#include <stdint.h>

namespace dk {

template <typename real>
struct RealBits;

template <>
struct RealBits<float> {
  // Binary exponent of a non-negative float (denormals and zero give -127).
  __device__ static __forceinline__ int exponent(float v) { return int((__float_as_uint(v) >> 23) & 0xffu) - 127; }
  // 2^-e for e in [-127, 126].
  __device__ static __forceinline__ float pow2_neg(int e) { return __uint_as_float(uint32_t(127 - e) << 23); }
};

template <>
struct RealBits<double> {
  __device__ static __forceinline__ int exponent(double v) {
    return int((__double_as_longlong(v) >> 52) & 0x7ffll) - 1023;
  }
  __device__ static __forceinline__ double pow2_neg(int e) {
    return __longlong_as_double(static_cast<long long>(1023 - e) << 52);
  }
};

template <typename real, int CHI>
struct Chain {
  real er[CHI][CHI];
  real ei[CHI][CHI];
  int e2;

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int a = 0; a < CHI; ++a)
#pragma unroll
      for (int b = 0; b < CHI; ++b) {
        er[a][b] = real(0);
        ei[a][b] = real(0);
      }
    er[0][0] = real(1);
    e2 = 0;
  }

  template <class LoadI, class LoadJ>
  __device__ __forceinline__ void step(const LoadI& ldi, const LoadJ& ldj) {
    real nr[CHI][CHI], ni[CHI][CHI];
#pragma unroll
    for (int a = 0; a < CHI; ++a)
#pragma unroll
      for (int b = 0; b < CHI; ++b) {
        nr[a][b] = real(0);
        ni[a][b] = real(0);
      }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      real fr[CHI][CHI], fi[CHI][CHI];
      // F_s[a][bp] = sum_b E[a][b] * A^j_s[b][bp]
#pragma unroll
      for (int bp = 0; bp < CHI; ++bp) {
        real cr[CHI], ci[CHI];
        ldj(s, bp, cr, ci);
#pragma unroll
        for (int a = 0; a < CHI; ++a) {
          real accr = er[a][0] * cr[0];
          real acci = er[a][0] * ci[0];
          accr = fma(-ei[a][0], ci[0], accr);
          acci = fma(ei[a][0], cr[0], acci);
#pragma unroll
          for (int b = 1; b < CHI; ++b) {
            accr = fma(er[a][b], cr[b], accr);
            accr = fma(-ei[a][b], ci[b], accr);
            acci = fma(er[a][b], ci[b], acci);
            acci = fma(ei[a][b], cr[b], acci);
          }
          fr[a][bp] = accr;
          fi[a][bp] = acci;
        }
      }
      // E'[ap][bp] += sum_a conj(A^i_s[a][ap]) * F_s[a][bp]
#pragma unroll
      for (int ap = 0; ap < CHI; ++ap) {
        real cr[CHI], ci[CHI];
        ldi(s, ap, cr, ci);
#pragma unroll
        for (int bp = 0; bp < CHI; ++bp) {
          real accr = nr[ap][bp];
          real acci = ni[ap][bp];
#pragma unroll
          for (int a = 0; a < CHI; ++a) {
            accr = fma(cr[a], fr[a][bp], accr);
            accr = fma(ci[a], fi[a][bp], accr);
            acci = fma(cr[a], fi[a][bp], acci);
            acci = fma(-ci[a], fr[a][bp], acci);
          }
          nr[ap][bp] = accr;
          ni[ap][bp] = acci;
        }
      }
    }
    // Exact power-of-two rescale: max(|Re|, |Im|) -> [1, 2).
    real mx = real(0);
#pragma unroll
    for (int a = 0; a < CHI; ++a)
#pragma unroll
      for (int b = 0; b < CHI; ++b) mx = fmax(mx, fmax(fabs(nr[a][b]), fabs(ni[a][b])));
    const int e = RealBits<real>::exponent(mx);
    const real sc = RealBits<real>::pow2_neg(e);
#pragma unroll
    for (int a = 0; a < CHI; ++a)
#pragma unroll
      for (int b = 0; b < CHI; ++b) {
        er[a][b] = nr[a][b] * sc;
        ei[a][b] = ni[a][b] * sc;
      }
    e2 += e;
  }

  // ln|a| = 0.5 ln(|mantissa|^2) + e2 ln 2, rounded to float (-inf for a = 0). The Gram
  // epilogue forms 2 * this - ln_norm_i - ln_norm_j, which is exactly 0 on the diagonal
  // because ln_norm_i is this same value from the self-overlap kernel.
  __device__ __forceinline__ float half_log_mod() const {
    const real re = er[0][0];
    const real im = ei[0][0];
    const real mod2 = fma(re, re, im * im);
    return float(fma(real(0.5), log(mod2), real(e2) * real(0.69314718055994530942)));
  }
};

}  // namespace dk
