// Left-to-right transfer contraction of one pair (§II-C, Eqs. 8-10), block-structured.
//
// For a pair (x_i, x_j) the amplitude a = <psi(x_i)|psi(x_j)> of two MPS is
//     E_0 = [1],   E_k = sum_{s in {0,1}} A_s^(k)(x_i)^dagger E_{k-1} A_s^(k)(x_j),   a = E_n,
// with E a chi x chi complex matrix (rows: bond of the conjugated row sample i, columns:
// bond of the column sample j).
//
// Block structure. In the ZZ-chain MPS every bond carries a copy of the computational
// value of the qubit to its left (the RZZ layers are diagonal), so with the bond index
// ordered as l = t * h + j (t = that copied bit, h = chi / 2) a site tensor A_s has
// non-zero columns only in block s, and consequently E_k is block diagonal,
// E = diag(E_0, E_1) with h x h blocks. Writing A_s[t] for the h x h sub-block of A_s
// with rows in block t and its block-s columns, one site is
//     E'_s = sum_{t in {0,1}} A_s[t](x_i)^dagger  E_t  A_s[t](x_j),     s = 0, 1,
// i.e. 8 h^3 complex multiply-adds instead of the 4 chi^3 = 32 h^3 of the dense form;
// the zeros skipped are exact zeros of the construction. At the last site the right bond
// is 1 and both s land in the same 1 x 1 entry: a = E'_0[0][0] + E'_1[0][0].
//
// Every 4 sites (and after the last) E is scaled by an exact power of two so that
// max(|Re|, |Im|) lies in [1, 2); the exponents are summed in e2, so a = mantissa * 2^e2
// never underflows (between rescales E shrinks by at most a few per-site overlap factors).
//
// All arithmetic is explicit fma() in a fixed order: the Gram kernels and the
// self-overlap kernel run this code on the same tensors and get bit-identical diagonal
// amplitudes.
#pragma once

#include <stdint.h>

namespace dk {

constexpr int RENORM_EVERY = 4;
static_assert((RENORM_EVERY & (RENORM_EVERY - 1)) == 0, "rescale interval must be a power of two");

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

// h x h complex block, split real / imaginary.
template <typename real, int H>
struct Blk {
  real r[H][H];
  real i[H][H];
};

// Transfer state of one pair: E = diag(b[0], b[1]) and the binary exponent.
template <typename real, int H>
struct PairE {
  Blk<real, H> b[2];
  int e2;

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int a = 0; a < H; ++a)
#pragma unroll
        for (int c = 0; c < H; ++c) {
          b[t].r[a][c] = real(0);
          b[t].i[a][c] = real(0);
        }
    b[0].r[0][0] = real(1);
    e2 = 0;
  }

  __device__ __forceinline__ void renorm() {
    real mx = real(0);
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int a = 0; a < H; ++a)
#pragma unroll
        for (int c = 0; c < H; ++c) mx = fmax(mx, fmax(fabs(b[t].r[a][c]), fabs(b[t].i[a][c])));
    const int e = RealBits<real>::exponent(mx);
    const real sc = RealBits<real>::pow2_neg(e);
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int a = 0; a < H; ++a)
#pragma unroll
        for (int c = 0; c < H; ++c) {
          b[t].r[a][c] *= sc;
          b[t].i[a][c] *= sc;
        }
    e2 += e;
  }

  // ln|a| with a = b[0][0][0] + b[1][0][0] (valid after the last site), rounded to float;
  // -inf for a = 0. The Gram epilogue forms 2 * this - ln_norm_i - ln_norm_j, which is
  // exactly 0 on the diagonal because ln_norm_i is this same value from the self-overlap
  // kernel.
  __device__ __forceinline__ float half_log_mod() const {
    const real re = b[0].r[0][0] + b[1].r[0][0];
    const real im = b[0].i[0][0] + b[1].i[0][0];
    const real mod2 = fma(re, re, im * im);
    return float(fma(real(0.5), log(mod2), real(e2) * real(0.69314718055994530942)));
  }
};

// acc += conj(ai)^T * (e * aj) for one (s, t) term of one pair:
//   F[a][c]   = sum_b e[a][b] aj[b][c]
//   acc[p][c] += sum_a conj(ai[a][p]) F[a][c]
// ai / aj are h x h sub-blocks indexed [row (bond l within block t)][column j].
template <typename real, int H>
__device__ __forceinline__ void term(Blk<real, H>& acc, const Blk<real, H>& e, const Blk<real, H>& ai,
                                     const Blk<real, H>& aj) {
  // one column of F at a time: each acc entry sees the same additions in the same order as
  // with the whole F formed first, with a quarter of the temporaries live
#pragma unroll
  for (int c = 0; c < H; ++c) {
    real fr_c[H], fi_c[H];
#pragma unroll
    for (int a = 0; a < H; ++a) {
      // operand order keeps each register in two consecutive FMAs (operand reuse)
      real fr = e.r[a][0] * aj.r[0][c];
      real fi = e.r[a][0] * aj.i[0][c];
      fr = fma(-e.i[a][0], aj.i[0][c], fr);
      fi = fma(e.i[a][0], aj.r[0][c], fi);
#pragma unroll
      for (int b = 1; b < H; ++b) {
        fr = fma(e.r[a][b], aj.r[b][c], fr);
        fi = fma(e.r[a][b], aj.i[b][c], fi);
        fr = fma(-e.i[a][b], aj.i[b][c], fr);
        fi = fma(e.i[a][b], aj.r[b][c], fi);
      }
      fr_c[a] = fr;
      fi_c[a] = fi;
    }
#pragma unroll
    for (int p = 0; p < H; ++p) {
      real ar = acc.r[p][c];
      real aim = acc.i[p][c];
#pragma unroll
      for (int a = 0; a < H; ++a) {
        ar = fma(ai.r[a][p], fr_c[a], ar);
        aim = fma(ai.r[a][p], fi_c[a], aim);
        ar = fma(ai.i[a][p], fi_c[a], ar);
        aim = fma(-ai.i[a][p], fr_c[a], aim);
      }
      acc.r[p][c] = ar;
      acc.i[p][c] = aim;
    }
  }
}

// One site for a PR x PC group of pairs (rows share A(x_i), columns share A(x_j)).
// The loaders fill one sub-block: ldi(pr, s, t, blk) / ldj(pc, s, t, blk).
template <typename real, int H, int PR, int PC, class LoadI, class LoadJ>
__device__ __forceinline__ void site_step(PairE<real, H> (&st)[PR][PC], const LoadI& ldi, const LoadJ& ldj,
                                          bool renorm) {
  Blk<real, H> nw[PR][PC][2];
#pragma unroll
  for (int pr = 0; pr < PR; ++pr)
#pragma unroll
    for (int pc = 0; pc < PC; ++pc)
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < H; ++a)
#pragma unroll
          for (int c = 0; c < H; ++c) {
            nw[pr][pc][s].r[a][c] = real(0);
            nw[pr][pc][s].i[a][c] = real(0);
          }
#pragma unroll
  for (int t = 0; t < 2; ++t) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      Blk<real, H> ai[PR], aj[PC];
#pragma unroll
      for (int pr = 0; pr < PR; ++pr) ldi(pr, s, t, ai[pr]);
#pragma unroll
      for (int pc = 0; pc < PC; ++pc) ldj(pc, s, t, aj[pc]);
#pragma unroll
      for (int pr = 0; pr < PR; ++pr)
#pragma unroll
        for (int pc = 0; pc < PC; ++pc) term<real, H>(nw[pr][pc][s], st[pr][pc].b[t], ai[pr], aj[pc]);
    }
  }
#pragma unroll
  for (int pr = 0; pr < PR; ++pr)
#pragma unroll
    for (int pc = 0; pc < PC; ++pc) {
      st[pr][pc].b[0] = nw[pr][pc][0];
      st[pr][pc].b[1] = nw[pr][pc][1];
      if (renorm) st[pr][pc].renorm();
    }
}

}  // namespace dk
