// FP64 products on FP16 tensor cores by exact integer slicing (the
// error-free splitting of Ozaki, Ogita, Oishi, Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012), with
// balanced (signed) base-256 digits.
//
// A value x of a row (or column) whose largest magnitude has biased FP64
// exponent Eref is rounded to the 63-bit fixed-point integer
//   I = round(|x| 2^(1085 - Eref)),   0 <= I < 2^63
// (exact for every x within 2^10 of the maximum), and I is written in eight
// signed base-256 digits
//   I = sum_{a=0..7} d_a 2^(56 - 8a),  d_0 in [0, 128], d_{a>0} in [-128, 127],
// each exact in FP16 (the sign of x is applied to every digit).  A product
// sum_k x_ik y_kj keeps the digit pairs with a + b <= 7; the pairs of one
// level L = a + b are accumulated together in FP32 by tcgen05.mma.  Per term
// a level sums at most 2^15 + 6 * 2^14 = 2^17 in magnitude, so a level
// accumulated over K <= 128 terms is an integer of magnitude <= 2^24, exact in
// FP32.  The levels are combined with 64-bit integer arithmetic into the
// 128-bit
//   T = sum_L acc_L 2^(8(7-L)) = (sum_{L<4} acc_L 2^(8(3-L))) 2^32 + sum_{L>=4} acc_L 2^(8(7-L))
// and T 2^(Erow + Ecol - 2114) is rounded once to FP64.  With R_i, C_j the
// row and column maxima (R_i >= 2^61 units of I), the rounding of I costs at
// most 2^-62 R_i per operand and the dropped pairs (a + b >= 8, at most
// 7 * 2^14 of their level units) at most 7.03 * 2^-60 R_i C_j per term, so
// one term is off by less than 2^-57 R_i C_j, 16 times below the unit
// roundoff; the sum is rounded once.  Everything outside the tensor cores is
// 32/64-bit integer work (FP64 instructions issue to a 1/64-rate pipe on this
// GPU).
#pragma once
#include <cstdint>
#include "common.cuh"

namespace mrcqr {
namespace oz {

constexpr int kSlices = 8;
constexpr int kLevels = 8;
constexpr int kScaleBias = 2114;   // T 2^(Erow + Ecol - kScaleBias) is the product

// Biased FP64 exponent field of |x| from its high word (0 for zero and
// subnormals, which slice to zero against any normal reference).
__device__ __forceinline__ uint32_t exp_field(uint32_t hi) { return (hi >> 20) & 0x7FFu; }

// The fixed-point integer I = round(|x| 2^eoff 2^(1085 - Eref)) of x (FP64
// bits hi:lo) against the reference exponent Eref (biased; >= the exponent of
// x 2^eoff), plus 128 at each of the seven low byte positions: the plain
// bytes of the result are the balanced digits (the top byte d_0, the others
// d_a + 128; the carries do the rest).  Zero and subnormal x give I = 0.  The
// power-of-two scale eoff (a diagonal scaling D of a product (X D)(D^-1 Y))
// never rounds.
__device__ __forceinline__ uint64_t biased_fixed63(uint32_t hi, uint32_t lo, int Eref, int eoff) {
  const int E = (int)exp_field(hi);
  uint64_t v = 0;
  if (E != 0) {
    const uint64_t M = ((uint64_t)(hi & 0xFFFFFu) << 32 | lo) | (1ull << 52);
    const int sh = E + eoff - Eref + 10;   // I = round(M 2^sh), sh <= 10
    if (sh >= 0) v = M << sh;
    else if (sh > -64) v = (M + (1ull << (-sh - 1))) >> (-sh);
  }
  return v + 0x0080808080808080ull;
}

// Signed digits d[0..7] of x 2^eoff (see biased_fixed63), sign of x included.
__device__ __forceinline__ void digits8(uint32_t hi, uint32_t lo, int Eref, int* d, int eoff = 0) {
  const uint64_t v = biased_fixed63(hi, lo, Eref, eoff);
  const uint32_t l = (uint32_t)v, h = (uint32_t)(v >> 32);
  d[0] = (int)(h >> 24);
  d[1] = (int)((h >> 16) & 255u) - 128;
  d[2] = (int)((h >> 8) & 255u) - 128;
  d[3] = (int)(h & 255u) - 128;
  d[4] = (int)(l >> 24) - 128;
  d[5] = (int)((l >> 16) & 255u) - 128;
  d[6] = (int)((l >> 8) & 255u) - 128;
  d[7] = (int)(l & 255u) - 128;
  if (hi >> 31) {
#pragma unroll
    for (int a = 0; a < kSlices; ++a) d[a] = -d[a];
  }
}

// The eight digits of two values as packed FP16 pairs (digit a of x0 in the
// low half of out[a], of x1 in the high half), straight from the bytes of
// their biased fixed-point words J0, J1 and their signs: FP16 bits
// 0x6580 + byte are the value 1536 + d_a (one binade, spacing 1), and one
// fused multiply-add (1536 + d) s - 1536 s = s d per pair applies the sign
// exactly.
__device__ __forceinline__ void digits8_pack(uint64_t J0, uint64_t J1, uint32_t neg0, uint32_t neg1, uint32_t* out) {
  const uint32_t l0 = (uint32_t)J0, h0 = (uint32_t)(J0 >> 32), l1 = (uint32_t)J1, h1 = (uint32_t)(J1 >> 32);
  const uint32_t sgn = (neg0 << 15) | (neg1 << 31);
  const uint32_t sb = 0x3C003C00u | sgn;   // (+-1, +-1)
  const uint32_t cb = 0xE600E600u ^ sgn;   // (-+1536, -+1536)
  const __half2 s2 = *reinterpret_cast<const __half2*>(&sb);
  const __half2 c2 = *reinterpret_cast<const __half2*>(&cb);
#pragma unroll
  for (int a = 0; a < kSlices; ++a) {
    const int k = a < 4 ? 3 - a : 7 - a;   // byte of the 32-bit word holding digit a
    const uint32_t w0 = a < 4 ? h0 : l0, w1 = a < 4 ? h1 : l1;
    uint32_t t = __byte_perm(w0, w1, (uint32_t)(k | (k << 4) | ((4 + k) << 8) | ((4 + k) << 12))) & 0x00FF00FFu;
    t += a == 0 ? 0x66006600u : 0x65806580u;
    const __half2 r = __hfma2(*reinterpret_cast<const __half2*>(&t), s2, c2);
    out[a] = *reinterpret_cast<const uint32_t*>(&r);
  }
}

// Exact float of a small signed integer (|v| < 2^22) without a conversion
// instruction: 1.5 * 2^23 + v has v in its low mantissa bits.
__device__ __forceinline__ float small_int_to_float(int v) {
  return __int_as_float(0x4B400000 + v) - 12582912.0f;
}

// Adds one level's exact FP32 accumulator (an integer, |v| <= 2^24) into the
// 64-bit halves of T.
// The shift is a multiply by 2^(8 (3 - L % 4)) fused with the 64-bit add
// (one mad.wide.s32: a sign-extended 32 x 32 -> 64-bit product plus the
// accumulator), exact for every |v| < 2^31.
__device__ __forceinline__ long long mad_wide_s32(int a, int b, long long c) {
  long long r;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(r) : "r"(a), "r"(b), "l"(c));
  return r;
}

__device__ __forceinline__ void add_level(int L, float v, long long& hi, long long& lo) {
  const int iv = __float2int_rn(v);
  if (L < 4) hi = mad_wide_s32(iv, 1 << (8 * (3 - L)), hi);
  else lo = mad_wide_s32(iv, 1 << (8 * (7 - L)), lo);
}

// Signed 128-bit integer as (high word th, low word tl): two's complement.
struct I128 {
  int64_t h;
  uint64_t l;
};

__device__ __forceinline__ I128 i128_from_parts(long long hi, long long lo) {   // hi 2^32 + lo
  I128 r;
  const uint64_t tl = (uint64_t)hi << 32;
  r.h = hi >> 32;
  r.l = tl + (uint64_t)lo;
  r.h += (lo >> 63) + (r.l < tl ? 1 : 0);
  return r;
}

__device__ __forceinline__ void i128_add(I128& a, const I128& b) {
  const uint64_t l = a.l + b.l;
  a.h += b.h + (l < a.l ? 1 : 0);
  a.l = l;
}

// T 2^scale rounded once to FP64 (round to nearest even).
__device__ __forceinline__ double i128_to_double(I128 t, int scale) {
  uint64_t tl = t.l;
  int64_t th = t.h;
  const bool neg = th < 0;
  if (neg) {
    tl = ~tl + 1ull;
    th = (int64_t)(~(uint64_t)th + (tl == 0 ? 1ull : 0ull));
  }
  const uint64_t uh = (uint64_t)th;
  if (uh == 0 && tl == 0) return neg ? -0.0 : 0.0;
  const int p = uh ? 127 - __clzll((long long)uh) : 63 - __clzll((long long)tl);   // msb position
  uint64_t m;
  int e2 = p;   // value = m 2^(p - 52) before scaling
  if (p <= 52) {
    m = tl << (52 - p);
  } else {
    const int sh = p - 52;   // 1 .. 75
    uint64_t q, rem_hi_bit, sticky;
    if (sh < 64) {
      q = (tl >> sh) | (uh << (64 - sh));
      rem_hi_bit = (tl >> (sh - 1)) & 1ull;
      sticky = tl & ((1ull << (sh - 1)) - 1ull);
    } else {
      const int s2 = sh - 64;   // 0 .. 11
      q = uh >> s2;
      if (s2 == 0) {
        rem_hi_bit = tl >> 63;
        sticky = tl & 0x7FFFFFFFFFFFFFFFull;
      } else {
        rem_hi_bit = (uh >> (s2 - 1)) & 1ull;
        sticky = (uh & ((1ull << (s2 - 1)) - 1ull)) | tl;
      }
    }
    m = q;
    if (rem_hi_bit && (sticky || (m & 1ull))) ++m;
    if (m >> 53) {
      m >>= 1;
      ++e2;
    }
  }
  const int E = e2 + scale + 1023;
  if (E <= 0 || E >= 2047) {   // outside the normal range (subnormal results are rounded twice)
    const double v = ldexp((double)(m & ((1ull << 53) - 1ull)), e2 - 52 + scale);
    return neg ? -v : v;
  }
  const uint64_t bits = ((uint64_t)(neg ? 1 : 0) << 63) | ((uint64_t)E << 52) | (m & ((1ull << 52) - 1ull));
  return __longlong_as_double((long long)bits);
}

// (hi 2^32 + lo) 2^scale rounded once to FP64.
__device__ __forceinline__ double i128_to_double(long long hi, long long lo, int scale) {
  return i128_to_double(i128_from_parts(hi, lo), scale);
}

}  // namespace oz
}  // namespace mrcqr
