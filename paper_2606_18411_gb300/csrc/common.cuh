// Shared device helpers of the MRCQR library: the per-factorization control
// block, Philox4x32-10, precision casts and small reductions.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

namespace mrcqr {

enum Prec : int { P_FP16 = 0, P_BF16 = 1, P_FP32 = 2, P_FP64 = 3, P_AUTO = 4 };
enum Status : int {
  ST_OK = 0, ST_INVALID = 1, ST_BREAKDOWN = 2, ST_NONFINITE = 3, ST_ORTHO = 4,
  ST_ALLOC = 5, ST_CUDA = 6, ST_TIMEOUT = 7
};

constexpr int kMaxLevels = 4;
constexpr int kNumFeatures = 16;

// Device-side control block of one factorization.  Every kernel of an
// escalation level L starts with `if (ctl->active != L) return;`, so the
// whole retry ladder (Sec. II-C: rerun at the next precision when the
// orthogonality check fails) is enqueued up front and needs no host sync.
struct Ctl {
  int active;          // level whose kernels run; -1 when finished
  int lvl_status;      // error raised inside the running level
  int final_status;    // mrcqr_status_t reported to the caller
  int prec_used;       // sketch precision of the accepted level
  int retries;         // escalations taken
  int prec_first;      // precision of level 0 (AUTO: the selector's choice)
  int nlevels;
  int input_nonfinite; // A holds NaN/Inf (no escalation can help)
  int lvl_prec[kMaxLevels];
  int mlp_choice;      // selector class (0 fp16, 1 fp32, 2 fp64), -1 if unused
  int pad0;
  double tol;          // acceptance threshold on ||I - Q^T Q||_F
  double ortho_fro;    // measured ||I - Q^T Q||_F of the accepted level
  float features[kNumFeatures];
};

__device__ __forceinline__ bool level_inactive(const Ctl* ctl, int level) {
  return ctl->active != level;
}

__device__ __forceinline__ void raise_level_status(Ctl* ctl, int code) {
  atomicCAS(&ctl->lvl_status, 0, code);
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
// (hi0,lo0)=M0*c0, (hi1,lo1)=M1*c2, c=(hi1^c1^k0, lo1, hi0^c3^k1, lo0),
// with the key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__host__ __device__ __forceinline__ uint2 seed_key(uint64_t seed) {
  return make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
}

// Rademacher sign of row i (Algorithm 2 step 1): +1 or -1.
__device__ __forceinline__ double row_sign(uint64_t i, uint2 key) {
  const uint4 r = philox4x32_10(make_uint4((uint32_t)i, 0u, 0u, 0u), key);
  return (r.x & 1u) ? -1.0 : 1.0;
}

// Single rounding FP64 -> precision p (fl_p of Algorithm 2 step 2), returned
// widened to float (exact).  FP64 passes through.
__device__ __forceinline__ float round_to_f16(double x) {
  unsigned short u;
  asm("cvt.rn.f16.f64 %0, %1;" : "=h"(u) : "d"(x));
  return __half2float(__ushort_as_half(u));
}
__device__ __forceinline__ float round_to_bf16(double x) {
  unsigned short u;
  asm("cvt.rn.bf16.f64 %0, %1;" : "=h"(u) : "d"(x));
  return __bfloat162float(__ushort_as_bfloat16(u));
}

template <int PREC>
__device__ __forceinline__ float round_to_p(double x) {
  if constexpr (PREC == P_FP16) return round_to_f16(x);
  else if constexpr (PREC == P_BF16) return round_to_bf16(x);
  else return (float)x;
}

// 2^e as a double for |e| <= 1022 (exact).
__device__ __forceinline__ double exp2i(int e) {
  e = max(-1022, min(1023, e));
  return __longlong_as_double((long long)(1023 + e) << 52);
}

// Exponent that brings max|x| into [2^13, 2^14): room for FP16 products
// with entries of magnitude <= 1 (the transform), zero columns get 0.
__device__ __forceinline__ int scale_exponent(double amax) {
  if (!(amax > 0.0) || !isfinite(amax)) return 0;
  int ex;
  frexp(amax, &ex);  // amax = f 2^ex, f in [0.5, 1)
  return 14 - ex;
}

// Sketch transforms (Sec. II-A).  Every entry of a transform row is
// cos(pi r / (2m)) for the integer phase r = (dk j + beta) mod 4m of column j:
//   T_DCT      DCT-II row k:             dk = 2k, beta = k  (cos(pi k (2j+1) / (2m)))
//   T_RFFT     Re of real-FFT bin k:     dk = 4k, beta = 0  (cos(2 pi k j / m))
//   T_RFFT_REIM Im rows of those bins:   dk = 4k, beta = m  (cos(2 pi k j / m + pi / 2)
//                                                           = -sin(2 pi k j / m))
// A row word holds k in bits 0..30 and, for the Im rows, kImRow.
enum Transform : int { T_DCT = 0, T_RFFT = 1, T_RFFT_REIM = 2 };
constexpr uint32_t kImRow = 0x80000000u;

struct RowPhase {
  uint64_t dk, beta;   // phase of column j: (dk j + beta) mod 4m, dk < 4m
};

__device__ __forceinline__ RowPhase row_phase(int tf, uint32_t word, uint64_t m) {
  const uint64_t k = word & ~kImRow, fm = 4ull * m;
  if (tf == T_DCT) return RowPhase{(2ull * k) % fm, k % fm};
  return RowPhase{(4ull * k) % fm, (word & kImRow) ? m : 0ull};
}

// (dk j + beta) mod 4m without overflow: dk < 4m <= 2^33, j < 2^31.
__device__ __forceinline__ uint64_t phase_at(const RowPhase& p, uint64_t j, uint64_t fm) {
  return (p.dk * j + p.beta) % fm;
}

// cos(pi r / (2m)) for an integer phase r in [0, 4m), from a table of
// cos(pi q / (2m)), q = 0..m (quarter-wave symmetry).
__device__ __forceinline__ double cos_phase(const double* __restrict__ tab, int64_t r, int64_t m) {
  if (r >= 2 * m) r = 4 * m - r;            // cos(2 pi - x) = cos x
  if (r > m) return -__ldg(tab + (2 * m - r));   // cos(pi - x) = -cos x
  return __ldg(tab + r);
}

// cos(pi r / (2m)) as FP64 bits (hi, lo) from the same table, the sign
// applied by XOR (no FP64 instruction).
__device__ __forceinline__ void cos_phase_bits(const double* __restrict__ tab, int64_t r, int64_t m, uint32_t& hi,
                                               uint32_t& lo) {
  uint32_t neg = 0u;
  if (r >= 2 * m) r = 4 * m - r;
  if (r > m) {
    r = 2 * m - r;
    neg = 0x80000000u;
  }
  const uint2 w = __ldg(reinterpret_cast<const uint2*>(tab) + r);
  lo = w.x;
  hi = w.y ^ neg;
}

// ---------------------------------------------------------------------------
// fl_p on the FP64 bit pattern with 32-bit integer operations only.  On this
// GPU every FP64 instruction (even a multiply by +-1, a compare or a
// conversion) issues to the 1/64-rate FP64 pipe, so the per-element work of
// the reduced-precision sketch avoids it: the Rademacher sign is an XOR of
// bit 63 (as the paper's DiagMult does), the 2^e scaling adds e to the
// exponent field, and rounding to FP16 / BF16 / FP32 is round-to-nearest-
// even computed from the 52-bit mantissa (one rounding, subnormal targets
// included).  x = (hi, lo) are the high and low words of the double.

// RNE of the 53-bit significand M (implicit bit set) shifted right by sh
// (1 <= sh <= 63): the subnormal-target path.
__device__ __forceinline__ uint32_t rne_shift(uint64_t M, int sh) {
  if (sh >= 64) return 0u;
  uint64_t q = M >> sh;
  const uint64_t rem = M & ((1ull << sh) - 1ull);
  const uint64_t half = 1ull << (sh - 1);
  q += (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;
  return (uint32_t)q;
}

// Target formats: mantissa bits MB, exponent bias BIAS, minimum normal
// unbiased exponent EMIN, maximum EMAX; returns the target bit pattern
// (FP16/BF16 in the low 16 bits, FP32 in 32 bits).
template <int MB, int BIAS, int EMIN, int EMAX, int SIGNSHIFT>
__device__ __forceinline__ uint32_t f64bits_to(uint32_t hi, uint32_t lo) {
  const uint32_t sign = (hi >> 31) << SIGNSHIFT;
  const int E = (int)((hi >> 20) & 0x7FFu);
  const uint32_t inf = (uint32_t)(EMAX + BIAS + 1) << MB;
  if (E == 0x7FF) return sign | inf | (((hi & 0xFFFFFu) | lo) ? (1u << (MB - 1)) : 0u);
  if (E == 0) return sign;   // FP64 zero or subnormal: below every target's range
  const int u = E - 1023;
  if (u > EMAX) return sign | inf;
  if (u >= EMIN) {
    // top MB mantissa bits: mantissa bits [51 .. 52-MB]
    uint32_t mant, rbit, sticky;
    if constexpr (MB <= 19) {
      mant = (hi >> (20 - MB)) & ((1u << MB) - 1u);
      rbit = (hi >> (19 - MB)) & 1u;
      sticky = (hi & ((1u << (19 - MB)) - 1u)) | lo;
    } else {   // FP32: 20 bits from hi, MB-20 from lo
      mant = ((hi & 0xFFFFFu) << (MB - 20)) | (lo >> (52 - MB));
      rbit = (lo >> (51 - MB)) & 1u;
      sticky = lo & ((1u << (51 - MB)) - 1u);
    }
    uint32_t q = ((uint32_t)(u + BIAS) << MB) | mant;
    q += rbit & ((sticky != 0u) | (q & 1u));   // carries into the exponent correctly
    return sign | q;
  }
  // subnormal target: units of 2^(EMIN - MB)
  const uint64_t M = (((uint64_t)(hi & 0xFFFFFu) << 32) | lo) | (1ull << 52);
  return sign | rne_shift(M, 52 - (u - (EMIN - MB)));
}

__device__ __forceinline__ uint32_t f64bits_to_f16(uint32_t hi, uint32_t lo) {
  return f64bits_to<10, 15, -14, 15, 15>(hi, lo);
}
__device__ __forceinline__ uint32_t f64bits_to_bf16(uint32_t hi, uint32_t lo) {
  return f64bits_to<7, 127, -126, 127, 15>(hi, lo);
}
__device__ __forceinline__ uint32_t f64bits_to_f32(uint32_t hi, uint32_t lo) {
  return f64bits_to<23, 127, -126, 127, 31>(hi, lo);
}

// x * 2^e on the bit pattern for finite normal x and a result that is still
// normal or underflows to a value below every target format (flushed to a
// signed zero, which the conversions above map to zero).  FP64 subnormal
// inputs take the slow FP64 path.
__device__ __forceinline__ void scale_bits(uint32_t& hi, uint32_t& lo, int e) {
  const int E = (int)((hi >> 20) & 0x7FFu);
  if (E == 0x7FF) return;
  if (E == 0) {
    if (((hi & 0xFFFFFu) | lo) == 0u) return;
    double v = __hiloint2double((int)hi, (int)lo) * exp2i(e);
    hi = (uint32_t)__double2hiint(v);
    lo = (uint32_t)__double2loint(v);
    return;
  }
  const int E2 = E + e;
  if (E2 <= 0) {
    hi &= 0x80000000u;
    lo = 0u;
    return;
  }
  hi = (hi & 0x800FFFFFu) | ((uint32_t)E2 << 20);
}

// x 2^e as FP32 bits, for x in the FP32 normal range after scaling, by
// rounding to odd (truncate, OR the sticky bit into the last place).  A
// later round-to-nearest-even to a format with at least two fewer bits
// (FP16, BF16) then equals one direct rounding of x 2^e.  Returns false when
// the scaled value leaves the FP32 normal range or x is not finite; the
// caller then takes the exact slow path.
__device__ __forceinline__ bool scaled_f32_rto(uint32_t hi, uint32_t lo, int e, uint32_t& out) {
  const int E = (int)((hi >> 20) & 0x7FFu);
  if (E == 0) {
    out = hi & 0x80000000u;
    return ((hi & 0xFFFFFu) | lo) == 0u;   // signed zero is fine, FP64 subnormal is not
  }
  const int u = E + e - 1023;
  if (E == 0x7FF || u < -126 || u > 127) return false;
  const uint32_t sticky = (lo & 0x1FFFFFFFu) != 0u ? 1u : 0u;
  out = (hi & 0x80000000u) | ((uint32_t)(u + 127) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29) | sticky;
  return true;
}

// Exponent e with max|x| 2^e in [2^13, 2^14), from the high word of max|x|
// (the exponent field orders like the value); zero or non-finite -> 0.
__device__ __forceinline__ int scale_exponent_bits(uint32_t hi_abs_max, uint32_t lo_of_max) {
  const int E = (int)(hi_abs_max >> 20);
  if (E == 0x7FF) return 0;
  if (E == 0) {
    if ((hi_abs_max | lo_of_max) == 0u) return 0;
    return scale_exponent(__hiloint2double((int)hi_abs_max, (int)lo_of_max));
  }
  return 1036 - E;   // frexp exponent ex = E - 1022, e = 14 - ex
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum (blockDim.x a multiple of 32, at most 1024); all threads get it.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* scratch /* >= 33 */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  if (wid == 0) {
    T t = lane < nw ? scratch[lane] : T(0);
    t = warp_sum(t);
    if (lane == 0) scratch[32] = t;
  }
  __syncthreads();
  return scratch[32];
}

}  // namespace mrcqr
