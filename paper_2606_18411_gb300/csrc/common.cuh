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
__device__ __forceinline__ unsigned short bits_f16(double x) {
  unsigned short u;
  asm("cvt.rn.f16.f64 %0, %1;" : "=h"(u) : "d"(x));
  return u;
}
__device__ __forceinline__ unsigned short bits_bf16(double x) {
  unsigned short u;
  asm("cvt.rn.bf16.f64 %0, %1;" : "=h"(u) : "d"(x));
  return u;
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

// cos(pi r / (2m)) for an integer phase r in [0, 4m), from a table of
// cos(pi q / (2m)), q = 0..m (quarter-wave symmetry).
__device__ __forceinline__ double cos_phase(const double* __restrict__ tab, int64_t r, int64_t m) {
  if (r >= 2 * m) r = 4 * m - r;            // cos(2 pi - x) = cos x
  if (r > m) return -__ldg(tab + (2 * m - r));   // cos(pi - x) = -cos x
  return __ldg(tab + r);
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
