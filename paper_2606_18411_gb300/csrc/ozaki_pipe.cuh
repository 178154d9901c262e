// The two-stage emulated-FP64 product pipeline shared by the kernels of
// ozaki.cu and ozaki_planes.cu: one CTA per SM, 512 threads, all 512 TMEM
// columns = 8 level accumulators of 128 x 64; digit panels of a K chunk (32
// deep, K-major SWIZZLE_64B) in shared memory, the 8 digits of the A operand
// against the N-stacked digits of the B operand in 12 MMAs per K step, and
// the exact level sums read out of TMEM into 64-bit integers every 4 chunks.
#pragma once
#include "kernels.h"
#include "ozaki.cuh"
#include "tc.cuh"

namespace mrcqr {
namespace {

constexpr int kOzThreads = 512;
constexpr int kM = 128;                     // MMA M: rows of the A operand
constexpr int kN = 64;                      // MMA N: rows of the B operand, TMEM columns per level
constexpr int kK = 32;                      // K depth of a chunk (one 64-byte FP16 row)
constexpr int kGroupChunks = 4;             // chunks per exact FP32 accumulation (K <= 128)
constexpr uint32_t kAPanel = kM * 64;       // one digit of a 128 x 32 FP16 block (8 KiB)
constexpr uint32_t kBPanel = kN * 64;       // one digit of a 64 x 32 FP16 block (4 KiB)
constexpr uint32_t kStage = oz::kSlices * (kAPanel + kBPanel);   // 96 KiB
constexpr size_t kSmem = 2 * (size_t)kStage + 1024;
constexpr size_t kPartElems = 2 * kM * kN;  // hi and lo of one 128 x 64 item

// The digit-pair products of one chunk (two K steps of 16).  Level L
// accumulates in TMEM columns [64 L, 64 L + 64).  The eight digit panels of B
// are contiguous, so digits 0 .. 7 - a stacked along N form one operand, and
// a single MMA of A digit a against it (N = 64 (8 - a), split at N = 256)
// written at TMEM column 64 a adds A_a B_b to level a + b for every b at once:
// 12 MMAs per K step instead of one per pair (36), with no discarded pairs.
// Issued by one thread; the first MMA (a = 0) of a group overwrites all eight
// levels.  ab / bb: shared addresses of digit 0 of the A and B panels.
__device__ __forceinline__ void oz_issue_chunk(uint32_t tmem, uint32_t ab, uint32_t bb, bool group_start) {
  const uint64_t da = tc::sw64_desc(ab), db = tc::sw64_desc(bb);
#pragma unroll
  for (int kk = 0; kk < kK; kk += 16) {
#pragma unroll
    for (int a = 0; a < oz::kLevels; ++a) {
      const uint64_t adesc = da + (uint64_t)((a * kAPanel + kk * 2) >> 4);
      const int ntot = kN * (oz::kLevels - a);
#pragma unroll
      for (int p0 = 0; p0 < ntot; p0 += 256) {
        const int nn = ntot - p0 < 256 ? ntot - p0 : 256;
        tc::mma_f16(tmem + (uint32_t)(kN * a + p0), adesc, db + (uint64_t)((p0 * 64 + kk * 2) >> 4),
                    tc::idesc(tc::F16, kM, nn), (kk == 0 && a == 0 && group_start) ? 0u : 1u);
      }
    }
  }
}

// Adds the exact level sums of TMEM lane 32 q + lane, columns 16 g .. 16 g + 15
// (warp w: q = w % 4, g = w / 4) into the 64-bit halves hi / lo.
__device__ __forceinline__ void oz_readout(uint32_t tmem, int q, int g, long long* hi, long long* lo) {
  const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(g * 16);
#pragma unroll 1
  for (int L = 0; L < oz::kLevels; ++L) {
    float v[16];
    tc::tmem_ld16(base + (uint32_t)(L * kN), v);
    tc::tmem_wait_ld();
#pragma unroll
    for (int c = 0; c < 16; ++c) oz::add_level(L, v[c], hi[c], lo[c]);
  }
}

// Digits of two values (FP64 bits, sign flips f0 / f1 applied, scaled by
// 2^eo0 / 2^eo1) against the reference exponent E, packed in pairs into the
// eight digit panels at dst.
__device__ __forceinline__ void oz_store_pair(double v0, double v1, uint32_t f0, uint32_t f1, int E,
                                              unsigned char* dst, uint32_t pstride, int eo0 = 0, int eo1 = 0,
                                              unsigned char* dst2 = nullptr, uint32_t pstride2 = 0) {
  const uint32_t h0 = (uint32_t)__double2hiint(v0), h1 = (uint32_t)__double2hiint(v1);
  const uint64_t J0 = oz::biased_fixed63(h0, (uint32_t)__double2loint(v0), E, eo0);
  const uint64_t J1 = oz::biased_fixed63(h1, (uint32_t)__double2loint(v1), E, eo1);
  uint32_t w[oz::kSlices];
  oz::digits8_pack(J0, J1, (h0 >> 31) ^ f0, (h1 >> 31) ^ f1, w);
#pragma unroll
  for (int a = 0; a < oz::kSlices; ++a) *reinterpret_cast<uint32_t*>(dst + a * pstride) = w[a];
  if (dst2) {
#pragma unroll
    for (int a = 0; a < oz::kSlices; ++a) *reinterpret_cast<uint32_t*>(dst2 + a * pstride2) = w[a];
  }
}

// A 32-row chunk of NC columns of a column-major matrix (column col0 + c,
// zero beyond n or r_end) in registers: lane l holds rows 2(l % 16) and
// 2(l % 16) + 1 of columns 32 it + 2 warp + l / 16.  Issued one chunk ahead
// of its use, so the loads are in flight during the MMAs.
template <int NC>
__device__ __forceinline__ void oz_load_cols(const double* __restrict__ X, int64_t ldx, int n, int col0, int64_t r0,
                                             int64_t r_end, int warp, int lane, double (&v)[NC / 32][2]) {
  const int p = lane & 15, h = lane >> 4;
  const int64_t ra = r0 + 2 * p;
#pragma unroll
  for (int it = 0; it < NC / 32; ++it) {
    const int col = col0 + 32 * it + 2 * warp + h;
    v[it][0] = v[it][1] = 0.0;
    if (col < n) {
      const double* src = X + (int64_t)col * ldx;
      if (ra < r_end) v[it][0] = __ldg(src + ra);
      if (ra + 1 < r_end) v[it][1] = __ldg(src + ra + 1);
    }
  }
}

// Digits of the values loaded by oz_load_cols (reference exponent E[c], sign
// flips f0 / f1 of the lane's two rows) into panel rows c.  With dup >= 0 the
// rows c in [dup, dup + kN) are also written to rows c - dup of the B panels
// at bpanel (a diagonal Gram tile, whose B operand is part of its A operand).
template <int NC>
__device__ __forceinline__ void oz_store_cols(const double (&v)[NC / 32][2], const uint32_t* E, uint32_t f0,
                                              uint32_t f1, unsigned char* panel, uint32_t pstride, int warp,
                                              int lane, int dup = -1, unsigned char* bpanel = nullptr) {
  const int p = lane & 15, h = lane >> 4;
#pragma unroll
  for (int it = 0; it < NC / 32; ++it) {
    const int c = 32 * it + 2 * warp + h;
    const bool d = dup >= 0 && c >= dup && c < dup + kN;   // uniform per it (dup a multiple of 64)
    oz_store_pair(v[it][0], v[it][1], f0, f1, E[c], panel + tc::sw64_offset(c, 2 * p, 2), pstride, 0, 0,
                  d ? bpanel + tc::sw64_offset(c - dup, 2 * p, 2) : nullptr, kBPanel);
  }
}

struct OzPipe {
  uint64_t* bar;      // [2]: oz_run commits every batch to bar[0]; two batches in flight alternate bar[0] / bar[1]
  uint32_t tmem, idesc;
  uint32_t mph;       // bit b: parity of the next completion of bar[b] (the same in every thread)
  uint32_t mopen;     // issuing thread: bit b = a batch committed to bar[b] and not yet waited for
  int tid, q, g;
};

// Waits (bounded) for the MMA batch of chunk ch (committed to bar[ch & 1]).
__device__ __forceinline__ bool oz_wait_mma(OzPipe& P, int ch) {
  const uint32_t b = (uint32_t)ch & 1u;
  const bool ok = tc::mbar_wait(&P.bar[b], (P.mph >> b) & 1u);
  if (ok) {
    P.mph ^= 1u << b;
    P.mopen &= ~(1u << b);
  }
  return ok;
}

// Runs nchunks chunks through the two stages: produce(ch, a, b) writes the
// digit panels of chunk ch (A at a, B at b, each digit's panel contiguous
// after the previous one) while the MMAs of chunk ch - 1 run; the batch of
// chunk ch is issued once that of ch - 1 is done (all batches commit to
// bar[0]).  Level sums are added into hi / lo after every kGroupChunks chunks
// (the exactness limit of the FP32 level sums) and after the last.  Issuing
// the next batch before the previous one completes (two barriers) was measured
// about 1% slower in these kernels, whose production overlaps the MMAs anyway.
// False when a wait timed out (every thread returns false together).
template <class Produce>
__device__ __forceinline__ bool oz_run(OzPipe& P, unsigned char* smem, int nchunks, Produce&& produce, long long* hi,
                                       long long* lo) {
  for (int ch = 0; ch < nchunks; ++ch) {
    unsigned char* a = smem + (ch & 1) * kStage;
    unsigned char* b = a + oz::kSlices * kAPanel;
    produce(ch, a, b);   // this stage was last read by the MMAs of chunk ch - 2, already complete
    tc::fence_proxy_async();
    bool ok = true;
    if (ch > 0) ok = oz_wait_mma(P, 0);
    if (__syncthreads_or(!ok)) return false;
    if (ch > 0 && (ch - 1) % kGroupChunks == kGroupChunks - 1) {   // group closed at ch - 1
      tc::fence_after();
      oz_readout(P.tmem, P.q, P.g, hi, lo);
      tc::fence_before();
      __syncthreads();
    }
    if (P.tid == 0) {
      tc::fence_after();
      oz_issue_chunk(P.tmem, tc::smem_u32(a), tc::smem_u32(b), ch % kGroupChunks == 0);
      tc::mma_commit(&P.bar[0]);
      P.mopen |= 1u;
    }
  }
  if (nchunks > 0) {
    const bool ok = oz_wait_mma(P, 0);
    if (__syncthreads_or(!ok)) return false;
    tc::fence_after();
    oz_readout(P.tmem, P.q, P.g, hi, lo);
    tc::fence_before();
    __syncthreads();
  }
  return true;
}

// CTA prologue / epilogue shared by the kernels: TMEM (512 columns) and the
// two MMA barriers (bar: a __shared__ uint64_t[2]).
__device__ __forceinline__ OzPipe oz_begin(uint32_t* tmem_slot, uint64_t* bar) {
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) tc::tmem_alloc(tmem_slot, 512);
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::mbar_fence_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  OzPipe P;
  P.bar = bar;
  P.tmem = *tmem_slot;
  P.idesc = tc::idesc(tc::F16, kM, kN);
  P.mph = 0;
  P.mopen = 0;
  P.tid = tid;
  P.q = warp & 3;
  P.g = warp >> 2;
  return P;
}

__device__ __forceinline__ void oz_end(const OzPipe& P, bool abort, Ctl* ctl) {
  if (abort && P.tid == 0) {
    raise_level_status(ctl, ST_TIMEOUT);
    // MMA batches may still run: wait for them (bounded) before the TMEM is freed
    for (uint32_t b = 0; b < 2; ++b)
      if ((P.mopen >> b) & 1u) tc::mbar_wait(&P.bar[b], (P.mph >> b) & 1u, 1u << 20);
  }
  tc::fence_before();
  __syncthreads();
  if ((P.tid >> 5) == 0) tc::tmem_dealloc(P.tmem, 512);
}

__device__ __forceinline__ unsigned char* oz_smem(unsigned char* raw) {
  return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
}

// One item's 128 x 64 partial (hi then lo, [column][row] so that a warp's
// stores are contiguous).
__device__ __forceinline__ void oz_store_partial(long long* out, int q, int g, int lane, const long long* hi,
                                                 const long long* lo) {
  const int il = q * 32 + lane;
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const int jl = g * 16 + c;
    out[jl * kM + il] = hi[c];
    out[kM * kN + jl * kM + il] = lo[c];
  }
}

__device__ __forceinline__ oz::I128 oz_sum_partials(const long long* part, int nslabs, size_t slab_stride, int il,
                                                    int jl) {
  oz::I128 acc{0, 0};
  for (int sl = 0; sl < nslabs; ++sl) {
    const long long* pp = part + (size_t)sl * slab_stride;
    oz::i128_add(acc, oz::i128_from_parts(pp[jl * kM + il], pp[kM * kN + jl * kM + il]));
  }
  return acc;
}

__device__ __forceinline__ double nan64() { return __longlong_as_double(0x7FF8000000000000ll); }

}  // namespace
}  // namespace mrcqr
