// FP64 products of the method on FP16 tensor cores with exact integer
// slicing (ozaki.cuh): the Gram matrix and the check Q^T Q (Algorithm 1
// step 1, Sec. II-C), the finalize Q = W R_c^{-1} (Algorithm 1 step 3) and
// the FP64 sketch (Algorithm 2 steps 2-4 at p = FP64).  Each result entry is
// the once-rounded value of a 63-bit fixed-point evaluation of its sum.
#include "kernels.h"
#include "ozaki.cuh"
#include "tc.cuh"

namespace mrcqr {

namespace {

constexpr int kOzThreads = 512;
constexpr int kRowsPerCta = 128;             // MMA M
constexpr int kTile = 64;                    // MMA N and K chunk
constexpr uint32_t kWPanel = kRowsPerCta * 128;   // one slice of a 128 x 64 FP16 block (16 KiB)
constexpr uint32_t kXPanel = kTile * 128;          // one slice of a 64 x 64 FP16 block (8 KiB)

constexpr int kGroupChunks = 2;             // K chunks per exact FP32 accumulation (K <= 128)

// The 36 digit-pair MMAs (levels 0..7, four K steps of 16) of one 64-deep K
// chunk; level L accumulates in TMEM columns [64 L, 64 L + 64).  ab / bb are
// the shared addresses of digit 0 of the A (128 rows) and B (64 rows) panels,
// astride / bstride the distance between digits.  Issued by one thread.
__device__ __forceinline__ void oz_issue_chunk(uint32_t tmem, uint32_t ab, uint32_t astride, uint32_t bb,
                                               uint32_t bstride, uint32_t idesc, bool group_start) {
#pragma unroll 1
  for (int L = 0; L < oz::kLevels; ++L) {
    const uint32_t d = tmem + (uint32_t)(L * kTile);
#pragma unroll 1
    for (int a = 0; a <= L; ++a) {
      const int b = L - a;
#pragma unroll
      for (int kk = 0; kk < kTile; kk += 16) {
        const uint32_t acc = (group_start && a == 0 && kk == 0) ? 0u : 1u;
        tc::mma_f16(d, tc::sw128_desc(ab + a * astride + kk * 2), tc::sw128_desc(bb + b * bstride + kk * 2), idesc,
                    acc);
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
    tc::tmem_ld16(base + (uint32_t)(L * kTile), v);
    tc::tmem_wait_ld();
#pragma unroll
    for (int c = 0; c < 16; ++c) oz::add_level(L, v[c], hi[c], lo[c]);
  }
}

// Digits of a 64-row chunk of one column of a column-major matrix, against
// the column's reference exponent E, into K-major SW128 panels: row `prow`
// of each digit panel (panel stride pstride).  Called by a full warp: lane
// l takes rows 2l and 2l + 1; flip64 (one bit per row) flips signs.
__device__ __forceinline__ void oz_slice_col_chunk(const double* __restrict__ col, int64_t r0, int64_t r_end,
                                                   uint32_t E, uint64_t flip64, unsigned char* panel, int prow,
                                                   uint32_t pstride, int lane) {
  const int64_t ra = r0 + 2 * lane;
  double v0 = 0.0, v1 = 0.0;
  if (col) {
    if (ra < r_end) v0 = col[ra];
    if (ra + 1 < r_end) v1 = col[ra + 1];
  }
  const uint32_t f0 = (uint32_t)(flip64 >> (2 * lane)) & 1u, f1 = (uint32_t)(flip64 >> (2 * lane + 1)) & 1u;
  int d0[oz::kSlices], d1[oz::kSlices];
  oz::digits8((uint32_t)__double2hiint(v0) ^ (f0 << 31), (uint32_t)__double2loint(v0), E, d0);
  oz::digits8((uint32_t)__double2hiint(v1) ^ (f1 << 31), (uint32_t)__double2loint(v1), E, d1);
  unsigned char* dst = panel + tc::sw128_offset(prow, 2 * lane, 2);
#pragma unroll
  for (int a = 0; a < oz::kSlices; ++a)
    *reinterpret_cast<uint32_t*>(dst + a * pstride) = oz::pack_f16x2(d0[a], d1[a]);
}

// One item's 128 x 64 partial (hi then lo, [column][row] so that a warp's
// stores are contiguous).
__device__ __forceinline__ void oz_store_partial(long long* out, int q, int g, int lane, const long long* hi,
                                                 const long long* lo) {
  const int il = q * 32 + lane;
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const int jl = g * 16 + c;
    out[jl * kRowsPerCta + il] = hi[c];
    out[kRowsPerCta * kTile + jl * kRowsPerCta + il] = lo[c];
  }
}

__device__ __forceinline__ oz::I128 oz_sum_partials(const long long* part, int nslabs, size_t slab_stride, int il,
                                                    int jl) {
  oz::I128 acc{0, 0};
  for (int sl = 0; sl < nslabs; ++sl) {
    const long long* pp = part + (size_t)sl * slab_stride;
    oz::i128_add(acc, oz::i128_from_parts(pp[jl * kRowsPerCta + il], pp[kRowsPerCta * kTile + jl * kRowsPerCta + il]));
  }
  return acc;
}

// X = R_c^{-1} (upper, XT[k][j] row-major with row stride npad): per column
// j the reference exponent of max_k |X[k][j]| and the eight digits of every
// X[k][j], stored as K-major SW128 panels: panel (b, t, kc) holds rows
// j in [64t, 64t+64) and k in [64kc, 64kc+64) of digit b.
__global__ void __launch_bounds__(512) k_oz_prep_x(int n, int npad, int n64, const double* __restrict__ XT,
                                                   uint32_t* __restrict__ colE, unsigned char* __restrict__ Xs,
                                                   const Ctl* ctl, int level) {
  if (ctl && (level_inactive(ctl, level) || ctl->lvl_status != 0)) return;
  const int j = blockIdx.x;   // column, < n64
  __shared__ uint32_t red[32];
  uint32_t mx = 0u;
  for (int k = threadIdx.x; k < n64; k += blockDim.x) {
    if (k < n && j < n) {
      const double v = XT[(int64_t)k * npad + j];
      mx = max(mx, (uint32_t)__double2hiint(v) & 0x7FFFFFFFu);
    }
  }
  mx = __reduce_max_sync(0xffffffffu, mx);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0u;
    v = __reduce_max_sync(0xffffffffu, v);
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  const uint32_t E = oz::exp_field(red[0]);
  if (threadIdx.x == 0) colE[j] = E;
  const int ntiles = n64 / kTile;
  const int t = j / kTile, jr = j % kTile;
  for (int k = threadIdx.x; k < n64; k += blockDim.x) {
    int d[oz::kSlices];
    const double v = (k < n && j < n) ? XT[(int64_t)k * npad + j] : 0.0;
    oz::digits8((uint32_t)__double2hiint(v), (uint32_t)__double2loint(v), E, d);
    const int kc = k / kTile, kr = k % kTile;
#pragma unroll
    for (int b = 0; b < oz::kSlices; ++b) {
      const __half h = __float2half_rn(oz::small_int_to_float(d[b]));
      unsigned char* panel = Xs + (size_t)((b * ntiles + t) * ntiles + kc) * kXPanel;
      *reinterpret_cast<__half*>(panel + tc::sw128_offset(jr, kr, 2)) = h;
    }
  }
}

// Q = W X in place, 128 rows per CTA, output tiles of 64 columns from right
// to left (a tile reads only W columns left of its right edge, which are
// still W).  X upper triangular: tile t needs K chunks 0..t.
__global__ void __launch_bounds__(kOzThreads, 1)
    k_finalize_oz(int64_t m, int n, int n64, double* __restrict__ Q, int64_t ldq, const uint32_t* __restrict__ colE,
                  const unsigned char* __restrict__ Xs, Ctl* ctl, int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* ws = smem;                                   // 8 slices x 16 KiB
  unsigned char* xs = smem + oz::kSlices * kWPanel;           // 8 slices x 8 KiB
  __shared__ __align__(8) uint64_t mma_bar;
  __shared__ uint32_t tmem_base;
  __shared__ uint32_t rowE[kRowsPerCta];
  __shared__ uint32_t redE[4][kRowsPerCta];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = n64 / kTile;
  if (warp == 0) tc::tmem_alloc(&tmem_base, 512);   // 8 levels x 64 columns
  if (tid == 0) {
    tc::mbar_init(&mma_bar, 1);
    tc::mbar_fence_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = tc::idesc(tc::F16, kRowsPerCta, kTile);
  const int q = warp & 3, g = warp >> 2;   // TMEM lane quarter, 16-column group
  uint32_t phase = 0;
  bool abort = false;
  const int64_t nblocks = (m + kRowsPerCta - 1) / kRowsPerCta;

  for (int64_t rb = blockIdx.x; rb < nblocks && !abort; rb += gridDim.x) {
    const int64_t r0 = rb * kRowsPerCta;
    // row reference exponents over all n columns of W
    {
      const int r = tid & (kRowsPerCta - 1), c0 = tid >> 7;
      uint32_t mx = 0u;
      if (r0 + r < m)
        for (int c = c0; c < n; c += 4) mx = max(mx, (uint32_t)__double2hiint(Q[r0 + r + (int64_t)c * ldq]) & 0x7FFFFFFFu);
      redE[c0][r] = mx;
      __syncthreads();
      if (tid < kRowsPerCta)
        rowE[tid] = oz::exp_field(max(max(redE[0][tid], redE[1][tid]), max(redE[2][tid], redE[3][tid])));
      __syncthreads();
    }
    for (int t = ntiles - 1; t >= 0 && !abort; --t) {
      long long hi[16], lo[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) hi[c] = lo[c] = 0;
      for (int kc = 0; kc <= t; ++kc) {
        const bool group_start = (kc % kGroupChunks) == 0;
        const bool group_end = (kc % kGroupChunks) == kGroupChunks - 1 || kc == t;
        // X digits of (t, kc)
        for (int i = tid; i < oz::kSlices * (int)(kXPanel / 16); i += kOzThreads) {
          const int b = i / (kXPanel / 16), o = i % (kXPanel / 16);
          const uint4* src = reinterpret_cast<const uint4*>(Xs + (size_t)((b * ntiles + t) * ntiles + kc) * kXPanel);
          reinterpret_cast<uint4*>(xs + b * kXPanel)[o] = src[o];
        }
        // W digits of columns [64 kc, 64 kc + 64): thread owns row r and column pairs
        {
          const int r = tid & (kRowsPerCta - 1);
          const uint32_t Er = rowE[r];
          const bool live = r0 + r < m;
#pragma unroll 2
          for (int p = tid >> 7; p < kTile / 2; p += 4) {
            const int k0 = kc * kTile + 2 * p;
            int d0[oz::kSlices], d1[oz::kSlices];
            double v0 = 0.0, v1 = 0.0;
            if (live && k0 < n) v0 = Q[r0 + r + (int64_t)k0 * ldq];
            if (live && k0 + 1 < n) v1 = Q[r0 + r + (int64_t)(k0 + 1) * ldq];
            oz::digits8((uint32_t)__double2hiint(v0), (uint32_t)__double2loint(v0), Er, d0);
            oz::digits8((uint32_t)__double2hiint(v1), (uint32_t)__double2loint(v1), Er, d1);
#pragma unroll
            for (int a = 0; a < oz::kSlices; ++a)
              *reinterpret_cast<uint32_t*>(ws + a * kWPanel + tc::sw128_offset(r, 2 * p, 2)) = oz::pack_f16x2(d0[a], d1[a]);
          }
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
          tc::fence_after();
          oz_issue_chunk(tmem, tc::smem_u32(ws), kWPanel, tc::smem_u32(xs), kXPanel, idesc, group_start);
          tc::mma_commit(&mma_bar);
        }
        const bool ok = tc::mbar_wait(&mma_bar, phase);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
          abort = true;
          break;
        }
        tc::fence_after();
        if (group_end) oz_readout(tmem, q, g, hi, lo);
        tc::fence_before();
        __syncthreads();
      }
      if (abort) break;
      // write Q[:, 64t + 16g + c] for this thread's row
      const int r = q * 32 + lane;
      if (r0 + r < m) {
        const int scale_r = (int)rowE[r] - oz::kScaleBias;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int j = t * kTile + g * 16 + c;
          if (j < n) {
            const uint32_t ce = colE[j];
            const double out = (rowE[r] == 2047u || ce == 2047u)   // non-finite operands
                                   ? __longlong_as_double(0x7FF8000000000000ll)
                                   : oz::i128_to_double(hi[c], lo[c], scale_r + (int)ce);
            Q[r0 + r + (int64_t)j * ldq] = out;
          }
        }
      }
      __syncthreads();
    }
  }
  if (abort && tid == 0) raise_level_status(ctl, ST_TIMEOUT);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}


// ---------------------------------------------------------------------------
// Gram G = W^T W (Algorithm 1 step 1) and the check matrix Q^T Q as emulated
// FP64.  Every column of W is sliced against the exponent of its maximum over
// all m rows, so the level sums of all rows share one scale: a work item
// (output tile of 128 x 64 entries, slab of rows) reads its exact level sums
// out of TMEM every 128 rows into 64-bit integer pairs, and a reduction adds
// the items' 128-bit values (exact, so the order does not matter) and rounds
// each entry once.

// Column maxima (as the high word of |x|, whose exponent field is the
// reference exponent) over all rows; colHi must be zero on entry.
__global__ void __launch_bounds__(256) k_col_hi(int64_t m, int n, const double* __restrict__ W, int64_t ldw,
                                                int64_t rows_per_cta, uint32_t* __restrict__ colHi, const Ctl* ctl,
                                                int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  const int j = blockIdx.x;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_cta;
  const int64_t r1 = min(m, r0 + rows_per_cta);
  const double* col = W + (int64_t)j * ldw;
  uint32_t mx = 0u;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += 256)
    mx = max(mx, (uint32_t)__double2hiint(__ldg(col + r)) & 0x7FFFFFFFu);
  __shared__ uint32_t red[8];
  mx = __reduce_max_sync(0xffffffffu, mx);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t v = red[0];
    for (int w = 1; w < 8; ++w) v = max(v, red[w]);
    if (v) atomicMax(colHi + j, v);
  }
}

__global__ void __launch_bounds__(kOzThreads, 1)
    k_syrk_oz(int64_t m, int n, const double* __restrict__ W, int64_t ldw, const uint32_t* __restrict__ colHi,
              SyrkOzPlan P, long long* __restrict__ part, Ctl* ctl, int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* as = smem;                                   // 8 digits x (128 columns x 64 rows)
  unsigned char* bs = smem + oz::kSlices * kWPanel;           // 8 digits x (64 columns x 64 rows)
  __shared__ __align__(8) uint64_t mma_bar;
  __shared__ uint32_t tmem_base;
  __shared__ uint32_t colE[kRowsPerCta + kTile];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
  if (tid == 0) {
    tc::mbar_init(&mma_bar, 1);
    tc::mbar_fence_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = tc::idesc(tc::F16, kRowsPerCta, kTile);
  const int q = warp & 3, g = warp >> 2;
  uint32_t phase = 0;
  bool abort = false;
  const int nitems = P.ntiles * P.slabs;

  for (int item = blockIdx.x; item < nitems && !abort; item += gridDim.x) {
    const int tile = item % P.ntiles, slab = item / P.ntiles;
    const int i0 = kRowsPerCta * P.ti[tile], j0 = kTile * P.tj[tile];
    const bool inner = (P.tj[tile] >> 1) == P.ti[tile];   // J block inside the I block
    const int64_t r_begin = (int64_t)slab * P.rows_per_slab;
    const int64_t r_end = min(m, r_begin + P.rows_per_slab);
    const int nchunks = r_end > r_begin ? (int)((r_end - r_begin + kTile - 1) / kTile) : 0;
    __syncthreads();
    if (tid < kRowsPerCta) colE[tid] = i0 + tid < n ? oz::exp_field(colHi[i0 + tid]) : 0u;
    else if (tid < kRowsPerCta + kTile) colE[tid] = j0 + tid - kRowsPerCta < n ? oz::exp_field(colHi[j0 + tid - kRowsPerCta]) : 0u;
    __syncthreads();
    long long hi[16], lo[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) hi[c] = lo[c] = 0;
    for (int ch = 0; ch < nchunks; ++ch) {
      const int64_t r0 = r_begin + (int64_t)ch * kTile;
      const bool group_start = (ch % kGroupChunks) == 0;
      const bool group_end = (ch % kGroupChunks) == kGroupChunks - 1 || ch == nchunks - 1;
      // digits of W[r0 .. r0+63, column]: one column per warp, two rows per lane
#pragma unroll 1
      for (int c = warp; c < kRowsPerCta + kTile; c += kOzThreads / 32) {
        if (c >= kRowsPerCta && inner) break;
        const int col = c < kRowsPerCta ? i0 + c : j0 + c - kRowsPerCta;
        const double* src = col < n ? W + (int64_t)col * ldw : nullptr;
        if (c < kRowsPerCta) oz_slice_col_chunk(src, r0, r_end, colE[c], 0ull, as, c, kWPanel, lane);
        else oz_slice_col_chunk(src, r0, r_end, colE[c], 0ull, bs, c - kRowsPerCta, kXPanel, lane);
      }
      tc::fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after();
        const uint32_t ab = tc::smem_u32(as);
        const uint32_t bb = inner ? ab + (uint32_t)(j0 - i0) * 128u : tc::smem_u32(bs);
        oz_issue_chunk(tmem, ab, kWPanel, bb, inner ? kWPanel : kXPanel, idesc, group_start);
        tc::mma_commit(&mma_bar);
      }
      const bool ok = tc::mbar_wait(&mma_bar, phase);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        abort = true;
        break;
      }
      tc::fence_after();
      if (group_end) oz_readout(tmem, q, g, hi, lo);
      tc::fence_before();
      __syncthreads();
    }
    if (abort) break;
    oz_store_partial(part + (size_t)item * (2 * kRowsPerCta * kTile), q, g, lane, hi, lo);
  }
  if (abort && tid == 0) raise_level_status(ctl, ST_TIMEOUT);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// Upper triangle of G from the items' partials (exact 128-bit sums over the
// slabs, one rounding); lower triangle zero.
__global__ void k_syrk_oz_reduce(int n, const uint32_t* __restrict__ colHi, SyrkOzPlan P,
                                 const long long* __restrict__ part, double* __restrict__ out, const Ctl* ctl,
                                 int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e % n), j = (int)(e / n);
  if (i > j) {
    out[e] = 0.0;
    return;
  }
  const int I = i / kRowsPerCta, J = j / kTile;
  const int tile = P.tile_of[I][J];
  const int il = i - I * kRowsPerCta, jl = j - J * kTile;
  const oz::I128 acc = oz_sum_partials(part + (size_t)tile * (2 * kRowsPerCta * kTile), P.slabs,
                                       (size_t)P.ntiles * (2 * kRowsPerCta * kTile), il, jl);
  const uint32_t Ei = oz::exp_field(colHi[i]), Ej = oz::exp_field(colHi[j]);
  out[e] = (Ei == 2047u || Ej == 2047u) ? __longlong_as_double(0x7FF8000000000000ll)
                                        : oz::i128_to_double(acc, (int)Ei + (int)Ej - oz::kScaleBias);
}

// ---------------------------------------------------------------------------
// FP64 sketch (Algorithm 2 steps 2-4 with p = FP64) as an emulated GEMM:
//   P[c][i] = sum_j (d_j A[j][c]) F[i][j],  F[i][j] = cos(pi r_ij / (2m)),
//   r_ij = k_i (2j + 1) mod 4m,
// with F[i][j] the FP64 quarter-wave table value (the value the FMA kernel
// multiplies with) and d_j the Rademacher sign; then Y[i][c] =
// sqrt(2/s) c_k(i) P[c][i].  A's columns are sliced against their maxima over
// all m rows, the table values against 2^0 (|F| <= 1).  Work item = (block of
// 128 columns of A, 64 sampled rows, slab of rows of A).
__global__ void __launch_bounds__(kOzThreads, 1)
    k_sketch_oz(int64_t m, int n, int s, const double* __restrict__ A, int64_t lda, const uint32_t* __restrict__ colHi,
                const uint32_t* __restrict__ idx, const double* __restrict__ tab, uint2 key, SketchOzPlan P,
                long long* __restrict__ part, Ctl* ctl, int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* as = smem;                                   // 8 digits x (128 columns x 64 rows)
  unsigned char* fs = smem + oz::kSlices * kWPanel;           // 8 digits x (64 samples x 64 rows)
  __shared__ __align__(8) uint64_t mma_bar;
  __shared__ uint32_t tmem_base;
  __shared__ uint32_t colE[kRowsPerCta];
  __shared__ uint32_t flips[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
  if (tid == 0) {
    tc::mbar_init(&mma_bar, 1);
    tc::mbar_fence_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = tc::idesc(tc::F16, kRowsPerCta, kTile);
  const int q = warp & 3, g = warp >> 2;
  const uint64_t four_m = 4ull * (uint64_t)m;
  uint32_t phase = 0;
  bool abort = false;
  const int ntiles_all = P.mblocks * P.ntiles;
  const int nitems = ntiles_all * P.slabs;
  // transform-panel role of this thread: sample fi, rows 8 fg .. 8 fg + 7
  const int fi = tid & (kTile - 1), fg = tid >> 6;

  for (int item = blockIdx.x; item < nitems && !abort; item += gridDim.x) {
    const int tile = item % ntiles_all, slab = item / ntiles_all;
    const int c0 = kRowsPerCta * (tile / P.ntiles), i0 = kTile * (tile % P.ntiles);
    const int64_t r_begin = (int64_t)slab * P.rows_per_slab;
    const int64_t r_end = min(m, r_begin + P.rows_per_slab);
    const int nchunks = r_end > r_begin ? (int)((r_end - r_begin + kTile - 1) / kTile) : 0;
    __syncthreads();
    if (tid < kRowsPerCta) colE[tid] = c0 + tid < n ? oz::exp_field(colHi[c0 + tid]) : 0u;
    // phase of (sample fi, row r_begin + 8 fg) and its advance per chunk
    const bool fval = i0 + fi < s;
    const uint64_t k = fval ? (uint64_t)idx[i0 + fi] : 0ull;
    uint64_t r = fval ? (k * (uint64_t)(2 * (r_begin + 8 * fg) + 1)) % four_m : 0ull;
    const uint64_t step_chunk = (k * (uint64_t)(2 * kTile)) % four_m;
    const uint64_t step_row = 2ull * k;   // < 4m
    long long hi[16], lo[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) hi[c] = lo[c] = 0;
    for (int ch = 0; ch < nchunks; ++ch) {
      const int64_t r0 = r_begin + (int64_t)ch * kTile;
      const bool group_start = (ch % kGroupChunks) == 0;
      const bool group_end = (ch % kGroupChunks) == kGroupChunks - 1 || ch == nchunks - 1;
      // Rademacher signs of the chunk's rows (bit t: d_{r0 + t} = -1)
      if (warp < 2) {
        const int64_t j0 = r0 + 32 * warp + lane;
        const bool neg = j0 < r_end && row_sign((uint64_t)j0, key) < 0.0;
        const uint32_t bits = __ballot_sync(0xffffffffu, neg);
        if (lane == 0) flips[warp] = bits;
      }
      // transform digits: sample fi, rows 8 fg .. 8 fg + 7
      {
        uint64_t rr = r;
        unsigned char* dst = fs + tc::sw128_offset(fi, 8 * fg, 2);
#pragma unroll
        for (int t2 = 0; t2 < 4; ++t2) {
          int d0[oz::kSlices], d1[oz::kSlices];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int64_t j = r0 + 8 * fg + 2 * t2 + h;
            uint32_t whi = 0u, wlo = 0u;
            if (fval && j < r_end) cos_phase_bits(tab, (int64_t)rr, m, whi, wlo);
            oz::digits8(whi, wlo, 1023u, h ? d1 : d0);
            rr += step_row;
            if (rr >= four_m) rr -= four_m;
          }
#pragma unroll
          for (int b = 0; b < oz::kSlices; ++b)
            *reinterpret_cast<uint32_t*>(dst + 4 * t2 + b * kXPanel) = oz::pack_f16x2(d0[b], d1[b]);
        }
        r += step_chunk;
        if (r >= four_m) r -= four_m;
      }
      __syncthreads();   // signs visible
      const uint64_t flip64 = (uint64_t)flips[0] | ((uint64_t)flips[1] << 32);
      // digits of d_j A[j][c]: one column per warp
#pragma unroll 1
      for (int c = warp; c < kRowsPerCta; c += kOzThreads / 32) {
        const int col = c0 + c;
        oz_slice_col_chunk(col < n ? A + (int64_t)col * lda : nullptr, r0, r_end, colE[c], flip64, as, c, kWPanel,
                           lane);
      }
      tc::fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after();
        oz_issue_chunk(tmem, tc::smem_u32(as), kWPanel, tc::smem_u32(fs), kXPanel, idesc, group_start);
        tc::mma_commit(&mma_bar);
      }
      const bool ok = tc::mbar_wait(&mma_bar, phase);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        abort = true;
        break;
      }
      tc::fence_after();
      if (group_end) oz_readout(tmem, q, g, hi, lo);
      tc::fence_before();
      __syncthreads();
    }
    if (abort) break;
    oz_store_partial(part + (size_t)item * (2 * kRowsPerCta * kTile), q, g, lane, hi, lo);
  }
  if (abort && tid == 0) raise_level_status(ctl, ST_TIMEOUT);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// Y (s x n, column-major) from the items' partials: exact sums over the
// slabs, one rounding, times sqrt(2/s) c_k.  A non-finite column of A gives a
// NaN column and raises NONFINITE.
__global__ void k_sketch_oz_reduce(int n, int s, const uint32_t* __restrict__ colHi, const uint32_t* __restrict__ idx,
                                   SketchOzPlan P, const long long* __restrict__ part, double* __restrict__ Y,
                                   Ctl* ctl, int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)s * n) return;
  const int i = (int)(e % s), c = (int)(e / s);
  const int tile = (c / kRowsPerCta) * P.ntiles + i / kTile;
  const size_t tstride = 2 * kRowsPerCta * kTile;
  const oz::I128 acc = oz_sum_partials(part + (size_t)tile * tstride, P.slabs,
                                       (size_t)P.mblocks * P.ntiles * tstride, c % kRowsPerCta, i % kTile);
  const uint32_t Ec = oz::exp_field(colHi[c]);
  const double coef = sqrt(2.0 / (double)s) * (idx[i] == 0 ? 0.70710678118654752440 : 1.0);
  const double y = Ec == 2047u ? __longlong_as_double(0x7FF8000000000000ll)
                               : oz::i128_to_double(acc, (int)Ec + 1023 - oz::kScaleBias) * coef;
  Y[e] = y;
  if (!isfinite(y)) {
    ctl->input_nonfinite = 1;
    raise_level_status(ctl, ST_NONFINITE);
  }
}

}  // namespace

size_t oz_xs_bytes(int n) {
  const int n64 = (n + kTile - 1) / kTile * kTile;
  const int nt = n64 / kTile;
  return (size_t)oz::kSlices * nt * nt * kXPanel;
}

void launch_finalize_oz(int64_t m, int n, double* Q, int64_t ldq, const double* XT, uint32_t* colE,
                        unsigned char* Xs, Ctl* ctl, int level, cudaStream_t st) {
  const int npad = (n + 31) / 32 * 32;
  const int n64 = (n + kTile - 1) / kTile * kTile;
  k_oz_prep_x<<<n64, 512, 0, st>>>(n, npad, n64, XT, colE, Xs, ctl, level);
  const size_t smem = (size_t)oz::kSlices * (kWPanel + kXPanel) + 1024;
  cudaFuncSetAttribute(k_finalize_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nblocks = (m + kRowsPerCta - 1) / kRowsPerCta;
  const unsigned grid = (unsigned)(nblocks < sms ? nblocks : sms);
  k_finalize_oz<<<grid, kOzThreads, smem, st>>>(m, n, n64, Q, ldq, colE, Xs, ctl, level);
}

static int num_sms() {
  static int cached = 0;
  if (!cached) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cached = sms > 0 ? sms : 152;
  }
  return cached;
}

static int gcd_int(int a, int b) { return b ? gcd_int(b, a % b) : a; }

SyrkOzPlan syrk_oz_plan(int64_t m, int n) {
  SyrkOzPlan P{};
  const int nI = (n + kRowsPerCta - 1) / kRowsPerCta, nJ = (n + kTile - 1) / kTile;
  for (int I = 0; I < 4; ++I)
    for (int J = 0; J < 8; ++J) P.tile_of[I][J] = -1;
  for (int I = 0; I < nI; ++I)
    for (int J = 0; J < nJ; ++J)
      if (kTile * J + kTile - 1 >= kRowsPerCta * I) {
        P.ti[P.ntiles] = (int8_t)I;
        P.tj[P.ntiles] = (int8_t)J;
        P.tile_of[I][J] = (int8_t)P.ntiles;
        ++P.ntiles;
      }
  // items = tiles x slabs a multiple of the SM count where the rows allow it
  const int sms = num_sms();
  int slabs = sms / gcd_int(P.ntiles, sms);
  const int64_t max_slabs = (m + 4 * kTile - 1) / (4 * kTile);   // at least 256 rows each
  if (slabs > max_slabs) slabs = (int)max_slabs;
  // at most 2^20 rows per slab: the 64-bit halves of an item stay below 2^61
  const int64_t min_slabs = (m + (1 << 20) - 1) >> 20;
  if (slabs < min_slabs) slabs = (int)min_slabs;
  if (slabs < 1) slabs = 1;
  int64_t rps = (m + slabs - 1) / slabs;
  rps = (rps + kTile - 1) / kTile * kTile;
  P.rows_per_slab = rps;
  P.slabs = (int)((m + rps - 1) / rps);
  return P;
}

size_t syrk_oz_part_bytes(const SyrkOzPlan& P) {
  return sizeof(long long) * 2 * kRowsPerCta * kTile * (size_t)P.ntiles * P.slabs;
}

size_t syrk_oz_colhi_bytes(int n) { return sizeof(uint32_t) * (size_t)((n + kRowsPerCta - 1) / kRowsPerCta * kRowsPerCta); }

void launch_syrk_oz(int64_t m, int n, const double* W, int64_t ldw, const SyrkOzPlan& P, uint32_t* colHi,
                    long long* part, double* out, Ctl* ctl, int level, cudaStream_t st) {
  cudaMemsetAsync(colHi, 0, syrk_oz_colhi_bytes(n), st);
  const int sms = num_sms();
  int ysplit = (4 * sms + n - 1) / n;
  const int64_t max_y = (m + 4095) / 4096;
  if (ysplit > max_y) ysplit = (int)max_y;
  if (ysplit < 1) ysplit = 1;
  const int64_t rpc = (m + ysplit - 1) / ysplit;
  k_col_hi<<<dim3(n, ysplit), 256, 0, st>>>(m, n, W, ldw, rpc, colHi, ctl, level);
  const size_t smem = (size_t)oz::kSlices * (kWPanel + kXPanel) + 1024;
  cudaFuncSetAttribute(k_syrk_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int nitems = P.ntiles * P.slabs;
  k_syrk_oz<<<nitems < sms ? nitems : sms, kOzThreads, smem, st>>>(m, n, W, ldw, colHi, P, part, ctl, level);
  const int64_t nn = (int64_t)n * n;
  k_syrk_oz_reduce<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(n, colHi, P, part, out, ctl, level);
}

SketchOzPlan sketch_oz_plan(int64_t m, int n, int s) {
  SketchOzPlan P{};
  P.mblocks = (n + kRowsPerCta - 1) / kRowsPerCta;
  P.ntiles = (s + kTile - 1) / kTile;
  const int tiles = P.mblocks * P.ntiles;
  const int sms = num_sms();
  int slabs = tiles >= sms ? 1 : sms / gcd_int(tiles, sms);
  const int64_t max_slabs = (m + 4 * kTile - 1) / (4 * kTile);
  if (slabs > max_slabs) slabs = (int)max_slabs;
  const int64_t min_slabs = (m + (1 << 20) - 1) >> 20;
  if (slabs < min_slabs) slabs = (int)min_slabs;
  if (slabs < 1) slabs = 1;
  int64_t rps = (m + slabs - 1) / slabs;
  rps = (rps + kTile - 1) / kTile * kTile;
  P.rows_per_slab = rps;
  P.slabs = (int)((m + rps - 1) / rps);
  return P;
}

size_t sketch_oz_part_bytes(const SketchOzPlan& P) {
  return sizeof(long long) * 2 * kRowsPerCta * kTile * (size_t)P.mblocks * P.ntiles * P.slabs;
}

void launch_sketch_oz(int64_t m, int n, int s, const double* A, int64_t lda, const uint32_t* idx, const double* tab,
                      uint64_t seed, const SketchOzPlan& P, uint32_t* colHi, long long* part, double* Y, Ctl* ctl,
                      int level, cudaStream_t st) {
  cudaMemsetAsync(colHi, 0, syrk_oz_colhi_bytes(n), st);
  const int sms = num_sms();
  int ysplit = (4 * sms + n - 1) / n;
  const int64_t max_y = (m + 4095) / 4096;
  if (ysplit > max_y) ysplit = (int)max_y;
  if (ysplit < 1) ysplit = 1;
  k_col_hi<<<dim3(n, ysplit), 256, 0, st>>>(m, n, A, lda, (m + ysplit - 1) / ysplit, colHi, ctl, level);
  const size_t smem = (size_t)oz::kSlices * (kWPanel + kXPanel) + 1024;
  cudaFuncSetAttribute(k_sketch_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int nitems = P.mblocks * P.ntiles * P.slabs;
  k_sketch_oz<<<nitems < sms ? nitems : sms, kOzThreads, smem, st>>>(m, n, s, A, lda, colHi, idx, tab, seed_key(seed),
                                                                      P, part, ctl, level);
  const int64_t total = (int64_t)s * n;
  k_sketch_oz_reduce<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(n, s, colHi, idx, P, part, Y, ctl, level);
}

}  // namespace mrcqr
