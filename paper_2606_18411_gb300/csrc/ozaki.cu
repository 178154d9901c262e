// FP64 products of the method on FP16 tensor cores with exact integer
// slicing (ozaki.cuh): the Gram matrix and the check Q^T Q (Algorithm 1
// step 1, Sec. II-C), the finalize Q = W R_c^{-1} (Algorithm 1 step 3) and
// the FP64 sketch (Algorithm 2 steps 2-4 at p = FP64).  Each result entry is
// the once-rounded value of a 63-bit fixed-point evaluation of its sum.
//
// All four run the same two-stage pipeline per CTA (one CTA per SM, 512
// threads, all 512 TMEM columns = 8 level accumulators of 128 x 64): the
// threads write the digit panels of K chunk c + 1 (32 deep, K-major
// SWIZZLE_64B) into one shared-memory stage while the tensor cores run the
// 36 digit-pair MMAs of chunk c from the other; every 4 chunks (K = 128, the
// exactness limit) the level sums are read out of TMEM into 64-bit integers.
#include "kernels.h"
#include "ozaki.cuh"
#include "tc.cuh"
#include "ozaki_pipe.cuh"

namespace mrcqr {

namespace {

// ---------------------------------------------------------------------------
// Finalize Q = W X in place (X = R_c^{-1} upper, Algorithm 1 step 3).
//
// Prep: per column j of X the reference exponent of max_k |X[k][j]| and the
// digits of every X[k][j] as K-major SWIZZLE_64B panels: panel
// ((b * ntiles + t) * nkc + kc) holds rows j in [64t, 64t+64) and k in
// [32kc, 32kc+32) of digit b.  XT[k][j] = X[k][j], row stride npad.
__device__ __forceinline__ void oz_prep_x_col(int n, int npad, int n64, const double* __restrict__ XT,
                                              uint32_t* __restrict__ colE, unsigned char* __restrict__ Xs,
                                              uint32_t* __restrict__ colHiOut, int nhi, int j, uint32_t* red) {
  if (colHiOut && j == 0)     // the finalize folds the column maxima of Q into these
    for (int i = threadIdx.x; i < nhi; i += blockDim.x) colHiOut[i] = 0u;
  __syncthreads();
  uint32_t mx = 0u;
  for (int k = threadIdx.x; k < n64; k += blockDim.x)
    if (k < n && j < n) mx = max(mx, (uint32_t)__double2hiint(XT[(int64_t)k * npad + j]) & 0x7FFFFFFFu);
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
  const int ntiles = n64 / kN, nkc = n64 / kK;
  const int t = j / kN, jr = j % kN;
  for (int k = threadIdx.x; k < n64; k += blockDim.x) {
    int d[oz::kSlices];
    const double v = (k < n && j < n) ? XT[(int64_t)k * npad + j] : 0.0;
    oz::digits8((uint32_t)__double2hiint(v), (uint32_t)__double2loint(v), E, d);
    const int kc = k / kK, kr = k % kK;
#pragma unroll
    for (int b = 0; b < oz::kSlices; ++b) {
      unsigned char* panel = Xs + (size_t)((b * ntiles + t) * nkc + kc) * kBPanel;
      *reinterpret_cast<__half*>(panel + tc::sw64_offset(jr, kr, 2)) = __float2half_rn(oz::small_int_to_float(d[b]));
    }
  }
}

__global__ void __launch_bounds__(512) k_oz_prep_x(int n, int npad, int n64, const double* __restrict__ XT,
                                                   uint32_t* __restrict__ colE, unsigned char* __restrict__ Xs,
                                                   uint32_t* __restrict__ colHiOut, int nhi, const Ctl* ctl,
                                                   int level) {
  if (ctl && (level_inactive(ctl, level) || ctl->lvl_status != 0)) return;
  __shared__ uint32_t red[32];
  oz_prep_x_col(n, npad, n64, XT, colE, Xs, colHiOut, nhi, blockIdx.x, red);
}

// Main kernel: 128 rows per work block, output tiles of 64 columns from right
// to left (a tile reads only W columns left of its right edge, still W).
// X upper triangular: tile t needs K chunks 0 .. 2t + 1.
// Q = W X for one problem: arguments of the kernel body.
struct FinOzArgs {
  int64_t m;
  int n, n64;
  double* Q;
  int64_t ldq;
  const uint32_t* colE;
  const unsigned char* Xs;
  uint32_t* colHiOut;
  Ctl* ctl;
};

// Shared-memory state of one CTA of the finalize (besides the pipeline).
struct FinOzCta {
  unsigned char* smem;
  uint32_t* rowE;
  uint32_t (*redE)[kM];
  uint32_t* cmax;   // column maxima of |Q| (high words) over this CTA's rows of the problem
};

__device__ __forceinline__ void fin_oz_begin(const FinOzArgs& a, FinOzCta& S) {
  __syncthreads();
  for (int j = threadIdx.x; j < a.n64; j += kOzThreads) S.cmax[j] = 0u;
  __syncthreads();
}

__device__ __forceinline__ void fin_oz_end(const FinOzArgs& a, FinOzCta& S) {
  __syncthreads();
  if (a.colHiOut)
    for (int j = threadIdx.x; j < a.n; j += kOzThreads)
      if (S.cmax[j]) atomicMax(a.colHiOut + j, S.cmax[j]);
  __syncthreads();
}

// One block of 128 rows starting at r0 (output tiles from right to left).
// False when a wait timed out (every thread together).
__device__ __forceinline__ bool fin_oz_block(const FinOzArgs& a, FinOzCta& S, OzPipe& P, int64_t r0) {
  const int64_t m = a.m;
  const int n = a.n;
  double* __restrict__ Q = a.Q;
  const int64_t ldq = a.ldq;
  const uint32_t* __restrict__ colE = a.colE;
  const unsigned char* __restrict__ Xs = a.Xs;
  uint32_t* colHiOut = a.colHiOut;
  unsigned char* smem = S.smem;
  uint32_t* rowE = S.rowE;
  uint32_t(*redE)[kM] = S.redE;
  uint32_t* cmax = S.cmax;
  const int tid = threadIdx.x, lane = tid & 31;
  const int ntiles = a.n64 / kN, nkc = a.n64 / kK;
  {   // row reference exponents over all n columns of W
    const int r = tid & (kM - 1), c0 = tid >> 7;
    uint32_t mx = 0u;
    if (r0 + r < m)
      for (int c = c0; c < n; c += 4) mx = max(mx, (uint32_t)__double2hiint(Q[r0 + r + (int64_t)c * ldq]) & 0x7FFFFFFFu);
    redE[c0][r] = mx;
    __syncthreads();
    if (tid < kM) rowE[tid] = oz::exp_field(max(max(redE[0][tid], redE[1][tid]), max(redE[2][tid], redE[3][tid])));
    __syncthreads();
  }
  const int r = tid & (kM - 1), pp = tid >> 7;   // producer role: row r, 16-byte chunk pp of each K chunk
  const bool live = r0 + r < m;
  for (int t = ntiles - 1; t >= 0; --t) {
    long long hi[16], lo[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) hi[c] = lo[c] = 0;
    double v[4][2];
    // row r, the four column pairs of 16-byte chunk pp of each 32-column chunk; lane group
    // lane / 8 starts at a different pair, so a warp's 4-byte panel stores hit 32 banks
    const int lg = lane >> 3;
    auto pair_of = [&](int i) { return 4 * pp + ((lg + i) & 3); };
    auto load_w = [&](int kc) {   // W of columns [32 kc, 32 kc + 32)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int k0 = kc * kK + 2 * pair_of(i);
        v[i][0] = (live && k0 < n) ? Q[r0 + r + (int64_t)k0 * ldq] : 0.0;
        v[i][1] = (live && k0 + 1 < n) ? Q[r0 + r + (int64_t)(k0 + 1) * ldq] : 0.0;
      }
    };
    load_w(0);
    const int nch = 2 * (t + 1);
    auto produce = [&](int kc, unsigned char* a, unsigned char* b) {
      // X digits of (t, kc): 32 KiB, four asynchronous 16-byte copies per thread
      const uint4* src = reinterpret_cast<const uint4*>(Xs);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int e = tid + kOzThreads * i;          // < 2048
        const int dg = e / (kBPanel / 16), o = e % (kBPanel / 16);
        tc::cp_async16(b + dg * kBPanel + 16 * o, src + (size_t)((dg * ntiles + t) * nkc + kc) * (kBPanel / 16) + o);
      }
      const uint32_t Er = rowE[r];
#pragma unroll
      for (int i = 0; i < 4; ++i)
        oz_store_pair(v[i][0], v[i][1], 0u, 0u, Er, a + tc::sw64_offset(r, 2 * pair_of(i), 2), kAPanel);
      if (kc + 1 < nch) load_w(kc + 1);
      tc::cp_async_wait_all();
    };
    if (!oz_run(P, smem, nch, produce, hi, lo)) return false;
    // write Q[:, 64t + 16g + c] for this thread's row (lane c keeps the warp's maximum of column c)
    const int rr = P.q * 32 + lane;
    const bool rlive = r0 + rr < m;
    const int scale_r = (int)rowE[rr] - oz::kScaleBias;
    uint32_t mine = 0u;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int j = t * kN + P.g * 16 + c;
      uint32_t h = 0u;
      if (rlive && j < n) {
        const uint32_t ce = colE[j];
        const double qv = (rowE[rr] == 2047u || ce == 2047u)   // non-finite operands
                              ? nan64()
                              : oz::i128_to_double(hi[c], lo[c], scale_r + (int)ce);
        Q[r0 + rr + (int64_t)j * ldq] = qv;
        h = (uint32_t)__double2hiint(qv) & 0x7FFFFFFFu;
      }
      if (colHiOut) {
        h = __reduce_max_sync(0xffffffffu, h);
        if (lane == c) mine = h;
      }
    }
    if (mine) atomicMax(&cmax[t * kN + P.g * 16 + lane], mine);
    __syncthreads();
  }
  return true;
}

#define MRCQR_FIN_OZ_CTA(S, P)                         \
  extern __shared__ unsigned char smem_raw[];          \
  __shared__ __align__(8) uint64_t mma_bar[2];         \
  __shared__ uint32_t tmem_slot;                       \
  __shared__ uint32_t rowE_s[kM];                      \
  __shared__ uint32_t redE_s[4][kM];                   \
  __shared__ uint32_t cmax_s[512];                     \
  OzPipe P = oz_begin(&tmem_slot, mma_bar);            \
  FinOzCta S{oz_smem(smem_raw), rowE_s, redE_s, cmax_s};

__global__ void __launch_bounds__(kOzThreads, 1)
    k_finalize_oz(int64_t m, int n, int n64, double* __restrict__ Q, int64_t ldq, const uint32_t* __restrict__ colE,
                  const unsigned char* __restrict__ Xs, uint32_t* __restrict__ colHiOut, Ctl* ctl, int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  MRCQR_FIN_OZ_CTA(S, P)
  const FinOzArgs a{m, n, n64, Q, ldq, colE, Xs, colHiOut, ctl};
  fin_oz_begin(a, S);
  bool abort = false;
  const int64_t nblocks = (m + kM - 1) / kM;
  for (int64_t rb = blockIdx.x; rb < nblocks; rb += gridDim.x)
    if (!fin_oz_block(a, S, P, rb * kM)) {
      abort = true;
      break;
    }
  if (!abort) fin_oz_end(a, S);
  oz_end(P, abort, ctl);
}

// ---------------------------------------------------------------------------
// Gram G = W^T W (Algorithm 1 step 1) and the check matrix Q^T Q.  Every
// column of W is sliced against the exponent of its maximum over all m rows,
// so the level sums of all rows share one scale: a work item (output tile of
// 128 x 64 entries, slab of rows) reads its exact level sums out of TMEM
// every 128 rows into 64-bit integer pairs, and a reduction adds the items'
// 128-bit values (exact, so the order does not matter) and rounds each entry
// once.

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

// One work item (output tile, row slab) of the Gram W^T W; false when a wait
// timed out (every thread together).
// ti, tj: the tile's I block (128 columns) and J block (64 columns); rows
// [r_begin, min(m, r_begin + rows_per_slab)); the partial goes to part_item.
__device__ __forceinline__ bool syrk_oz_item(int64_t m, int n, const double* __restrict__ W, int64_t ldw,
                                             const uint32_t* __restrict__ colHi, int ti, int tj, int64_t r_begin,
                                             int64_t rows_per_slab, long long* __restrict__ part_item, OzPipe& P,
                                             unsigned char* smem, uint32_t* colE) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = kM * ti, j0 = kN * tj;
  const bool inner = (tj >> 1) == ti;   // J block inside the I block
  const int64_t r_end = min(m, r_begin + rows_per_slab);
  const int nchunks = r_end > r_begin ? (int)((r_end - r_begin + kK - 1) / kK) : 0;
  __syncthreads();
  if (tid < kM) colE[tid] = i0 + tid < n ? oz::exp_field(colHi[i0 + tid]) : 0u;
  else if (tid < kM + kN) colE[tid] = j0 + tid - kM < n ? oz::exp_field(colHi[j0 + tid - kM]) : 0u;
  __syncthreads();
  long long hi[16], lo[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) hi[c] = lo[c] = 0;
  double va[kM / 32][2];
  oz_load_cols<kM>(W, ldw, n, i0, r_begin, r_end, warp, lane, va);
  auto produce = [&](int ch, unsigned char* a, unsigned char* b) {
    const int64_t r0 = r_begin + (int64_t)ch * kK;
    oz_store_cols<kM>(va, colE, 0u, 0u, a, kAPanel, warp, lane, inner ? j0 - i0 : -1, b);
    if (ch + 1 < nchunks) oz_load_cols<kM>(W, ldw, n, i0, r0 + kK, r_end, warp, lane, va);
    if (!inner) {   // second operand of an off-diagonal tile: loaded and sliced at once
      double vb[kN / 32][2];
      oz_load_cols<kN>(W, ldw, n, j0, r0, r_end, warp, lane, vb);
      oz_store_cols<kN>(vb, colE + kM, 0u, 0u, b, kBPanel, warp, lane);
    }
  };
  if (!oz_run(P, smem, nchunks, produce, hi, lo)) return false;
  oz_store_partial(part_item, P.q, P.g, lane, hi, lo);
  return true;
}

__global__ void __launch_bounds__(kOzThreads, 1)
    k_syrk_oz(int64_t m, int n, const double* __restrict__ W, int64_t ldw, const uint32_t* __restrict__ colHi,
              SyrkOzPlan SP, long long* __restrict__ part, Ctl* ctl, int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = oz_smem(smem_raw);
  __shared__ __align__(8) uint64_t mma_bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ uint32_t colE[kM + kN];
  OzPipe P = oz_begin(&tmem_slot, mma_bar);
  bool abort = false;
  const int nitems = SP.ntiles * SP.slabs;
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int tile = item % SP.ntiles, slab = item / SP.ntiles;
    if (!syrk_oz_item(m, n, W, ldw, colHi, SP.ti[tile], SP.tj[tile], (int64_t)slab * SP.rows_per_slab,
                      SP.rows_per_slab, part + (size_t)item * kPartElems, P, smem, colE)) {
      abort = true;
      break;
    }
  }
  oz_end(P, abort, ctl);
}

// Upper triangle of G from the items' partials (exact 128-bit sums over the
// slabs, one rounding); lower triangle zero.
template <class Plan>
__device__ __forceinline__ void syrk_oz_reduce_entry(int n, const uint32_t* __restrict__ colHi, const Plan& SP,
                                                     const long long* __restrict__ part, double* __restrict__ out,
                                                     int64_t e) {
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e % n), j = (int)(e / n);
  if (i > j) {
    out[e] = 0.0;
    return;
  }
  const int I = i / kM, J = j / kN;
  const int tile = SP.tile_of[I][J];
  const oz::I128 acc =
      oz_sum_partials(part + (size_t)tile * kPartElems, SP.slabs, (size_t)SP.ntiles * kPartElems, i - I * kM, j - J * kN);
  const uint32_t Ei = oz::exp_field(colHi[i]), Ej = oz::exp_field(colHi[j]);
  out[e] = (Ei == 2047u || Ej == 2047u) ? nan64() : oz::i128_to_double(acc, (int)Ei + (int)Ej - oz::kScaleBias);
}

__global__ void k_syrk_oz_reduce(int n, const uint32_t* __restrict__ colHi, SyrkOzPlan SP,
                                 const long long* __restrict__ part, double* __restrict__ out, const Ctl* ctl,
                                 int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  syrk_oz_reduce_entry(n, colHi, SP, part, out, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
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
// One work item (128 columns of A, 64 sampled rows, row slab) of the FP64
// sketch; false when a wait timed out (every thread together).
__device__ __forceinline__ bool sketch_oz_item(int64_t m, int n, int s, const double* __restrict__ A, int64_t lda,
                                               const uint32_t* __restrict__ colHi, const uint32_t* __restrict__ idx,
                                               const double* __restrict__ tab, uint2 key, const SketchOzPlan& SP,
                                               long long* __restrict__ part, int tf, OzPipe& P,
                                               unsigned char* smem, uint32_t* colE, uint32_t* sgn, int item) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint64_t four_m = 4ull * (uint64_t)m;
  // signs of the rows r0 .. r0 + 31 as a bit mask, one Philox draw per lane of warp 1
  auto sign_mask = [&](int64_t r0, int64_t r_end) {
    const int64_t j = r0 + lane;
    const bool neg = j < r_end && row_sign((uint64_t)j, key) < 0.0;
    return __ballot_sync(0xffffffffu, neg);
  };
  const int ntiles_all = SP.mblocks * SP.ntiles;
  const int nitems = ntiles_all * SP.slabs;
  // transform-panel role: sample fi, rows 4 fg .. 4 fg + 3 of each chunk
  const int fi = tid & (kN - 1), fg = tid >> 6;
  // sign role: rows 2 (lane % 16), 2 (lane % 16) + 1 of each chunk
  const int sp = lane & 15;

  const int tile = item % ntiles_all, slab = item / ntiles_all;
  const int c0 = kM * (tile / SP.ntiles), i0 = kN * (tile % SP.ntiles);
  const int64_t r_begin = (int64_t)slab * SP.rows_per_slab;
  const int64_t r_end = min(m, r_begin + SP.rows_per_slab);
  const int nchunks = r_end > r_begin ? (int)((r_end - r_begin + kK - 1) / kK) : 0;
  __syncthreads();
  if (tid < kM) colE[tid] = c0 + tid < n ? oz::exp_field(colHi[c0 + tid]) : 0u;
  if (warp == 1) {
    const uint32_t mk = sign_mask(r_begin, r_end);
    if (lane == 0) sgn[0] = mk;
  }
  __syncthreads();
  // phase of (sample fi, row r_begin + 4 fg), its advance per chunk and per row
  const bool fval = i0 + fi < s;
  const RowPhase rp = row_phase(tf, fval ? idx[i0 + fi] : 0u, (uint64_t)m);
  uint64_t r = fval ? phase_at(rp, (uint64_t)(r_begin + 4 * fg), four_m) : 0ull;
  const uint64_t step_chunk = (rp.dk * (uint64_t)kK) % four_m;
  const uint64_t step_row = rp.dk;   // < 4m
  long long hi[16], lo[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) hi[c] = lo[c] = 0;
  // chunk 0 ahead: A values, table values of this thread's four rows
  double va[kM / 32][2];
  uint32_t whi[4], wlo[4];
  auto load_chunk = [&](int64_t r0) {
    oz_load_cols<kM>(A, lda, n, c0, r0, r_end, warp, lane, va);
    uint64_t rr = r;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      whi[t] = wlo[t] = 0u;
      if (fval && r0 + 4 * fg + t < r_end) cos_phase_bits(tab, (int64_t)rr, m, whi[t], wlo[t]);
      rr += step_row;
      if (rr >= four_m) rr -= four_m;
    }
    r += step_chunk;
    if (r >= four_m) r -= four_m;
  };
  load_chunk(r_begin);
  auto produce = [&](int ch, unsigned char* a, unsigned char* b) {
    const int64_t r0 = r_begin + (int64_t)ch * kK;
    // Rademacher signs of this lane's two rows (mask of this chunk made one chunk ahead by warp 1;
    // the pipeline's barrier between chunks publishes it)
    const uint32_t mk = sgn[ch & 1];
    const uint32_t f0 = (mk >> (2 * sp)) & 1u, f1 = (mk >> (2 * sp + 1)) & 1u;
    if (warp == 1 && ch + 1 < nchunks) {
      const uint32_t mk1 = sign_mask(r0 + kK, r_end);
      if (lane == 0) sgn[(ch + 1) & 1] = mk1;
    }
    oz_store_cols<kM>(va, colE, f0, f1, a, kAPanel, warp, lane);
#pragma unroll
    for (int t2 = 0; t2 < 2; ++t2)
      oz_store_pair(__hiloint2double((int)whi[2 * t2], (int)wlo[2 * t2]),
                    __hiloint2double((int)whi[2 * t2 + 1], (int)wlo[2 * t2 + 1]), 0u, 0u, 1023u,
                    b + tc::sw64_offset(fi, 4 * fg + 2 * t2, 2), kBPanel);
    if (ch + 1 < nchunks) load_chunk(r0 + kK);
  };
  if (!oz_run(P, smem, nchunks, produce, hi, lo)) return false;
  oz_store_partial(part + (size_t)item * kPartElems, P.q, P.g, lane, hi, lo);
  return true;
}

__global__ void __launch_bounds__(kOzThreads, 1)
    k_sketch_oz(int64_t m, int n, int s, const double* __restrict__ A, int64_t lda, const uint32_t* __restrict__ colHi,
                const uint32_t* __restrict__ idx, const double* __restrict__ tab, uint2 key, SketchOzPlan SP,
                long long* __restrict__ part, Ctl* ctl, int level, int tf) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = oz_smem(smem_raw);
  __shared__ __align__(8) uint64_t mma_bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ uint32_t colE[kM];
  __shared__ uint32_t sgn[2];   // Rademacher signs of a chunk's 32 rows (bit i: row r0 + i), by chunk parity
  OzPipe P = oz_begin(&tmem_slot, mma_bar);
  bool abort = false;
  const int nitems = SP.mblocks * SP.ntiles * SP.slabs;
  for (int item = blockIdx.x; item < nitems; item += gridDim.x)
    if (!sketch_oz_item(m, n, s, A, lda, colHi, idx, tab, key, SP, part, tf, P, smem, colE, sgn, item)) {
      abort = true;
      break;
    }
  oz_end(P, abort, ctl);
}

// Y (s x n, column-major) from the items' partials: exact sums over the
// slabs, one rounding, times the row's scale (DCT: sqrt(2/s) c_k; real FFT:
// sqrt(c/m) for c bins).  A non-finite column of A gives a NaN column and
// raises NONFINITE.
__device__ __forceinline__ void sketch_oz_reduce_entry(int n, int s, const uint32_t* __restrict__ colHi,
                                                       const uint32_t* __restrict__ idx, const SketchOzPlan& SP,
                                                       const long long* __restrict__ part, double* __restrict__ Y,
                                                       Ctl* ctl, int tf, int64_t m, int64_t e) {
  if (e >= (int64_t)s * n) return;
  const int i = (int)(e % s), c = (int)(e / s);
  const int tile = (c / kM) * SP.ntiles + i / kN;
  const oz::I128 acc = oz_sum_partials(part + (size_t)tile * kPartElems, SP.slabs,
                                       (size_t)SP.mblocks * SP.ntiles * kPartElems, c % kM, i % kN);
  const uint32_t Ec = oz::exp_field(colHi[c]);
  const double coef = tf == T_DCT ? sqrt(2.0 / (double)s) * (idx[i] == 0 ? 0.70710678118654752440 : 1.0)
                                  : sqrt((double)(tf == T_RFFT_REIM ? s / 2 : s) / (double)m);
  const double y = Ec == 2047u ? nan64() : oz::i128_to_double(acc, (int)Ec + 1023 - oz::kScaleBias) * coef;
  Y[e] = y;
  if (!isfinite(y)) {
    ctl->input_nonfinite = 1;
    raise_level_status(ctl, ST_NONFINITE);
  }
}

__global__ void k_sketch_oz_reduce(int n, int s, const uint32_t* __restrict__ colHi, const uint32_t* __restrict__ idx,
                                   SketchOzPlan SP, const long long* __restrict__ part, double* __restrict__ Y,
                                   Ctl* ctl, int level, int tf, int64_t m) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  sketch_oz_reduce_entry(n, s, colHi, idx, SP, part, Y, ctl, tf, m, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// W = A R^{-1} (Algorithm 2 step 7, R = R_s upper triangular; rows of W by
// substitution, Sec. II-A), blocked by 16 columns.  For sub-block J:
//   B_J = A_J - W_{<J} R_{<J,J}   emulated FP64 product (one rounding), then
//                                  one FP64 subtraction;
//   W_J = B_J R_JJ^{-1}           substitution in FP64 on the 16 x 16 block,
//                                  as the FMA kernel does it.
// The FP64 work falls from n^2/2 to 8n fused multiply-adds per row.  128 rows
// per work block, 256 threads, two CTAs per SM (one CTA's substitution runs
// while the other's MMAs do).  The product is formed as (W D)(D^-1 R) with
// D = diag(2^e_k), 2^e_k the binade of the largest entry of row k of R: a
// graded R (rows falling by many orders, the usual shape of R_s) then pairs
// balanced operands, and the digit error stays relative to |W| |R| as in
// substitution.  W's digits are taken against the running maxima of the rows
// of W D, R's against the column maxima of D^-1 R above the diagonal block.
constexpr int kTB = 16;                           // sub-block width = MMA N
constexpr int kTThreads = 256;
constexpr uint32_t kTAPanel = kM * 64;            // one digit, 128 rows x 32 K (8 KiB)
constexpr uint32_t kTBPanel = kTB * 64;           // one digit, 16 rows x 32 K (1 KiB)
constexpr size_t kTSmem = (size_t)oz::kSlices * (kTAPanel + kTBPanel) + sizeof(double) * kM * kTB + 1024;

// e_k = unbiased exponent of max_c |R[k][c]| (0 for a zero row): the
// diagonal scaling of the product.  One warp per row.
__device__ __forceinline__ void oz_row_scale_block(int n, int npad, const double* __restrict__ RT,
                                                   int* __restrict__ eR, int blk) {
  const int k = blk * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (k >= n) return;
  uint32_t mx = 0u;
  for (int c = lane; c < n; c += 32) mx = max(mx, (uint32_t)__double2hiint(RT[(int64_t)k * npad + c]) & 0x7FFFFFFFu);
  mx = __reduce_max_sync(0xffffffffu, mx);
  if (lane == 0) {
    const int E = (int)oz::exp_field(mx);
    eR[k] = (E == 0 || E == 2047) ? 0 : E - 1023;
  }
}

__global__ void __launch_bounds__(256) k_oz_row_scale(int n, int npad, const double* __restrict__ RT,
                                                      int* __restrict__ eR, const Ctl* ctl, int level) {
  if (ctl && (level_inactive(ctl, level) || ctl->lvl_status != 0)) return;
  oz_row_scale_block(n, npad, RT, eR, blockIdx.x);
}

// Digits of D^-1 R: panel (J, kc) holds columns [16J, 16J+16) (as rows) and
// rows k in [32kc, 32kc+32) of R 2^-e_k, zero for k >= 16J; colE[c] = the
// largest exponent of R[k][c] 2^-e_k over k < 16 (c / 16) (2047 when a used
// entry is not finite).  RT[k][c] = R[k][c], row stride npad.
__device__ __forceinline__ void oz_prep_r_col(int n, int npad, int nkc, const double* __restrict__ RT,
                                              const int* __restrict__ eR, int* __restrict__ colE,
                                              unsigned char* __restrict__ Rd, uint32_t* __restrict__ colHiOut, int nhi,
                                              int c, int* red, int* bad) {
  // c: column, < 16 ceil(n / 16)
  if (colHiOut && c == 0)     // the TRSM folds the column maxima of W into these
    for (int i = threadIdx.x; i < nhi; i += blockDim.x) colHiOut[i] = 0u;
  const int J = c / kTB, kend = kTB * J;
  __syncthreads();
  int mx = -100000, nf = 0;
  for (int k = threadIdx.x; k < kend; k += blockDim.x)
    if (c < n) {
      const int E = (int)oz::exp_field((uint32_t)__double2hiint(RT[(int64_t)k * npad + c]));
      if (E == 2047) nf = 1;
      else if (E != 0) mx = max(mx, E - eR[k]);
    }
  mx = __reduce_max_sync(0xffffffffu, mx);
  nf = __reduce_or_sync(0xffffffffu, nf);
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = mx;
    bad[threadIdx.x >> 5] = nf;
  }
  __syncthreads();
  int E = red[0], anybad = bad[0];
  for (int w = 1; w < 8; ++w) {
    E = max(E, red[w]);
    anybad |= bad[w];
  }
  if (E == -100000) E = 0;   // no nonzero entry: every digit is zero
  if (threadIdx.x == 0) colE[c] = anybad ? 2047 : E;
  const int nch = (kend + kK - 1) / kK;
  for (int k = threadIdx.x; k < nch * kK; k += blockDim.x) {
    int d[oz::kSlices];
    const double x = (c < n && k < kend) ? RT[(int64_t)k * npad + c] : 0.0;
    oz::digits8((uint32_t)__double2hiint(x), (uint32_t)__double2loint(x), E, d, k < n ? -eR[k] : 0);
    unsigned char* panel = Rd + (size_t)(J * nkc + k / kK) * oz::kSlices * kTBPanel;
#pragma unroll
    for (int b = 0; b < oz::kSlices; ++b)
      *reinterpret_cast<__half*>(panel + b * kTBPanel + tc::sw64_offset(c % kTB, k % kK, 2)) =
          __float2half_rn(oz::small_int_to_float(d[b]));
  }
}

__global__ void __launch_bounds__(256) k_oz_prep_r(int n, int npad, int nkc, const double* __restrict__ RT,
                                                   const int* __restrict__ eR, int* __restrict__ colE,
                                                   unsigned char* __restrict__ Rd, uint32_t* __restrict__ colHiOut,
                                                   int nhi, const Ctl* ctl, int level) {
  if (ctl && (level_inactive(ctl, level) || ctl->lvl_status != 0)) return;
  __shared__ int red[8];
  __shared__ int bad[8];
  oz_prep_r_col(n, npad, nkc, RT, eR, colE, Rd, colHiOut, nhi, blockIdx.x, red, bad);
}

// W = A R^{-1} for one problem: arguments of the kernel body.
struct TrsmOzArgs {
  int64_t m;
  int n;
  const double* A;
  int64_t lda;
  const double* RT;
  const double* rinv;
  const int* eR;
  const int* colE;
  const unsigned char* Rd;
  int nkc;
  double* W;
  int64_t ldw;
  uint32_t* colHiOut;
  Ctl* ctl;
};

// Shared-memory state of one CTA of the TRSM.
struct TrsmOzCta {
  unsigned char* as;     // 8 digit panels of W, 128 rows x 32 K
  unsigned char* bs;     // 8 digit panels of D^-1 R, 16 rows x 32 K
  double* Bblk;          // [16][128] right-hand sides of the diagonal block
  uint64_t* bar;
  uint32_t tmem;
  uint32_t commits;      // MMA batches committed (the same count in every thread)
  int* rowX;             // running max exponent of W D per row (kNonfinite: a non-finite entry)
  int* eRs;              // e_k of the problem
  double (*Rd16)[kTB + 1];
  double* rinv16;
  uint32_t* cmax;        // column maxima of |W| (high words) over this CTA's rows of the problem
};

constexpr int kNoEntry = -100000, kNonfinite = 100000;

// The problem's e_k into shared memory, column maxima cleared.
__device__ __forceinline__ void trsm_oz_begin(const TrsmOzArgs& a, TrsmOzCta& S) {
  __syncthreads();
  for (int k = threadIdx.x; k < a.n; k += kTThreads) {
    S.eRs[k] = a.eR[k];
    S.cmax[k] = 0u;
  }
  __syncthreads();
}

// This CTA's column maxima of W folded into the problem's.
__device__ __forceinline__ void trsm_oz_end(const TrsmOzArgs& a, TrsmOzCta& S) {
  __syncthreads();
  if (a.colHiOut)
    for (int k = threadIdx.x; k < a.n; k += kTThreads)
      if (S.cmax[k]) atomicMax(a.colHiOut + k, S.cmax[k]);
  __syncthreads();
}

// One block of 128 rows starting at r0.  False when a wait timed out (every
// thread returns false together).
__device__ __forceinline__ bool trsm_oz_block(const TrsmOzArgs& a, TrsmOzCta& S, int64_t r0) {
  const int64_t m = a.m;
  const int n = a.n;
  const double* __restrict__ A = a.A;
  const int64_t lda = a.lda;
  const double* __restrict__ RT = a.RT;
  const double* __restrict__ rinv = a.rinv;
  const int* __restrict__ colE = a.colE;
  const unsigned char* __restrict__ Rd = a.Rd;
  const int nkc = a.nkc;
  double* W = a.W;
  const int64_t ldw = a.ldw;
  uint32_t* colHiOut = a.colHiOut;
  unsigned char* as = S.as;
  unsigned char* bs = S.bs;
  double* Bblk = S.Bblk;
  const uint32_t tmem = S.tmem;
  uint32_t& commits = S.commits;
  int* rowX = S.rowX;
  int* eRs = S.eRs;
  double(*Rd16)[kTB + 1] = S.Rd16;
  double* rinv16 = S.rinv16;
  uint32_t* cmax = S.cmax;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3, g = warp >> 2;   // readout: lanes 32 q.., columns 8 g..8 g + 7
  const int npad = (n + 31) / 32 * 32;
  const int nsub = (n + kTB - 1) / kTB;
  const int pr = tid & (kM - 1), ph = tid >> 7;   // producer role: row pr, 16-byte chunks 2 ph, 2 ph + 1
  if (tid < kM) rowX[tid] = kNoEntry;
  __syncthreads();
  for (int J = 0; J < nsub; ++J) {
    const int c0 = J * kTB;
    // diagonal block and reciprocals of this sub-block
    {
      const int a = tid / kTB, b = tid % kTB;   // 256 threads = 16 x 16
      Rd16[a][b] = (c0 + a < n && c0 + b < n) ? RT[(int64_t)(c0 + a) * npad + c0 + b] : 0.0;
      if (tid < kTB) rinv16[tid] = rinv[c0 + tid];
    }
    // B_J = A_J - W_{<J} R_{<J,J}, thread (row 32 q + lane, columns 8 g .. 8 g + 7)
    const int rr = q * 32 + lane;
    const bool rlive = r0 + rr < m;
    double bv[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int col = c0 + 8 * g + c;
      bv[c] = (rlive && col < n) ? A[r0 + rr + (int64_t)col * lda] : 0.0;
    }
    if (J > 0) {
      long long hi[8], lo[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) hi[c] = lo[c] = 0;
      const int nch = (c0 + kK - 1) / kK;
      const bool plive = r0 + pr < m;
      const int Er = rowX[pr];
      for (int kc = 0; kc < nch; ++kc) {
        // R digits of (J, kc): 8 KiB, two asynchronous 16-byte copies per thread
        const uint4* src = reinterpret_cast<const uint4*>(Rd + (size_t)(J * nkc + kc) * oz::kSlices * kTBPanel);
#pragma unroll
        for (int i = 0; i < 2; ++i) tc::cp_async16(bs + 16 * (tid + kTThreads * i), src + tid + kTThreads * i);
        // W digits of columns [32 kc, 32 kc + 32) (zero from c0 on): row pr, the eight column
        // pairs of 16-byte chunks 2 ph and 2 ph + 1; lane group lane / 8 rotates through the
        // chunk's four pairs, so a warp's 4-byte panel stores hit 32 banks
        const int lg = lane >> 3;
        auto pair_of = [&](int i) { return 4 * (2 * ph + (i & 1)) + ((lg + (i >> 1)) & 3); };
        double v[8][2];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int k0 = kc * kK + 2 * pair_of(i);
          v[i][0] = (plive && k0 < c0) ? W[r0 + pr + (int64_t)k0 * ldw] : 0.0;
          v[i][1] = (plive && k0 + 1 < c0) ? W[r0 + pr + (int64_t)(k0 + 1) * ldw] : 0.0;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int k0 = kc * kK + 2 * pair_of(i);
          oz_store_pair(v[i][0], v[i][1], 0u, 0u, Er, as + tc::sw64_offset(pr, 2 * pair_of(i), 2), kTAPanel,
                        k0 < n ? eRs[k0] : 0, k0 + 1 < n ? eRs[k0 + 1] : 0);
        }
        tc::cp_async_wait_all();
        tc::fence_proxy_async();
        tc::fence_before();
        __syncthreads();
        if (tid == 0) {
          tc::fence_after();
          const uint64_t da = tc::sw64_desc(tc::smem_u32(as)), db = tc::sw64_desc(tc::smem_u32(bs));
          const uint32_t first = (kc % kGroupChunks) == 0 ? 0u : 1u;
          // one MMA per A digit against the stacked R digits 0 .. 7 - a (N = 16 (8 - a))
#pragma unroll
          for (int kk = 0; kk < kK; kk += 16)
#pragma unroll
            for (int a = 0; a < oz::kLevels; ++a)
              tc::mma_f16(tmem + (uint32_t)(a * kTB), da + (uint64_t)((a * kTAPanel + kk * 2) >> 4),
                          db + (uint64_t)((kk * 2) >> 4), tc::idesc(tc::F16, kM, kTB * (oz::kLevels - a)),
                          (a == 0 && kk == 0) ? first : 1u);
          tc::mma_commit(S.bar);
        }
        const bool ok = tc::mbar_wait(S.bar, commits & 1u);
        ++commits;
        if (__syncthreads_or(!ok)) return false;
        tc::fence_after();
        if (kc % kGroupChunks == kGroupChunks - 1 || kc == nch - 1) {
          const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(g * 8);
#pragma unroll 1
          for (int L = 0; L < oz::kLevels; ++L) {
            float f[8];
            tc::tmem_ld8(base + (uint32_t)(L * kTB), f);
            tc::tmem_wait_ld();
#pragma unroll
            for (int c = 0; c < 8; ++c) oz::add_level(L, f[c], hi[c], lo[c]);
          }
        }
        tc::fence_before();
        __syncthreads();   // panels and accumulators free for the next chunk
      }
      const int Erow = rowX[rr];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int col = c0 + 8 * g + c;
        if (col < n) {
          const int ce = colE[col];
          const double p = (Erow == kNonfinite || ce == 2047)
                               ? nan64()
                               : oz::i128_to_double(hi[c], lo[c], Erow + ce - oz::kScaleBias);
          bv[c] -= p;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) Bblk[(8 * g + c) * kM + rr] = bv[c];
    __syncthreads();
    // substitution on the diagonal block, one thread per row
    if (tid < kM) {
      double t[kTB];
#pragma unroll
      for (int c = 0; c < kTB; ++c) t[c] = Bblk[c * kM + tid];
      int mx = rowX[tid];
#pragma unroll
      for (int c = 0; c < kTB; ++c) {
        t[c] *= rinv16[c];
#pragma unroll
        for (int c2 = c + 1; c2 < kTB; ++c2) t[c2] = fma(-t[c], Rd16[c][c2], t[c2]);
      }
      if (r0 + tid < m) {
#pragma unroll
        for (int c = 0; c < kTB; ++c)
          if (c0 + c < n) {
            W[r0 + tid + (int64_t)(c0 + c) * ldw] = t[c];
            const int E = (int)oz::exp_field((uint32_t)__double2hiint(t[c]));
            if (E == 2047) mx = kNonfinite;
            else if (E != 0 && mx != kNonfinite) mx = max(mx, E + eRs[c0 + c]);
          }
      }
      rowX[tid] = mx;
      if (colHiOut) {   // lane c keeps the warp's maximum of column c0 + c
        uint32_t mine = 0u;
#pragma unroll
        for (int c = 0; c < kTB; ++c) {
          const uint32_t h = (r0 + tid < m && c0 + c < n) ? ((uint32_t)__double2hiint(t[c]) & 0x7FFFFFFFu) : 0u;
          const uint32_t wm = __reduce_max_sync(0xffffffffu, h);
          if (lane == c) mine = wm;
        }
        if (mine) atomicMax(&cmax[c0 + lane], mine);
      }
    }
    __syncthreads();
  }
  return true;
}

// CTA prologue of the TRSM kernels: shared-memory state, TMEM (128 columns)
// and the MMA barrier, gathered in the TrsmOzCta named S.
#define MRCQR_TRSM_OZ_CTA(S)                                                   \
  extern __shared__ unsigned char smem_raw[];                                  \
  unsigned char* smem = oz_smem(smem_raw);                                     \
  __shared__ __align__(8) uint64_t mma_bar;                                    \
  __shared__ uint32_t tmem_slot;                                               \
  __shared__ int rowX_s[kM];                                                   \
  __shared__ int eRs_s[512];                                                   \
  __shared__ double Rd16_s[kTB][kTB + 1];                                      \
  __shared__ double rinv16_s[kTB];                                             \
  __shared__ uint32_t cmax_s[512];                                             \
  if ((threadIdx.x >> 5) == 0) tc::tmem_alloc(&tmem_slot, 128);                \
  if (threadIdx.x == 0) {                                                      \
    tc::mbar_init(&mma_bar, 1);                                                \
    tc::mbar_fence_init();                                                     \
  }                                                                            \
  tc::fence_before();                                                          \
  __syncthreads();                                                             \
  tc::fence_after();                                                           \
  TrsmOzCta S;                                                                 \
  S.as = smem;                                                                 \
  S.bs = smem + oz::kSlices * kTAPanel;                                        \
  S.Bblk = reinterpret_cast<double*>(S.bs + oz::kSlices * kTBPanel);           \
  S.bar = &mma_bar;                                                            \
  S.tmem = tmem_slot;                                                          \
  S.commits = 0;                                                               \
  S.rowX = rowX_s;                                                             \
  S.eRs = eRs_s;                                                               \
  S.Rd16 = Rd16_s;                                                             \
  S.rinv16 = rinv16_s;                                                         \
  S.cmax = cmax_s;

__device__ __forceinline__ void trsm_oz_cta_end(TrsmOzCta& S, bool abort, Ctl* ctl) {
  if (abort && threadIdx.x == 0 && ctl) raise_level_status(ctl, ST_TIMEOUT);
  tc::fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(S.tmem, 128);
}

__global__ void __launch_bounds__(kTThreads, 2)
    k_trsm_oz(int64_t m, int n, const double* __restrict__ A, int64_t lda, const double* __restrict__ RT,
              const double* __restrict__ rinv, const int* __restrict__ eR, const int* __restrict__ colE,
              const unsigned char* __restrict__ Rd, int nkc, double* W, int64_t ldw, uint32_t* __restrict__ colHiOut,
              Ctl* ctl, int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  MRCQR_TRSM_OZ_CTA(S)
  const TrsmOzArgs a{m, n, A, lda, RT, rinv, eR, colE, Rd, nkc, W, ldw, colHiOut, ctl};
  trsm_oz_begin(a, S);
  bool abort = false;
  const int64_t nblocks = (m + kM - 1) / kM;
  for (int64_t rb = blockIdx.x; rb < nblocks; rb += gridDim.x)
    if (!trsm_oz_block(a, S, rb * kM)) {
      abort = true;
      break;
    }
  if (!abort) trsm_oz_end(a, S);
  trsm_oz_cta_end(S, abort, ctl);
}


// ---------------------------------------------------------------------------
// Grouped forms for batched plans (many problems of uneven m and n): one
// persistent launch per kernel walks a work list of {problem, block} items
// with a grid-stride loop; an item whose problem is not active at this
// escalation level, or has raised a status, is skipped.  The per-item work is
// the single-problem kernels' body; a CTA that moves on to another problem
// folds its column maxima into the previous one's first.

__device__ __forceinline__ bool oz_live(const Prob& P, int level) {
  return P.ctl->active == level && P.ctl->lvl_status == 0;
}

__device__ __forceinline__ int oz_nhi(int n) { return (n + kM - 1) / kM * kM; }

// Column maxima of A (high words of |a|), one column per item, entries
// n .. nhi - 1 zero.
__global__ void __launch_bounds__(256) kg_oz_colhi(Group g, int level) {
  __shared__ uint32_t red[8];
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (!oz_live(P, level)) continue;
    const int j = w.y;
    uint32_t mx = 0u;
    if (j < P.n) {
      const double* col = P.A + (int64_t)j * P.lda;
      for (int64_t r = threadIdx.x; r < P.m; r += 256)
        mx = max(mx, (uint32_t)__double2hiint(__ldg(col + r)) & 0x7FFFFFFFu);
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t v = red[0];
      for (int k = 1; k < 8; ++k) v = max(v, red[k]);
      P.oz_colhi[j] = v;
    }
  }
}

__global__ void __launch_bounds__(kOzThreads, 1) kg_oz_sketch(Group g, int level) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = oz_smem(smem_raw);
  __shared__ __align__(8) uint64_t mma_bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ uint32_t colE[kM];
  __shared__ uint32_t sgn[2];
  OzPipe pipe = oz_begin(&tmem_slot, mma_bar);
  bool abort = false;
  Ctl* actl = nullptr;
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (!oz_live(P, level)) continue;
    if (!sketch_oz_item(P.m, P.n, P.s, P.A, P.lda, P.oz_colhi, P.idx, P.tab, P.key, P.oz_kp, P.oz_part, P.tf, pipe,
                        smem, colE, sgn, w.y)) {
      abort = true;
      actl = P.ctl;
      break;
    }
  }
  oz_end(pipe, abort, actl);
}

__global__ void __launch_bounds__(256) kg_oz_sketch_reduce(Group g, int level) {
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (!oz_live(P, level)) continue;
    sketch_oz_reduce_entry(P.n, P.s, P.oz_colhi, P.idx, P.oz_kp, P.oz_part, P.y, P.ctl, P.tf, P.m,
                           (int64_t)w.y * 256 + threadIdx.x);
  }
}

__global__ void __launch_bounds__(256) kg_oz_row_scale(Group g, int level) {
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (!oz_live(P, level)) continue;
    oz_row_scale_block(P.n, P.npad, P.rst, P.oz_cole + (P.n + kTB - 1) / kTB * kTB, w.y);
  }
}

__global__ void __launch_bounds__(256) kg_oz_prep_r(Group g, int level) {
  __shared__ int red[8];
  __shared__ int bad[8];
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (!oz_live(P, level)) continue;
    const int n16 = (P.n + kTB - 1) / kTB * kTB;
    oz_prep_r_col(P.n, P.npad, (P.n + kK - 1) / kK, P.rst, P.oz_cole + n16, P.oz_cole, P.oz_rd, P.oz_colhi,
                  oz_nhi(P.n), w.y, red, bad);
  }
}

__device__ __forceinline__ TrsmOzArgs trsm_args_of(const Prob& P) {
  const int n16 = (P.n + kTB - 1) / kTB * kTB;
  return TrsmOzArgs{P.m, P.n, P.A, P.lda, P.rst, P.rinv, P.oz_cole + n16, P.oz_cole, P.oz_rd, (P.n + kK - 1) / kK,
                    P.Q, P.ldq, P.oz_colhi, P.ctl};
}

__global__ void __launch_bounds__(kTThreads, 2) kg_oz_trsm(Group g, int level) {
  MRCQR_TRSM_OZ_CTA(S)
  __shared__ TrsmOzArgs a;   // the current problem's arguments (shared: not held in registers)
  bool abort = false;
  int cur = -1;
  Ctl* actl = nullptr;
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (!oz_live(P, level)) continue;
    if (w.x != cur) {
      if (cur >= 0) trsm_oz_end(a, S);
      __syncthreads();
      if (threadIdx.x == 0) a = trsm_args_of(P);
      trsm_oz_begin(a, S);
      cur = w.x;
    }
    if (!trsm_oz_block(a, S, (int64_t)w.y * kM)) {
      abort = true;
      actl = P.ctl;
      break;
    }
  }
  if (!abort && cur >= 0) trsm_oz_end(a, S);
  trsm_oz_cta_end(S, abort, actl);
}

__global__ void __launch_bounds__(kOzThreads, 1) kg_oz_syrk(Group g, int level) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = oz_smem(smem_raw);
  __shared__ __align__(8) uint64_t mma_bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ uint32_t colE[kM + kN];
  OzPipe pipe = oz_begin(&tmem_slot, mma_bar);
  bool abort = false;
  Ctl* actl = nullptr;
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (!oz_live(P, level)) continue;
    const int tile = w.y % P.oz_sp.ntiles, slab = w.y / P.oz_sp.ntiles;
    if (!syrk_oz_item(P.m, P.n, P.Q, P.ldq, P.oz_colhi, P.oz_sp.ti[tile], P.oz_sp.tj[tile],
                      (int64_t)slab * P.oz_sp.rows_per_slab, P.oz_sp.rows_per_slab,
                      P.oz_part + (size_t)w.y * kPartElems, pipe, smem, colE)) {
      abort = true;
      actl = P.ctl;
      break;
    }
  }
  oz_end(pipe, abort, actl);
}

__global__ void __launch_bounds__(256) kg_oz_syrk_reduce(Group g, int check, int level) {
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (!oz_live(P, level)) continue;
    syrk_oz_reduce_entry(P.n, P.oz_colhi, P.oz_sp, P.oz_part, check ? P.e : P.rc, (int64_t)w.y * 256 + threadIdx.x);
  }
}

__global__ void __launch_bounds__(512) kg_oz_prep_x(Group g, int level) {
  __shared__ uint32_t red[32];
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (!oz_live(P, level)) continue;
    oz_prep_x_col(P.n, P.npad, (P.n + kN - 1) / kN * kN, P.xt, P.oz_xe, P.oz_xs, P.check ? P.oz_colhi : nullptr,
                  oz_nhi(P.n), w.y, red);
  }
}

__global__ void __launch_bounds__(kOzThreads, 1) kg_oz_finalize(Group g, int level) {
  MRCQR_FIN_OZ_CTA(S, pipe)
  __shared__ FinOzArgs a;   // the current problem's arguments (shared: not held in registers)
  bool abort = false;
  int cur = -1;
  Ctl* actl = nullptr;
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (!oz_live(P, level)) continue;
    if (w.x != cur) {
      if (cur >= 0) fin_oz_end(a, S);
      __syncthreads();
      if (threadIdx.x == 0)
        a = FinOzArgs{P.m, P.n, (P.n + kN - 1) / kN * kN, P.Q, P.ldq, P.oz_xe, P.oz_xs,
                      P.check ? P.oz_colhi : nullptr, P.ctl};
      fin_oz_begin(a, S);
      cur = w.x;
    }
    if (!fin_oz_block(a, S, pipe, (int64_t)w.y * kM)) {
      abort = true;
      actl = P.ctl;
      break;
    }
  }
  if (!abort && cur >= 0) fin_oz_end(a, S);
  oz_end(pipe, abort, actl);
}

int num_sms() {
  static int cached = 0;
  if (!cached) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cached = sms > 0 ? sms : 152;
  }
  return cached;
}

int gcd_int(int a, int b) { return b ? gcd_int(b, a % b) : a; }

// Row slabs so that tiles x slabs is a multiple of the SM count where the
// rows allow it; at least 256 rows per slab, at most 2^20 (the 64-bit halves
// of an item stay below 2^61).
int choose_slabs(int64_t m, int tiles, int64_t* rows_per_slab) {
  const int sms = num_sms();
  int slabs = tiles >= sms ? 1 : sms / gcd_int(tiles, sms);
  const int64_t max_slabs = (m + 255) / 256;
  if (slabs > max_slabs) slabs = (int)max_slabs;
  const int64_t min_slabs = (m + (1 << 20) - 1) >> 20;
  if (slabs < min_slabs) slabs = (int)min_slabs;
  if (slabs < 1) slabs = 1;
  int64_t rps = (m + slabs - 1) / slabs;
  rps = (rps + kK - 1) / kK * kK;
  *rows_per_slab = rps;
  return (int)((m + rps - 1) / rps);
}

void launch_col_hi(int64_t m, int n, const double* X, int64_t ldx, uint32_t* colHi, const Ctl* ctl, int level,
                   cudaStream_t st);

template <class K>
void set_smem(K kernel) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
}

}  // namespace

int oz_x_cols(int n) { return (n + kN - 1) / kN * kN; }

size_t oz_xs_bytes(int n) {
  const int n64 = oz_x_cols(n);
  return (size_t)oz::kSlices * (n64 / kN) * (n64 / kK) * kBPanel;
}

size_t syrk_oz_colhi_bytes(int n) { return sizeof(uint32_t) * (size_t)((n + kM - 1) / kM * kM); }

namespace {
void launch_col_hi(int64_t m, int n, const double* X, int64_t ldx, uint32_t* colHi, const Ctl* ctl, int level,
                   cudaStream_t st) {
  cudaMemsetAsync(colHi, 0, syrk_oz_colhi_bytes(n), st);
  int ysplit = (4 * num_sms() + n - 1) / n;
  const int64_t max_y = (m + 4095) / 4096;
  if (ysplit > max_y) ysplit = (int)max_y;
  if (ysplit < 1) ysplit = 1;
  { ::mrcqr::note_launch(); k_col_hi<<<dim3(n, ysplit), 256, 0, st>>>(m, n, X, ldx, (m + ysplit - 1) / ysplit, colHi, ctl, level); }
}
}  // namespace

void launch_oz_col_hi(int64_t m, int n, const double* X, int64_t ldx, uint32_t* colHi, const Ctl* ctl, int level,
                      cudaStream_t st) {
  launch_col_hi(m, n, X, ldx, colHi, ctl, level, st);
}

void launch_sketch_oz_reduce(int n, int s, const uint32_t* colHi, const uint32_t* idx, const SketchOzPlan& P,
                             const long long* part, double* Y, Ctl* ctl, int level, cudaStream_t st, int tf,
                             int64_t m) {
  const int64_t total = (int64_t)s * n;
  { ::mrcqr::note_launch(); k_sketch_oz_reduce<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(n, s, colHi, idx, P, part, Y, ctl, level, tf, m); }
}

void launch_finalize_oz(int64_t m, int n, double* Q, int64_t ldq, const double* XT, uint32_t* colE,
                        unsigned char* Xs, Ctl* ctl, int level, cudaStream_t st, uint32_t* colHiOut) {
  const int npad = (n + 31) / 32 * 32;
  const int n64 = (n + kN - 1) / kN * kN;
  const int nhi = (int)(syrk_oz_colhi_bytes(n) / sizeof(uint32_t));
  { ::mrcqr::note_launch(); k_oz_prep_x<<<n64, 512, 0, st>>>(n, npad, n64, XT, colE, Xs, colHiOut, nhi, ctl, level); }
  set_smem(k_finalize_oz);
  const int64_t nblocks = (m + kM - 1) / kM;
  const unsigned grid = (unsigned)(nblocks < num_sms() ? nblocks : num_sms());
  { ::mrcqr::note_launch(); k_finalize_oz<<<grid, kOzThreads, kSmem, st>>>(m, n, n64, Q, ldq, colE, Xs, colHiOut, ctl, level); }
}

SyrkOzPlan syrk_oz_plan(int64_t m, int n, int64_t rows_per_slab) {
  SyrkOzPlan P{};
  const int nI = (n + kM - 1) / kM, nJ = (n + kN - 1) / kN;
  for (int I = 0; I < 4; ++I)
    for (int J = 0; J < 8; ++J) P.tile_of[I][J] = -1;
  for (int I = 0; I < nI; ++I)
    for (int J = 0; J < nJ; ++J)
      if (kN * J + kN - 1 >= kM * I) {
        P.ti[P.ntiles] = (int8_t)I;
        P.tj[P.ntiles] = (int8_t)J;
        P.tile_of[I][J] = (int8_t)P.ntiles;
        ++P.ntiles;
      }
  if (rows_per_slab > 0) {   // a given slab height (32-row multiple, at most 2^20 rows: the 64-bit halves stay exact)
    int64_t rps = (rows_per_slab + kK - 1) / kK * kK;
    if (rps > (int64_t(1) << 20)) rps = int64_t(1) << 20;
    P.rows_per_slab = rps;
    P.slabs = (int)((m + rps - 1) / rps);
    if (P.slabs < 1) P.slabs = 1;
  } else {
    P.slabs = choose_slabs(m, P.ntiles, &P.rows_per_slab);
  }
  return P;
}

size_t syrk_oz_part_bytes(const SyrkOzPlan& P) { return sizeof(long long) * kPartElems * (size_t)P.ntiles * P.slabs; }

void launch_syrk_oz(int64_t m, int n, const double* W, int64_t ldw, const SyrkOzPlan& P, uint32_t* colHi,
                    long long* part, double* out, Ctl* ctl, int level, cudaStream_t st, bool colhi_ready) {
  if (!colhi_ready) launch_col_hi(m, n, W, ldw, colHi, ctl, level, st);
  set_smem(k_syrk_oz);
  const int nitems = P.ntiles * P.slabs;
  { ::mrcqr::note_launch(); k_syrk_oz<<<nitems < num_sms() ? nitems : num_sms(), kOzThreads, kSmem, st>>>(m, n, W, ldw, colHi, P, part, ctl,
                                                                               level); }
  const int64_t nn = (int64_t)n * n;
  { ::mrcqr::note_launch(); k_syrk_oz_reduce<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(n, colHi, P, part, out, ctl, level); }
}


SketchOzPlan sketch_oz_plan(int64_t m, int n, int s) {
  SketchOzPlan P{};
  P.mblocks = (n + kM - 1) / kM;
  P.ntiles = (s + kN - 1) / kN;
  P.slabs = choose_slabs(m, P.mblocks * P.ntiles, &P.rows_per_slab);
  return P;
}

size_t sketch_oz_part_bytes(const SketchOzPlan& P) {
  return sizeof(long long) * kPartElems * (size_t)P.mblocks * P.ntiles * P.slabs;
}

void launch_sketch_oz(int64_t m, int n, int s, const double* A, int64_t lda, const uint32_t* idx, const double* tab,
                      uint64_t seed, const SketchOzPlan& P, uint32_t* colHi, long long* part, double* Y, Ctl* ctl,
                      int level, cudaStream_t st, int tf) {
  launch_col_hi(m, n, A, lda, colHi, ctl, level, st);
  set_smem(k_sketch_oz);
  const int nitems = P.mblocks * P.ntiles * P.slabs;
  { ::mrcqr::note_launch(); k_sketch_oz<<<nitems < num_sms() ? nitems : num_sms(), kOzThreads, kSmem, st>>>(m, n, s, A, lda, colHi, idx, tab,
                                                                                 seed_key(seed), P, part, ctl, level, tf); }
  launch_sketch_oz_reduce(n, s, colHi, idx, P, part, Y, ctl, level, st, tf, m);
}

size_t trsm_oz_rd_bytes(int n) {
  const int nsub = (n + kTB - 1) / kTB, nkc = (n + kK - 1) / kK;
  return (size_t)nsub * nkc * oz::kSlices * kTBPanel;
}

size_t trsm_oz_cole_bytes(int n) { return 2 * sizeof(int) * (size_t)((n + kTB - 1) / kTB * kTB); }

void launch_trsm_oz(int64_t m, int n, const double* A, int64_t lda, const double* RT, const double* rinv,
                    uint32_t* colE_ws, unsigned char* Rd, double* W, int64_t ldw, Ctl* ctl, int level, cudaStream_t st,
                    uint32_t* colHiOut) {
  const int npad = (n + 31) / 32 * 32;
  const int nkc = (n + kK - 1) / kK;
  const int nhi = (int)(syrk_oz_colhi_bytes(n) / sizeof(uint32_t));
  const int64_t nblocks = (m + kM - 1) / kM;
  const int64_t slots = 2 * (int64_t)num_sms();
  const unsigned grid = (unsigned)(nblocks < slots ? nblocks : slots);
  const int n16 = (n + kTB - 1) / kTB * kTB;
  int* colE = reinterpret_cast<int*>(colE_ws);
  int* eR = colE + n16;
  { ::mrcqr::note_launch(); k_oz_row_scale<<<(n + 7) / 8, 256, 0, st>>>(n, npad, RT, eR, ctl, level); }
  { ::mrcqr::note_launch(); k_oz_prep_r<<<n16, 256, 0, st>>>(n, npad, nkc, RT, eR, colE, Rd, colHiOut, nhi, ctl, level); }
  cudaFuncSetAttribute(k_trsm_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTSmem);
  { ::mrcqr::note_launch(); k_trsm_oz<<<grid, kTThreads, kTSmem, st>>>(m, n, A, lda, RT, rinv, eR, colE, Rd, nkc, W, ldw,
                                                                  colHiOut, ctl, level); }
}

// ---- grouped launches -------------------------------------------------------
namespace {
unsigned grid_oz(int nitems, int per_sm) {
  const int cap = num_sms() * per_sm;
  return (unsigned)(nitems < cap ? nitems : cap);
}
}  // namespace

void prepare_g_oz_kernels() {
  cudaFuncSetAttribute(kg_oz_sketch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  cudaFuncSetAttribute(kg_oz_syrk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  cudaFuncSetAttribute(kg_oz_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  cudaFuncSetAttribute(kg_oz_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTSmem);
}

void launch_g_oz_colhi(const Group& g, int level, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_oz_colhi<<<grid_oz(g.nitems, 16), 256, 0, st>>>(g, level); }
}
void launch_g_oz_sketch(const Group& g, int level, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_oz_sketch<<<grid_oz(g.nitems, 1), kOzThreads, kSmem, st>>>(g, level); }
}
void launch_g_oz_sketch_reduce(const Group& g, int level, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_oz_sketch_reduce<<<grid_oz(g.nitems, 16), 256, 0, st>>>(g, level); }
}
void launch_g_oz_row_scale(const Group& g, int level, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_oz_row_scale<<<grid_oz(g.nitems, 16), 256, 0, st>>>(g, level); }
}
void launch_g_oz_prep_r(const Group& g, int level, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_oz_prep_r<<<grid_oz(g.nitems, 16), 256, 0, st>>>(g, level); }
}
void launch_g_oz_trsm(const Group& g, int level, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_oz_trsm<<<grid_oz(g.nitems, 2), kTThreads, kTSmem, st>>>(g, level); }
}
void launch_g_oz_syrk(const Group& g, bool check, int level, cudaStream_t st) {
  (void)check;   // the item's problem record names W or Q (the Q buffer holds W before the finalize)
  if (g.nitems) { ::mrcqr::note_launch(); kg_oz_syrk<<<grid_oz(g.nitems, 1), kOzThreads, kSmem, st>>>(g, level); }
}
void launch_g_oz_syrk_reduce(const Group& g, bool check, int level, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_oz_syrk_reduce<<<grid_oz(g.nitems, 16), 256, 0, st>>>(g, check ? 1 : 0, level); }
}
void launch_g_oz_prep_x(const Group& g, int level, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_oz_prep_x<<<grid_oz(g.nitems, 8), 512, 0, st>>>(g, level); }
}
void launch_g_oz_finalize(const Group& g, int level, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_oz_finalize<<<grid_oz(g.nitems, 1), kOzThreads, kSmem, st>>>(g, level); }
}

}  // namespace mrcqr
