// Stage 2 and 3 of MRCQR (Algorithm 2 steps 7-9, Algorithm 1, Sec. II-A), all
// in FP64: W = A R_s^{-1} by substitution, G = W^T W, R_c = chol(G), the
// orthogonal factor Q = W R_c^{-1}, R = R_c R_s, and the orthogonality check
// E = Q^T Q that judges the result (Sec. II-C: a precision that was too low
// shows as ||I - Q^T Q|| >> u and triggers a rerun at the next precision).
//
// FP64 on this GPU runs at ~1/64 of the FP32 rate and has no tensor-core
// path, so these kernels are FP64-pipe bound for every n >= 4: each one is a
// plain SIMT kernel that keeps the DFMA pipe fed (independent accumulators,
// broadcast operand loads), and memory traffic is secondary.
#include "kernels.h"

namespace mrcqr {

constexpr int kNC = 32;   // column chunk of the row-per-thread kernels
constexpr int kPad = 32;  // row stride padding of the transposed triangles

static inline int padded(int n) { return (n + kPad - 1) / kPad * kPad; }

// ---------------------------------------------------------------------------
// W = A R_s^{-1}: every row w of W solves w R_s = a by substitution
// (Algorithm 2 step 7, the paper's dtrsm), w_j = (a_j - sum_{k<j} w_k R_kj) / R_jj.
// One thread per row; columns in chunks of 32 held in registers; finished
// columns are read back from W (the Q buffer).  R_s comes transposed
// (row-major, row stride npad, zero padding) so a row segment is one
// contiguous uniform load.
__device__ __forceinline__ void trsm_row(int64_t r, int n, const double* __restrict__ A, int64_t lda,
                                         const double* __restrict__ RT, const double* __restrict__ rinv,
                                         double* __restrict__ W, int64_t ldw) {
  const int npad = (n + kPad - 1) / kPad * kPad;
  for (int J0 = 0; J0 < n; J0 += kNC) {
    double t[kNC];
#pragma unroll
    for (int c = 0; c < kNC; ++c) t[c] = (J0 + c < n) ? A[r + (int64_t)(J0 + c) * lda] : 0.0;
    for (int k = 0; k < J0; ++k) {
      const double wk = W[r + (int64_t)k * ldw];
      const double2* Rk = reinterpret_cast<const double2*>(RT + (int64_t)k * npad + J0);
#pragma unroll
      for (int c2 = 0; c2 < kNC / 2; ++c2) {
        const double2 rv = __ldg(Rk + c2);
        t[2 * c2] = fma(-wk, rv.x, t[2 * c2]);
        t[2 * c2 + 1] = fma(-wk, rv.y, t[2 * c2 + 1]);
      }
    }
#pragma unroll
    for (int c = 0; c < kNC; ++c) {
      t[c] *= __ldg(rinv + J0 + c);
      const double* Rc = RT + (int64_t)(J0 + c) * npad + J0;
      if (J0 + c < n) {
#pragma unroll
        for (int c2 = c + 1; c2 < kNC; ++c2) t[c2] = fma(-t[c], __ldg(Rc + c2), t[c2]);
      }
    }
#pragma unroll
    for (int c = 0; c < kNC; ++c)
      if (J0 + c < n) W[r + (int64_t)(J0 + c) * ldw] = t[c];
  }
}

__global__ void __launch_bounds__(128) k_trsm(int64_t m, int n, const double* __restrict__ A, int64_t lda,
                                              const double* __restrict__ RT, const double* __restrict__ rinv,
                                              double* __restrict__ W, int64_t ldw, const Ctl* ctl, int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < m) trsm_row(r, n, A, lda, RT, rinv, W, ldw);
}

void launch_trsm(int64_t m, int n, const double* A, int64_t lda, const double* RT, const double* rinv, double* W,
                 int64_t ldw, const Ctl* ctl, int level, cudaStream_t st) {
  { ::mrcqr::note_launch(); k_trsm<<<(unsigned)((m + 127) / 128), 128, 0, st>>>(m, n, A, lda, RT, rinv, W, ldw, ctl, level); }
}

// ---------------------------------------------------------------------------
// Partial Gram matrices X^T X (upper triangle) over row splits: the Gram
// step of Algorithm 1 (the paper uses dgemm; computing only the upper
// triangle is the same arithmetic per entry).  A CTA owns one TN x TN tile
// (ti <= tj) and one row split; each warp owns a 16 x 16 block and skips it
// when it lies strictly below the diagonal.  Lane (li, lj) computes rows
// li*4..+4 and columns lj*2..+2 of its block.  Partials are summed in a
// fixed order by the consumer (deterministic).
template <int TN>
__device__ __forceinline__ void syrk_block(int64_t m, int n, const double* __restrict__ X, int64_t ldx,
                                           int64_t rows_per_split, int ntile, double* __restrict__ Gpart,
                                           int tile, int split) {
  constexpr int KB = 32;
  constexpr int NB = TN / 16;          // 16x16 blocks per tile side
  constexpr int NT = 32 * NB * NB;     // threads
  __shared__ __align__(16) double Xi[KB][TN];
  __shared__ __align__(16) double Xj[KB][TN];
  // tile index -> (ti, tj), ti <= tj, row-major over the upper triangle
  int t = tile, ti = 0;
  while (t >= ntile - ti) { t -= ntile - ti; ++ti; }
  const int tj = ti + t;
  const int i0 = ti * TN, j0 = tj * TN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int bi = warp / NB, bj = warp % NB;
  const bool active = !(ti == tj && bi > bj);
  const int li = lane & 3, lj = lane >> 2;
  const int rbase = bi * 16 + li * 4, cbase = bj * 16 + lj * 2;
  const int64_t k_begin = (int64_t)split * rows_per_split;
  const int64_t k_end = min(m, k_begin + rows_per_split);
  double acc[4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = 0.0;
  for (int64_t k0 = k_begin; k0 < k_end; k0 += KB) {
    __syncthreads();
    for (int e = tid; e < KB * TN; e += NT) {
      const int kk = e % KB, c = e / KB;
      const int64_t row = k0 + kk;
      const bool okr = row < k_end;
      Xi[kk][c] = (okr && i0 + c < n) ? X[row + (int64_t)(i0 + c) * ldx] : 0.0;
      if (ti != tj) Xj[kk][c] = (okr && j0 + c < n) ? X[row + (int64_t)(j0 + c) * ldx] : 0.0;
    }
    __syncthreads();
    if (active) {
      const double(*Xb)[TN] = (ti == tj) ? Xi : Xj;
#pragma unroll 8
      for (int kk = 0; kk < KB; ++kk) {
        const double2 b = *reinterpret_cast<const double2*>(&Xb[kk][cbase]);
        double a[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) a[q] = Xi[kk][rbase + q];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[q][0] = fma(a[q], b.x, acc[q][0]);
          acc[q][1] = fma(a[q], b.y, acc[q][1]);
        }
      }
    }
  }
  __syncthreads();
  if (!active) return;
  double* out = Gpart + (size_t)split * (size_t)n * (size_t)n;
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int gi = i0 + rbase + q, gj = j0 + cbase + c;
      if (gi < n && gj < n && gi <= gj) out[(int64_t)gj * n + gi] = acc[q][c];
    }
}

template <int TN>
__global__ void __launch_bounds__(32 * (TN / 16) * (TN / 16)) k_syrk(int64_t m, int n, const double* __restrict__ X,
                                                                      int64_t ldx, int64_t rows_per_split, int ntile,
                                                                      double* __restrict__ Gpart, const Ctl* ctl,
                                                                      int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  syrk_block<TN>(m, n, X, ldx, rows_per_split, ntile, Gpart, blockIdx.x, blockIdx.y);
}

static int syrk_tile(int n) { return n <= 16 ? 16 : (n <= 32 ? 32 : 64); }
int syrk_tile_for(int n) { return syrk_tile(n); }

// CTAs of k_syrk<TN> that fit on the GPU at once (SMs x resident CTAs per SM).
static int syrk_slots(int TN) {
  static int cached[3] = {0, 0, 0};
  const int slot = TN == 16 ? 0 : (TN == 32 ? 1 : 2);
  if (cached[slot] == 0) {
    int dev = 0, sms = 152, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int threads = 32 * (TN / 16) * (TN / 16);
    if (TN == 16) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_syrk<16>, threads, 0);
    else if (TN == 32) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_syrk<32>, threads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_syrk<64>, threads, 0);
    cudaGetLastError();
    cached[slot] = sms * (per > 0 ? per : 1);
  }
  return cached[slot];
}

int syrk_splits(int64_t m, int n) {
  const int TN = syrk_tile(n);
  const int nt = (n + TN - 1) / TN;
  const int tiles = nt * (nt + 1) / 2;
  // about eight full waves of CTAs, so the last partial wave costs little;
  // each split keeps at least 64 rows
  int splits = (8 * syrk_slots(TN) + tiles - 1) / tiles;
  const int64_t maxs = (m + 63) / 64;
  if (splits > maxs) splits = (int)maxs;
  return splits < 1 ? 1 : splits;
}

void launch_syrk(int64_t m, int n, const double* X, int64_t ldx, int splits, double* Gpart, const Ctl* ctl, int level,
                 cudaStream_t st) {
  const int TN = syrk_tile(n);
  const int nt = (n + TN - 1) / TN;
  const int tiles = nt * (nt + 1) / 2;
  int64_t rps = (m + splits - 1) / splits;
  rps = (rps + 31) / 32 * 32;
  const dim3 grid(tiles, splits);
  if (TN == 16) { ::mrcqr::note_launch(); k_syrk<16><<<grid, 32, 0, st>>>(m, n, X, ldx, rps, nt, Gpart, ctl, level); }
  else if (TN == 32) { ::mrcqr::note_launch(); k_syrk<32><<<grid, 128, 0, st>>>(m, n, X, ldx, rps, nt, Gpart, ctl, level); }
  else { ::mrcqr::note_launch(); k_syrk<64><<<grid, 512, 0, st>>>(m, n, X, ldx, rps, nt, Gpart, ctl, level); }
}

// ---------------------------------------------------------------------------
// Sum of the per-split Gram partials, upper triangle, in a fixed order (one
// thread per entry; deterministic).  Lower triangle set to zero.
__device__ __forceinline__ void reduce_partial_entry(int n, int splits, const double* __restrict__ part,
                                                     double* __restrict__ out, int64_t e) {
  const int64_t nn = (int64_t)n * n;
  const int i = (int)(e % n), j = (int)(e / n);
  double v = 0.0;
  if (i <= j)
    for (int sp = 0; sp < splits; ++sp) v += part[(size_t)sp * nn + e];
  out[e] = v;
}

__global__ void k_reduce_partials(int n, int splits, const double* __restrict__ part, double* __restrict__ out,
                                  const Ctl* ctl, int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < (int64_t)n * n) reduce_partial_entry(n, splits, part, out, e);
}

void launch_reduce_partials(int n, int splits, const double* part, double* out, const Ctl* ctl, int level,
                            cudaStream_t st) {
  const int64_t nn = (int64_t)n * n;
  { ::mrcqr::note_launch(); k_reduce_partials<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(n, splits, part, out, ctl, level); }
}

// ---------------------------------------------------------------------------
// Cholesky of the Gram matrix (Algorithm 1 step 2): G = R_c^T R_c, R_c
// upper with positive diagonal, in place on the reduced upper triangle with
// right-looking elimination (one CTA).  A non-positive or non-finite pivot
// raises BREAKDOWN for this level.
// Returns false (for every thread) on breakdown.
__device__ __forceinline__ bool chol_block(int n, double* __restrict__ G) {
  const int tid = threadIdx.x;
  const int64_t nn = (int64_t)n * n;
  __shared__ double piv, ipiv;
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      const double d = G[(int64_t)k * n + k];
      piv = (d > 0.0 && isfinite(d)) ? sqrt(d) : -1.0;
      ipiv = piv > 0.0 ? 1.0 / piv : 0.0;
      if (piv > 0.0) G[(int64_t)k * n + k] = piv;
    }
    __syncthreads();
    const double p = piv;
    if (!(p > 0.0)) {
      __syncthreads();
      return false;
    }
    const double ip = ipiv;
    for (int j = k + 1 + tid; j < n; j += blockDim.x) G[(int64_t)j * n + k] *= ip;   // row k
    __syncthreads();
    // trailing update G[i][j] -= R[k][i] R[k][j], k < i <= j: lanes over
    // rows i (coalesced within a column), warps over columns j
    const int tx = tid & 31, ty = tid >> 5;
    for (int j = k + 1 + ty; j < n; j += 32) {
      const double rkj = G[(int64_t)j * n + k];
      for (int i = k + 1 + tx; i <= j; i += 32)
        G[(int64_t)j * n + i] = fma(-G[(int64_t)i * n + k], rkj, G[(int64_t)j * n + i]);
    }
    __syncthreads();
  }
  for (int64_t e = tid; e < nn; e += blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (i > j) G[e] = 0.0;
  }
  __syncthreads();
  return true;
}

__global__ void __launch_bounds__(1024) k_chol(int n, double* __restrict__ G, Ctl* ctl, int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  if (!chol_block(n, G) && threadIdx.x == 0) raise_level_status(ctl, ST_BREAKDOWN);
}

// The same elimination with the upper triangle of G held in shared memory
// (n <= kCholSmemN); the finished row k of R_c goes straight to G.
constexpr int kCholSmemN = 160;

__global__ void __launch_bounds__(1024) k_chol_smem(int n, double* __restrict__ G, Ctl* ctl, int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  extern __shared__ double S[];   // S[j n + i] = G[i][j], i <= j
  __shared__ double piv, ipiv;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int64_t nn = (int64_t)n * n;
  for (int64_t e = tid; e < nn; e += blockDim.x) S[e] = G[e];
  __syncthreads();
  bool ok = true;
  for (int k = 0; k < n; ++k) {
    // one thread forms the pivot and its reciprocal: the FP64 sqrt and division are
    // long sequences on a 1/64-rate pipe, not to be repeated by every warp
    if (tid == 0) {
      const double d = S[(int64_t)k * n + k];
      piv = (d > 0.0 && isfinite(d)) ? sqrt(d) : -1.0;
      ipiv = piv > 0.0 ? 1.0 / piv : 0.0;
    }
    __syncthreads();
    const double p = piv;
    if (!(p > 0.0)) {
      ok = false;
      break;
    }
    const double ip = ipiv;
    for (int j = k + 1 + tid; j < n; j += blockDim.x) {
      const double r = S[(int64_t)j * n + k] * ip;
      S[(int64_t)j * n + k] = r;
      G[(int64_t)j * n + k] = r;
    }
    if (tid == 0) G[(int64_t)k * n + k] = p;
    __syncthreads();
    for (int j = k + 1 + ty; j < n; j += 32) {
      const double rkj = S[(int64_t)j * n + k];
      for (int i = k + 1 + tx; i <= j; i += 32)
        S[(int64_t)j * n + i] = fma(-S[(int64_t)i * n + k], rkj, S[(int64_t)j * n + i]);
    }
    __syncthreads();
  }
  if (!ok) {
    if (tid == 0) raise_level_status(ctl, ST_BREAKDOWN);
    return;
  }
  for (int64_t e = tid; e < nn; e += blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (i > j) G[e] = 0.0;
  }
}

// Blocked right-looking Cholesky over many CTAs (n > kCholBlockedMin): the
// single-CTA elimination puts all n^3/3 FP64 flops on one SM's 1/64-rate
// FP64 pipe (5.4 ms at n = 512), here the trailing updates spread over the
// GPU.  Panels of kCB = 32 columns; for the panel at columns c0 .. c0 + 31:
//   k_chol_diag    R_pp = chol(G_pp): one warp, lane j holds column j of the
//                  block, pivots broadcast by shuffles (no block barriers);
//   k_chol_panel   R_{p,j} = R_pp^{-T} G_{p,j} for the columns j beyond the
//                  panel: forward substitution, one warp per column;
//   k_chol_update  G_ij -= R_{p,i}^T R_{p,j} on the trailing upper triangle,
//                  one CTA per 32 x 32 tile.
// Same arithmetic per entry as the elimination (a sum over k of products,
// one FMA each), a different order of the updates.  A pivot that is not
// positive and finite raises BREAKDOWN; the later launches then return.
constexpr int kCB = 32;
constexpr int kCholBlockedMin = 64;

__global__ void __launch_bounds__(32) k_chol_diag(int n, int c0, double* __restrict__ G, Ctl* ctl, int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  const int lane = threadIdx.x;
  const int w = min(kCB, n - c0);
  const int64_t col = (int64_t)(c0 + lane) * n + c0;   // column c0 + lane, row c0
  double g[kCB];
#pragma unroll
  for (int i = 0; i < kCB; ++i) g[i] = (lane < w && i <= lane) ? G[col + i] : 0.0;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < kCB; ++k) {
    if (k >= w) break;
    const double d = __shfl_sync(0xffffffffu, g[k], k);
    const double piv = (d > 0.0 && isfinite(d)) ? sqrt(d) : -1.0;
    if (!(piv > 0.0)) {
      ok = false;
      break;
    }
    const double ip = 1.0 / piv;
    if (lane == k) g[k] = piv;
    else if (lane > k) g[k] *= ip;                      // r_k,lane
#pragma unroll
    for (int i = k + 1; i < kCB; ++i) {
      const double rki = __shfl_sync(0xffffffffu, g[k], i);
      if (i <= lane) g[i] = fma(-rki, g[k], g[i]);
    }
  }
  if (!ok) {
    if (lane == 0) raise_level_status(ctl, ST_BREAKDOWN);
    return;
  }
  if (lane < w) {
#pragma unroll
    for (int i = 0; i < kCB; ++i)
      if (i < w) G[col + i] = i <= lane ? g[i] : 0.0;
  }
}

__global__ void __launch_bounds__(256) k_chol_panel(int n, int c0, double* __restrict__ G, const Ctl* ctl,
                                                    int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  __shared__ double Rp[kCB][kCB + 1];   // Rp[t][i] = R[c0 + t][c0 + i]
  __shared__ double rdiag[kCB];
  const int tid = threadIdx.x, lane = tid & 31;
  for (int e = tid; e < kCB * kCB; e += blockDim.x) {
    const int t = e % kCB, i = e / kCB;
    Rp[t][i] = G[(int64_t)(c0 + i) * n + c0 + t];
  }
  __syncthreads();
  if (tid < kCB) rdiag[tid] = 1.0 / Rp[tid][tid];
  __syncthreads();
  const int j = c0 + kCB + blockIdx.x * 8 + (tid >> 5);
  if (j >= n) return;
  double* colj = G + (int64_t)j * n + c0;
  double b = colj[lane];
#pragma unroll
  for (int t = 0; t < kCB; ++t) {
    const double xt = __shfl_sync(0xffffffffu, b, t) * rdiag[t];
    if (lane == t) b = xt;
    else if (lane > t) b = fma(-Rp[t][lane], xt, b);
  }
  colj[lane] = b;
  G[(int64_t)(c0 + lane) * n + j] = 0.0;   // strict lower triangle of the panel columns
}

__global__ void __launch_bounds__(256) k_chol_update(int n, int c0, double* __restrict__ G, const Ctl* ctl,
                                                     int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  const int c1 = c0 + kCB;
  // tile (I, J), I <= J, of the trailing upper triangle, numbered column by column
  int J = 0, b = blockIdx.x;
  while (b > J) {
    b -= J + 1;
    ++J;
  }
  const int I = b;
  __shared__ double PI[kCB][kCB], PJ[kCB][kCB];   // P[t][i] = R[c0 + t][c1 + 32 X + i]
  const int tid = threadIdx.x;
  for (int e = tid; e < kCB * kCB; e += blockDim.x) {
    const int t = e % kCB, i = e / kCB;
    const int ci = c1 + kCB * I + i, cj = c1 + kCB * J + i;
    PI[t][i] = ci < n ? G[(int64_t)ci * n + c0 + t] : 0.0;
    PJ[t][i] = cj < n ? G[(int64_t)cj * n + c0 + t] : 0.0;
  }
  __syncthreads();
  const int ii = tid & 31, gi = c1 + kCB * I + ii;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int jj = (tid >> 5) + 8 * q, gj = c1 + kCB * J + jj;
    if (gi >= n || gj >= n || gi > gj) continue;
    double acc = G[(int64_t)gj * n + gi];
#pragma unroll 8
    for (int t = 0; t < kCB; ++t) acc = fma(-PI[t][ii], PJ[t][jj], acc);
    G[(int64_t)gj * n + gi] = acc;
  }
}

void launch_chol(int n, double* G, Ctl* ctl, int level, cudaStream_t st) {
  if (n > kCholBlockedMin) {
    for (int c0 = 0; c0 < n; c0 += kCB) {
      { ::mrcqr::note_launch(); k_chol_diag<<<1, 32, 0, st>>>(n, c0, G, ctl, level); }
      const int ncols = n - c0 - kCB;
      if (ncols <= 0) break;
      { ::mrcqr::note_launch(); k_chol_panel<<<(ncols + 7) / 8, 256, 0, st>>>(n, c0, G, ctl, level); }
      const int T = (ncols + kCB - 1) / kCB;
      { ::mrcqr::note_launch(); k_chol_update<<<T * (T + 1) / 2, 256, 0, st>>>(n, c0, G, ctl, level); }
    }
    return;
  }
  if (n <= kCholSmemN) {
    const size_t smem = sizeof(double) * (size_t)n * n;
    cudaFuncSetAttribute(k_chol_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(double) * kCholSmemN * kCholSmemN));
    { ::mrcqr::note_launch(); k_chol_smem<<<1, 1024, smem, st>>>(n, G, ctl, level); }
    return;
  }
  { ::mrcqr::note_launch(); k_chol<<<1, 1024, 0, st>>>(n, G, ctl, level); }
}

// ---------------------------------------------------------------------------
// X = R_c^{-1} (upper): column j by back substitution, one thread per column.
// R_c is well conditioned after preconditioning, so forming its inverse and
// applying it as a product (instead of a second substitution) keeps FP64
// orthogonality; the paper's warning against explicit inverses concerns the
// ill-conditioned R_s (Sec. II-A).  Output transposed: XT[k][j] = X[k][j]
// stored row-major with row stride npad, zeros below the diagonal and in
// the padding.
__device__ __forceinline__ void trinv_column(int n, const double* __restrict__ Rc, double* __restrict__ XT, int j) {
  const int npad = (n + kPad - 1) / kPad * kPad;
  for (int i = j + 1; i < n; ++i) XT[(int64_t)i * npad + j] = 0.0;
  if (j >= n) {
    for (int i = 0; i < n; ++i) XT[(int64_t)i * npad + j] = 0.0;
    return;
  }
  XT[(int64_t)j * npad + j] = 1.0 / Rc[(int64_t)j * n + j];
  for (int i = j - 1; i >= 0; --i) {
    double acc = 0.0;
    for (int k = i + 1; k <= j; ++k) acc = fma(Rc[(int64_t)k * n + i], XT[(int64_t)k * npad + j], acc);
    XT[(int64_t)i * npad + j] = -acc / Rc[(int64_t)i * n + i];
  }
}

// Single-problem form: one warp per column j, which solves R_c x = e_j by a
// backward column sweep (x_i = b_i / R_ii, then b_k -= R_ki x_i for k < i);
// lane l holds rows l + 32 t (t < NT, 32 NT >= n), so every step is one
// broadcast and NT independent FMAs instead of a serial dot product.
template <int NT>
__global__ void __launch_bounds__(128) k_trinv(int n, const double* __restrict__ Rc, double* __restrict__ XT,
                                               const Ctl* ctl, int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  __shared__ double rdiag[32 * NT];
  for (int i = threadIdx.x; i < n; i += blockDim.x) rdiag[i] = 1.0 / Rc[(int64_t)i * n + i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int npad = (n + kPad - 1) / kPad * kPad;
  if (j >= npad) return;
  if (j >= n) {
    for (int i = lane; i < n; i += 32) XT[(int64_t)i * npad + j] = 0.0;
    return;
  }
  for (int i = j + 1 + lane; i < n; i += 32) XT[(int64_t)i * npad + j] = 0.0;
  double b[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) b[t] = (lane + 32 * t == j) ? 1.0 : 0.0;
  for (int i = j; i >= 0; --i) {
    const int ti = i >> 5, li = i & 31;
    double bi = 0.0;
#pragma unroll
    for (int t = 0; t < NT; ++t)
      if (t == ti) bi = b[t];
    const double xi = __shfl_sync(0xffffffffu, bi, li) * rdiag[i];
    const double* col = Rc + (int64_t)i * n;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int k = lane + 32 * t;
      if (k < i) b[t] = fma(-col[k], xi, b[t]);
      else if (k == i) b[t] = xi;
    }
  }
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int k = lane + 32 * t;
    if (k <= j) XT[(int64_t)k * npad + j] = b[t];
  }
}

void launch_trinv(int n, const double* Rc, double* RcinvT, const Ctl* ctl, int level, cudaStream_t st) {
  const int npad = padded(n);
  const unsigned grid = (unsigned)((npad + 3) / 4);
  if (n <= 64) { ::mrcqr::note_launch(); k_trinv<2><<<grid, 128, 0, st>>>(n, Rc, RcinvT, ctl, level); }
  else if (n <= 128) { ::mrcqr::note_launch(); k_trinv<4><<<grid, 128, 0, st>>>(n, Rc, RcinvT, ctl, level); }
  else if (n <= 256) { ::mrcqr::note_launch(); k_trinv<8><<<grid, 128, 0, st>>>(n, Rc, RcinvT, ctl, level); }
  else { ::mrcqr::note_launch(); k_trinv<16><<<grid, 128, 0, st>>>(n, Rc, RcinvT, ctl, level); }
}

// R = R_c R_s (Algorithm 2 step 9), upper x upper; R col-major with ld ldr,
// strict lower triangle set to zero.
__device__ __forceinline__ void rmul_entry(int n, const double* __restrict__ Rc, const double* __restrict__ Rs,
                                           double* __restrict__ R, int64_t ldr, int64_t e) {
  const int i = (int)(e % n), j = (int)(e / n);
  double acc = 0.0;
  for (int k = i; k <= j; ++k) acc = fma(Rc[(int64_t)k * n + i], Rs[(int64_t)j * n + k], acc);
  R[(int64_t)j * ldr + i] = (i <= j) ? acc : 0.0;
}

__global__ void k_rmul(int n, const double* __restrict__ Rc, const double* __restrict__ Rs, double* __restrict__ R,
                       int64_t ldr, const Ctl* ctl, int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < (int64_t)n * n) rmul_entry(n, Rc, Rs, R, ldr, e);
}

void launch_rmul(int n, const double* Rc, const double* Rs, double* R, int64_t ldr, const Ctl* ctl, int level,
                 cudaStream_t st) {
  const int64_t nn = (int64_t)n * n;
  { ::mrcqr::note_launch(); k_rmul<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(n, Rc, Rs, R, ldr, ctl, level); }
}

// ---------------------------------------------------------------------------
// Q = W X in place (X = R_c^{-1} upper): q_j = sum_{k<=j} w_k X_kj.  One
// thread per row; column chunks right to left so every chunk reads only
// columns that are still W.
__device__ __forceinline__ void finalize_row(int64_t r, int n, double* __restrict__ Q, int64_t ldq,
                                             const double* __restrict__ XT) {
  const int npad = (n + kPad - 1) / kPad * kPad;
  const int last = (n - 1) / kNC * kNC;
  for (int J0 = last; J0 >= 0; J0 -= kNC) {
    double acc[kNC];
#pragma unroll
    for (int c = 0; c < kNC; ++c) acc[c] = 0.0;
    for (int k = 0; k < J0; ++k) {
      const double wk = Q[r + (int64_t)k * ldq];
      const double2* Xk = reinterpret_cast<const double2*>(XT + (int64_t)k * npad + J0);
#pragma unroll
      for (int c2 = 0; c2 < kNC / 2; ++c2) {
        const double2 xv = __ldg(Xk + c2);
        acc[2 * c2] = fma(wk, xv.x, acc[2 * c2]);
        acc[2 * c2 + 1] = fma(wk, xv.y, acc[2 * c2 + 1]);
      }
    }
#pragma unroll
    for (int kc = 0; kc < kNC; ++kc) {
      if (J0 + kc < n) {
        const double wk = Q[r + (int64_t)(J0 + kc) * ldq];
        const double* Xk = XT + (int64_t)(J0 + kc) * npad + J0;
#pragma unroll
        for (int c = kc; c < kNC; ++c) acc[c] = fma(wk, __ldg(Xk + c), acc[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < kNC; ++c)
      if (J0 + c < n) Q[r + (int64_t)(J0 + c) * ldq] = acc[c];
  }
}

__global__ void __launch_bounds__(128) k_finalize(int64_t m, int n, double* __restrict__ Q, int64_t ldq,
                                                  const double* __restrict__ XT, const Ctl* ctl, int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < m) finalize_row(r, n, Q, ldq, XT);
}

// X (column-major, ld ldx, upper triangle read) into the transposed padded
// triangle XT[k][j] = X[k][j] (k <= j), zero elsewhere.
__global__ void k_upper_to_xt(int n, int npad, const double* __restrict__ X, int64_t ldx, double* __restrict__ XT) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * npad) return;
  const int k = (int)(e / npad), j = (int)(e % npad);
  XT[e] = (j < n && k <= j) ? X[k + (int64_t)j * ldx] : 0.0;
}

void launch_upper_to_xt(int n, const double* X, int64_t ldx, double* XT, cudaStream_t st) {
  const int npad = padded(n);
  const int64_t total = (int64_t)n * npad;
  { ::mrcqr::note_launch(); k_upper_to_xt<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(n, npad, X, ldx, XT); }
}

void launch_finalize(int64_t m, int n, double* Q, int64_t ldq, const double* XT, const Ctl* ctl, int level,
                     cudaStream_t st) {
  { ::mrcqr::note_launch(); k_finalize<<<(unsigned)((m + 127) / 128), 128, 0, st>>>(m, n, Q, ldq, XT, ctl, level); }
}

// ---------------------------------------------------------------------------
// Judge (Sec. II-C): e = ||I - Q^T Q||_F from the check partials (fixed
// order); accept, or escalate to the next level, or give up.
// One CTA: ||I - E||_F from the reduced check matrix, then accept / escalate /
// give up (thread 0 writes the control block).
__device__ __forceinline__ void judge_block(int n, const double* __restrict__ E, int check, Ctl* ctl, int level) {
  __shared__ double red[33];
  const int64_t nn = (int64_t)n * n;
  double part = 0.0;
  const bool run_check = check && ctl->lvl_status == 0;
  if (run_check) {
    for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) {
      const int i = (int)(e % n), j = (int)(e / n);
      if (i > j) continue;
      const double v = E[e] - (i == j ? 1.0 : 0.0);
      part += (i == j ? 1.0 : 2.0) * v * v;
    }
  }
  const double ss = block_sum(part, red);
  if (threadIdx.x == 0) {
    const double e = run_check ? sqrt(ss) : 0.0;
    const bool ok = ctl->lvl_status == 0 && e <= ctl->tol;   // NaN fails
    if (ok) {
      ctl->final_status = ST_OK;
      ctl->prec_used = ctl->lvl_prec[level];
      ctl->ortho_fro = e;
      ctl->active = -1;
    } else if (ctl->input_nonfinite) {
      ctl->final_status = ST_NONFINITE;
      ctl->prec_used = ctl->lvl_prec[level];
      ctl->ortho_fro = e;
      ctl->active = -1;
    } else if (level + 1 < ctl->nlevels) {
      ctl->retries += 1;
      ctl->lvl_status = 0;
      ctl->active = level + 1;
    } else {
      ctl->final_status = ctl->lvl_status ? ctl->lvl_status : ST_ORTHO;
      ctl->prec_used = ctl->lvl_prec[level];
      ctl->ortho_fro = e;
      ctl->active = -1;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(1024) k_judge(int n, const double* __restrict__ E, int check, Ctl* ctl,
                                                int level) {
  if (level_inactive(ctl, level)) return;
  judge_block(n, E, check, ctl, level);
}

void launch_judge(int n, const double* E, int check, Ctl* ctl, int level, cudaStream_t st) {
  { ::mrcqr::note_launch(); k_judge<<<1, 1024, 0, st>>>(n, E, check, ctl, level); }
}

// ---------------------------------------------------------------------------
// Grouped kernels (batched factorizations): the same bodies over a work list.
namespace {

constexpr int kGridCap = 152 * 8;

inline unsigned grid_for(int nitems) { return (unsigned)(nitems < kGridCap ? (nitems > 0 ? nitems : 1) : kGridCap); }

__device__ __forceinline__ bool item_live(const Prob& P, int level) {
  return P.ctl->active == level && P.ctl->lvl_status == 0;
}

__global__ void __launch_bounds__(128) kg_trsm(Group g, int level) {
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (!item_live(P, level)) continue;
    const int64_t r = (int64_t)w.y * 128 + threadIdx.x;
    if (r < P.m) trsm_row(r, P.n, P.A, P.lda, P.rst, P.rinv, P.Q, P.ldq);
  }
}

template <int TN>
__global__ void __launch_bounds__(32 * (TN / 16) * (TN / 16)) kg_syrk(Group g, int level) {
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (!item_live(P, level)) continue;
    syrk_block<TN>(P.m, P.n, P.Q, P.ldq, P.rows_per_split, P.ntile_syrk, P.gpart, w.y, w.z);
  }
}

__global__ void kg_reduce(Group g, int check, int level) {
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (!item_live(P, level)) continue;
    const int64_t e = (int64_t)w.y * 256 + threadIdx.x;
    if (e < (int64_t)P.n * P.n) reduce_partial_entry(P.n, P.splits, P.gpart, check ? P.e : P.rc, e);
  }
}

__global__ void __launch_bounds__(1024) kg_chol(Group g, int level) {
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (!item_live(P, level)) continue;
    if (!chol_block(P.n, P.rc) && threadIdx.x == 0) raise_level_status(P.ctl, ST_BREAKDOWN);
    __syncthreads();
  }
}

__global__ void kg_trinv(Group g, int level) {
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (!item_live(P, level)) continue;
    const int j = w.y * 64 + threadIdx.x;
    if (j < P.npad) trinv_column(P.n, P.rc, P.xt, j);
  }
}

__global__ void kg_rmul(Group g, int level) {
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (!item_live(P, level)) continue;
    const int64_t e = (int64_t)w.y * 256 + threadIdx.x;
    if (e < (int64_t)P.n * P.n) rmul_entry(P.n, P.rc, P.rs, P.R, P.ldr, e);
  }
}

__global__ void __launch_bounds__(128) kg_finalize(Group g, int level) {
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (!item_live(P, level)) continue;
    const int64_t r = (int64_t)w.y * 128 + threadIdx.x;
    if (r < P.m) finalize_row(r, P.n, P.Q, P.ldq, P.xt);
  }
}

__global__ void __launch_bounds__(1024) kg_judge(Group g, int level) {
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (P.ctl->active != level) continue;
    judge_block(P.n, P.e, P.check, P.ctl, level);
  }
}

__global__ void kg_publish(Group g) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.nitems) return;
  const Prob& P = g.probs[p];
  if (P.status) *P.status = P.ctl->final_status;
}

}  // namespace

void launch_g_trsm(const Group& g, int level, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_trsm<<<grid_for(g.nitems), 128, 0, st>>>(g, level); }
}
void launch_g_syrk(const Group& g, int tn, bool check, int level, cudaStream_t st) {
  (void)check;
  if (!g.nitems) return;
  if (tn == 16) { ::mrcqr::note_launch(); kg_syrk<16><<<grid_for(g.nitems), 32, 0, st>>>(g, level); }
  else if (tn == 32) { ::mrcqr::note_launch(); kg_syrk<32><<<grid_for(g.nitems), 128, 0, st>>>(g, level); }
  else { ::mrcqr::note_launch(); kg_syrk<64><<<grid_for(g.nitems), 512, 0, st>>>(g, level); }
}
void launch_g_reduce(const Group& g, bool check, int level, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_reduce<<<grid_for(g.nitems), 256, 0, st>>>(g, check ? 1 : 0, level); }
}
void launch_g_chol(const Group& g, int level, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_chol<<<grid_for(g.nitems), 1024, 0, st>>>(g, level); }
}
void launch_g_trinv(const Group& g, int level, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_trinv<<<grid_for(g.nitems), 64, 0, st>>>(g, level); }
}
void launch_g_rmul(const Group& g, int level, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_rmul<<<grid_for(g.nitems), 256, 0, st>>>(g, level); }
}
void launch_g_finalize(const Group& g, int level, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_finalize<<<grid_for(g.nitems), 128, 0, st>>>(g, level); }
}
void launch_g_judge(const Group& g, int level, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_judge<<<grid_for(g.nitems), 1024, 0, st>>>(g, level); }
}
void launch_g_publish(const Group& g, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_publish<<<(g.nitems + 127) / 128, 128, 0, st>>>(g); }
}

}  // namespace mrcqr
