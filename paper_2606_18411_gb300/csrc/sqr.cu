// SketchQR (Algorithm 2 step 5, Sec. II-A): thin Householder QR of the s x n
// sketch Y, in FP32 for the FP16/BF16/FP32 sketches (the paper promotes the
// half-precision sketch to single for the QR) and in FP64 for the FP64
// sketch; R_s is normalised to a positive diagonal (rows flipped) and
// promoted to FP64 (Algorithm 2 step 6).
//
// Sketches of up to 1024 rows take the blocked form (panel kernel + trailing
// updates, below); larger ones, and the batched path, one CTA of 1024 threads
// that walks the columns with the working copy of Y in global memory
// (L2-resident).  Output: R_s
// column-major (n x n), its transpose padded to a row stride npad (for the
// TRSM's uniform row loads, zeros in the padding) and 1/diag(R_s).
#include <type_traits>
#include "kernels.h"

namespace mrcqr {

constexpr int kSqrThreads = 1024;
constexpr int kPadCols = 32;

__host__ __device__ inline int padded(int n) { return (n + kPadCols - 1) / kPadCols * kPadCols; }

template <typename T>
__device__ __forceinline__ void sketch_qr_block(int n, int s, const double* __restrict__ Y, T* __restrict__ W,
                                                double* __restrict__ Rs, double* __restrict__ RsT,
                                                double* __restrict__ rinv) {
  __shared__ T red[33];
  __shared__ T diag[512];
  __shared__ T sh_inv, sh_tau;   // per-column scalars, formed once (FP64 division and sqrt are long sequences)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int64_t total = (int64_t)s * n;
  for (int64_t e = tid; e < total; e += blockDim.x) W[e] = (T)Y[e];
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    T* col = W + (int64_t)j * s;
    // 2-norm of col[j..s) with scaling by the max (no over/underflow)
    T amax = T(0);
    for (int i = j + tid; i < s; i += blockDim.x) amax = max(amax, (T)fabs(col[i]));
    amax = warp_max(amax);
    __syncthreads();
    if (lane == 0) red[warp] = amax;
    __syncthreads();
    if (warp == 0) {
      T t = lane < nwarps ? red[lane] : T(0);
      t = warp_max(t);
      if (lane == 0) {
        red[32] = t;
        sh_inv = t > T(0) ? T(1) / t : T(0);
      }
    }
    __syncthreads();
    amax = red[32];
    T part = T(0);
    if (amax > T(0)) {
      const T inv = sh_inv;
      for (int i = j + tid; i < s; i += blockDim.x) {
        const T v = col[i] * inv;
        part = fma(v, v, part);
      }
    }
    const T ss = block_sum(part, red);
    if (tid == 0) {
      const T nrm = amax * sqrt(ss);
      const T x0 = col[j];
      const T alpha = (x0 >= T(0)) ? -nrm : nrm;
      // ||v||^2 = 2 nrm (nrm + |x0|), so tau = 2/||v||^2 = 1/(nrm (nrm + |x0|))
      sh_tau = (nrm > T(0)) ? T(1) / (nrm * (nrm + (T)fabs(x0))) : T(0);
      col[j] = x0 - alpha;
      diag[j] = alpha;
    }
    __syncthreads();
    const T tau = sh_tau;
    for (int c = j + 1 + warp; c < n; c += nwarps) {
      T* cc = W + (int64_t)c * s;
      T d = T(0);
      for (int i = j + lane; i < s; i += 32) d = fma(col[i], cc[i], d);
      d = warp_sum(d);
      const T f = tau * d;
      for (int i = j + lane; i < s; i += 32) cc[i] = fma(-f, col[i], cc[i]);
    }
    __syncthreads();
  }
  const int npad = padded(n);
  for (int e = tid; e < npad * n; e += blockDim.x) {
    // e indexes RsT row-major: row r (< n), column c (< npad)
    const int r = e / npad, c = e % npad;
    const double sg = diag[r] < T(0) ? -1.0 : 1.0;
    double v = 0.0;
    if (c < n) {
      if (r < c) v = (double)W[(int64_t)c * s + r] * sg;
      else if (r == c) v = fabs((double)diag[r]);
    }
    RsT[(int64_t)r * npad + c] = v;
    if (c < n) Rs[(int64_t)c * n + r] = v;
  }
  for (int r = tid; r < npad; r += blockDim.x) rinv[r] = r < n ? 1.0 / fabs((double)diag[r]) : 0.0;
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kSqrThreads) k_sketch_qr(int n, int s, const double* __restrict__ Y,
                                                           T* __restrict__ W, double* __restrict__ Rs,
                                                           double* __restrict__ RsT, double* __restrict__ rinv,
                                                           Ctl* ctl, int level) {
  if (level_inactive(ctl, level)) return;
  if (ctl->lvl_status != 0) return;
  sketch_qr_block<T>(n, s, Y, W, Rs, RsT, rinv);
}


// ---------------------------------------------------------------------------
// Blocked form for s <= 1024 (the single-CTA kernel above keeps the larger
// sketches): panels of kQB columns are factored by one CTA in shared memory,
// and the columns right of a panel are updated by one warp per column (the
// column in registers), so the O(s n^2) reflector applications are spread
// over the GPU instead of one SM (FP64 issues at 1/64 of the FP32 rate here).
// The working copy holds LAPACK's geqrf layout: beta_j = +-||x|| on the
// diagonal, the reflector v (v_j = 1 implicit) below it; tau = 2 / ||v||^2
// is recomputed from v where it is needed, so no extra storage is used.
constexpr int kQB = 16;          // panel width
constexpr int kQMaxS = 1024;     // rows handled by the blocked form
constexpr int kQPanelThreads = 512;

__global__ void k_sqr_copy(int64_t total, const double* __restrict__ Y, void* __restrict__ Wk, int fp64,
                           const Ctl* ctl, int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    if (fp64) static_cast<double*>(Wk)[e] = Y[e];
    else static_cast<float*>(Wk)[e] = (float)Y[e];
  }
}

// Warp-wide sum and max.
template <typename T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T wmax(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Householder reflector of x[jj..rows) by one warp (the column's owner):
// beta = -sign(x0) ||x||, v = (1, x[jj+1..] / (x0 - beta)), tau = 2 / ||v||^2.
// x[jj] <- beta, x[jj+1..] <- v[1..]; returns tau (0 for a zero column).
// FP32 scales the norm by the column maximum so it neither overflows nor
// underflows; FP64 does so only when the plain sum of squares leaves
// [1e-250, 1e250] (each FP64 operation is a long-latency step on this GPU).
template <typename T>
__device__ __forceinline__ T house_warp(T* x, int jj, int rows, int lane) {
  if constexpr (sizeof(T) == 8) {   // FP64: unscaled sums of squares unless they leave the normal range
    T t0 = T(0), t1 = T(0);
    int i = jj + 1 + lane;
    for (; i + 32 < rows; i += 64) {
      t0 = fma(x[i], x[i], t0);
      t1 = fma(x[i + 32], x[i + 32], t1);
    }
    if (i < rows) t0 = fma(x[i], x[i], t0);
    const T tail = wsum(t0 + t1);
    const T x0 = x[jj];
    const T ss = fma(x0, x0, tail);
    if (ss > T(1e-250) && ss < T(1e250)) {
      const T nrm = sqrt(ss);
      const T beta = x0 >= T(0) ? -nrm : nrm;
      const T d = x0 - beta;
      const T scale = T(1) / d;
      const T tau = T(2) / fma(tail * scale, scale, T(1));
      __syncwarp();
      for (int k = jj + 1 + lane; k < rows; k += 32) x[k] *= scale;
      if (lane == 0) x[jj] = beta;
      __syncwarp();
      return tau;
    }
    if (!(ss > T(0))) return T(0);   // zero column (or NaN: left as it is)
  }
  T amax = T(0);
  for (int i = jj + lane; i < rows; i += 32) amax = max(amax, (T)fabs(x[i]));
  amax = wmax(amax);
  if (!(amax > T(0))) return T(0);
  const T inv = T(1) / amax;
  T t0 = T(0), t1 = T(0);
  int i = jj + 1 + lane;
  for (; i + 32 < rows; i += 64) {
    const T a = x[i] * inv, b = x[i + 32] * inv;
    t0 = fma(a, a, t0);
    t1 = fma(b, b, t1);
  }
  if (i < rows) {
    const T a = x[i] * inv;
    t0 = fma(a, a, t0);
  }
  const T tail = wsum(t0 + t1);   // sum of (x_i / amax)^2 over i > jj
  const T x0 = x[jj], y0 = x0 * inv;
  const T nrm = amax * sqrt(fma(y0, y0, tail));
  const T beta = x0 >= T(0) ? -nrm : nrm;
  const T d = x0 - beta;   // |d| = |x0| + nrm: no cancellation
  const T scale = T(1) / d;
  const T r = amax * scale;
  const T tau = T(2) / fma(tail * r, r, T(1));
  __syncwarp();
  for (int k = jj + 1 + lane; k < rows; k += 32) x[k] *= scale;
  if (lane == 0) x[jj] = beta;
  __syncwarp();
  return tau;
}

// y <- (I - tau v v^T) y over rows jj..rows-1, v = (1, x[jj+1..]), one warp.
template <typename T>
__device__ __forceinline__ void house_apply_warp(const T* x, T* y, T tau, int jj, int rows, int lane) {
  T d0 = lane == 0 ? y[jj] : T(0), d1 = T(0);
  int i = jj + 1 + lane;
  for (; i + 32 < rows; i += 64) {
    d0 = fma(x[i], y[i], d0);
    d1 = fma(x[i + 32], y[i + 32], d1);
  }
  if (i < rows) d0 = fma(x[i], y[i], d0);
  const T f = tau * wsum(d0 + d1);
  if (lane == 0) y[jj] -= f;
  for (int k = jj + 1 + lane; k < rows; k += 32) y[k] = fma(-f, x[k], y[k]);
  __syncwarp();
}

// Panel [c0, c1) of the s x n working copy (column-major, ld s), rows c0 .. s-1,
// factored in shared memory; warp w owns panel column w.  Step jj: the owner
// of column jj has already applied reflectors 0 .. jj-1 to it and forms
// reflector jj; after one barrier every warp right of it applies it to its own
// column, the owner of jj+1 first and then straight on to its reflector.
template <typename T>
__global__ void __launch_bounds__(kQPanelThreads) k_sqr_panel(int s, int c0, int c1, T* __restrict__ Wk,
                                                              const Ctl* ctl, int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  extern __shared__ unsigned char sqr_smem[];
  T* P = reinterpret_cast<T*>(sqr_smem);   // [kQB][rows]
  __shared__ T taus[kQB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rows = s - c0, b = c1 - c0;
  for (int e = tid; e < b * rows; e += blockDim.x) {
    const int c = e / rows, i = e % rows;
    P[c * rows + i] = Wk[(int64_t)(c0 + c) * s + c0 + i];
  }
  __syncthreads();
  if (warp == 0) {
    const T t = house_warp(P, 0, rows, lane);
    if (lane == 0) taus[0] = t;
  }
  __syncthreads();
  for (int jj = 0; jj < b; ++jj) {
    if (warp > jj && warp < b) {
      T* y = P + warp * rows;
      house_apply_warp(P + jj * rows, y, taus[jj], jj, rows, lane);
      if (warp == jj + 1) {
        const T t = house_warp(y, jj + 1, rows, lane);
        if (lane == 0) taus[jj + 1] = t;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < b * rows; e += blockDim.x) {
    const int c = e / rows, i = e % rows;
    Wk[(int64_t)(c0 + c) * s + c0 + i] = P[c * rows + i];
  }
}

// Columns c >= c1: apply the panel's reflectors j = c0 .. c1-1 in order
// (one warp per column; lane l holds rows c0 + l + 32 t, t < kR, with
// 32 kR >= s - c0).
template <typename T, int kR>
__global__ void __launch_bounds__(32) k_sqr_update(int s, int c0, int c1, T* __restrict__ Wk, const Ctl* ctl,
                                                   int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  const int lane = threadIdx.x;
  const int c = c1 + blockIdx.x;
  T* y = Wk + (int64_t)c * s;
  const T* V = Wk;
  T xr[kR];
#pragma unroll
  for (int t = 0; t < kR; ++t) {
    const int i = c0 + lane + 32 * t;
    xr[t] = i < s ? y[i] : T(0);
  }
  for (int j = c0; j < c1; ++j) {
    const T* v = V + (int64_t)j * s;
    T d[2] = {T(0), T(0)}, vv[2] = {T(0), T(0)};
#pragma unroll
    for (int t = 0; t < kR; ++t) {
      const int i = c0 + lane + 32 * t;
      if (i > j && i < s) {
        const T vi = v[i];
        d[t & 1] = fma(vi, xr[t], d[t & 1]);
        vv[t & 1] = fma(vi, vi, vv[t & 1]);
      } else if (i == j) {
        d[t & 1] += xr[t];
      }
    }
    const T dd = wsum(d[0] + d[1]), vs = wsum(vv[0] + vv[1]);
    const T f = (T(2) / (T(1) + vs)) * dd;
#pragma unroll
    for (int t = 0; t < kR; ++t) {
      const int i = c0 + lane + 32 * t;
      if (i > j && i < s) xr[t] = fma(-f, v[i], xr[t]);
      else if (i == j) xr[t] -= f;
    }
  }
#pragma unroll
  for (int t = 0; t < kR; ++t) {
    const int i = c0 + lane + 32 * t;
    if (i < s) y[i] = xr[t];
  }
}

// R_s (column-major), its padded transpose and 1/diag from the factored
// working copy, rows flipped to a positive diagonal.
template <typename T>
__global__ void k_sqr_out(int n, int s, const T* __restrict__ Wk, double* __restrict__ Rs, double* __restrict__ RsT,
                          double* __restrict__ rinv, const Ctl* ctl, int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  const int npad = padded(n);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < (int64_t)npad * n) {
    const int r = (int)(e / npad), c = (int)(e % npad);
    const double beta = (double)Wk[(int64_t)r * s + r];
    const double sg = beta < 0.0 ? -1.0 : 1.0;
    double v = 0.0;
    if (c < n) {
      if (r < c) v = (double)Wk[(int64_t)c * s + r] * sg;
      else if (r == c) v = fabs(beta);
    }
    RsT[(int64_t)r * npad + c] = v;
    if (c < n) Rs[(int64_t)c * n + r] = v;
  }
  if (e < npad) rinv[e] = e < n ? 1.0 / fabs((double)Wk[e * s + e]) : 0.0;
}

template <typename T>
void launch_sqr_blocked(int n, int s, const double* Y, T* Wk, double* Rs, double* RsT, double* rinv, Ctl* ctl,
                        int level, cudaStream_t st) {
  const int64_t total = (int64_t)s * n;
  { ::mrcqr::note_launch(); k_sqr_copy<<<(unsigned)((total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024), 256, 0, st>>>(
      total, Y, Wk, std::is_same<T, double>::value ? 1 : 0, ctl, level); }
  cudaFuncSetAttribute(k_sqr_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(sizeof(T) * (size_t)kQB * (size_t)kQMaxS));
  for (int c0 = 0; c0 < n; c0 += kQB) {
    const int c1 = c0 + kQB < n ? c0 + kQB : n;
    const size_t smem = sizeof(T) * (size_t)kQB * (size_t)(s - c0);
    { ::mrcqr::note_launch(); k_sqr_panel<T><<<1, kQPanelThreads, smem, st>>>(s, c0, c1, Wk, ctl, level); }
    if (c1 < n) {
      const int rows = s - c0;
      const unsigned g = (unsigned)(n - c1);
      if (rows <= 256) { ::mrcqr::note_launch(); k_sqr_update<T, 8><<<g, 32, 0, st>>>(s, c0, c1, Wk, ctl, level); }
      else if (rows <= 512) { ::mrcqr::note_launch(); k_sqr_update<T, 16><<<g, 32, 0, st>>>(s, c0, c1, Wk, ctl, level); }
      else { ::mrcqr::note_launch(); k_sqr_update<T, 32><<<g, 32, 0, st>>>(s, c0, c1, Wk, ctl, level); }
    }
  }
  const int64_t tot = (int64_t)padded(n) * n;
  { ::mrcqr::note_launch(); k_sqr_out<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, s, Wk, Rs, RsT, rinv, ctl, level); }
}

size_t sqr_workspace_bytes(int n, int s) { return (size_t)n * (size_t)s * sizeof(double); }

void launch_sketch_qr(int prec, int n, int s, const double* Y, void* work, double* Rs, double* RsT, double* rinv,
                      Ctl* ctl, int level, cudaStream_t st) {
  if (s <= kQMaxS) {
    if (prec == P_FP64) launch_sqr_blocked<double>(n, s, Y, (double*)work, Rs, RsT, rinv, ctl, level, st);
    else launch_sqr_blocked<float>(n, s, Y, (float*)work, Rs, RsT, rinv, ctl, level, st);
    return;
  }
  if (prec == P_FP64)
    { ::mrcqr::note_launch(); k_sketch_qr<double><<<1, kSqrThreads, 0, st>>>(n, s, Y, (double*)work, Rs, RsT, rinv, ctl, level); }
  else
    { ::mrcqr::note_launch(); k_sketch_qr<float><<<1, kSqrThreads, 0, st>>>(n, s, Y, (float*)work, Rs, RsT, rinv, ctl, level); }
}

}  // namespace mrcqr

namespace mrcqr {

// R_s given by the caller (column-major n x n): its padded transpose and
// 1/diag for the substitution kernel.
__global__ void k_rs_prepare(int n, const double* __restrict__ Rs, double* __restrict__ RsT,
                             double* __restrict__ rinv) {
  const int npad = padded(n);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < (int64_t)n * npad) {
    const int r = (int)(e / npad), c = (int)(e % npad);
    RsT[e] = (c < n && r <= c) ? Rs[(int64_t)c * n + r] : 0.0;
  }
  if (e < npad) rinv[e] = e < n ? 1.0 / Rs[e * n + e] : 0.0;
}

void launch_rs_prepare(int n, const double* Rs, double* RsT, double* rinv, cudaStream_t st) {
  const int64_t tot = (int64_t)n * padded(n);
  { ::mrcqr::note_launch(); k_rs_prepare<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, Rs, RsT, rinv); }
}

// Grouped sketch QR: one CTA per problem.
namespace {

template <typename T>
__global__ void __launch_bounds__(kSqrThreads) kg_sketch_qr(Group g, int level) {
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const Prob& P = g.probs[g.items[it].x];
    if (P.ctl->active != level || P.ctl->lvl_status != 0) continue;
    sketch_qr_block<T>(P.n, P.s, P.y, static_cast<T*>(P.sqrw), P.rs, P.rst, P.rinv);
  }
}

}  // namespace

void launch_g_sketch_qr(const Group& g, bool fp64, int level, cudaStream_t st) {
  if (!g.nitems) return;
  const unsigned grid = (unsigned)(g.nitems < 152 * 2 ? g.nitems : 152 * 2);
  if (fp64) { ::mrcqr::note_launch(); kg_sketch_qr<double><<<grid, kSqrThreads, 0, st>>>(g, level); }
  else { ::mrcqr::note_launch(); kg_sketch_qr<float><<<grid, kSqrThreads, 0, st>>>(g, level); }
}

}  // namespace mrcqr
