// SketchQR (Algorithm 2 step 5, Sec. II-A): thin Householder QR of the s x n
// sketch Y, in FP32 for the FP16/BF16/FP32 sketches (the paper promotes the
// half-precision sketch to single for the QR) and in FP64 for the FP64
// sketch; R_s is normalised to a positive diagonal (rows flipped) and
// promoted to FP64 (Algorithm 2 step 6).
//
// One CTA of 1024 threads walks the columns; the working copy of Y stays in
// global memory (L2-resident: at most 1024 x 512 words).  Output: R_s
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
      if (lane == 0) red[32] = t;
    }
    __syncthreads();
    amax = red[32];
    T part = T(0);
    if (amax > T(0)) {
      const T inv = T(1) / amax;
      for (int i = j + tid; i < s; i += blockDim.x) {
        const T v = col[i] * inv;
        part = fma(v, v, part);
      }
    }
    const T ss = block_sum(part, red);
    const T nrm = amax * sqrt(ss);
    const T x0 = col[j];
    const T alpha = (x0 >= T(0)) ? -nrm : nrm;
    const T v0 = x0 - alpha;
    // ||v||^2 = 2 nrm (nrm + |x0|), so tau = 2/||v||^2 = 1/(nrm (nrm + |x0|))
    const T tau = (nrm > T(0)) ? T(1) / (nrm * (nrm + (T)fabs(x0))) : T(0);
    __syncthreads();
    if (tid == 0) {
      col[j] = v0;
      diag[j] = alpha;
    }
    __syncthreads();
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

size_t sqr_workspace_bytes(int n, int s) { return (size_t)n * (size_t)s * sizeof(double); }

void launch_sketch_qr(int prec, int n, int s, const double* Y, void* work, double* Rs, double* RsT, double* rinv,
                      Ctl* ctl, int level, cudaStream_t st) {
  if (prec == P_FP64)
    k_sketch_qr<double><<<1, kSqrThreads, 0, st>>>(n, s, Y, (double*)work, Rs, RsT, rinv, ctl, level);
  else
    k_sketch_qr<float><<<1, kSqrThreads, 0, st>>>(n, s, Y, (float*)work, Rs, RsT, rinv, ctl, level);
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
  k_rs_prepare<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, Rs, RsT, rinv);
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
  if (fp64) kg_sketch_qr<double><<<grid, kSqrThreads, 0, st>>>(g, level);
  else kg_sketch_qr<float><<<grid, kSqrThreads, 0, st>>>(g, level);
}

}  // namespace mrcqr
