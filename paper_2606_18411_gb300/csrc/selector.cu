// Learned sketch-precision selector (the paper's Sec. II-C leaves choosing
// the precision to a coarse estimate of kappa_2(A) and names machine-learned
// estimators as one option).
//
//  * k_features: 16 features of the R_s an FP16 sketch produced (one CTA,
//    FP64): log-diagonal ratios and quantiles, 3-step power-iteration
//    condition estimates of R_s and R_s diag(R_s)^{-1}, column-norm spread,
//    off-diagonal mass, fractions of diagonals under the FP16 / FP32 noise
//    floors, the log-diagonal decay slope, shape.
//  * an MLP 16-64-64-3 (ReLU) with BF16 weights and FP32 accumulation;
//    k_mlp_select (one CTA, inside MRCQR_PREC_AUTO) picks the start of the
//    precision ladder that minimises the expected cost
//    sum_y p(y|x) C[k][y], C[k][y] = cost(k) if k >= y else the cost of every
//    run from k up to y.
//  * training kernels: per-CTA gradient partials of the class-weighted
//    cross-entropy (forward and backward in FP32 on the BF16 weights), then
//    a fixed-order reduction fused with AdamW on FP32 master weights that
//    also refreshes the BF16 copies.  Deterministic (no atomics).
#include <cstdio>
#include <mutex>
#include <vector>

#include "kernels.h"

namespace mrcqr {

namespace {

constexpr int kF = kNumFeatures, kH = 64, kC = 3;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kF, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kC * kH, kNParams = kOffB3 + kC;
constexpr int kFeatThreads = 256;
constexpr int kMaxN = 512;

// ---------------------------------------------------------------------------
// features

__device__ double block_sum_d(double v, double* red) { return block_sum(v, red); }

__device__ double block_max_d(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double t = lane < nw ? red[lane] : -INFINITY;
    t = warp_max(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// The reciprocals of the diagonal (rd = 1 / |R_jj|, rdg = 1 / R_jj) are formed
// once: FP64 division is a long sequence on this GPU's 1/64-rate pipe, and the
// sweeps below would otherwise divide at every step in every thread.

// y = M x (M = R or R diag(R)^-1), x and y in shared memory
__device__ void mat_vec(const double* R, const double* rd, bool unit, int n, const double* x, double* y) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double acc = 0.0;
    for (int j = i; j < n; ++j) acc = fma(R[(int64_t)j * n + i] * (unit ? rd[j] : 1.0), x[j], acc);
    y[i] = acc;
  }
  __syncthreads();
}

// y = M^T x
__device__ void mat_t_vec(const double* R, const double* rd, bool unit, int n, const double* x, double* y) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i <= j; ++i) acc = fma(R[(int64_t)j * n + i], x[i], acc);
    y[j] = unit ? acc * rd[j] : acc;
  }
  __syncthreads();
}

// x <- M^{-1} x (column sweep from the last column)
__device__ void solve(const double* R, const double* rd, const double* rdg, bool unit, int n, double* x) {
  for (int j = n - 1; j >= 0; --j) {
    const double xj = unit ? x[j] : x[j] * rdg[j];
    __syncthreads();
    for (int i = threadIdx.x; i < j; i += blockDim.x)
      x[i] = fma(-R[(int64_t)j * n + i] * (unit ? rd[j] : 1.0), xj, x[i]);
    if (threadIdx.x == 0) x[j] = xj;
    __syncthreads();
  }
}

// x <- M^{-T} x (forward sweep)
__device__ void solve_t(const double* R, const double* rd, const double* rdg, bool unit, int n, double* x) {
  for (int j = 0; j < n; ++j) {
    const double xj = unit ? x[j] : x[j] * rdg[j];
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x)
      x[i] = fma(-R[(int64_t)i * n + j] * (unit ? rd[i] : 1.0), xj, x[i]);
    if (threadIdx.x == 0) x[j] = xj;
    __syncthreads();
  }
}

__device__ double vec_norm(const double* x, int n, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s = fma(x[i], x[i], s);
  return sqrt(block_sum_d(s, red));
}

// 3-step power iteration for ||M|| (inverse = false) or ||M^{-1}|| (true).
__device__ double power_norm(const double* R, const double* rd, const double* rdg, bool unit, bool inverse, int n,
                             double* x, double* y, double* red) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = 1.0 / sqrt((double)n);
  __syncthreads();
  double nrm = 0.0;
  for (int it = 0; it < 3; ++it) {
    if (!inverse) {
      mat_vec(R, rd, unit, n, x, y);
      mat_t_vec(R, rd, unit, n, y, x);
    } else {
      solve(R, rd, rdg, unit, n, x);
      solve_t(R, rd, rdg, unit, n, x);
    }
    nrm = vec_norm(x, n, red);
    if (!(nrm > 0.0) || !isfinite(nrm)) return nrm;
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] /= nrm;
    __syncthreads();
  }
  return sqrt(nrm);
}

__global__ void __launch_bounds__(kFeatThreads) k_features(const double* __restrict__ R, int n, int64_t m,
                                                          float* __restrict__ out, const Ctl* ctl, int level) {
  if (ctl && (ctl->active != level || ctl->lvl_status != 0)) return;
  __shared__ double d[kMaxN], L[kMaxN], Ls[kMaxN], x[kMaxN], y[kMaxN], rd[kMaxN], rdg[kMaxN];
  __shared__ double red[33];
  const double tiny = 2.2250738585072014e-308;
  const int tid = threadIdx.x;
  for (int i = tid; i < kMaxN; i += blockDim.x) {
    if (i < n) {
      d[i] = fabs(R[(int64_t)i * n + i]);
      rd[i] = 1.0 / d[i];
      rdg[i] = 1.0 / R[(int64_t)i * n + i];
      L[i] = log10(fmax(d[i], tiny));
      Ls[i] = L[i];
    } else {
      Ls[i] = INFINITY;
    }
  }
  __syncthreads();
  // bitonic sort of Ls (ascending, padding +inf last)
  for (int k = 2; k <= kMaxN; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < kMaxN; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const double a = Ls[i], b = Ls[l];
          if ((a > b) == ((i & k) == 0)) { Ls[i] = b; Ls[l] = a; }
        }
      }
      __syncthreads();
    }
  double lmax = -INFINITY, lsum = 0.0;
  for (int i = tid; i < n; i += blockDim.x) { lmax = fmax(lmax, L[i]); lsum += L[i]; }
  lmax = block_max_d(lmax, red);
  const double lmean = block_sum_d(lsum, red) / n;
  const double lmin = Ls[0];
  double dev = 0.0, gap = 0.0;
  for (int i = tid; i < n; i += blockDim.x) {
    dev += (L[i] - lmean) * (L[i] - lmean);
    gap += lmax - L[i];
  }
  const double lstd = sqrt(block_sum_d(dev, red) / n);
  const double gapm = block_sum_d(gap, red) / n;
  const double dmax = pow(10.0, lmax);
  // condition estimates of R and of R diag(R)^-1
  const double nr = power_norm(R, rd, rdg, false, false, n, x, y, red);
  const double ni = power_norm(R, rd, rdg, false, true, n, x, y, red);
  const double ur = power_norm(R, rd, rdg, true, false, n, x, y, red);
  const double ui = power_norm(R, rd, rdg, true, true, n, x, y, red);
  // column norms, off-diagonal mass, noise-floor fractions
  double cmax = 0.0, cmin = INFINITY, off = 0.0, dsq = 0.0, f16 = 0.0, f32 = 0.0;
  for (int j = tid; j < n; j += blockDim.x) {
    double c = 0.0;
    for (int i = 0; i <= j; ++i) {
      const double v = R[(int64_t)j * n + i];
      c = fma(v, v, c);
      if (i < j) off = fma(v, v, off);
    }
    c = sqrt(c);
    cmax = fmax(cmax, c);
    cmin = fmin(cmin, c);
    dsq = fma(d[j], d[j], dsq);
    f16 += d[j] < ldexp(dmax, -11) ? 1.0 : 0.0;
    f32 += d[j] < ldexp(dmax, -20) ? 1.0 : 0.0;
  }
  cmax = block_max_d(cmax, red);
  cmin = -block_max_d(-cmin, red);
  off = block_sum_d(off, red);
  dsq = block_sum_d(dsq, red);
  f16 = block_sum_d(f16, red);
  f32 = block_sum_d(f32, red);
  // least-squares slope of L over the first half
  const int h = max(n / 2, 2);
  const double imean = 0.5 * (h - 1);
  double lh = 0.0;
  for (int i = tid; i < h; i += blockDim.x) lh += L[i];
  const double lhm = block_sum_d(lh, red) / h;
  double sxy = 0.0, sxx = 0.0;
  for (int i = tid; i < h; i += blockDim.x) {
    sxy += (i - imean) * (L[i] - lhm);
    sxx += (i - imean) * (i - imean);
  }
  sxy = block_sum_d(sxy, red);
  sxx = block_sum_d(sxx, red);
  if (tid == 0) {
    const int q10 = (int)floor(0.10 * (n - 1)), q50 = (int)floor(0.50 * (n - 1));
    out[0] = (float)(lmax - lmin);
    out[1] = (float)(lmax - Ls[q10]);
    out[2] = (float)(lmax - Ls[q50]);
    out[3] = (float)gapm;
    out[4] = (float)lstd;
    out[5] = (float)log10(fmax(nr * ni, 1.0));
    out[6] = (float)log10(fmax(ur * ui, 1.0));
    out[7] = (float)log10(fmax(cmax, tiny) / fmax(cmin, tiny));
    out[8] = (float)(sqrt(off) / fmax(sqrt(dsq), tiny));
    out[9] = (float)(n / 512.0);
    out[10] = (float)(log2((double)m) / 22.0);
    out[11] = (float)(f16 / n);
    out[12] = (float)(f32 / n);
    out[13] = (float)(-(sxy / sxx) * (n - 1));
    out[14] = (float)(lmax - L[n - 1]);
    out[15] = 1.0f;
  }
}

// ---------------------------------------------------------------------------
// MLP

struct Sel {
  const unsigned short* w;   // BF16 parameters (kNParams)
  const float* mu;           // feature mean (16)
  const float* sd;           // feature scale (16)
  const float* costs;        // ladder costs (3)
};

__device__ __forceinline__ float wv(const unsigned short* w, int i) { return __bfloat162float(__ushort_as_bfloat16(w[i])); }

// Forward of one sample by a 64-thread group; logits in z (shared).
__device__ void mlp_forward64(const Sel& S, const float* feat, float* xs, float* h1, float* h2, float* a1, float* a2,
                              float* z) {
  const int j = threadIdx.x;
  if (j < kF) xs[j] = (feat[j] - S.mu[j]) / S.sd[j];
  __syncthreads();
  float acc = wv(S.w, kOffB1 + j);
#pragma unroll
  for (int k = 0; k < kF; ++k) acc = fmaf(wv(S.w, kOffW1 + j * kF + k), xs[k], acc);
  a1[j] = acc;
  h1[j] = fmaxf(acc, 0.f);
  __syncthreads();
  acc = wv(S.w, kOffB2 + j);
  for (int k = 0; k < kH; ++k) acc = fmaf(wv(S.w, kOffW2 + j * kH + k), h1[k], acc);
  a2[j] = acc;
  h2[j] = fmaxf(acc, 0.f);
  __syncthreads();
  if (j < kC) {
    float zz = wv(S.w, kOffB3 + j);
    for (int k = 0; k < kH; ++k) zz = fmaf(wv(S.w, kOffW3 + j * kH + k), h2[k], zz);
    z[j] = zz;
  }
  __syncthreads();
}

__device__ int expected_cost_choice(const float* z, const float* costs) {
  const float zm = fmaxf(z[0], fmaxf(z[1], z[2]));
  float p[kC], s = 0.f;
  for (int c = 0; c < kC; ++c) { p[c] = __expf(z[c] - zm); s += p[c]; }
  int best = kC - 1;
  float bestc = INFINITY;
  for (int k = 0; k < kC; ++k) {
    float e = 0.f;
    for (int t = 0; t < kC; ++t) {
      float ck = 0.f;
      if (k >= t) ck = costs[k];
      else for (int u = k; u <= t; ++u) ck += costs[u];
      e += p[t] / s * ck;
    }
    if (e < bestc) { bestc = e; best = k; }
  }
  return best;
}

// AUTO: choose the start of the ladder (levels 0/1/2 = fp16/fp32/fp64).
__global__ void __launch_bounds__(64) k_mlp_select(Sel S, const float* __restrict__ feat, Ctl* ctl) {
  if (ctl->active != 0 || ctl->lvl_status != 0) return;
  __shared__ float xs[kF], h1[kH], h2[kH], a1[kH], a2[kH], z[kC];
  mlp_forward64(S, feat, xs, h1, h2, a1, a2, z);
  if (threadIdx.x == 0) {
    const int k = expected_cost_choice(z, S.costs);
    ctl->mlp_choice = k;
    ctl->prec_first = ctl->lvl_prec[k];
    for (int i = 0; i < kF; ++i) ctl->features[i] = feat[i];
    ctl->active = k;
  }
}

__global__ void __launch_bounds__(64) k_mlp_forward(Sel S, int batch, const float* __restrict__ X,
                                                    float* __restrict__ logits, int32_t* __restrict__ choice) {
  __shared__ float xs[kF], h1[kH], h2[kH], a1[kH], a2[kH], z[kC];
  for (int b = blockIdx.x; b < batch; b += gridDim.x) {
    mlp_forward64(S, X + (size_t)b * kF, xs, h1, h2, a1, a2, z);
    if (threadIdx.x < kC) logits[(size_t)b * kC + threadIdx.x] = z[threadIdx.x];
    if (threadIdx.x == 0 && choice) choice[b] = expected_cost_choice(z, S.costs);
    __syncthreads();
  }
}

// Gradient partial of the class-weighted mean cross-entropy over the samples
// [blk * per, (blk+1) * per): thread j owns hidden unit j of both layers.
__global__ void __launch_bounds__(64) k_mlp_grad_partial(Sel S, int batch, int per, const float* __restrict__ X,
                                                         const int32_t* __restrict__ y,
                                                         const float* __restrict__ class_w,
                                                         float* __restrict__ part, float* __restrict__ loss_part) {
  __shared__ float xs[kF], h1[kH], h2[kH], a1[kH], a2[kH], z[kC], dz[kC], dh2[kH], W2s[kH * kH];
  const int j = threadIdx.x;
  for (int i = j; i < kH * kH; i += kH) W2s[i] = wv(S.w, kOffW2 + i);
  float gW1[kF], gW2[kH], gW3[kC], gb1 = 0.f, gb2 = 0.f, gb3 = 0.f, loss = 0.f;
#pragma unroll
  for (int k = 0; k < kF; ++k) gW1[k] = 0.f;
#pragma unroll
  for (int k = 0; k < kH; ++k) gW2[k] = 0.f;
#pragma unroll
  for (int c = 0; c < kC; ++c) gW3[c] = 0.f;
  __syncthreads();
  const int b0 = blockIdx.x * per, b1 = min(batch, b0 + per);
  const float invB = 1.0f / (float)batch;
  for (int b = b0; b < b1; ++b) {
    mlp_forward64(S, X + (size_t)b * kF, xs, h1, h2, a1, a2, z);
    const int yb = y[b];
    const float wb = class_w[yb];
    if (j == 0) {
      const float zm = fmaxf(z[0], fmaxf(z[1], z[2]));
      float e[kC], s = 0.f;
      for (int c = 0; c < kC; ++c) { e[c] = __expf(z[c] - zm); s += e[c]; }
      for (int c = 0; c < kC; ++c) dz[c] = wb * (e[c] / s - (c == yb ? 1.f : 0.f)) * invB;
      loss += wb * -(z[yb] - zm - __logf(s)) * invB;
    }
    __syncthreads();
    // layer 3
#pragma unroll
    for (int c = 0; c < kC; ++c) gW3[c] = fmaf(dz[c], h2[j], gW3[c]);
    if (j < kC) gb3 += dz[j];
    float g2 = 0.f;
#pragma unroll
    for (int c = 0; c < kC; ++c) g2 = fmaf(wv(S.w, kOffW3 + c * kH + j), dz[c], g2);
    g2 = a2[j] > 0.f ? g2 : 0.f;
    dh2[j] = g2;
    __syncthreads();
    // layer 2
#pragma unroll
    for (int k = 0; k < kH; ++k) gW2[k] = fmaf(g2, h1[k], gW2[k]);
    gb2 += g2;
    float g1 = 0.f;
    for (int i = 0; i < kH; ++i) g1 = fmaf(W2s[i * kH + j], dh2[i], g1);
    g1 = a1[j] > 0.f ? g1 : 0.f;
    // layer 1
#pragma unroll
    for (int k = 0; k < kF; ++k) gW1[k] = fmaf(g1, xs[k], gW1[k]);
    gb1 += g1;
    __syncthreads();
  }
  float* P = part + (size_t)blockIdx.x * kNParams;
#pragma unroll
  for (int k = 0; k < kF; ++k) P[kOffW1 + j * kF + k] = gW1[k];
  P[kOffB1 + j] = gb1;
#pragma unroll
  for (int k = 0; k < kH; ++k) P[kOffW2 + j * kH + k] = gW2[k];
  P[kOffB2 + j] = gb2;
#pragma unroll
  for (int c = 0; c < kC; ++c) P[kOffW3 + c * kH + j] = gW3[c];
  if (j < kC) P[kOffB3 + j] = gb3;
  if (j == 0) loss_part[blockIdx.x] = loss;
}

// Fixed-order sum of the partials, then AdamW (decoupled decay) on the FP32
// master weights and refresh of the BF16 copies.  grad_out / loss_out get
// the summed gradient and loss when non-null.
__global__ void k_mlp_reduce_adamw(int nparts, const float* __restrict__ part, const float* __restrict__ loss_part,
                                   float* __restrict__ master, float* __restrict__ mom, float* __restrict__ var,
                                   unsigned short* __restrict__ wbf16, float lr, float beta1, float beta2, float eps,
                                   float wd, int step, int apply, float* __restrict__ grad_out,
                                   float* __restrict__ loss_out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0 && loss_out) {
    float l = 0.f;
    for (int b = 0; b < nparts; ++b) l += loss_part[b];
    *loss_out = l;
  }
  if (p >= kNParams) return;
  float g = 0.f;
  for (int b = 0; b < nparts; ++b) g += part[(size_t)b * kNParams + p];
  if (grad_out) grad_out[p] = g;
  if (!apply) return;
  const float m1 = beta1 * mom[p] + (1.f - beta1) * g;
  const float v1 = beta2 * var[p] + (1.f - beta2) * g * g;
  mom[p] = m1;
  var[p] = v1;
  const float mh = m1 / (1.f - powf(beta1, (float)step));
  const float vh = v1 / (1.f - powf(beta2, (float)step));
  const float w = master[p] - lr * (mh / (sqrtf(vh) + eps) + wd * master[p]);
  master[p] = w;
  wbf16[p] = __bfloat16_as_ushort(__float2bfloat16_rn(w));
}

// Per-device selector weights used by MRCQR_PREC_AUTO.
struct DevSel {
  unsigned short* w = nullptr;
  float* aux = nullptr;   // mu[16], sd[16], costs[3]
};
std::mutex g_sel_mu;
std::vector<DevSel> g_sel;

}  // namespace

int selector_num_params() { return kNParams; }

bool selector_ready() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_sel_mu);
  return dev < (int)g_sel.size() && g_sel[dev].w != nullptr;
}

int selector_set(const float* params, const float* mu, const float* sd, const float* costs) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_sel_mu);
  if ((int)g_sel.size() <= dev) g_sel.resize(dev + 1);
  DevSel& s = g_sel[dev];
  if (!s.w && cudaMalloc(&s.w, sizeof(unsigned short) * kNParams) != cudaSuccess) return ST_ALLOC;
  if (!s.aux && cudaMalloc(&s.aux, sizeof(float) * 35) != cudaSuccess) return ST_ALLOC;
  std::vector<unsigned short> wb(kNParams);
  for (int i = 0; i < kNParams; ++i) wb[i] = __bfloat16_as_ushort(__float2bfloat16_rn(params[i]));
  std::vector<float> aux(35);
  for (int i = 0; i < 16; ++i) { aux[i] = mu[i]; aux[16 + i] = sd[i] > 0 ? sd[i] : 1.f; }
  for (int i = 0; i < 3; ++i) aux[32 + i] = costs[i];
  if (cudaMemcpy(s.w, wb.data(), sizeof(unsigned short) * kNParams, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s.aux, aux.data(), sizeof(float) * 35, cudaMemcpyHostToDevice) != cudaSuccess)
    return ST_CUDA;
  return ST_OK;
}

void launch_features(const double* Rs, int n, int64_t m, float* out, const Ctl* ctl, int level, cudaStream_t st) {
  { ::mrcqr::note_launch(); k_features<<<1, kFeatThreads, 0, st>>>(Rs, n, m, out, ctl, level); }
}

bool launch_mlp_select(const float* feat, Ctl* ctl, cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  Sel S;
  {
    std::lock_guard<std::mutex> lk(g_sel_mu);
    if (dev >= (int)g_sel.size() || !g_sel[dev].w) return false;
    S = Sel{g_sel[dev].w, g_sel[dev].aux, g_sel[dev].aux + 16, g_sel[dev].aux + 32};
  }
  { ::mrcqr::note_launch(); k_mlp_select<<<1, 64, 0, st>>>(S, feat, ctl); }
  return true;
}

void launch_mlp_forward(const unsigned short* w, const float* mu, const float* sd, const float* costs, int batch,
                        const float* X, float* logits, int32_t* choice, cudaStream_t st) {
  const Sel S{w, mu, sd, costs};
  const int grid = batch < 152 * 16 ? batch : 152 * 16;
  if (batch > 0) { ::mrcqr::note_launch(); k_mlp_forward<<<grid, 64, 0, st>>>(S, batch, X, logits, choice); }
}

void launch_mlp_grad(const unsigned short* w, const float* mu, const float* sd, int batch, const float* X,
                     const int32_t* y, const float* class_w, float* part, float* loss_part, int nparts,
                     cudaStream_t st) {
  const Sel S{w, mu, sd, nullptr};
  const int per = (batch + nparts - 1) / nparts;
  { ::mrcqr::note_launch(); k_mlp_grad_partial<<<nparts, 64, 0, st>>>(S, batch, per, X, y, class_w, part, loss_part); }
}

void launch_mlp_reduce_adamw(int nparts, const float* part, const float* loss_part, float* master, float* mom,
                             float* var, unsigned short* wbf16, float lr, float beta1, float beta2, float eps,
                             float wd, int step, int apply, float* grad_out, float* loss_out, cudaStream_t st) {
  { ::mrcqr::note_launch(); k_mlp_reduce_adamw<<<(kNParams + 255) / 256, 256, 0, st>>>(nparts, part, loss_part, master, mom, var, wbf16, lr,
                                                             beta1, beta2, eps, wd, step, apply, grad_out, loss_out); }
}

}  // namespace mrcqr
