// Regime classification without learning (Sec. II-C): estimates of
// kappa_2(A) that pick the sketch precision before a factorization (half up
// to 1e4, single up to 1e8, double beyond).
//
//   CholQR probe: Algorithm 1 on A (G = A^T A, Cholesky R, Q = A R^{-1}),
//     q = ||I - Q^T Q||_2, and kappa_2(A) >= sqrt(q / (u (1 + q))).
//   Block 1-norm estimate: kappa_2(A)^2 <= n ||G||_1 ||G^{-1}||_1, with
//     ||G^{-1}||_1 from the block estimator of Higham and Tisseur (SIAM J.
//     Matrix Anal. Appl. 21 (2000), Algorithm 2.4; t = 2 columns, at most 5
//     iterations, +-1 columns from Philox), G^{-1} applied through the
//     Cholesky factor by two substitutions.
//
// The m-row work (Gram matrices, Q = A R^{-1}) runs in the emulated-FP64
// tensor-core kernels of the factorization; the n x n work runs in one CTA.
// A Cholesky breakdown (kappa_2(A) beyond about u^-1/2) gives kappa = inf and
// the double-precision regime.
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace mrcqr {
namespace {

constexpr int kRegThreads = 1024;
constexpr int kRegMaxN = 512;
constexpr int kPowerIters = 40;
constexpr int kT = 2;               // columns of the estimator's blocks
constexpr int kItMax = 5;
constexpr int kMaxResample = 100;
constexpr double kUnitRoundoff = 1.1102230246251565404e-16;   // 2^-53

__device__ __forceinline__ double regime_of(double kappa) {
  if (kappa <= 1e4) return 0.0;
  if (kappa <= 1e8) return 1.0;
  return 2.0;   // beyond 1e8, inf and NaN
}

__device__ __forceinline__ double sym_at(const double* __restrict__ E, int n, int i, int j) {
  return i <= j ? E[i + (int64_t)j * n] : E[j + (int64_t)i * n];
}

// q = ||E - I||_2 for the Gram E = Q^T Q (upper triangle, ld n) by power
// iteration from a fixed start (a lower bound that rises to q), then the
// probe bound.  out = {kappa, regime, q, 0}.
__global__ void __launch_bounds__(kRegThreads) k_probe(int n, const double* __restrict__ E, const Ctl* ctl,
                                                       double* __restrict__ out) {
  __shared__ double x[kRegMaxN], y[kRegMaxN];
  __shared__ double scratch[33];
  const int tid = threadIdx.x;
  if (ctl->lvl_status != 0) {
    if (tid == 0) {
      out[0] = INFINITY;
      out[1] = 2.0;
      out[2] = INFINITY;
      out[3] = 0.0;
    }
    return;
  }
  for (int i = tid; i < n; i += blockDim.x) x[i] = 1.0 + (double)((i * 7919) % 97) / 194.0;
  __syncthreads();
  double q = 0.0;
  for (int it = 0; it < kPowerIters; ++it) {
    double yy = 0.0, xx = 0.0;
    if (tid < n) {
      double acc = -x[tid];
      for (int j = 0; j < n; ++j) acc = fma(sym_at(E, n, tid, j), x[j], acc);
      y[tid] = acc;
      yy = acc * acc;
      xx = x[tid] * x[tid];
    }
    const double ny2 = block_sum(yy, scratch);
    const double nx2 = block_sum(xx, scratch);
    q = ny2 > 0.0 ? sqrt(ny2 / nx2) : 0.0;
    if (ny2 == 0.0) break;
    const double inv = 1.0 / sqrt(ny2);
    if (tid < n) x[tid] = y[tid] * inv;
    __syncthreads();
  }
  if (tid == 0) {
    const double kappa = sqrt(q / (kUnitRoundoff * (1.0 + q)));
    out[0] = kappa;
    out[1] = regime_of(kappa);
    out[2] = q;
    out[3] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// Block 1-norm estimate of G^{-1} = R^{-1} R^{-T} (G = R^T R), thread (c, i)
// = (tid / 512, tid % 512) owns entry i of block column c.  The control flow
// of the algorithm runs in thread 0 on shared state, the products in all
// threads; every loop is bounded.
struct Est {
  double X[kT][kRegMaxN];     // current block (unit 1-norm columns)
  double V[kT][kRegMaxN];     // substitution workspace
  double Y[kT][kRegMaxN];     // B X, then B S
  signed char S[kT][kRegMaxN], So[kT][kRegMaxN];
  double h[kRegMaxN];
  int hist[kT * (kItMax + 2)];
  int nhist, ind[kT], ind_best, draw, stop, flag;
  double est, est_old;
};

// Y[c] = G^{-1} X[c] for both columns: R^T v = x (forward, rows of R from RT),
// then R y = v (backward, columns of R).  One barrier per step.
__device__ void apply_ginv(Est& e, int n, const double* __restrict__ R, const double* __restrict__ RT, int npad,
                           const double* __restrict__ rinv) {
  const int c = threadIdx.x / kRegMaxN, i = threadIdx.x % kRegMaxN;
  const bool live = i < n;
  double* w = e.Y[c];      // running right-hand side of the forward sweep
  double* v = e.V[c];
  if (live) w[i] = e.X[c][i];
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const double vj = w[j] * rinv[j];
    if (live) {
      if (i == j) v[j] = vj;
      else if (i > j) w[i] = fma(-RT[(int64_t)j * npad + i], vj, w[i]);
    }
    __syncthreads();
  }
  // backward: running right-hand side in v, solution into Y
  for (int j = n - 1; j >= 0; --j) {
    const double yj = v[j] * rinv[j];
    if (live) {
      if (i == j) w[j] = yj;
      else if (i < j) v[i] = fma(-R[i + (int64_t)j * n], yj, v[i]);
    }
    __syncthreads();
  }
}

// Two +-1 columns are parallel when they are equal or opposite; a zero column
// (S before the first iteration) is parallel to none.
__device__ __forceinline__ bool parallel_cols(const signed char* a, const signed char* b, int n) {
  int eq = 0, opp = 0;
  for (int i = 0; i < n; ++i) {
    eq += a[i] == b[i];
    opp += a[i] == -b[i];
  }
  return eq == n || opp == n;
}

__device__ __forceinline__ bool all_same_sign(const signed char* a, int n) {
  int pos = 0;
  for (int i = 0; i < n; ++i) pos += a[i] > 0;
  return pos == n || pos == 0;
}

// Column c of S := the next random +-1 column (draw e.draw), all threads.
__device__ __forceinline__ void fill_random(Est& e, int col, int n, uint2 key) {
  const int c = threadIdx.x / kRegMaxN, i = threadIdx.x % kRegMaxN;
  if (c == 0 && i < n) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)i, 2u, (uint32_t)e.draw, 0u), key);
    e.S[col][i] = (r.x & 1u) ? -1 : 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) ++e.draw;
  __syncthreads();
}

// out = {kappa, regime, ||G||_1, est ||G^-1||_1}; G upper triangle (ld n),
// R upper (ld n), RT[k][c] = R[k][c] (row stride npad), rinv = 1/diag(R).
__global__ void __launch_bounds__(kRegThreads) k_onenorm(int n, const double* __restrict__ G,
                                                         const double* __restrict__ R, const double* __restrict__ RT,
                                                         int npad, const double* __restrict__ rinv, uint2 key,
                                                         const Ctl* ctl, double* __restrict__ out) {
  __shared__ Est e;
  __shared__ double colsum[kRegMaxN];
  const int tid = threadIdx.x, c = tid / kRegMaxN, i = tid % kRegMaxN;
  // ||G||_1 = largest column sum of |G| (G symmetric, upper triangle stored)
  if (c == 0 && i < n) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += fabs(sym_at(G, n, k, i));
    colsum[i] = s;
  }
  __syncthreads();
  if (ctl->lvl_status != 0) {
    if (tid == 0) {
      double g1 = 0.0;
      for (int k = 0; k < n; ++k) g1 = fmax(g1, colsum[k]);
      out[0] = INFINITY;
      out[1] = 2.0;
      out[2] = g1;
      out[3] = INFINITY;
    }
    return;
  }
  if (tid == 0) {
    e.draw = 0;
    e.nhist = 0;
    e.stop = 0;
    e.est = e.est_old = 0.0;
    e.ind[0] = e.ind[1] = 0;
    e.ind_best = 0;
  }
  __syncthreads();
  if (n <= 4) {
    // exact: G^{-1} applied to the unit vectors (two per pass)
    double best = 0.0;
    for (int p = 0; p < n; p += kT) {
      if (i < n) e.X[c][i] = (i == p + c) ? 1.0 : 0.0;
      __syncthreads();
      apply_ginv(e, n, R, RT, npad, rinv);
      if (tid == 0)
        for (int cc = 0; cc < kT && p + cc < n; ++cc) {
          double s = 0.0;
          for (int k = 0; k < n; ++k) s += fabs(e.Y[cc][k]);
          best = fmax(best, s);
        }
      __syncthreads();
    }
    if (tid == 0) e.est = best;
  } else {
    // starting block: e / n and a random +-1 / n column not parallel to it
    fill_random(e, 1, n, key);
    for (int a = 0; a < kMaxResample; ++a) {
      if (tid == 0) e.flag = all_same_sign(e.S[1], n);
      __syncthreads();
      const int redraw = e.flag;
      __syncthreads();   // every thread has read the flag before thread 0 writes it again
      if (!redraw) break;
      fill_random(e, 1, n, key);
    }
    if (i < n) e.X[c][i] = (c == 0 ? 1.0 : (double)e.S[1][i]) / (double)n;
    if (i < n) e.S[c][i] = 0;   // S = 0 before the first iteration
    __syncthreads();
    for (int k = 1; k <= kItMax + 1; ++k) {
      apply_ginv(e, n, R, RT, npad, rinv);
      if (tid == 0) {
        double nrm[kT];
        for (int cc = 0; cc < kT; ++cc) {
          double s = 0.0;
          for (int r = 0; r < n; ++r) s += fabs(e.Y[cc][r]);
          nrm[cc] = s;
        }
        const int jb = nrm[1] > nrm[0] ? 1 : 0;
        double est = nrm[jb];
        if (est > e.est_old || k == 2) e.ind_best = e.ind[jb];
        if (k >= 2 && est <= e.est_old) {   // no increase: keep the previous estimate
          est = e.est_old;
          e.stop = 1;
        } else {
          e.est_old = est;
          if (k > kItMax) e.stop = 1;
        }
        e.est = est;
      }
      __syncthreads();
      if (e.stop) break;
      // S_old = S, S = sign(Y) (sign 0 = +1)
      if (i < n) {
        e.So[c][i] = e.S[c][i];
        e.S[c][i] = e.Y[c][i] >= 0.0 ? 1 : -1;
      }
      __syncthreads();
      if (tid == 0) {   // every column of S parallel to a column of S_old: converged
        bool all = true;
        for (int j = 0; j < kT && all; ++j) {
          bool any = false;
          for (int o = 0; o < kT; ++o) any = any || parallel_cols(e.S[j], e.So[o], n);
          all = any;
        }
        e.stop = all;
      }
      __syncthreads();
      if (e.stop) break;
      // no column parallel to an earlier column of S or to a column of S_old
      for (int j = 0; j < kT; ++j)
        for (int a = 0; a < kMaxResample; ++a) {
          if (tid == 0) {
            bool par = false;
            for (int o = 0; o < j; ++o) par = par || parallel_cols(e.S[j], e.S[o], n);
            for (int o = 0; o < kT; ++o) par = par || parallel_cols(e.S[j], e.So[o], n);
            e.flag = par;
          }
          __syncthreads();
          const int redraw = e.flag;
          __syncthreads();
          if (!redraw) break;
          fill_random(e, j, n, key);
        }
      // Z = B^T S = B S (B symmetric), h_r = max_c |Z[r][c]|
      if (i < n) e.X[c][i] = (double)e.S[c][i];
      __syncthreads();
      apply_ginv(e, n, R, RT, npad, rinv);
      if (c == 0 && i < n) e.h[i] = fmax(fabs(e.Y[0][i]), fabs(e.Y[1][i]));
      __syncthreads();
      if (tid == 0) {
        double hmax = 0.0;
        for (int r = 0; r < n; ++r) hmax = fmax(hmax, e.h[r]);
        if (k >= 2 && hmax == e.h[e.ind_best]) e.stop = 1;
        if (!e.stop) {
          // the t largest h (ties by index) among all rows, then among rows not used before
          auto in_hist = [&](int r) {
            for (int q = 0; q < e.nhist; ++q)
              if (e.hist[q] == r) return true;
            return false;
          };
          auto top = [&](bool skip_hist, int* pick) {
            int got = 0;
            for (int t = 0; t < kT; ++t) {
              int best = -1;
              for (int r = 0; r < n; ++r) {
                if (skip_hist && in_hist(r)) continue;
                bool taken = false;
                for (int q = 0; q < got; ++q) taken = taken || pick[q] == r;
                if (taken) continue;
                if (best < 0 || e.h[r] > e.h[best]) best = r;
              }
              if (best < 0) break;
              pick[got++] = best;
            }
            return got;
          };
          int lead[kT], fresh[kT];
          const int nl = top(false, lead);
          bool all_used = nl == kT;
          for (int t = 0; t < nl; ++t) all_used = all_used && in_hist(lead[t]);
          if (all_used) {
            e.stop = 1;
          } else if (top(true, fresh) < kT) {
            e.stop = 1;
          } else {
            for (int t = 0; t < kT; ++t) {
              e.ind[t] = fresh[t];
              e.hist[e.nhist++] = fresh[t];
            }
          }
        }
      }
      __syncthreads();
      if (e.stop) break;
      if (i < n) e.X[c][i] = (i == e.ind[c]) ? 1.0 : 0.0;
      __syncthreads();
    }
  }
  if (tid == 0) {
    double g1 = 0.0;
    for (int k = 0; k < n; ++k) g1 = fmax(g1, colsum[k]);
    const double kappa = sqrt((double)n * g1 * e.est);
    out[0] = kappa;
    out[1] = regime_of(kappa);
    out[2] = g1;
    out[3] = e.est;
  }
}

}  // namespace

void launch_probe(int n, const double* E, const Ctl* ctl, double* out, cudaStream_t st) {
  { ::mrcqr::note_launch(); k_probe<<<1, kRegThreads, 0, st>>>(n, E, ctl, out); }
}

void launch_onenorm(int n, const double* G, const double* R, const double* RT, const double* rinv, uint64_t seed,
                    const Ctl* ctl, double* out, cudaStream_t st) {
  const int npad = (n + 31) / 32 * 32;
  { ::mrcqr::note_launch(); k_onenorm<<<1, kRegThreads, 0, st>>>(n, G, R, RT, npad, rinv, seed_key(seed), ctl, out); }
}

}  // namespace mrcqr
