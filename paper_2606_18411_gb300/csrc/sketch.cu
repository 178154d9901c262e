// Stage 1 of MRCQR (Algorithm 2 steps 1-4, Sec. II-A): random signs D, the
// sample set S, and the sketch Y = sqrt(m/s) P F D A with F the orthonormal
// DCT-II, computed in the sketch precision p.
//
// This file holds the SIMT kernels (every precision; the FP64 sketch always
// runs here because FP64 has no tensor-core path on this GPU) and the sketch
// dispatch; the tensor-core FP16/BF16/FP32 sketch lives in sketch_tc.cu.
#include <type_traits>
#include "kernels.h"

namespace mrcqr {

// ---------------------------------------------------------------------------
// Sample set (Algorithm 2 step 1): s distinct rows of {0..m-1}, uniform
// without replacement by Floyd's algorithm, sorted ascending.  The draw for
// j in [m-s, m) is r_j = (Philox(key, (j,1,0,0)).x * (j+1)) >> 32, uniform on
// {0..j}; Floyd keeps r_j unless it was already chosen, in which case it
// keeps j (never chosen before, since all earlier values are < j).
constexpr uint32_t kEmpty = 0xffffffffu;

// m is the population: the rows of the transform (DCT) or its floor(m/2) + 1
// bins (real FFT).  reim: idx[s + t] = idx[t] | kImRow, the Im rows of the
// same bins.
__device__ __forceinline__ void sample_block(int64_t m, int s, uint2 key, uint32_t* __restrict__ idx, int reim = 0) {
  extern __shared__ uint32_t sm[];
  int H = 1;
  while (H < 2 * s) H <<= 1;
  uint32_t* draws = sm;            // s
  uint32_t* hash = sm + s;         // H
  uint32_t* keys = hash + H;       // P (power of two >= s) for the sort
  int P = 1;
  while (P < s) P <<= 1;
  for (int t = threadIdx.x; t < s; t += blockDim.x) {
    const uint64_t j = (uint64_t)(m - s + t);
    const uint4 r = philox4x32_10(make_uint4((uint32_t)j, 1u, 0u, 0u), key);
    draws[t] = (uint32_t)(((uint64_t)r.x * (j + 1)) >> 32);
  }
  for (int h = threadIdx.x; h < H; h += blockDim.x) hash[h] = kEmpty;
  for (int p = threadIdx.x; p < P; p += blockDim.x) keys[p] = kEmpty;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int hb = __ffs(H) - 1;
    for (int t = 0; t < s; ++t) {
      const uint32_t j = (uint32_t)(m - s + t);
      uint32_t v = draws[t];
      // lookup v
      uint32_t h = (v * 2654435761u) >> (32 - max(hb, 1));
      h &= (H - 1);
      bool found = false;
      while (hash[h] != kEmpty) {
        if (hash[h] == v) { found = true; break; }
        h = (h + 1) & (H - 1);
      }
      if (found) {
        v = j;
        h = ((v * 2654435761u) >> (32 - max(hb, 1))) & (H - 1);
        while (hash[h] != kEmpty) h = (h + 1) & (H - 1);
      }
      hash[h] = v;
      keys[t] = v;
    }
  }
  __syncthreads();
  // bitonic sort of keys[0..P) ascending (padding kEmpty sorts last)
  for (int k = 2; k <= P; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int l = i ^ jj;
        if (l > i) {
          const uint32_t a = keys[i], b = keys[l];
          const bool up = (i & k) == 0;
          if ((a > b) == up) { keys[i] = b; keys[l] = a; }
        }
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < s; t += blockDim.x) {
    idx[t] = keys[t];
    if (reim) idx[s + t] = keys[t] | kImRow;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(1024) k_sample(int64_t m, int s, uint2 key, uint32_t* __restrict__ idx,
                                                  const Ctl* ctl, int reim) {
  (void)ctl;
  sample_block(m, s, key, idx, reim);
}

// s = the number of sampled rows (DCT) or bins (real FFT); the real-FFT
// transforms draw from the floor(m/2) + 1 bins of a real column.
void launch_sample(int64_t m, int s, uint64_t seed, uint32_t* idx, const Ctl* ctl, cudaStream_t st, int tf) {
  if (tf != T_DCT) m = m / 2 + 1;
  int H = 1;
  while (H < 2 * s) H <<= 1;
  int P = 1;
  while (P < s) P <<= 1;
  const size_t smem = sizeof(uint32_t) * (size_t)(s + H + P);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_sample, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  { ::mrcqr::note_launch(); k_sample<<<1, 1024, smem, st>>>(m, s, seed_key(seed), idx, ctl, tf == T_RFFT_REIM); }
}

// ---------------------------------------------------------------------------
// Quarter-wave table cos(pi q / (2m)), q = 0..m, in FP64.
__global__ void k_costab(int64_t m, double* __restrict__ tab) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q <= m) {
    const double c = cospi((double)q / (2.0 * (double)m));
    tab[q] = c;
  }
}

void launch_costab(int64_t m, double* tab, cudaStream_t st) {
  const int64_t nq = m + 1;
  { ::mrcqr::note_launch(); k_costab<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(m, tab); }
}

// fl_p exactly as the tensor-core sketch computes it (integer RNE on the
// FP64 bits), widened back to FP64.
__global__ void k_round(int prec, int64_t count, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double v = x[i];
  const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
  double r;
  if (prec == P_FP16) r = (double)__half2float(__ushort_as_half((unsigned short)f64bits_to_f16(hi, lo)));
  else if (prec == P_BF16) r = (double)__bfloat162float(__ushort_as_bfloat16((unsigned short)f64bits_to_bf16(hi, lo)));
  else if (prec == P_FP32) r = (double)__uint_as_float(f64bits_to_f32(hi, lo));
  else r = v;
  y[i] = r;
}

void launch_round(int prec, int64_t count, const double* x, double* y, cudaStream_t st) {
  { ::mrcqr::note_launch(); k_round<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(prec, count, x, y); }
}

__global__ void k_signs(int64_t m, uint2 key, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = row_sign((uint64_t)i, key);
}

void launch_signs(int64_t m, uint64_t seed, double* out, cudaStream_t st) {
  { ::mrcqr::note_launch(); k_signs<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(m, seed_key(seed), out); }
}

// ---------------------------------------------------------------------------
// SIMT sketch: a CTA owns a 64 (sample rows) x 64 (columns) tile of Y over
// one chunk of m and walks it in slabs of 32 rows.  Per slab: Rademacher
// signs from Philox, the sign-flipped A tile scaled per column by 2^e so
// that max |.| lies in [2^13, 2^14) (keeps FP16 clear of underflow), one
// rounding to p (fl_p), the transform entries cos(pi k (2j+1) / (2m))
// rounded to p, products accumulated in FP32 (FP64 for the FP64 sketch) and
// the scale undone.  Partials of every chunk go to Ypart and are summed in a
// fixed order by k_sketch_reduce (deterministic).
constexpr int kSkST = 64, kSkNT = 64, kSkT = 32;

template <int PREC>
__device__ __forceinline__ void sketch_simt_block(const double* __restrict__ A, int64_t lda, int64_t m, int n, int s,
                                                  const uint32_t* __restrict__ idx, const double* __restrict__ tab,
                                                  uint2 key, int64_t rows_per_chunk, double* __restrict__ Ypart,
                                                  int bx, int by, int bz, int tf) {
  using Acc = std::conditional_t<PREC == P_FP64, double, float>;
  constexpr int ST = kSkST, NT = kSkNT, T = kSkT;
  __shared__ double Xd[T][NT + 1];
  // FP64 reads its operand straight from Xd; the others round into Xs
  __shared__ __align__(16) Acc Xs[T][PREC == P_FP64 ? 1 : NT];
  __shared__ __align__(16) Acc Ss[T][ST];
  __shared__ Acc colscale[NT];
  __shared__ double sg[T];
  __shared__ uint32_t ks[ST];
  __shared__ uint64_t r0[ST], dks[ST];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int s0 = by * ST, n0 = bz * NT;
  const int64_t j_begin = (int64_t)bx * rows_per_chunk;
  const int64_t j_end = min(m, j_begin + rows_per_chunk);
  const uint64_t four_m = 4ull * (uint64_t)m;
  if (tid < ST) {
    ks[tid] = (s0 + tid < s) ? idx[s0 + tid] : kEmpty;
    dks[tid] = ks[tid] == kEmpty ? 0ull : row_phase(tf, ks[tid], (uint64_t)m).dk;
  }

  Acc acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = Acc(0);

  for (int64_t j0 = j_begin; j0 < j_end; j0 += T) {
    __syncthreads();
    if (tid < T) sg[tid] = (j0 + tid < j_end) ? row_sign((uint64_t)(j0 + tid), key) : 0.0;
    if (tid >= 64 && tid < 64 + ST) {
      const int i = tid - 64;
      r0[i] = ks[i] == kEmpty ? 0 : phase_at(row_phase(tf, ks[i], (uint64_t)m), (uint64_t)j0, four_m);
    }
    __syncthreads();
    for (int e = tid; e < T * NT; e += 256) {
      const int t = e % T, c = e / T;
      const int64_t j = j0 + t;
      const int col = n0 + c;
      double v = 0.0;
      if (j < j_end && col < n) v = A[j + (int64_t)col * lda] * sg[t];
      Xd[t][c] = v;
    }
    for (int e = tid; e < T * ST; e += 256) {
      const int i = e % ST, t = e / ST;
      const uint32_t k = ks[i];
      double v = 0.0;
      if (k != kEmpty && j0 + t < j_end) {
        const uint64_t r = (r0[i] + dks[i] * (uint64_t)t) % four_m;
        v = cos_phase(tab, (int64_t)r, m);
      }
      if constexpr (PREC == P_FP64) Ss[t][i] = v;
      else Ss[t][i] = round_to_p<PREC>(v);
    }
    __syncthreads();
    if constexpr (PREC != P_FP64) {
      if (tid < NT) {
        double amax = 0.0;
#pragma unroll 8
        for (int t = 0; t < T; ++t) amax = fmax(amax, fabs(Xd[t][tid]));
        const int e = scale_exponent(amax);
        colscale[tid] = (Acc)exp2i(-e);
        const double up = exp2i(e);
#pragma unroll 8
        for (int t = 0; t < T; ++t) Xs[t][tid] = round_to_p<PREC>(Xd[t][tid] * up);
      }
    }
    __syncthreads();
    Acc tmp[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) tmp[r][c] = Acc(0);
#pragma unroll 4
    for (int t = 0; t < T; ++t) {
      Acc a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = Ss[t][ty * 4 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if constexpr (PREC == P_FP64) b[c] = Xd[t][tx * 4 + c];
        else b[c] = Xs[t][tx * 4 + c];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) tmp[r][c] = fma(a[r], b[c], tmp[r][c]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if constexpr (PREC == P_FP64) acc[r][c] += tmp[r][c];
        else acc[r][c] = fma(tmp[r][c], colscale[tx * 4 + c], acc[r][c]);
      }
  }
  double* out = Ypart + (size_t)bx * (size_t)s * (size_t)n;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = s0 + ty * 4 + r, col = n0 + tx * 4 + c;
      if (i < s && col < n) out[(size_t)col * s + i] = (double)acc[r][c];
    }
  __syncthreads();
}

template <int PREC>
__global__ void __launch_bounds__(256) k_sketch_simt(const double* __restrict__ A, int64_t lda, int64_t m, int n,
                                                      int s, const uint32_t* __restrict__ idx,
                                                      const double* __restrict__ tab, uint2 key,
                                                      int64_t rows_per_chunk, double* __restrict__ Ypart,
                                                      const Ctl* ctl, int level, int tf) {
  if (level_inactive(ctl, level)) return;
  sketch_simt_block<PREC>(A, lda, m, n, s, idx, tab, key, rows_per_chunk, Ypart, blockIdx.x, blockIdx.y, blockIdx.z,
                          tf);
}

int sketch_chunks(int64_t m, int n, int s) {
  const int tiles = ((s + kSkST - 1) / kSkST) * ((n + kSkNT - 1) / kSkNT);
  int chunks = (4 * 152 + tiles - 1) / tiles;
  const int64_t max_chunks = (m + kSkT - 1) / kSkT;
  if (chunks > max_chunks) chunks = (int)max_chunks;
  if (chunks < 1) chunks = 1;
  return chunks;
}

static int64_t rows_per_chunk(int64_t m, int chunks) {
  int64_t r = (m + chunks - 1) / chunks;
  return (r + 63) / 64 * 64;
}

int sketch_max_chunks(int64_t m, int n, int s) {
  int c = sketch_chunks(m, n, s);
  for (int prec : {P_FP16, P_FP32}) {
    const int f = sketch_fs_chunks(prec, m, n);
    if (f > c) c = f;
  }
  return c;
}

// The faster tensor-core variant by measurement (dense rows V1 against the
// four-step V2) for precision prec at n columns (s = 2n); true picks the
// four-step.  Measured at m = 2^20 on GB300 (ms, V1 / V2, CUDA events over
// five calls): FP16 n = 128: 0.92 / 1.45, 192: 3.27 / 1.83, 256: 2.97 /
// 2.50, 320: 8.16 / 3.81, 512: 19.6 / 6.78 (BF16 within 1% of FP16); FP32
// n = 128: 1.93 / 2.16, 192: 7.80 / 3.14, 256: 7.12 / 4.24, 320: 20.1 /
// 6.10.  The dense-row variant's work grows as s n, the four-step's as n; the
// switch point sits between the measured sizes.
static bool four_step_preferred(int prec, int64_t m, int n) {
  (void)m;
  (void)prec;
  return n >= 160;
}

int launch_sketch(int prec, int variant, const double* A, int64_t lda, int64_t m, int n, int s,
                  const uint32_t* idx, const double* tab, uint64_t seed, int chunks,
                  double* Ypart, Ctl* ctl, int level, cudaStream_t st, int tf, int* chunks_used) {
  if (chunks_used) *chunks_used = chunks;
  const bool fs_ok = (variant == 0 || variant == 4) && sketch_fs_eligible(prec, tf, A, lda, m, n, s);
  if (fs_ok && (variant == 4 || four_step_preferred(prec, m, n))) {
    const int fc = sketch_fs_chunks(prec, m, n);
    if (launch_sketch_fs(prec, A, lda, m, n, s, idx, tab, seed, fc, Ypart, ctl, level, st)) {
      if (chunks_used) *chunks_used = fc;
      return 4;
    }
  }
  if (variant != 1 && sketch_tc_eligible(prec, A, lda) &&
      launch_sketch_tc(prec, A, lda, m, n, s, idx, tab, seed, chunks, Ypart, ctl, level, st, tf))
    return 2;
  const dim3 grid(chunks, (s + kSkST - 1) / kSkST, (n + kSkNT - 1) / kSkNT);
  const int64_t rpc = rows_per_chunk(m, chunks);
  const uint2 key = seed_key(seed);
  switch (prec) {
    case P_FP16: { ::mrcqr::note_launch(); k_sketch_simt<P_FP16><<<grid, 256, 0, st>>>(A, lda, m, n, s, idx, tab, key, rpc, Ypart, ctl, level, tf); } break;
    case P_BF16: { ::mrcqr::note_launch(); k_sketch_simt<P_BF16><<<grid, 256, 0, st>>>(A, lda, m, n, s, idx, tab, key, rpc, Ypart, ctl, level, tf); } break;
    case P_FP32: { ::mrcqr::note_launch(); k_sketch_simt<P_FP32><<<grid, 256, 0, st>>>(A, lda, m, n, s, idx, tab, key, rpc, Ypart, ctl, level, tf); } break;
    default: { ::mrcqr::note_launch(); k_sketch_simt<P_FP64><<<grid, 256, 0, st>>>(A, lda, m, n, s, idx, tab, key, rpc, Ypart, ctl, level, tf); } break;
  }
  return 1;
}

// Y = coef_i * sum over chunks (fixed order).  DCT: coef = sqrt(2/s) c_k with
// c_0 = 1/sqrt(2), the sqrt(m/s) sketch scale times the sqrt(2/m) c_k of the
// orthonormal DCT-II.  Real FFT: coef = sqrt(c/m) for c sampled bins (the
// unnormalised transform, Algorithm 2 as printed).
__device__ __forceinline__ void sketch_reduce_entry(int n, int s, int chunks, const double* __restrict__ Ypart,
                                                    const uint32_t* __restrict__ idx, double* __restrict__ Y,
                                                    Ctl* ctl, int64_t e, int tf = T_DCT, int64_t m = 0) {
  const int64_t total = (int64_t)s * n;
  const int i = (int)(e % s);
  double acc = 0.0;
  for (int c = 0; c < chunks; ++c) acc += Ypart[(size_t)c * total + e];
  const double coef = tf == T_DCT ? sqrt(2.0 / (double)s) * (idx[i] == 0 ? 0.70710678118654752440 : 1.0)
                                  : sqrt((double)(tf == T_RFFT_REIM ? s / 2 : s) / (double)m);
  const double y = acc * coef;
  Y[e] = y;
  if (!isfinite(y)) {
    ctl->input_nonfinite = 1;
    raise_level_status(ctl, ST_NONFINITE);
  }
}

__global__ void k_sketch_reduce(int n, int s, int chunks, const double* __restrict__ Ypart,
                                const uint32_t* __restrict__ idx, double* __restrict__ Y, Ctl* ctl, int level, int tf,
                                int64_t m) {
  if (level_inactive(ctl, level)) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < (int64_t)s * n) sketch_reduce_entry(n, s, chunks, Ypart, idx, Y, ctl, e, tf, m);
}

void launch_sketch_reduce(int64_t m, int n, int s, int chunks, const double* Ypart, const uint32_t* idx, double* Y,
                          Ctl* ctl, int level, cudaStream_t st, int tf) {
  const int64_t total = (int64_t)s * n;
  { ::mrcqr::note_launch(); k_sketch_reduce<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(n, s, chunks, Ypart, idx, Y, ctl, level, tf, m); }
}

// ---------------------------------------------------------------------------
// Grouped kernels (batched factorizations).
namespace {

constexpr int kGridCapS = 152 * 8;
inline unsigned gridS(int nitems) { return (unsigned)(nitems < kGridCapS ? (nitems > 0 ? nitems : 1) : kGridCapS); }

__global__ void kg_init(Group g) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.nitems) return;
  const Prob& P = g.probs[p];
  Ctl* c = P.ctl;
  c->active = 0;
  c->lvl_status = 0;
  c->final_status = ST_OK;
  c->prec_used = P.lvl_prec[0];
  c->retries = 0;
  c->prec_first = P.lvl_prec[0];
  c->nlevels = P.nlevels;
  c->input_nonfinite = 0;
  for (int i = 0; i < kMaxLevels; ++i) c->lvl_prec[i] = P.lvl_prec[i];
  c->mlp_choice = -1;
  c->pad0 = 0;
  c->tol = P.tol;
  c->ortho_fro = 0.0;
  for (int i = 0; i < kNumFeatures; ++i) c->features[i] = 0.f;
}

__global__ void __launch_bounds__(1024) kg_sample(Group g) {
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const Prob& P = g.probs[g.items[it].x];
    sample_block(P.tf == T_DCT ? P.m : P.m / 2 + 1, P.bins, P.key, P.idx, P.tf == T_RFFT_REIM);
  }
}

__global__ void kg_costab(Group g) {
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    const int64_t q = (int64_t)w.y * 256 + threadIdx.x;
    if (q <= P.m) {
      const double c = cospi((double)q / (2.0 * (double)P.m));
      P.tab[q] = c;
    }
  }
}

template <int PREC>
__global__ void __launch_bounds__(256) kg_sketch(Group g, int level) {
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (P.ctl->active != level) continue;
    sketch_simt_block<PREC>(P.A, P.lda, P.m, P.n, P.s, P.idx, P.tab, P.key, P.rows_per_chunk, P.ypart, w.y, w.z,
                            w.w, P.tf);
  }
}

__global__ void kg_sketch_reduce(Group g, int level) {
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (P.ctl->active != level) continue;
    const int64_t e = (int64_t)w.y * 256 + threadIdx.x;
    if (e < (int64_t)P.s * P.n) sketch_reduce_entry(P.n, P.s, P.chunks, P.ypart, P.idx, P.y, P.ctl, e, P.tf, P.m);
  }
}

}  // namespace

void launch_g_init(const Group& g, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_init<<<(g.nitems + 127) / 128, 128, 0, st>>>(g); }
}
static size_t g_sample_smem(int max_s) {
  int H = 1;
  while (H < 2 * max_s) H <<= 1;
  int P = 1;
  while (P < max_s) P <<= 1;
  return sizeof(uint32_t) * (size_t)(max_s + H + P);
}

void prepare_g_kernels(int max_s) {
  cudaFuncSetAttribute(kg_sample, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g_sample_smem(max_s));
}

void launch_g_sample(const Group& g, int max_s, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_sample<<<gridS(g.nitems), 1024, g_sample_smem(max_s), st>>>(g); }
}
void launch_g_costab(const Group& g, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_costab<<<gridS(g.nitems), 256, 0, st>>>(g); }
}
void launch_g_sketch(const Group& g, int prec, int level, cudaStream_t st) {
  if (!g.nitems) return;
  switch (prec) {
    case P_FP16: { ::mrcqr::note_launch(); kg_sketch<P_FP16><<<gridS(g.nitems), 256, 0, st>>>(g, level); } break;
    case P_BF16: { ::mrcqr::note_launch(); kg_sketch<P_BF16><<<gridS(g.nitems), 256, 0, st>>>(g, level); } break;
    case P_FP32: { ::mrcqr::note_launch(); kg_sketch<P_FP32><<<gridS(g.nitems), 256, 0, st>>>(g, level); } break;
    default: { ::mrcqr::note_launch(); kg_sketch<P_FP64><<<gridS(g.nitems), 256, 0, st>>>(g, level); } break;
  }
}
void launch_g_sketch_reduce(const Group& g, int level, cudaStream_t st) {
  if (g.nitems) { ::mrcqr::note_launch(); kg_sketch_reduce<<<gridS(g.nitems), 256, 0, st>>>(g, level); }
}

}  // namespace mrcqr
