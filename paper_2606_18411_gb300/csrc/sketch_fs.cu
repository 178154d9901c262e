// Four-step sketch: variant V2 of Algorithm 2 steps 2-4 (a fast transform,
// the butterfly route of Sec. II-A and Table 3, in place of the dense row
// evaluation of sketch_tc.cu) for the DCT-II and the FP16, BF16 and FP32
// sketch precisions, m a multiple of 1024.
//
// With m = 64 m1 and the row index j = j1 + m1 j2 (j1 < m1, j2 < 64),
//   y_k = sum_j x_j cos(pi k (2j + 1) / (2m))
//       = sum_{j1} Re( e^{i phi(k, j1)} U[j1][k mod 128] ),
//   phi(k, j1) = pi k (2 j1 + 1) / (2m),
//   U[j1][r]   = sum_{j2 < 64} x_{j1 + m1 j2} e^{i pi r j2 / 64},
// because pi k (2j + 1) / (2m) = phi(k, j1) + pi k j2 / 64.  x is real, so
// U[j1][128 - r] = conj(U[j1][r]): 65 real parts (r = 0..64) and 63
// imaginary parts (r = 1..63) hold all of U[j1].
//
// Step 1, the first butterfly level (a radix-64 DFT of the strided
// subsequences), runs on the tensor cores: D = W X with W the 128 x 64 real
// DFT matrix (rows cos(pi r j2 / 64), r = 0..64, then sin(pi r j2 / 64),
// r = 1..63) rounded to p, and X the sign-flipped, per-tile per-column 2^e
// scaled, p-rounded values of A (the fl_p of sketch_tc.cu; FP32 as 3xTF32).
// A tile is 16 consecutive j1 x 64 j2 x C columns of A, brought by one 3-D
// TMA copy (16 rows of 128 contiguous bytes per j2 and column), so A is
// read from HBM once.
// Step 2 is pruned to the s sampled k: each sample reads its residue row
// pair of U from shared memory, applies the twiddle e^{i phi(k, j1)}
// (FP32, exact integer phase, sincospi every four j1 and exact rotations in
// between) and the inverse column scale, and accumulates in FP32 registers
// over the CTA's j1 range; partial sums per j1 chunk go to the same FP64
// reduction as the other variants.
//
// Per tile: TMA (3 stages) -> convert into the MMA operand (2 buffers) ->
// one thread issues the MMAs into TMEM (2 buffers) -> while those run, the
// previous tile's D is copied to shared memory and step 2 runs on it.  Every
// wait is bounded; on a timeout the CTA waits (bounded) for its own copies
// in flight, frees its TMEM, raises TIMEOUT and returns.
#include <mutex>

#include "kernels.h"
#include "tc.cuh"

namespace mrcqr {

namespace {

constexpr int kB = 16;           // j1 per tile
constexpr int kM2 = 64;          // length of the strided DFT
constexpr int kRows = 2 * kM2;   // real rows of W = MMA M
constexpr int kThreads = 512;
constexpr int kMaxS = 1024;
constexpr int kKpt = kMaxS / kThreads;   // samples per thread at most

template <int PREC>
struct Fs {
  static constexpr int C = (PREC == P_FP32) ? 2 : 4;          // columns per tile
  static constexpr int N = kB * C;                            // MMA N: (j1, column) pairs
  static constexpr int EB = (PREC == P_FP32) ? 4 : 2;         // operand bytes
  static constexpr int PARTS = (PREC == P_FP32) ? 2 : 1;      // big (+ small) parts
  static constexpr int KSTEP = (PREC == P_FP32) ? 8 : 16;     // K per instruction
  static constexpr int KPANELS = kM2 * EB / 128;              // 128-byte SW128 panels along K
  static constexpr int KPER = 128 / EB;                       // K per panel
  static constexpr uint32_t FMT = (PREC == P_FP32) ? tc::TF32 : (PREC == P_BF16 ? tc::BF16 : tc::F16);
  static constexpr uint32_t W_PANEL = kRows * 128;
  static constexpr uint32_t X_PANEL = N * 128;
  static constexpr uint32_t XD_BYTES = kB * kM2 * C * 8;      // one FP64 tile
  static constexpr int STAGES = 3;
  static constexpr int USTR = N + 1;                          // U row stride (floats), conflict-free columns
  static constexpr uint32_t W_OFF = 0;                                   // [PARTS][KPANELS]
  static constexpr uint32_t X_OFF = W_OFF + PARTS * KPANELS * W_PANEL;   // [2][PARTS][KPANELS]
  static constexpr uint32_t XD_OFF = X_OFF + 2 * PARTS * KPANELS * X_PANEL;
  static constexpr uint32_t U_OFF = XD_OFF + STAGES * XD_BYTES;          // (kRows + 1) x USTR floats
  static constexpr uint32_t SMEM = U_OFF + (kRows + 1) * USTR * 4;
  static constexpr uint32_t TMEM_COLS = 2 * N <= 64 ? 64 : 128;
};

// fl_p of a table entry (FP64 bits) at (r, k) of the W operand.
template <int PREC>
__device__ __forceinline__ void store_w(unsigned char* w, int r, int k, uint32_t hi, uint32_t lo) {
  using F = Fs<PREC>;
  unsigned char* panel = w + (k / F::KPER) * F::W_PANEL;
  const int kk = k % F::KPER;
  if constexpr (PREC == P_FP16) {
    *reinterpret_cast<unsigned short*>(panel + tc::sw128_offset(r, kk, 2)) = (unsigned short)f64bits_to_f16(hi, lo);
  } else if constexpr (PREC == P_BF16) {
    *reinterpret_cast<unsigned short*>(panel + tc::sw128_offset(r, kk, 2)) = (unsigned short)f64bits_to_bf16(hi, lo);
  } else {
    const float f = __uint_as_float(f64bits_to_f32(hi, lo));
    const uint32_t b = tc::to_tf32(f);
    *reinterpret_cast<uint32_t*>(panel + tc::sw128_offset(r, kk, 4)) = b;
    *reinterpret_cast<uint32_t*>(panel + F::KPANELS * F::W_PANEL + tc::sw128_offset(r, kk, 4)) =
        tc::to_tf32(f - __uint_as_float(b));
  }
}

__device__ __forceinline__ uint64_t u64_max_warp(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

template <int PREC>
__global__ void __launch_bounds__(kThreads, 1)
    k_sketch_fs(const __grid_constant__ CUtensorMap tmap, int64_t m, int n, int s, const uint32_t* __restrict__ idx,
                const double* __restrict__ tab, uint2 key, int chunks, int tiles_per_chunk,
                double* __restrict__ Ypart, Ctl* ctl, int level) {
  using F = Fs<PREC>;
  constexpr int C = F::C, N = F::N;
  if (level_inactive(ctl, level)) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* wop = smem + F::W_OFF;
  unsigned char* xop = smem + F::X_OFF;
  double* xd = reinterpret_cast<double*>(smem + F::XD_OFF);
  float* U = reinterpret_cast<float*>(smem + F::U_OFF);
  __shared__ __align__(8) uint64_t tma_bar[F::STAGES];
  __shared__ __align__(8) uint64_t mma_bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ float colscale[2][C];
  __shared__ uint32_t red32[kThreads / 32][C];
  __shared__ uint64_t redmax[kThreads / 32];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t m1 = m / kM2;
  const uint64_t four_m = 4ull * (uint64_t)m;
  const int ncb = (n + C - 1) / C;
  const int nitems = ncb * chunks;
  // this CTA's items: blockIdx.x, blockIdx.x + gridDim.x, ...; every item has tiles_per_chunk tiles
  const int my_items = blockIdx.x < nitems ? (nitems - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int total = my_items * tiles_per_chunk;

  if (warp == 0) tc::tmem_alloc(&tmem_base, F::TMEM_COLS);
  if (tid == 0) {
    for (int st = 0; st < F::STAGES; ++st) tc::mbar_init(&tma_bar[st], 1);
    tc::mbar_init(&mma_bar[0], 1);
    tc::mbar_init(&mma_bar[1], 1);
    tc::mbar_fence_init();
  }
  // W: cos / sin(pi r j2 / 64) as phases of the quarter-wave table, P = r j2 m / 32
  for (int e = tid; e < kRows * kM2; e += kThreads) {
    const int row = e / kM2, j2 = e % kM2;
    const bool im = row > 64;
    const int r = im ? row - 64 : row;
    const uint64_t P = ((uint64_t)r * (uint64_t)j2 * (uint64_t)(m / 32)) % four_m;
    const uint64_t Pq = im ? (P <= (uint64_t)m ? (uint64_t)m - P : (uint64_t)m + four_m - P) : P;   // pi/2 - x
    uint32_t hi, lo;
    cos_phase_bits(tab, (int64_t)Pq, m, hi, lo);
    store_w<PREC>(wop, row, j2, hi, lo);
  }
  for (int e = tid; e < F::USTR; e += kThreads) U[kRows * F::USTR + e] = 0.f;   // the zero row (no Im part)
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;

  auto tile_of = [&](int u, int& item, int& j1_0) {
    const int il = u / tiles_per_chunk, ti = u % tiles_per_chunk;
    item = (int)blockIdx.x + il * (int)gridDim.x;
    j1_0 = ((item / ncb) * tiles_per_chunk + ti) * kB;
  };
  auto issue_tma = [&](int u) {
    int item, j1_0;
    tile_of(u, item, j1_0);
    const int st = u % F::STAGES;
    tc::mbar_expect_tx(&tma_bar[st], F::XD_BYTES);
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(tc::smem_u32(xd + st * (F::XD_BYTES / 8))),
        "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(j1_0), "r"(0), "r"((item % ncb) * C),
        "r"(tc::smem_u32(&tma_bar[st]))
        : "memory");
  };
  int issued = 0;
  if (tid == 0)
    for (; issued < F::STAGES && issued < total; ++issued) issue_tma(issued);

  // step-2 sample order: the samples sorted by the U row they read (a counting sort over the 65 real
  // rows), so a warp's samples read one or two neighbouring rows (broadcasts and distinct banks, where
  // random rows collide on a bank about 3.5-fold); each sample is still summed by one thread in the
  // same order, so Y does not change
  __shared__ uint16_t sorder[kMaxS];
  __shared__ int sbucket[66];
  if (tid < 66) sbucket[tid] = 0;
  __syncthreads();
  auto row_of = [&](int e) {
    const int r = (int)(idx[e] & 127u);
    return r <= 64 ? r : 128 - r;
  };
  for (int e = tid; e < s; e += kThreads) atomicAdd(&sbucket[row_of(e) + 1], 1);
  __syncthreads();
  if (tid == 0)
    for (int b = 1; b < 66; ++b) sbucket[b] += sbucket[b - 1];
  __syncthreads();
  for (int e = tid; e < s; e += kThreads) sorder[atomicAdd(&sbucket[row_of(e)], 1)] = (uint16_t)e;
  __syncthreads();

  // step-2 identity: G thread groups share the samples when s is small (each group takes C / G of
  // the tile's columns, so every thread works); thread t: group t / SPT, sample slots t % SPT + SPT i,
  // slot v taking sample sorder[v]
  int G = 1;
  while (G < C && s * (G * 2) <= kThreads) G *= 2;
  const int SPT = kThreads / G;
  const int grp = tid / SPT, slot = tid % SPT;
  const int cg_lo = grp * (C / G), cg_hi = cg_lo + C / G;
  const float inv2m = 1.0f / (2.0f * (float)m);
  const uint32_t fm32 = (uint32_t)four_m;   // 4m <= 2^24
  int srow_r[kKpt], srow_i[kKpt];
  float ssig[kKpt], rot_c[kKpt], rot_s[kKpt];
  uint32_t sk[kKpt], sk2[kKpt], sk32[kKpt], ph[kKpt];   // k, 2k, 32k mod 4m, phase k (2 j1_0 + 1) mod 4m
#pragma unroll
  for (int i = 0; i < kKpt; ++i) {
    const int sv = slot + SPT * i;
    srow_r[i] = srow_i[i] = kRows;
    ssig[i] = 0.f;
    rot_c[i] = 1.f;
    rot_s[i] = 0.f;
    sk[i] = sk2[i] = sk32[i] = ph[i] = 0u;
    if (sv < s) {
      const uint32_t k = idx[sorder[sv]];
      const int r = (int)(k & 127u);
      const int rp = r <= 64 ? r : 128 - r;
      srow_r[i] = rp;
      srow_i[i] = (rp == 0 || rp == 64) ? kRows : 64 + rp;
      ssig[i] = r <= 64 ? 1.f : -1.f;
      sk[i] = k;
      sk2[i] = 2u * k;
      sk32[i] = (uint32_t)((32ull * k) % four_m);
      // rotation by pi k / m per j1 step (exact argument for power-of-two m; otherwise within an ulp)
      sincospif((float)sk2[i] * inv2m, &rot_s[i], &rot_c[i]);
    }
  }
  float acc[kKpt][C];
#pragma unroll
  for (int i = 0; i < kKpt; ++i)
#pragma unroll
    for (int c = 0; c < C; ++c) acc[i][c] = 0.f;

  // conversion identity: j1 = tid % 16, j2 pair (2p, 2p + 1) with p = tid / 16, every column
  const int cj1 = tid & 15, cp = tid >> 4;
  const uint32_t idesc = tc::idesc(F::FMT, kRows, N);
  bool abort = false;
  int consumed = 0, mma_issued = 0, mma_done = 0;

  auto step2 = [&](int u) {   // U holds the tile u products; column c, j1 jj at U column c kB + jj
    int item, j1_0;
    tile_of(u, item, j1_0);
    const int b = u & 1;
    const bool first = u % tiles_per_chunk == 0;
#pragma unroll
    for (int i = 0; i < kKpt; ++i) {
      if (slot + SPT * i >= s) continue;
      // phase at this tile's first j1: from scratch at an item's first tile, else advanced by 16 j1
      if (first) ph[i] = (uint32_t)(((uint64_t)sk[i] * (uint64_t)(2 * j1_0 + 1)) % four_m);
      uint32_t P = ph[i];
      const float* ur = U + srow_r[i] * F::USTR;
      const float* ui = U + srow_i[i] * F::USTR;
      const float sg = ssig[i];
      float cph = 0.f, sph = 0.f;
#pragma unroll
      for (int jj = 0; jj < kB; ++jj) {
        if ((jj & 3) == 0) {   // exact twiddle every four j1, the phase an integer below 2^24
          sincospif((float)P * inv2m, &sph, &cph);
        } else {
          const float c2 = cph * rot_c[i] - sph * rot_s[i];
          sph = sph * rot_c[i] + cph * rot_s[i];
          cph = c2;
        }
        P += sk2[i];
        if (P >= fm32) P -= fm32;
        const float ss = sg * sph;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          if (c < cg_lo || c >= cg_hi) continue;
          const float t = fmaf(cph, ur[c * kB + jj], -ss * ui[c * kB + jj]);
          acc[i][c] = fmaf(t, colscale[b][c], acc[i][c]);
        }
      }
      uint32_t nx = ph[i] + sk32[i];
      if (nx >= fm32) nx -= fm32;
      ph[i] = nx;
    }
    if (u % tiles_per_chunk == tiles_per_chunk - 1) {   // last tile of the item: write its partial sums
      const int ch = item / ncb, c0 = (item % ncb) * C;
      double* out = Ypart + (size_t)ch * (size_t)s * (size_t)n;
#pragma unroll
      for (int i = 0; i < kKpt; ++i) {
        const int sv = slot + SPT * i;
        const int si = sv < s ? (int)sorder[sv] : 0;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          if (sv < s && c >= cg_lo && c < cg_hi && c0 + c < n) out[(size_t)(c0 + c) * s + si] = (double)acc[i][c];
          acc[i][c] = 0.f;
        }
      }
    }
  };

  auto d_to_smem = [&](int u) {   // TMEM buffer of tile u -> U (rows 32 q + lane, columns of group g)
    const int q = warp & 3, g = warp >> 2;
    constexpr int CW = N / 4;
    const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((u & 1) * N + g * CW);
    float v[CW];
    if constexpr (CW == 16) tc::tmem_ld16(base, v);
    else tc::tmem_ld8(base, v);
    tc::tmem_wait_ld();
    float* dst = U + (q * 32 + lane) * F::USTR + g * CW;
#pragma unroll
    for (int j = 0; j < CW; ++j) dst[j] = v[j];
  };

  for (int u = 0; u < total; ++u) {
    const int stage = u % F::STAGES;
    const uint32_t par = (uint32_t)((u / F::STAGES) & 1);
    const int buf = u & 1;
    int item, j1_0;
    tile_of(u, item, j1_0);
    // signs of this thread's two rows j = j1_0 + cj1 + m1 (2 cp + h)
    uint32_t sgn[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint64_t j = (uint64_t)(j1_0 + cj1) + (uint64_t)m1 * (uint64_t)(2 * cp + h);
      sgn[h] = (philox4x32_10(make_uint4((uint32_t)j, 0u, 0u, 0u), key).x & 1u) << 31;
    }
    const bool ok_tma = tc::mbar_wait(&tma_bar[stage], par);
    if (__syncthreads_or(!ok_tma)) {
      abort = true;
      break;
    }
    consumed = u + 1;
    const uint2* X = reinterpret_cast<const uint2*>(xd + stage * (F::XD_BYTES / 8));
    uint32_t vh[C][2], vl[C][2];
#pragma unroll
    for (int c = 0; c < C; ++c) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint2 w = X[(c * kM2 + 2 * cp + h) * kB + cj1];
        vh[c][h] = w.y ^ sgn[h];
        vl[c][h] = w.x;
      }
      // the exponent field orders |x| like the value: the high words' maximum gives the scale
      const uint32_t mx = __reduce_max_sync(0xffffffffu, max(vh[c][0] & 0x7FFFFFFFu, vh[c][1] & 0x7FFFFFFFu));
      if (lane == 0) red32[warp][c] = mx;
    }
    __syncthreads();
    if (tid < C) {
      uint32_t mx = 0u;
      for (int w = 0; w < kThreads / 32; ++w) mx = max(mx, red32[w][tid]);
      red32[0][tid] = mx;
    }
    __syncthreads();
    unsigned char* xb = xop + buf * F::PARTS * F::KPANELS * F::X_PANEL;
    const int c0t = (item % ncb) * C;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const uint32_t hmx = red32[0][c];
      int e = 0;
      if (c0t + c < n) {
        if ((hmx >> 20) != 0u) {
          e = scale_exponent_bits(hmx, 1u);
        } else {   // no normal value in this tile column: the exact 64-bit maximum (uniform branch)
          const uint64_t a0 = ((uint64_t)(vh[c][0] & 0x7FFFFFFFu) << 32) | vl[c][0];
          const uint64_t a1 = ((uint64_t)(vh[c][1] & 0x7FFFFFFFu) << 32) | vl[c][1];
          const uint64_t mw = u64_max_warp(a0 > a1 ? a0 : a1);
          __syncthreads();
          if (lane == 0) redmax[warp] = mw;
          __syncthreads();
          uint64_t mb = 0;
          for (int w = 0; w < kThreads / 32; ++w) mb = redmax[w] > mb ? redmax[w] : mb;
          e = scale_exponent_bits((uint32_t)(mb >> 32), (uint32_t)mb);
        }
      }
      if (tid == 0) colscale[buf][c] = ldexpf(1.0f, -e);
      const int row = c * kB + cj1;   // MMA N index: (column, j1)
      if constexpr (PREC == P_FP32) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t hh = vh[c][h], ll = vl[c][h];
          scale_bits(hh, ll, e);
          const float f = __uint_as_float(f64bits_to_f32(hh, ll));
          const uint32_t bg = tc::to_tf32(f);
          const int k = 2 * cp + h;
          unsigned char* pan = xb + (k / F::KPER) * F::X_PANEL;
          *reinterpret_cast<uint32_t*>(pan + tc::sw128_offset(row, k % F::KPER, 4)) = bg;
          *reinterpret_cast<uint32_t*>(pan + F::KPANELS * F::X_PANEL + tc::sw128_offset(row, k % F::KPER, 4)) =
              tc::to_tf32(f - __uint_as_float(bg));
        }
      } else {
        uint32_t pk;
        uint32_t f0, f1;
        const bool ok0 = scaled_f32_rto(vh[c][0], vl[c][0], e, f0);
        const bool ok1 = scaled_f32_rto(vh[c][1], vl[c][1], e, f1);
        if (ok0 && ok1) {
          if constexpr (PREC == P_FP16) {
            const __half2 v2 = __floats2half2_rn(__uint_as_float(f0), __uint_as_float(f1));
            pk = *reinterpret_cast<const uint32_t*>(&v2);
          } else {
            const __nv_bfloat162 v2 = __floats2bfloat162_rn(__uint_as_float(f0), __uint_as_float(f1));
            pk = *reinterpret_cast<const uint32_t*>(&v2);
          }
        } else {
          uint32_t h0 = vh[c][0], l0 = vl[c][0], h1 = vh[c][1], l1 = vl[c][1];
          scale_bits(h0, l0, e);
          scale_bits(h1, l1, e);
          if constexpr (PREC == P_FP16) pk = f64bits_to_f16(h0, l0) | (f64bits_to_f16(h1, l1) << 16);
          else pk = f64bits_to_bf16(h0, l0) | (f64bits_to_bf16(h1, l1) << 16);
        }
        *reinterpret_cast<uint32_t*>(xb + tc::sw128_offset(row, 2 * cp, 2)) = pk;
      }
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      if (issued < total) issue_tma(issued++);   // refill the stage just consumed
      tc::fence_after();
      const uint32_t d = tmem + (uint32_t)(buf * N);
      const uint32_t wb = tc::smem_u32(wop), xbs = tc::smem_u32(xb);
#pragma unroll
      for (int kk = 0; kk < kM2 / F::KSTEP; ++kk) {
        const int k = kk * F::KSTEP;
        const uint32_t po = (uint32_t)(k / F::KPER), koff = (uint32_t)((k % F::KPER) * F::EB);
        const uint32_t wa = wb + po * F::W_PANEL + koff, xa = xbs + po * F::X_PANEL + koff;
        if constexpr (PREC == P_FP32) {
          const uint32_t ws = F::KPANELS * F::W_PANEL, xs = F::KPANELS * F::X_PANEL;
          tc::mma_tf32(d, tc::sw128_desc(wa), tc::sw128_desc(xa), idesc, kk > 0);
          tc::mma_tf32(d, tc::sw128_desc(wa), tc::sw128_desc(xa + xs), idesc, 1);
          tc::mma_tf32(d, tc::sw128_desc(wa + ws), tc::sw128_desc(xa), idesc, 1);
        } else {
          tc::mma_f16(d, tc::sw128_desc(wa), tc::sw128_desc(xa), idesc, kk > 0);
        }
      }
      tc::mma_commit(&mma_bar[buf]);
      mma_issued = u + 1;
    }
    if (u > 0) {   // step 2 of the previous tile while this tile's MMAs run
      const bool ok_mma = tc::mbar_wait(&mma_bar[buf ^ 1], (uint32_t)(((u - 1) >> 1) & 1));
      if (__syncthreads_or(!ok_mma)) {
        abort = true;
        break;
      }
      mma_done = u;
      tc::fence_after();
      d_to_smem(u - 1);
      tc::fence_before();
      __syncthreads();
      step2(u - 1);
      __syncthreads();   // U is rewritten by the next tile
    }
  }
  if (!abort && total > 0) {
    const int u = total - 1;
    const bool ok_mma = tc::mbar_wait(&mma_bar[u & 1], (uint32_t)((u >> 1) & 1));
    if (__syncthreads_or(!ok_mma)) {
      abort = true;
    } else {
      mma_done = total;
      tc::fence_after();
      d_to_smem(u);
      tc::fence_before();
      __syncthreads();
      step2(u);
    }
  }
  if (abort && tid == 0) {
    // let this CTA's own copies and MMAs in flight finish before its shared memory and TMEM go away
    for (int v = consumed; v < issued; ++v)
      tc::mbar_wait(&tma_bar[v % F::STAGES], (uint32_t)((v / F::STAGES) & 1), 1u << 20);
    for (int v = mma_done; v < mma_issued; ++v) tc::mbar_wait(&mma_bar[v & 1], (uint32_t)((v >> 1) & 1), 1u << 20);
    raise_level_status(ctl, ST_TIMEOUT);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, F::TMEM_COLS);
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn fs_encode_fn() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
    cudaGetLastError();
  });
  return fn;
}

int sms() {
  static int cached = 0;
  if (!cached) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached = v > 0 ? v : 152;
  }
  return cached;
}

template <int PREC>
bool launch_fs(const double* A, int64_t lda, int64_t m, int n, int s, const uint32_t* idx, const double* tab,
               uint64_t seed, int chunks, double* Ypart, Ctl* ctl, int level, cudaStream_t st) {
  using F = Fs<PREC>;
  EncodeFn enc = fs_encode_fn();
  if (!enc) return false;
  const int64_t m1 = m / kM2;
  CUtensorMap map;
  const cuuint64_t dims[3] = {(cuuint64_t)m1, (cuuint64_t)kM2, (cuuint64_t)n};
  const cuuint64_t strides[2] = {(cuuint64_t)m1 * sizeof(double), (cuuint64_t)lda * sizeof(double)};
  const cuuint32_t box[3] = {(cuuint32_t)kB, (cuuint32_t)kM2, (cuuint32_t)F::C};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<double*>(A), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  const size_t smem = F::SMEM + 1024;
  if (cudaFuncSetAttribute(k_sketch_fs<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return false;
  const int ntiles = (int)(m1 / kB);
  const int tpc = ntiles / chunks;
  const int nitems = ((n + F::C - 1) / F::C) * chunks;
  const int grid = nitems < sms() ? nitems : sms();
  { ::mrcqr::note_launch(); k_sketch_fs<PREC><<<grid, kThreads, smem, st>>>(map, m, n, s, idx, tab, seed_key(seed), chunks, tpc, Ypart, ctl, level); }
  return true;
}

}  // namespace

bool sketch_fs_eligible(int prec, int tf, const double* A, int64_t lda, int64_t m, int n, int s) {
  if (prec != P_FP16 && prec != P_BF16 && prec != P_FP32) return false;
  if (tf != T_DCT || s < 1 || s > kMaxS || n < 1) return false;
  if (m < 2048 || (m % 1024) != 0 || m > (int64_t(1) << 22)) return false;   // m1 = m / 64 a multiple of 16
  if ((reinterpret_cast<uintptr_t>(A) & 15) != 0 || (lda & 1) != 0) return false;
  return fs_encode_fn() != nullptr;
}

// j1 chunks (a power of two dividing the m / 1024 tiles) so that column
// blocks x chunks gives about eight work items per SM.
int sketch_fs_chunks(int prec, int64_t m, int n) {
  const int C = prec == P_FP32 ? Fs<P_FP32>::C : Fs<P_FP16>::C;
  const int ncb = (n + C - 1) / C;
  const int64_t ntiles = m / (kM2 * kB);
  int chunks = 1;
  while ((int64_t)chunks * 2 <= ntiles && ntiles % (chunks * 2) == 0 && ncb * chunks < 8 * 152) chunks *= 2;
  return chunks;
}

bool launch_sketch_fs(int prec, const double* A, int64_t lda, int64_t m, int n, int s, const uint32_t* idx,
                      const double* tab, uint64_t seed, int chunks, double* Ypart, Ctl* ctl, int level,
                      cudaStream_t st) {
  switch (prec) {
    case P_FP16: return launch_fs<P_FP16>(A, lda, m, n, s, idx, tab, seed, chunks, Ypart, ctl, level, st);
    case P_BF16: return launch_fs<P_BF16>(A, lda, m, n, s, idx, tab, seed, chunks, Ypart, ctl, level, st);
    case P_FP32: return launch_fs<P_FP32>(A, lda, m, n, s, idx, tab, seed, chunks, Ypart, ctl, level, st);
    default: return false;
  }
}

}  // namespace mrcqr
