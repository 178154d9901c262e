// Tensor-core sketch (Algorithm 2 steps 2-4) for the FP16, BF16 and FP32
// sketch precisions.
//
// Y_i = sqrt(2/s) c_{k_i} sum_j cos(pi k_i (2j+1) / (2m)) d_j A_j.  For a slab
// of T rows starting at j0 the phase splits as theta_i + beta_it with
// theta_i = pi k_i (2 j0 + 1) / (2m) and beta_it = pi k_i t / m, so
//   sum_t cos(theta_i + beta_it) x_t = cos(theta_i) (C x)_i - sin(theta_i) (S x)_i
// with C_it = cos(pi k_i t/m), S_it = sin(pi k_i t/m) independent of the
// slab.  The real-FFT transforms of Algorithm 2 as printed take the same
// path with the phase 2 pi k j / m (plus pi / 2 on the Im rows, which turns
// the cosine into -sin), i.e. C_it = cos(2 pi k_i t / m) and theta_i the phase
// of j0 (the row words and phases of common.cuh).
// A CTA keeps C and S (rounded to the sketch precision) in shared
// memory for up to 256 sampled rows (one or two MMA tiles of 128) and 64
// columns of A, and per slab:
//   1. TMA brings the FP64 tile A[j0 : j0+T, n0 : n0+64] (3-4 stages); where
//      no TMA map can describe A (base not 16-byte aligned or lda odd: the
//      copy engine needs 16-byte strides) the converting warps load their
//      values from global memory instead, one slab ahead, into registers;
//   2. the tile is sign-flipped (Philox; XOR of the sign bit), scaled per
//      column by 2^e so that max |.| lies in [2^13, 2^14), rounded once to p
//      (fl_p) and written as a K-major SWIZZLE_128B operand -- all in 32-bit
//      integer operations, because every FP64 instruction runs on this
//      GPU's 1/64-rate FP64 pipe;
//   3. one thread issues tcgen05.mma for C x and S x of every tile into TMEM
//      (FP32; operand and accumulators double-buffered);
//   4. while those MMAs run, every thread reads its row of the previous
//      slab's products from TMEM, applies the rotation cos/sin(theta_i) and
//      the inverse scale, and accumulates in registers.
// FP16/BF16 use kind::f16 with T = 64.  FP32 uses kind::tf32 with T = 32 and
// the 3xTF32 split (big*big + big*small + small*big) so that the products
// keep about 22 bits.
//
// Every wait is bounded; on a timeout the CTA waits (bounded) for its own
// copies in flight, frees its TMEM, raises TIMEOUT and returns.
#include <cstring>
#include <mutex>

#include "kernels.h"
#include "tc.cuh"

namespace mrcqr {

namespace {

constexpr int kM = 128;          // sampled rows per MMA tile (MMA M)
constexpr int kN = 64;           // columns per CTA (MMA N)
constexpr int kThreads = 512;

template <int PREC, int MT>
struct Cfg {
  static constexpr int T = (PREC == P_FP32) ? 32 : 64;      // slab rows = MMA K per slab
  static constexpr int EB = (PREC == P_FP32) ? 4 : 2;       // operand element bytes
  static constexpr int PARTS = (PREC == P_FP32) ? 2 : 1;    // big (+ small) parts
  static constexpr int KSTEP = (PREC == P_FP32) ? 8 : 16;   // K per instruction
  static constexpr uint32_t FMT = (PREC == P_FP32) ? tc::TF32 : (PREC == P_BF16 ? tc::BF16 : tc::F16);
  static constexpr uint32_t PANEL = kM * 128;               // one 128-row operand panel
  static constexpr uint32_t XT_BYTES = kN * 128;            // one 64-row operand panel
  static constexpr uint32_t XD_BYTES = kN * T * 8;          // FP64 stage
  static constexpr int STAGES = (PREC == P_FP32) ? 3 : 4;   // TMA stages of the FP64 A tile
  // tables: [MT][C, S][PARTS] panels; operand X: [2 buffers][PARTS]; FP64 stages
  static constexpr uint32_t TAB_OFF = 0;
  static constexpr uint32_t XT_OFF = MT * 2 * PARTS * PANEL;
  static constexpr uint32_t XD_OFF = XT_OFF + 2 * PARTS * XT_BYTES;
  static constexpr uint32_t SMEM = XD_OFF + STAGES * XD_BYTES;
  // TMEM: [2 buffers][MT][C, S] accumulators of kN columns
  static constexpr uint32_t TMEM_COLS = 2 * MT * 2 * kN;
  static constexpr int ACC = (MT == 2) ? 32 : 16;           // accumulator columns per thread
};

// fl_p of the transform entry with FP64 bits (hi, lo) at (r, k) of a K-major
// SW128 panel (exact rounding; used once per CTA for the tables).
template <uint32_t FMT>
__device__ __forceinline__ void store_table(unsigned char* big, unsigned char* small, int r, int k, uint32_t hi,
                                            uint32_t lo) {
  if constexpr (FMT == tc::F16) {
    *reinterpret_cast<unsigned short*>(big + tc::sw128_offset(r, k, 2)) = (unsigned short)f64bits_to_f16(hi, lo);
  } else if constexpr (FMT == tc::BF16) {
    *reinterpret_cast<unsigned short*>(big + tc::sw128_offset(r, k, 2)) = (unsigned short)f64bits_to_bf16(hi, lo);
  } else {
    const float f = __uint_as_float(f64bits_to_f32(hi, lo));
    const uint32_t b = tc::to_tf32(f);
    *reinterpret_cast<uint32_t*>(big + tc::sw128_offset(r, k, 4)) = b;
    *reinterpret_cast<uint32_t*>(small + tc::sw128_offset(r, k, 4)) = tc::to_tf32(f - __uint_as_float(b));
  }
}

// fl_p of two consecutive entries (k, k+1) of row r of the X operand, given
// as FP64 bits scaled by 2^e: round to odd into FP32 (integer ops), then one
// packed round-to-nearest-even; exact slow path outside the FP32 range.
template <uint32_t FMT>
__device__ __forceinline__ uint32_t pack2(uint32_t h0, uint32_t l0, uint32_t h1, uint32_t l1, int e) {
  uint32_t f0, f1;
  const bool ok0 = scaled_f32_rto(h0, l0, e, f0);
  const bool ok1 = scaled_f32_rto(h1, l1, e, f1);
  if (ok0 && ok1) {
    if constexpr (FMT == tc::F16) {
      const __half2 v = __floats2half2_rn(__uint_as_float(f0), __uint_as_float(f1));
      return *reinterpret_cast<const uint32_t*>(&v);
    } else {
      const __nv_bfloat162 v = __floats2bfloat162_rn(__uint_as_float(f0), __uint_as_float(f1));
      return *reinterpret_cast<const uint32_t*>(&v);
    }
  }
  scale_bits(h0, l0, e);
  scale_bits(h1, l1, e);
  if constexpr (FMT == tc::F16) return f64bits_to_f16(h0, l0) | (f64bits_to_f16(h1, l1) << 16);
  else return f64bits_to_bf16(h0, l0) | (f64bits_to_bf16(h1, l1) << 16);
}

// Phase (dk j0 + beta) mod 4m of a row at slab start j0, advanced by slabs of
// T rows: adds dk T mod 4m.
struct Phase {
  uint64_t r, step, four_m;
  __device__ void init(const RowPhase& p, int64_t j0, int T, uint64_t fm) {
    four_m = fm;
    r = phase_at(p, (uint64_t)j0, fm);
    step = (p.dk * (uint64_t)T) % fm;
  }
  __device__ void advance() {
    r += step;
    if (r >= four_m) r -= four_m;
  }
};

// Shared state of one CTA of the tensor-core sketch (kept across work items).
template <int PREC, int MT>
struct TcCta {
  unsigned char* tabs;
  unsigned char* xt;
  double* xd;
  uint64_t* tma_bar;
  uint64_t* mma_bar;
  uint32_t tmem;
  float (*colscale)[kN];
  uint32_t (*sgnmask)[Cfg<PREC, MT>::T];
  uint32_t seq;    // slabs this CTA has run: the MMA barriers' phases and the operand/TMEM buffers
  uint32_t tseq;   // slabs this CTA has loaded by TMA: the copy barriers' stages and phases (a
                   // plain-copy item completes no copy-barrier phase, so it must not advance them)
};

// One work item: sampled rows s0 .. s0 + 128 MT - 1, columns n0 .. n0 + 63,
// rows [j_begin, j_end) of A (TMA map tmap, or with tmap null plain copies
// of A with leading dimension lda); the partial sums go to out[col s + row].
// False when a wait timed out (every thread together; this CTA's copies and
// MMAs in flight are awaited first).
template <int PREC, int MT>
__device__ __forceinline__ bool sketch_tc_item(const CUtensorMap* tmap, const double* __restrict__ A, int64_t lda,
                                               int64_t m, int n, int s,
                                               const uint32_t* __restrict__ idx, const double* __restrict__ tab,
                                               uint2 key, int64_t j_begin, int64_t j_end, int s0, int n0,
                                               double* __restrict__ out, int tf, TcCta<PREC, MT>& S) {
  using C = Cfg<PREC, MT>;
  constexpr int T = C::T;
  unsigned char* tabs = S.tabs;
  unsigned char* xt = S.xt;
  double* xd = S.xd;
  uint64_t* tma_bar = S.tma_bar;
  uint64_t* mma_bar = S.mma_bar;
  const uint32_t tmem = S.tmem;
  float(*colscale)[kN] = S.colscale;
  uint32_t(*sgnmask)[T] = S.sgnmask;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nslabs = j_begin < j_end ? (int)((j_end - j_begin + T - 1) / T) : 0;
  const uint64_t four_m = 4ull * (uint64_t)m;
  __syncthreads();   // the previous item's MMAs and epilogue are done with the tables
  // slab-invariant transform tables: two threads per sampled row (halves of
  // t), phases dk t mod 4m advanced by additions along t
  for (int w = tid; w < 2 * kM * MT; w += kThreads) {
    const int ri = w >> 1, half = w & 1;
    const int mt = ri / kM, i = ri % kM;
    unsigned char* cb = tabs + (mt * 2 + 0) * C::PARTS * C::PANEL;
    unsigned char* sb = tabs + (mt * 2 + 1) * C::PARTS * C::PANEL;
    const bool ok = s0 + ri < s;
    const uint64_t d = row_phase(tf, ok ? idx[s0 + ri] : 0u, (uint64_t)m).dk;
    const int t0 = half * (T / 2);
    uint64_t rc = (d * (uint64_t)t0) % four_m;
#pragma unroll 8
    for (int t = t0; t < t0 + T / 2; ++t) {
      uint32_t chi = 0u, clo = 0u, shi = 0u, slo = 0u;
      if (ok) {
        cos_phase_bits(tab, (int64_t)rc, m, chi, clo);
        const uint64_t rsn = rc <= (uint64_t)m ? (uint64_t)m - rc : (uint64_t)m + four_m - rc;   // pi/2 - x
        cos_phase_bits(tab, (int64_t)rsn, m, shi, slo);
      }
      store_table<C::FMT>(cb, cb + C::PANEL, i, t, chi, clo);
      store_table<C::FMT>(sb, sb + C::PANEL, i, t, shi, slo);
      rc += d;
      if (rc >= four_m) rc -= four_m;
    }
  }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();

  // plain loads (no TMA map): every thread copies its share of the slab's
  // FP64 tile into the stage with 8-byte cp.async, in the layout the TMA box
  // has ([column][row], zero outside the chunk and n), one commit group per
  // slab; a thread waits for its own groups before the barrier that precedes
  // the conversion
  auto dcopy = [&](int sl, int sg) {
    const int64_t j0 = j_begin + (int64_t)sl * T;
    double* dst = xd + sg * (C::XD_BYTES / 8);
    for (int e = tid; e < T * kN; e += kThreads) {
      const int c = e / T, r = e % T;
      const int col = n0 + c;
      const int64_t j = j0 + r;
      const bool ok = col < n && j < j_end;
      tc::cp_async8_zfill(dst + e, ok ? A + j + (int64_t)col * lda : A, ok ? 8u : 0u);
    }
    tc::cp_async_commit();
  };

  int issued = 0;   // slab loads of this item issued (the same count in every thread)
  const uint32_t cbase = tmap ? S.tseq : 0u;   // copy-stage index of this item's slab 0
  for (int st = 0; st < C::STAGES && st < nslabs; ++st) {
    const int sg = (int)((cbase + (uint32_t)st) % C::STAGES);
    if (!tmap) {
      dcopy(st, sg);
    } else if (tid == 0) {
      tc::mbar_expect_tx(&tma_bar[sg], C::XD_BYTES);
      tc::tma_load_2d(xd + sg * (C::XD_BYTES / 8), tmap, (int)(j_begin + st * T), n0, &tma_bar[sg]);
    }
    ++issued;
  }

  // epilogue identity
  // TMEM lane quarter q (warp % 4); MT = 2: tile (warp / 4) % 2 and column
  // half warp / 8; MT = 1: column quarter warp / 4
  int mt_e, q, c_lo;
  if constexpr (MT == 2) { mt_e = (warp >> 2) & 1; q = warp & 3; c_lo = (warp >> 3) * 32; }
  else { mt_e = 0; q = warp & 3; c_lo = (warp >> 2) * 16; }
  const int erow = mt_e * kM + q * 32 + lane;
  const bool row_ok = s0 + erow < s;
  Phase ph;
  ph.init(row_phase(tf, row_ok ? idx[s0 + erow] : 0u, (uint64_t)m), j_begin, T, four_m);
  const uint32_t idesc = tc::idesc(C::FMT, kM, kN);
  float acc[C::ACC];
#pragma unroll
  for (int c = 0; c < C::ACC; ++c) acc[c] = 0.f;
  bool abort = false;
  int consumed = 0, mma_issued = 0, mma_done = 0;

  // rotation factors cos/sin(theta_i) of slab sl, theta_i = pi r / (2m) with
  // the exact integer phase r: computed at the start of iteration sl (no
  // memory access; r / (2m) is exact in FP32 for power-of-two m <= 2^22) and
  // used by the slab's epilogue one iteration later
  const float inv2m = 1.0f / (2.0f * (float)m);
  float rc0 = 0.f, rs0 = 0.f, rc1 = 0.f, rs1 = 0.f;   // even / odd slabs
  auto prefetch_rotation = [&](int sl) {
    float c = 0.f, sn = 0.f;
    if (row_ok) sincospif((float)ph.r * inv2m, &sn, &c);
    if (sl & 1) { rc1 = c; rs1 = sn; }
    else { rc0 = c; rs0 = sn; }
    ph.advance();
  };

  auto epilogue = [&](int sl) {
    const int buf = sl & 1;
    const float cf = buf ? rc1 : rc0, sf = buf ? rs1 : rs0;
    const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((buf * MT + mt_e) * 2 * kN);
#pragma unroll
    for (int c0 = 0; c0 < C::ACC; c0 += 16) {
      float pc[16], ps[16];
      tc::tmem_ld16(base + c_lo + c0, pc);
      tc::tmem_ld16(base + kN + c_lo + c0, ps);
      tc::tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j)
        acc[c0 + j] = fmaf(fmaf(cf, pc[j], -sf * ps[j]), colscale[buf][c_lo + c0 + j], acc[c0 + j]);
    }
    tc::fence_before();
  };

  for (int sl = 0; sl < nslabs; ++sl) {
    const uint32_t u = S.seq + (uint32_t)sl;   // slab index over the CTA's items: MMA parity, buffer
    const uint32_t cu = cbase + (uint32_t)sl;   // copy stage and its barrier parity
    const int stage = (int)(cu % C::STAGES);
    const uint32_t par = (cu / C::STAGES) & 1u;
    const int buf = (int)(u & 1u);
    const int64_t j0 = j_begin + (int64_t)sl * T;
    prefetch_rotation((int)u);
    if (tid < T) {
      const int64_t j = j0 + tid;
      sgnmask[buf][tid] = j < j_end ? (philox4x32_10(make_uint4((uint32_t)j, 0u, 0u, 0u), key).x & 1u) << 31
                                    : 0xFFFFFFFFu;   // all ones marks a row outside the chunk
    }
    bool ok_tma = true;
    if (tmap) {
      ok_tma = tc::mbar_wait(&tma_bar[stage], par);
    } else {   // slab sl's group complete: at most issued - sl - 1 younger groups pending
      const int younger = issued - sl - 1;   // <= STAGES - 1 <= 3
      if (younger >= 3) tc::cp_async_wait_group<3>();
      else if (younger == 2) tc::cp_async_wait_group<2>();
      else if (younger == 1) tc::cp_async_wait_group<1>();
      else tc::cp_async_wait_group<0>();
    }
    if (__syncthreads_or(!ok_tma)) { abort = true; break; }
    consumed = sl + 1;
    // convert the FP64 tile: warp w owns columns 4w..4w+3
    const uint2* X = reinterpret_cast<const uint2*>(xd + stage * (C::XD_BYTES / 8));
    unsigned char* xb = xt + buf * C::PARTS * C::XT_BYTES;
    if constexpr (PREC == P_FP32) {
      const uint32_t sm = sgnmask[buf][lane];
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int col = warp * 4 + cc;
        const uint2 w = X[col * T + lane];
        const uint32_t hi = sm == 0xFFFFFFFFu ? 0u : (w.y ^ sm), lo = sm == 0xFFFFFFFFu ? 0u : w.x;
        uint32_t amax = __reduce_max_sync(0xffffffffu, hi & 0x7FFFFFFFu);
        int e;
        if ((amax >> 20) != 0u) e = scale_exponent_bits(amax, 1u);
        else e = scale_exponent(warp_max(fabs(__hiloint2double((int)hi, (int)lo))));
        if (lane == 0) colscale[buf][col] = ldexpf(1.0f, -e);
        uint32_t h = hi, l = lo;
        scale_bits(h, l, e);
        const float f = __uint_as_float(f64bits_to_f32(h, l));   // fl_32
        const uint32_t b = tc::to_tf32(f);
        *reinterpret_cast<uint32_t*>(xb + tc::sw128_offset(col, lane, 4)) = b;
        *reinterpret_cast<uint32_t*>(xb + C::XT_BYTES + tc::sw128_offset(col, lane, 4)) =
            tc::to_tf32(f - __uint_as_float(b));
      }
    } else {
      const uint32_t sm0 = sgnmask[buf][2 * lane], sm1 = sgnmask[buf][2 * lane + 1];
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int col = warp * 4 + cc;
        const uint4 w = reinterpret_cast<const uint4*>(X)[(col * T) / 2 + lane];   // rows 2 lane, 2 lane + 1
        const uint32_t h0 = sm0 == 0xFFFFFFFFu ? 0u : (w.y ^ sm0), l0 = sm0 == 0xFFFFFFFFu ? 0u : w.x;
        const uint32_t h1 = sm1 == 0xFFFFFFFFu ? 0u : (w.w ^ sm1), l1 = sm1 == 0xFFFFFFFFu ? 0u : w.z;
        uint32_t amax = __reduce_max_sync(0xffffffffu, max(h0 & 0x7FFFFFFFu, h1 & 0x7FFFFFFFu));
        int e;
        if ((amax >> 20) != 0u) e = scale_exponent_bits(amax, 1u);
        else e = scale_exponent(warp_max(fmax(fabs(__hiloint2double((int)h0, (int)l0)),
                                              fabs(__hiloint2double((int)h1, (int)l1)))));
        if (lane == 0) colscale[buf][col] = ldexpf(1.0f, -e);
        *reinterpret_cast<uint32_t*>(xb + tc::sw128_offset(col, 2 * lane, 2)) = pack2<C::FMT>(h0, l0, h1, l1, e);
      }
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (issued < nslabs) {   // refill the stage just consumed
      if (!tmap) {
        dcopy(issued, stage);
      } else if (tid == 0) {
        tc::mbar_expect_tx(&tma_bar[stage], C::XD_BYTES);
        tc::tma_load_2d(xd + stage * (C::XD_BYTES / 8), tmap, (int)(j_begin + (int64_t)issued * T), n0,
                        &tma_bar[stage]);
      }
      ++issued;
    }
    if (tid == 0) {
      tc::fence_after();
      const uint32_t tb = tc::smem_u32(tabs), xbs = tc::smem_u32(xb);
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
#pragma unroll
        for (int tbl = 0; tbl < 2; ++tbl) {
          const uint32_t d = tmem + (uint32_t)(((buf * MT + mt) * 2 + tbl) * kN);
          const uint32_t big = tb + (mt * 2 + tbl) * C::PARTS * C::PANEL;
#pragma unroll
          for (int k = 0; k < T; k += C::KSTEP) {
            const uint32_t koff = k * C::EB;
            if constexpr (PREC == P_FP32) {
              tc::mma_tf32(d, tc::sw128_desc(big + koff), tc::sw128_desc(xbs + koff), idesc, k > 0);
              tc::mma_tf32(d, tc::sw128_desc(big + koff), tc::sw128_desc(xbs + C::XT_BYTES + koff), idesc, 1);
              tc::mma_tf32(d, tc::sw128_desc(big + C::PANEL + koff), tc::sw128_desc(xbs + koff), idesc, 1);
            } else {
              tc::mma_f16(d, tc::sw128_desc(big + koff), tc::sw128_desc(xbs + koff), idesc, k > 0);
            }
          }
        }
      }
      tc::mma_commit(&mma_bar[buf]);
      mma_issued = sl + 1;
    }
    // the previous slab's products are read while this slab's MMAs run
    if (sl > 0) {
      const bool ok_mma = tc::mbar_wait(&mma_bar[buf ^ 1], ((u - 1) >> 1) & 1u);
      if (__syncthreads_or(!ok_mma)) { abort = true; break; }
      mma_done = sl;
      tc::fence_after();
      epilogue((int)(u - 1));
    }
  }
  if (!abort && nslabs > 0) {
    const uint32_t u = S.seq + (uint32_t)(nslabs - 1);
    const bool ok_mma = tc::mbar_wait(&mma_bar[u & 1u], (u >> 1) & 1u);
    if (__syncthreads_or(!ok_mma)) abort = true;
    else {
      mma_done = nslabs;
      tc::fence_after();
      epilogue((int)u);
    }
  }

  if (abort) {
    if (!tmap) tc::cp_async_wait_all();
    if (tid == 0) {   // this CTA's own copies and MMAs in flight land before its shared memory and TMEM go away
      for (int v = consumed; v < issued && tmap; ++v) {
        const uint32_t cu = cbase + (uint32_t)v;
        tc::mbar_wait(&tma_bar[cu % C::STAGES], (cu / C::STAGES) & 1u, 1u << 20);
      }
      for (int v = mma_done; v < mma_issued; ++v) {
        const uint32_t u = S.seq + (uint32_t)v;
        tc::mbar_wait(&mma_bar[u & 1u], (u >> 1) & 1u, 1u << 20);
      }
    }
    return false;
  }
  S.seq += (uint32_t)nslabs;
  if (tmap) S.tseq += (uint32_t)nslabs;
#pragma unroll
  for (int c = 0; c < C::ACC; ++c) {
    const int col = n0 + c_lo + c;
    if (row_ok && col < n) out[(size_t)col * s + s0 + erow] = (double)acc[c];
  }
  return true;
}

// CTA prologue of the tensor-core sketch kernels: shared memory, TMEM and
// barriers, gathered in the TcCta named S.
#define MRCQR_SKETCH_TC_CTA(S)                                                                        \
  using C = Cfg<PREC, MT>;                                                                            \
  extern __shared__ unsigned char smem_raw[];                                                         \
  unsigned char* smem =                                                                               \
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023)); \
  __shared__ __align__(8) uint64_t tma_bar_s[C::STAGES];                                              \
  __shared__ __align__(8) uint64_t mma_bar_s[2];                                                      \
  __shared__ uint32_t tmem_base;                                                                      \
  __shared__ float colscale_s[2][kN];                                                                 \
  __shared__ uint32_t sgnmask_s[2][C::T];                                                             \
  if ((threadIdx.x >> 5) == 0) tc::tmem_alloc(&tmem_base, C::TMEM_COLS);                              \
  if (threadIdx.x == 0) {                                                                             \
    for (int st = 0; st < C::STAGES; ++st) tc::mbar_init(&tma_bar_s[st], 1);                          \
    tc::mbar_init(&mma_bar_s[0], 1);                                                                  \
    tc::mbar_init(&mma_bar_s[1], 1);                                                                  \
    tc::mbar_fence_init();                                                                            \
  }                                                                                                   \
  tc::fence_before();                                                                                 \
  __syncthreads();                                                                                    \
  tc::fence_after();                                                                                  \
  TcCta<PREC, MT> S{smem + C::TAB_OFF, smem + C::XT_OFF, reinterpret_cast<double*>(smem + C::XD_OFF), \
                    tma_bar_s,          mma_bar_s,         tmem_base, colscale_s, sgnmask_s, 0u, 0u};

template <int PREC, int MT>
__device__ __forceinline__ void sketch_tc_cta_end(TcCta<PREC, MT>& S, bool abort, Ctl* ctl) {
  if (abort && threadIdx.x == 0 && ctl) raise_level_status(ctl, ST_TIMEOUT);
  tc::fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(S.tmem, Cfg<PREC, MT>::TMEM_COLS);
}

template <int PREC, int MT>
__global__ void __launch_bounds__(kThreads, 1)
    k_sketch_tc(const __grid_constant__ CUtensorMap tmapA, int use_map, const double* __restrict__ A, int64_t lda,
                int64_t m, int n, int s, const uint32_t* __restrict__ idx,
                const double* __restrict__ tab, uint2 key, int64_t rows_per_chunk,
                double* __restrict__ Ypart, Ctl* ctl, int level, int tf) {
  if (level_inactive(ctl, level)) return;
  MRCQR_SKETCH_TC_CTA(S)
  const int64_t j_begin = (int64_t)blockIdx.z * rows_per_chunk;
  const bool ok = sketch_tc_item<PREC, MT>(use_map ? &tmapA : nullptr, A, lda, m, n, s, idx, tab, key, j_begin,
                                           min(m, j_begin + rows_per_chunk),
                                           blockIdx.x * (kM * MT), blockIdx.y * kN,
                                           Ypart + (size_t)blockIdx.z * (size_t)s * (size_t)n, tf, S);
  sketch_tc_cta_end(S, !ok, ctl);
}

// Grouped form for batched plans: items {problem, chunk, 128 MT-row sample
// tile, 64-column block}; each problem's TMA maps (slabs of 64 and of 32 rows)
// sit in the plan's workspace (null where A has no map: plain loads).
template <int PREC, int MT>
__global__ void __launch_bounds__(kThreads, 1) kg_sketch_tc(Group g, int level) {
  MRCQR_SKETCH_TC_CTA(S)
  bool abort = false;
  Ctl* actl = nullptr;
  for (int it = blockIdx.x; it < g.nitems; it += gridDim.x) {
    const int4 w = g.items[it];
    const Prob& P = g.probs[w.x];
    if (level_inactive(P.ctl, level)) continue;
    const CUtensorMap* map = reinterpret_cast<const CUtensorMap*>(PREC == P_FP32 ? P.tmap32 : P.tmap64);
    const int64_t j_begin = (int64_t)w.y * P.rows_per_chunk;
    if (!sketch_tc_item<PREC, MT>(map, P.A, P.lda, P.m, P.n, P.s, P.idx, P.tab, P.key, j_begin,
                                  min(P.m, j_begin + P.rows_per_chunk),
                                  w.z * (kM * MT), w.w * kN, P.ypart + (size_t)w.y * (size_t)P.s * (size_t)P.n, P.tf,
                                  S)) {
      abort = true;
      actl = P.ctl;
      break;
    }
  }
  sketch_tc_cta_end(S, abort, actl);
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
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

template <int PREC, int MT>
bool launch_tc(const CUtensorMap& map, bool use_map, const double* A, int64_t lda, int64_t m, int n, int s,
               const uint32_t* idx, const double* tab, uint64_t seed, int chunks, double* Ypart, Ctl* ctl, int level,
               cudaStream_t st, int tf) {
  using C = Cfg<PREC, MT>;
  const size_t smem = C::SMEM + 1024;
  if (cudaFuncSetAttribute(k_sketch_tc<PREC, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return false;
  int64_t rpc = (m + chunks - 1) / chunks;
  rpc = (rpc + 63) / 64 * 64;
  const dim3 grid((s + kM * MT - 1) / (kM * MT), (n + kN - 1) / kN, chunks);
  { ::mrcqr::note_launch(); k_sketch_tc<PREC, MT><<<grid, kThreads, smem, st>>>(map, use_map ? 1 : 0, A, lda, m, n, s, idx, tab,
                                                                               seed_key(seed), rpc, Ypart, ctl, level, tf); }
  return true;
}

template <int PREC>
bool launch_prec(const double* A, int64_t lda, int64_t m, int n, int s, const uint32_t* idx, const double* tab,
                 uint64_t seed, int chunks, double* Ypart, Ctl* ctl, int level, cudaStream_t st,
                 int tf) {
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  const bool use_map = sketch_tc_encode(Cfg<PREC, 1>::T, A, lda, m, n, &map);   // else plain loads
  if (s > kM) return launch_tc<PREC, 2>(map, use_map, A, lda, m, n, s, idx, tab, seed, chunks, Ypart, ctl, level, st, tf);
  return launch_tc<PREC, 1>(map, use_map, A, lda, m, n, s, idx, tab, seed, chunks, Ypart, ctl, level, st, tf);
}

}  // namespace

bool sketch_tc_encode(int rows, const double* A, int64_t lda, int64_t m, int n, void* map_out) {
  EncodeFn enc = encode_fn();
  if (!enc || (reinterpret_cast<uintptr_t>(A) & 15) != 0 || (lda & 1) != 0) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)lda * sizeof(double)};
  const cuuint32_t box[2] = {(cuuint32_t)rows, (cuuint32_t)kN};
  const cuuint32_t estr[2] = {1, 1};
  return enc(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(A), dims,
             strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t sketch_tc_map_bytes() { return sizeof(CUtensorMap); }

void prepare_g_sketch_tc() {
  cudaFuncSetAttribute(kg_sketch_tc<P_FP16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg<P_FP16, 1>::SMEM + 1024);
  cudaFuncSetAttribute(kg_sketch_tc<P_FP16, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg<P_FP16, 2>::SMEM + 1024);
  cudaFuncSetAttribute(kg_sketch_tc<P_BF16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg<P_BF16, 1>::SMEM + 1024);
  cudaFuncSetAttribute(kg_sketch_tc<P_BF16, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg<P_BF16, 2>::SMEM + 1024);
  cudaFuncSetAttribute(kg_sketch_tc<P_FP32, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg<P_FP32, 1>::SMEM + 1024);
  cudaFuncSetAttribute(kg_sketch_tc<P_FP32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg<P_FP32, 2>::SMEM + 1024);
}

void launch_g_sketch_tc(const Group& g, int prec, int mt, int level, cudaStream_t st) {
  if (!g.nitems) return;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)(g.nitems < sms ? g.nitems : sms);
#define MRCQR_G_TC(PR, MTV)                                                                                \
  { ::mrcqr::note_launch(); kg_sketch_tc<PR, MTV><<<grid, kThreads, Cfg<PR, MTV>::SMEM + 1024, st>>>(g, level); }
  if (prec == P_FP16) { if (mt == 2) MRCQR_G_TC(P_FP16, 2) else MRCQR_G_TC(P_FP16, 1) }
  else if (prec == P_BF16) { if (mt == 2) MRCQR_G_TC(P_BF16, 2) else MRCQR_G_TC(P_BF16, 1) }
  else { if (mt == 2) MRCQR_G_TC(P_FP32, 2) else MRCQR_G_TC(P_FP32, 1) }
#undef MRCQR_G_TC
}

bool sketch_tc_eligible(int prec, const double* A, int64_t lda) {
  (void)lda;   // any leading dimension: plain loads where no TMA map fits
  if (prec != P_FP16 && prec != P_BF16 && prec != P_FP32) return false;
  return (reinterpret_cast<uintptr_t>(A) & 7) == 0;
}

bool launch_sketch_tc(int prec, const double* A, int64_t lda, int64_t m, int n, int s, const uint32_t* idx,
                      const double* tab, uint64_t seed, int chunks, double* Ypart, Ctl* ctl,
                      int level, cudaStream_t st, int tf) {
  switch (prec) {
    case P_FP16: return launch_prec<P_FP16>(A, lda, m, n, s, idx, tab, seed, chunks, Ypart, ctl, level, st, tf);
    case P_BF16: return launch_prec<P_BF16>(A, lda, m, n, s, idx, tab, seed, chunks, Ypart, ctl, level, st, tf);
    case P_FP32: return launch_prec<P_FP32>(A, lda, m, n, s, idx, tab, seed, chunks, Ypart, ctl, level, st, tf);
    default: return false;
  }
}

}  // namespace mrcqr
