// The FP64 sketch (Algorithm 2 steps 2-4 at p = FP64) as an emulated-FP64
// product whose operands need no slicing inside the product kernel.
//
// The per-item kernel of ozaki.cu slices the 128 columns of A of its work
// item for every tile of 64 sampled rows, so each value of A is sliced s / 64
// times (16 times at n = 512), and the transform entries once per 128-column
// block; digit production, not the tensor cores, bounds it.  Here:
//  - the eight balanced base-256 digits of d_j A[j][c], sliced once against
//    the column maxima of A, are written as eight FP16 planes
//    plane[a][c][j] (k_oz_planes_a), and one 3-D TMA copy brings the eight
//    128 x 32 digit panels of a K chunk into shared memory in the K-major
//    SWIZZLE_64B layout the MMAs read;
//  - the eight digits of every quarter-wave table value cos(pi q / (2m)),
//    sliced once against 2^0 (k_oz_tab_digits), are gathered per transform
//    entry with the sign of its quadrant applied by XOR.
// The digits are those the per-item kernel forms, the level sums are exact
// integers and the slab partials are summed exactly, so Y is bit for bit the
// same as that kernel's for any split into row chunks or slabs.
//
// The planes take 16 bytes per entry of A.  A factorization lends them the
// Q buffer (free until stage 2 of the level writes W into it, and 8 bytes
// per entry), so A is processed in row chunks of at most half the rows: per
// chunk the planes, then the products of that chunk's slabs; one reduction
// at the end.  Every kernel returns at once unless the level is the active
// one, so an inactive FP64 level never writes into Q.
#include <algorithm>
#include <mutex>
#include <vector>

#include "ozaki_pipe.cuh"

namespace mrcqr {

namespace {

// FP16 digits of the quarter-wave table: tabd[q] holds digit a of
// cos(pi q / (2m)) (sliced against 2^0, the transform operand's reference) in
// 16-bit lane a.  Two entries per thread.
__global__ void __launch_bounds__(256) k_oz_tab_digits(int64_t m, const double* __restrict__ tab,
                                                       uint4* __restrict__ tabd, const Ctl* ctl, int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  const int64_t q = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (q > m) return;
  const double x0 = tab[q];
  const double x1 = q + 1 <= m ? tab[q + 1] : 0.0;
  const uint32_t h0 = (uint32_t)__double2hiint(x0), h1 = (uint32_t)__double2hiint(x1);
  const uint64_t J0 = oz::biased_fixed63(h0, (uint32_t)__double2loint(x0), 1023, 0);
  const uint64_t J1 = oz::biased_fixed63(h1, (uint32_t)__double2loint(x1), 1023, 0);
  uint32_t w[oz::kSlices];
  oz::digits8_pack(J0, J1, h0 >> 31, h1 >> 31, w);   // w[a]: digit a of x0 (low half), of x1 (high half)
  tabd[q] = make_uint4(__byte_perm(w[0], w[1], 0x5410), __byte_perm(w[2], w[3], 0x5410),
                       __byte_perm(w[4], w[5], 0x5410), __byte_perm(w[6], w[7], 0x5410));
  if (q + 1 <= m)
    tabd[q + 1] = make_uint4(__byte_perm(w[0], w[1], 0x7632), __byte_perm(w[2], w[3], 0x7632),
                             __byte_perm(w[4], w[5], 0x7632), __byte_perm(w[6], w[7], 0x7632));
}

// Digit planes of rows [row0, row0 + mc) of D A (d_j the Rademacher sign of
// row j): plane a, column c, local row j at ((a n + c) R + j), FP16, each
// value sliced against the exponent of its column's maximum over all m rows
// (colHi).  A thread takes a pair of rows and kPlaneCols columns; a warp's
// loads and stores are contiguous along the rows.
constexpr int kPlaneCols = 16;

__global__ void __launch_bounds__(256) k_oz_planes_a(int64_t row0, int64_t mc, int n, const double* __restrict__ A,
                                                     int64_t lda, const uint32_t* __restrict__ colHi, uint2 key,
                                                     uint32_t* __restrict__ planes, int64_t R, const Ctl* ctl,
                                                     int level) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  const int64_t jp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = 2 * jp;
  if (j >= mc) return;
  const bool has1 = j + 1 < mc;
  const uint32_t f0 = philox4x32_10(make_uint4((uint32_t)(row0 + j), 0u, 0u, 0u), key).x & 1u;
  const uint32_t f1 = has1 ? philox4x32_10(make_uint4((uint32_t)(row0 + j + 1), 0u, 0u, 0u), key).x & 1u : 0u;
  const int c0 = blockIdx.y * kPlaneCols;
  double v[kPlaneCols][2];
#pragma unroll
  for (int t = 0; t < kPlaneCols; ++t) {
    const int c = c0 + t;
    v[t][0] = v[t][1] = 0.0;
    if (c < n) {
      const double* col = A + (int64_t)c * lda + row0 + j;
      v[t][0] = __ldg(col);
      if (has1) v[t][1] = __ldg(col + 1);
    }
  }
  const int64_t half = R / 2;   // u32 words per plane row
#pragma unroll
  for (int t = 0; t < kPlaneCols; ++t) {
    const int c = c0 + t;
    if (c >= n) break;
    const int E = (int)oz::exp_field(colHi[c]);
    const uint32_t h0 = (uint32_t)__double2hiint(v[t][0]), h1 = (uint32_t)__double2hiint(v[t][1]);
    const uint64_t J0 = oz::biased_fixed63(h0, (uint32_t)__double2loint(v[t][0]), E, 0);
    const uint64_t J1 = oz::biased_fixed63(h1, (uint32_t)__double2loint(v[t][1]), E, 0);
    uint32_t w[oz::kSlices];
    oz::digits8_pack(J0, J1, (h0 >> 31) ^ f0, (h1 >> 31) ^ f1, w);
#pragma unroll
    for (int a = 0; a < oz::kSlices; ++a) planes[((int64_t)a * n + c) * half + jp] = w[a];
  }
}

// One work item (128 columns of A, 64 sampled rows, row slab of the chunk)
// of the FP64 sketch from the planes.  The A panels of a chunk come by TMA;
// thread (fi, fg) gathers the table digits of sample fi at rows 4 fg .. 4 fg
// + 3 of the chunk.  The stages alternate by the CTA's running chunk count
// gch.  False when a wait timed out (every thread together).
struct OzpState {
  uint64_t* tma_bar;   // [2], one per stage
  int* abort_flag;     // set by the issuing thread when a TMA wait timed out
  uint32_t tma_phase;  // thread 0: bit st = parity of the next completion of stage st
  uint32_t pend;       // thread 0: bit st = a copy into stage st issued and not yet waited for
  uint32_t gch;        // chunks this CTA has run (stage of chunk c of an item: (gch + c) & 1)
};

__device__ __forceinline__ bool sketch_ozp_item(const CUtensorMap* tmap, int64_t row0, int64_t mc, int n, int s,
                                                const uint32_t* __restrict__ idx, const uint4* __restrict__ tabd,
                                                const SketchOzPlan& SP, long long* __restrict__ part, int tf,
                                                int64_t m, OzPipe& P, OzpState& S, unsigned char* smem, int item) {
  const int tid = threadIdx.x, lane = tid & 31;
  const uint64_t four_m = 4ull * (uint64_t)m;
  const int ntiles_all = SP.mblocks * SP.ntiles;
  const int tile = item % ntiles_all, slab = item / ntiles_all;
  const int c0 = kM * (tile / SP.ntiles), i0 = kN * (tile % SP.ntiles);
  const int64_t r_begin = (int64_t)slab * SP.rows_per_slab;
  const int64_t r_end = min(mc, r_begin + SP.rows_per_slab);
  const int nchunks = r_end > r_begin ? (int)((r_end - r_begin + kK - 1) / kK) : 0;
  long long hi[16], lo[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) hi[c] = lo[c] = 0;
  if (nchunks > 0) {
    const int fi = tid & (kN - 1), fg = tid >> 6;
    const bool fval = i0 + fi < s;
    const RowPhase rp = row_phase(tf, fval ? idx[i0 + fi] : 0u, (uint64_t)m);
    uint64_t r = fval ? phase_at(rp, (uint64_t)(row0 + r_begin + 4 * fg), four_m) : 0ull;
    const uint64_t step_chunk = (rp.dk * (uint64_t)kK) % four_m;
    const uint64_t step_row = rp.dk;
    uint4 u[4];
    // table digits of this thread's four rows of the chunk at local row r0 (zero past the slab)
    auto gather = [&](int64_t r0) {
      uint64_t rr = r;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        u[t] = make_uint4(0u, 0u, 0u, 0u);
        if (fval && r0 + 4 * fg + t < r_end) {
          int64_t q = (int64_t)rr;
          uint32_t neg = 0u;
          if (q >= 2 * m) q = 4 * m - q;   // cos(2 pi - x) = cos x
          if (q > m) {                      // cos(pi - x) = -cos x
            q = 2 * m - q;
            neg = 0x80008000u;
          }
          const uint4 d = __ldg(tabd + q);
          u[t] = make_uint4(d.x ^ neg, d.y ^ neg, d.z ^ neg, d.w ^ neg);
        }
        rr += step_row;
        if (rr >= four_m) rr -= four_m;
      }
      r += step_chunk;
      if (r >= four_m) r -= four_m;
    };
    auto issue_tma = [&](int ch) {
      const uint32_t st = (S.gch + (uint32_t)ch) & 1u;
      unsigned char* a = smem + st * kStage;
      S.pend |= 1u << st;
      tc::mbar_expect_tx(&S.tma_bar[st], oz::kSlices * kAPanel);
      tc::tma_load_3d(a, tmap, (int)(r_begin + (int64_t)ch * kK), c0, 0, &S.tma_bar[st]);
    };
    // Two MMA batches in flight (bar[0] / bar[1] by chunk parity): the batch of chunk ch is issued while that of
    // ch - 1 runs; the copy of chunk ch + 1 and the production of its transform digits go into the
    // stage chunk ch - 1 read, once that batch is done.  The stage of chunk 0 was last read by
    // batches that completed before this item.
    if (tid == 0) issue_tma(0);
    gather(r_begin);
    bool ok = true;
    for (int ch = 0; ch < nchunks; ++ch) {
      const uint32_t st = (S.gch + (uint32_t)ch) & 1u;
      unsigned char* a = smem + st * kStage;
      unsigned char* b = a + oz::kSlices * kAPanel;
      // transform digits of chunk ch: rows 4 fg + 2 t2, + 1 of sample fi
#pragma unroll
      for (int t2 = 0; t2 < 2; ++t2) {
        const uint4 x0 = u[2 * t2], x1 = u[2 * t2 + 1];
        const uint32_t w0[4] = {x0.x, x0.y, x0.z, x0.w}, w1[4] = {x1.x, x1.y, x1.z, x1.w};
        unsigned char* dst = b + tc::sw64_offset(fi, 4 * fg + 2 * t2, 2);
#pragma unroll
        for (int d = 0; d < oz::kSlices; ++d)
          *reinterpret_cast<uint32_t*>(dst + d * kBPanel) =
              __byte_perm(w0[d >> 1], w1[d >> 1], (d & 1) ? 0x7632 : 0x5410);
      }
      if (ch + 1 < nchunks) gather(r_begin + (int64_t)(ch + 1) * kK);
      tc::fence_proxy_async();
      const bool gstart = ch % kGroupChunks == 0;
      if (gstart && ch > 0) ok = oz_wait_mma(P, (int)(S.gch + ch - 1)) && ok;
      // the flag is read after the barrier, so every thread sees the issuing thread's last write
      if (__syncthreads_or(!ok) || *S.abort_flag) return false;
      if (gstart && ch > 0) {   // group closed at ch - 1: its level sums before the next group overwrites them
        tc::fence_after();
        oz_readout(P.tmem, P.q, P.g, hi, lo);
        tc::fence_before();
        __syncthreads();
      }
      if (tid == 0) {
        const bool tok = tc::mbar_wait(&S.tma_bar[st], (S.tma_phase >> st) & 1u);
        if (tok) {
          S.tma_phase ^= 1u << st;
          S.pend &= ~(1u << st);
        }
        tc::fence_after();
        if (tok) oz_issue_chunk(P.tmem, tc::smem_u32(a), tc::smem_u32(b), gstart);
        else *S.abort_flag = 1;
        tc::mma_commit(&P.bar[(S.gch + ch) & 1u]);   // with no MMA issued it arrives once the earlier ones are done
        P.mopen |= 1u << ((S.gch + ch) & 1u);
      }
      if (!gstart) ok = oz_wait_mma(P, (int)(S.gch + ch - 1));   // frees the stage of chunk ch + 1
      if (tid == 0 && ok && ch + 1 < nchunks) issue_tma(ch + 1);
    }
    ok = oz_wait_mma(P, (int)(S.gch + nchunks - 1)) && ok;
    if (__syncthreads_or(!ok) || *S.abort_flag) return false;
    tc::fence_after();
    oz_readout(P.tmem, P.q, P.g, hi, lo);
    tc::fence_before();
    __syncthreads();
    S.gch += (uint32_t)nchunks;
  }
  oz_store_partial(part + (size_t)item * kPartElems, P.q, P.g, lane, hi, lo);
  return true;
}

__global__ void __launch_bounds__(kOzThreads, 1)
    k_sketch_ozp(const __grid_constant__ CUtensorMap tmap, int64_t row0, int64_t mc, int n, int s,
                 const uint32_t* __restrict__ idx, const uint4* __restrict__ tabd, SketchOzPlan SP,
                 long long* __restrict__ part, Ctl* ctl, int level, int tf, int64_t m) {
  if (level_inactive(ctl, level) || ctl->lvl_status != 0) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = oz_smem(smem_raw);
  __shared__ __align__(8) uint64_t mma_bar[2];
  __shared__ __align__(8) uint64_t tma_bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    tc::mbar_init(&tma_bar[0], 1);
    tc::mbar_init(&tma_bar[1], 1);
    abort_flag = 0;
  }
  OzPipe P = oz_begin(&tmem_slot, mma_bar);   // initialises the MMA barriers and fences the inits
  OzpState S{tma_bar, &abort_flag, 0u, 0u, 0u};
  bool abort = false;
  const int nitems = SP.mblocks * SP.ntiles * SP.slabs;
  for (int item = blockIdx.x; item < nitems; item += gridDim.x)
    if (!sketch_ozp_item(&tmap, row0, mc, n, s, idx, tabd, SP, part, tf, m, P, S, smem, item)) {
      abort = true;
      break;
    }
  if (abort && threadIdx.x == 0) {
    // copies may still be in flight into shared memory: wait for them (bounded) before leaving
    for (uint32_t st = 0; st < 2; ++st)
      if ((S.pend >> st) & 1u) tc::mbar_wait(&tma_bar[st], (S.tma_phase >> st) & 1u, 1u << 20);
  }
  oz_end(P, abort, ctl);
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

int sm_count() {
  static int cached = 0;
  if (!cached) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached = v > 0 ? v : 152;
  }
  return cached;
}

constexpr int64_t kMinChunkRows = 1024;

}  // namespace

int64_t sketch_ozp_chunk_rows(int64_t m, int n, size_t scratch_bytes) {
  int64_t R = (int64_t)(scratch_bytes / (16ull * (uint64_t)n)) / kK * kK;
  const int64_t mr = (m + kK - 1) / kK * kK;
  if (R > mr) R = mr;
  return R >= kMinChunkRows || R >= mr ? R : 0;
}

size_t sketch_ozp_part_bytes(int64_t m, int n, int s, size_t scratch_bytes) {
  const int64_t R = sketch_ozp_chunk_rows(m, n, scratch_bytes);
  if (R <= 0) return 0;
  const int64_t nch = (m + R - 1) / R;
  return (size_t)nch * sketch_oz_part_bytes(sketch_oz_plan(R, n, s));
}

bool sketch_ozp_eligible(int64_t m, int n, const void* scratch, size_t scratch_bytes) {
  if (!scratch || (reinterpret_cast<uintptr_t>(scratch) & 15) != 0) return false;
  if (sketch_ozp_chunk_rows(m, n, scratch_bytes) <= 0) return false;
  return encode_fn() != nullptr;
}

bool launch_sketch_ozp(int64_t m, int n, int s, const double* A, int64_t lda, const uint32_t* idx, const double* tab,
                       uint4* tabd, uint64_t seed, uint32_t* colHi, long long* part, size_t part_bytes, double* Y,
                       void* scratch, size_t scratch_bytes, Ctl* ctl, int level, cudaStream_t st, int tf) {
  if (!sketch_ozp_eligible(m, n, scratch, scratch_bytes)) return false;
  const int64_t R = sketch_ozp_chunk_rows(m, n, scratch_bytes);
  const int64_t nch = (m + R - 1) / R;
  const SketchOzPlan Pc = sketch_oz_plan(R, n, s);
  const int items = Pc.mblocks * Pc.ntiles * Pc.slabs;
  if ((size_t)nch * sketch_oz_part_bytes(Pc) > part_bytes) return false;
  if (cudaFuncSetAttribute(k_sketch_ozp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem) != cudaSuccess)
    return false;
  // every tensor map first: nothing is enqueued when one cannot be encoded
  std::vector<CUtensorMap> maps((size_t)nch);
  for (int64_t k = 0; k < nch; ++k) {
    const int64_t mc = std::min(R, m - k * R);
    const cuuint64_t dims[3] = {(cuuint64_t)mc, (cuuint64_t)n, (cuuint64_t)oz::kSlices};
    const cuuint64_t strides[2] = {(cuuint64_t)R * 2, (cuuint64_t)R * 2 * (cuuint64_t)n};
    const cuuint32_t box[3] = {(cuuint32_t)kK, (cuuint32_t)kM, (cuuint32_t)oz::kSlices};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (encode_fn()(&maps[(size_t)k], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, scratch, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  launch_oz_col_hi(m, n, A, lda, colHi, ctl, level, st);
  const int64_t tq = (m + 2) / 2;   // table entries 0 .. m, two per thread
  { ::mrcqr::note_launch(); k_oz_tab_digits<<<(unsigned)((tq + 255) / 256), 256, 0, st>>>(m, tab, tabd, ctl, level); }
  const uint2 key = seed_key(seed);
  const int grid = items < sm_count() ? items : sm_count();
  for (int64_t k = 0; k < nch; ++k) {
    const int64_t row0 = k * R, mc = std::min(R, m - row0);
    const int64_t pairs = (mc + 1) / 2;
    const dim3 pg((unsigned)((pairs + 255) / 256), (unsigned)((n + kPlaneCols - 1) / kPlaneCols));
    { ::mrcqr::note_launch(); k_oz_planes_a<<<pg, 256, 0, st>>>(row0, mc, n, A, lda, colHi, key,
                                                                static_cast<uint32_t*>(scratch), R, ctl, level); }
    { ::mrcqr::note_launch(); k_sketch_ozp<<<grid, kOzThreads, kSmem, st>>>(maps[(size_t)k], row0, mc, n, s, idx,
                                                                              tabd, Pc, part + (size_t)k * items * kPartElems,
                                                                              ctl, level, tf, m); }
  }
  SketchOzPlan Pall = Pc;
  Pall.slabs = Pc.slabs * (int)nch;
  launch_sketch_oz_reduce(n, s, colHi, idx, Pall, part, Y, ctl, level, st, tf, m);
  return true;
}

}  // namespace mrcqr
