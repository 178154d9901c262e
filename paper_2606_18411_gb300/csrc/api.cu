// C ABI of the MRCQR library: argument checks, the workspace plan, the
// escalation ladder of Sec. II-C and the per-stream status records.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "../../include/mrcqr.h"
#include "kernels.h"

using namespace mrcqr;

namespace {

constexpr int kVersion = 10000;
constexpr int kMaxN = 512;
constexpr double kDefaultTol = 1e-13;

size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Workspace of one factorization.
struct Plan {
  int64_t m = 0;
  int n = 0, s = 0, npad = 0, chunks = 0, splits = 0;
  int tf = T_DCT;   // sketch transform; s counts the rows of Y (2 x bins for T_RFFT_REIM)
  size_t off_ctl = 0, off_idx = 0, off_tab = 0, off_ypart = 0, off_y = 0, off_sqr = 0, off_rs = 0, off_rst = 0,
         off_rinv = 0, off_gpart = 0, off_rc = 0, off_xt = 0, off_e = 0, off_feat = 0, off_oze = 0, off_ozx = 0,
         off_colhi = 0, off_ozpart = 0, off_tcole = 0, off_trd = 0, off_tabd = 0, off_planes = 0, total = 0;
  size_t ozpart_bytes = 0, planes_bytes = 0;
  SyrkOzPlan oz{};
  SketchOzPlan sk{};
};

// planes: reserve the digit planes of the FP64 sketch in the workspace (the step-level sketch call,
// which has no Q buffer to lend them); a factorization lends them its Q buffer.
Plan make_plan(int64_t m, int n, int s, int tf = T_DCT, bool planes = false) {
  Plan p;
  p.tf = tf;
  p.m = m;
  p.n = n;
  p.s = s;
  p.npad = (n + 31) / 32 * 32;
  p.chunks = sketch_chunks(m, n, s);
  p.splits = syrk_splits(m, n);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  p.off_ctl = take(sizeof(Ctl));
  p.off_idx = take(sizeof(uint32_t) * (size_t)s);
  p.off_tab = take(sizeof(double) * (size_t)(m + 1));
  p.off_ypart = take(sizeof(double) * (size_t)sketch_max_chunks(m, n, s) * s * n);
  p.off_y = take(sizeof(double) * (size_t)s * n);
  p.off_sqr = take(sqr_workspace_bytes(n, s));
  p.off_rs = take(sizeof(double) * (size_t)n * n);
  p.off_rst = take(sizeof(double) * (size_t)n * p.npad);
  p.off_rinv = take(sizeof(double) * (size_t)p.npad);
  p.off_gpart = take(sizeof(double) * (size_t)p.splits * n * n);
  p.off_rc = take(sizeof(double) * (size_t)n * n);
  p.off_xt = take(sizeof(double) * (size_t)n * p.npad);
  p.off_e = take(sizeof(double) * (size_t)n * n);
  p.off_feat = take(sizeof(float) * kNumFeatures);
  p.off_oze = take(sizeof(uint32_t) * (size_t)oz_x_cols(n));
  p.off_ozx = take(oz_xs_bytes(n));
  p.oz = syrk_oz_plan(m, n);
  p.sk = sketch_oz_plan(m, n, s);
  p.off_colhi = take(syrk_oz_colhi_bytes(n));
  // the FP64 sketch from digit planes in row chunks: at most the chunks of a Q buffer with ldq = m, or
  // one chunk in the workspace's own planes
  const size_t q_bytes = sizeof(double) * (size_t)m * n;
  const int64_t mr = (m + 31) / 32 * 32;
  if (planes) p.planes_bytes = 16ull * (size_t)n * (size_t)mr;
  p.ozpart_bytes = std::max({syrk_oz_part_bytes(p.oz), sketch_oz_part_bytes(p.sk), sketch_ozp_part_bytes(m, n, s, q_bytes),
                             planes ? sketch_ozp_part_bytes(m, n, s, p.planes_bytes) : size_t(0)});
  p.off_ozpart = take(p.ozpart_bytes);   // the Gram, the check and the FP64 sketch use it one after the other
  p.off_tcole = take(trsm_oz_cole_bytes(n));
  p.off_trd = take(trsm_oz_rd_bytes(n));
  p.off_tabd = take(16ull * (size_t)(m + 1));   // FP16 digits of the quarter-wave table
  if (planes) p.off_planes = take(p.planes_bytes);
  p.total = o;
  return p;
}

template <typename T>
T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

__global__ void k_init_ctl(Ctl* ctl, int nlevels, int p0, int p1, int p2, int p3, double tol) {
  ctl->active = 0;
  ctl->lvl_status = 0;
  ctl->final_status = ST_OK;
  ctl->prec_used = p0;
  ctl->retries = 0;
  ctl->prec_first = p0;
  ctl->nlevels = nlevels;
  ctl->input_nonfinite = 0;
  ctl->lvl_prec[0] = p0;
  ctl->lvl_prec[1] = p1;
  ctl->lvl_prec[2] = p2;
  ctl->lvl_prec[3] = p3;
  ctl->mlp_choice = -1;
  ctl->pad0 = 0;
  ctl->tol = tol;
  ctl->ortho_fro = 0.0;
  for (int i = 0; i < kNumFeatures; ++i) ctl->features[i] = 0.f;
}

__global__ void k_write_stats(const Ctl* ctl, mrcqr_stats_t* out) {
  out->status = ctl->final_status;
  out->prec_used = ctl->prec_used;
  out->retries = ctl->retries;
  out->prec_first = ctl->prec_first;
  out->selector_choice = ctl->mlp_choice;
  out->reserved[0] = out->reserved[1] = out->reserved[2] = 0;
  out->ortho_fro = ctl->ortho_fro;
}

// Instrumentation: a host-side count of kernel launches and, between
// mrcqr_profile_begin/end, a CUDA-event pair around every launch group.
std::atomic<uint64_t> g_kernels{0};

struct ProfRec {
  int stage, level;
  cudaEvent_t a, b;
};

struct Prof {
  std::mutex mu;
  bool on = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
} g_prof;

template <typename F>
void launch(int stage, int level, cudaStream_t st, F&& f) {
  if (g_prof.on) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    ProfRec r{stage, level, g_prof.get(), g_prof.get()};
    cudaEventRecord(r.a, st);
    f();
    cudaEventRecord(r.b, st);
    g_prof.recs.push_back(r);
  } else {
    f();
  }
}

enum Stage {
  SG_INIT = 0, SG_SAMPLE, SG_COSTAB, SG_SKETCH, SG_SKREDUCE, SG_SQR, SG_TRSM, SG_SYRK, SG_CHOL, SG_TRINV, SG_RMUL,
  SG_FINALIZE, SG_CHECK, SG_JUDGE, SG_STATS, SG_PREP, SG_GREDUCE, SG_EREDUCE, SG_FEATURES, SG_SELECT, SG_MLP,
  SG_COUNT
};
const char* kStageNames[SG_COUNT] = {"init", "sample", "costab", "sketch", "sketch_reduce", "sketch_qr", "trsm",
                                     "syrk", "chol", "trinv", "rmul", "finalize", "check", "judge", "stats",
                                     "prepare", "gram_reduce", "check_reduce", "features", "select", "mlp"};

// Per-(device, stream) status records for mrcqr_get_last_status.
std::mutex g_mu;
std::map<std::pair<int, void*>, mrcqr_stats_t*> g_slots;

mrcqr_stats_t* status_slot(cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  auto key = std::make_pair(dev, (void*)st);
  auto it = g_slots.find(key);
  if (it != g_slots.end()) return it->second;
  mrcqr_stats_t* p = nullptr;
  if (cudaMalloc(&p, sizeof(mrcqr_stats_t)) != cudaSuccess) return nullptr;
  g_slots[key] = p;
  return p;
}

mrcqr_stats_t* find_slot(cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_slots.find(std::make_pair(dev, (void*)st));
  return it == g_slots.end() ? nullptr : it->second;
}

bool overlaps(const void* a, size_t abytes, const void* b, size_t bbytes) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + bbytes && pb < pa + abytes;
}

// Rows of Y for c sampled rows or bins; INVALID (-1) when c does not fit the
// transform: at most m rows of the DCT, floor(m/2) + 1 bins of the real FFT,
// at most 8192 rows of Y.
int64_t sketch_rows(int64_t m, int64_t c, int tf) {
  if (tf < T_DCT || tf > T_RFFT_REIM || c < 1) return -1;
  if (c > (tf == T_DCT ? m : m / 2 + 1)) return -1;
  const int64_t rows = tf == T_RFFT_REIM ? 2 * c : c;
  return rows > 8192 ? -1 : rows;
}

int validate(int64_t m, int64_t n, const double* A, int64_t lda, const double* Q, int64_t ldq, const double* R,
             int64_t ldr, int s_factor, int tf = T_DCT) {
  if (!A || !Q || !R) return MRCQR_ERR_INVALID;
  if (n < 1 || n > kMaxN || m < 1 || m >= (int64_t(1) << 31)) return MRCQR_ERR_INVALID;
  if (s_factor < 1 || s_factor > 16) return MRCQR_ERR_INVALID;
  if (sketch_rows(m, (int64_t)s_factor * n, tf) < 0) return MRCQR_ERR_INVALID;
  if (lda < m || ldq < m || ldr < n) return MRCQR_ERR_INVALID;
  const size_t abytes = sizeof(double) * (size_t)((n - 1) * lda + m);
  const size_t qbytes = sizeof(double) * (size_t)((n - 1) * ldq + m);
  const size_t rbytes = sizeof(double) * (size_t)((n - 1) * ldr + n);
  if (overlaps(A, abytes, Q, qbytes) || overlaps(A, abytes, R, rbytes) || overlaps(Q, qbytes, R, rbytes))
    return MRCQR_ERR_INVALID;
  return MRCQR_OK;
}

// Precision ladder starting at p (Sec. II-C): FP16/BF16 -> FP32 -> FP64.
int make_ladder(int p, bool escalate, int* lv) {
  int k = 0;
  lv[k++] = p;
  if (escalate) {
    if (p == P_FP16 || p == P_BF16) lv[k++] = P_FP32;
    if (p != P_FP64) lv[k++] = P_FP64;
  }
  return k;
}

// Stage 2 + 3 for level `lvl` (R_s already in the workspace).
int g_sketch_variant_last = 0;

// Sketch Y of level `lvl` (Algorithm 2 steps 2-4).  FP64: emulated FP64 on the
// tensor cores unless the SIMT variant or FP64-FMA products are asked for,
// from digit planes written into `scratch` (variant 5) where it is large and
// aligned enough and the variant allows, else sliced per work item (3).
// Returns the variant that ran (1 SIMT, 2 tensor-core dense rows, 3 emulated
// FP64 sliced per item, 4 four-step, 5 emulated FP64 from digit planes).
int enqueue_sketch(const Plan& p, void* ws, int prec, int variant, int fp64_products, const double* A, int64_t lda,
                   uint64_t seed, double* Y, Ctl* ctl, int lvl, cudaStream_t st, void* scratch = nullptr,
                   size_t scratch_bytes = 0) {
  const uint32_t* idx = at<uint32_t>(ws, p.off_idx);
  const double* tab = at<double>(ws, p.off_tab);
  int used = 0;
  if (prec == P_FP64 && variant != 1 && fp64_products == 0) {
    uint32_t* colhi = at<uint32_t>(ws, p.off_colhi);
    long long* part = at<long long>(ws, p.off_ozpart);
    const bool planes = variant != 3 && sketch_ozp_eligible(p.m, p.n, scratch, scratch_bytes) &&
                        sketch_ozp_part_bytes(p.m, p.n, p.s, scratch_bytes) <= p.ozpart_bytes;
    used = 3;
    launch(SG_SKETCH, lvl, st, [&] {
      if (planes && launch_sketch_ozp(p.m, p.n, p.s, A, lda, idx, tab, at<uint4>(ws, p.off_tabd), seed, colhi, part,
                                      p.ozpart_bytes, Y, scratch, scratch_bytes, ctl, lvl, st, p.tf))
        used = 5;
      else
        launch_sketch_oz(p.m, p.n, p.s, A, lda, idx, tab, seed, p.sk, colhi, part, Y, ctl, lvl, st, p.tf);
    });
    return used;
  }
  double* ypart = at<double>(ws, p.off_ypart);
  int chunks = p.chunks;
  launch(SG_SKETCH, lvl, st, [&] {
    used = launch_sketch(prec, variant, A, lda, p.m, p.n, p.s, idx, tab, seed, p.chunks,
                         ypart, ctl, lvl, st, p.tf, &chunks);
  });
  launch(SG_SKREDUCE, lvl, st, [&] {
    launch_sketch_reduce(p.m, p.n, p.s, chunks, ypart, idx, Y, ctl, lvl, st, p.tf);
  });
  return used;
}

void enqueue_stage2(const Plan& p, void* ws, const double* A, int64_t lda, double* Q, int64_t ldq, double* R,
                    int64_t ldr, int check, Ctl* ctl, int lvl, cudaStream_t st, int fp64_products = 0) {
  double* RsT = at<double>(ws, p.off_rst);
  double* rinv = at<double>(ws, p.off_rinv);
  double* Gpart = at<double>(ws, p.off_gpart);
  double* Rc = at<double>(ws, p.off_rc);
  double* XT = at<double>(ws, p.off_xt);
  double* Rs = at<double>(ws, p.off_rs);
  const bool emu = fp64_products == 0;
  uint32_t* colhi = at<uint32_t>(ws, p.off_colhi);
  long long* ozpart = at<long long>(ws, p.off_ozpart);
  if (emu)
    launch(SG_TRSM, lvl, st, [&] {
      launch_trsm_oz(p.m, p.n, A, lda, RsT, rinv, at<uint32_t>(ws, p.off_tcole), at<unsigned char>(ws, p.off_trd), Q,
                     ldq, ctl, lvl, st, colhi);
    });
  else
    launch(SG_TRSM, lvl, st, [&] { launch_trsm(p.m, p.n, A, lda, RsT, rinv, Q, ldq, ctl, lvl, st); });
  double* E = at<double>(ws, p.off_e);
  if (emu) {
    launch(SG_SYRK, lvl, st, [&] { launch_syrk_oz(p.m, p.n, Q, ldq, p.oz, colhi, ozpart, Rc, ctl, lvl, st, true); });
  } else {
    launch(SG_SYRK, lvl, st, [&] { launch_syrk(p.m, p.n, Q, ldq, p.splits, Gpart, ctl, lvl, st); });
    launch(SG_GREDUCE, lvl, st, [&] { launch_reduce_partials(p.n, p.splits, Gpart, Rc, ctl, lvl, st); });
  }
  launch(SG_CHOL, lvl, st, [&] { launch_chol(p.n, Rc, ctl, lvl, st); });
  launch(SG_TRINV, lvl, st, [&] { launch_trinv(p.n, Rc, XT, ctl, lvl, st); });
  launch(SG_RMUL, lvl, st, [&] { launch_rmul(p.n, Rc, Rs, R, ldr, ctl, lvl, st); });
  if (!emu)
    launch(SG_FINALIZE, lvl, st, [&] { launch_finalize(p.m, p.n, Q, ldq, XT, ctl, lvl, st); });
  else
    launch(SG_FINALIZE, lvl, st, [&] {
      launch_finalize_oz(p.m, p.n, Q, ldq, XT, at<uint32_t>(ws, p.off_oze), at<unsigned char>(ws, p.off_ozx), ctl,
                         lvl, st, check ? colhi : nullptr);
    });
  if (check && emu) {
    launch(SG_CHECK, lvl, st, [&] { launch_syrk_oz(p.m, p.n, Q, ldq, p.oz, colhi, ozpart, E, ctl, lvl, st, true); });
  } else if (check) {
    launch(SG_CHECK, lvl, st, [&] { launch_syrk(p.m, p.n, Q, ldq, p.splits, Gpart, ctl, lvl, st); });
    launch(SG_EREDUCE, lvl, st, [&] { launch_reduce_partials(p.n, p.splits, Gpart, E, ctl, lvl, st); });
  }
  launch(SG_JUDGE, lvl, st, [&] { launch_judge(p.n, E, check, ctl, lvl, st); });
}

int finish(cudaStream_t st) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "mrcqr: CUDA error %s\n", cudaGetErrorString(e));
    return MRCQR_ERR_CUDA;
  }
  (void)st;
  return MRCQR_OK;
}

}  // namespace

void mrcqr::note_launch() { g_kernels.fetch_add(1, std::memory_order_relaxed); }

extern "C" {

int mrcqr_version(void) { return kVersion; }

const char* mrcqr_status_string(int status) {
  switch (status) {
    case MRCQR_OK: return "ok";
    case MRCQR_ERR_INVALID: return "invalid argument";
    case MRCQR_ERR_BREAKDOWN: return "Cholesky breakdown (Gram matrix not positive definite)";
    case MRCQR_ERR_NONFINITE: return "non-finite input";
    case MRCQR_ERR_ORTHO: return "orthogonality check failed at the highest precision";
    case MRCQR_ERR_ALLOC: return "workspace allocation failed";
    case MRCQR_ERR_CUDA: return "CUDA error";
    case MRCQR_ERR_TIMEOUT: return "bounded device wait timed out";
    default: return "unknown status";
  }
}

int mrcqr_factor_ex(int64_t m, int64_t n, const double* A, int64_t lda, double* Q, int64_t ldq, double* R,
                    int64_t ldr, int sketch_prec, uint64_t seed, const mrcqr_opts_t* opts, mrcqr_stream_t stream) {
  const int s_factor = (opts && opts->s_factor > 0) ? opts->s_factor : 2;
  const int check = opts ? (opts->check != 0) : 1;
  const bool escalate = opts ? (opts->escalate != 0) : true;
  const double tol = (opts && opts->ortho_tol > 0) ? opts->ortho_tol : kDefaultTol;
  const int variant = opts ? opts->sketch_variant : 0;
  const int fp64p = opts ? opts->fp64_products : 0;
  const int tf = opts ? opts->transform : T_DCT;
  int rc = validate(m, n, A, lda, Q, ldq, R, ldr, s_factor, tf);
  if (rc != MRCQR_OK) return rc;
  if (sketch_prec < P_FP16 || sketch_prec > P_AUTO) return MRCQR_ERR_INVALID;
  const bool autosel = sketch_prec == P_AUTO;
  if (autosel && !selector_ready()) {
    fprintf(stderr, "mrcqr: MRCQR_PREC_AUTO needs selector weights (mrcqr_selector_load / mrcqr_selector_set)\n");
    return MRCQR_ERR_INVALID;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int bins = s_factor * (int)n;                 // sampled rows (DCT) or bins (real FFT)
  const int s = (int)sketch_rows(m, bins, tf);        // rows of Y
  const Plan p = make_plan(m, (int)n, s, tf);
  int lv[kMaxLevels] = {P_FP64, P_FP64, P_FP64, P_FP64};
  // AUTO: the ladder fp16 -> fp32 -> fp64 always; the selector picks where it starts
  const int nlevels = make_ladder(autosel ? (int)P_FP16 : sketch_prec, autosel || escalate, lv);
  mrcqr_stats_t* slot = status_slot(st);
  if (!slot) return MRCQR_ERR_ALLOC;
  void* ws = nullptr;
  if (cudaMallocAsync(&ws, p.total, st) != cudaSuccess) {
    cudaGetLastError();
    return MRCQR_ERR_ALLOC;
  }
  Ctl* ctl = at<Ctl>(ws, p.off_ctl);
  uint32_t* idx = at<uint32_t>(ws, p.off_idx);
  double* tab = at<double>(ws, p.off_tab);
  launch(SG_INIT, 0, st, [&] { { ::mrcqr::note_launch(); k_init_ctl<<<1, 1, 0, st>>>(ctl, nlevels, lv[0], lv[1], lv[2], lv[3], tol); } });
  launch(SG_SAMPLE, 0, st, [&] { launch_sample(m, bins, seed, idx, ctl, st, tf); });
  launch(SG_COSTAB, 0, st, [&] { launch_costab(m, tab, st); });
  for (int L = 0; L < nlevels; ++L) {
    double* y = at<double>(ws, p.off_y);
    // the FP64 sketch borrows the Q buffer for its digit planes (stage 2 of the level writes W there later)
    g_sketch_variant_last = enqueue_sketch(p, ws, lv[L], variant, fp64p, A, lda, seed, y, ctl, L, st, Q,
                                           sizeof(double) * (size_t)((n - 1) * ldq + m));
    launch(SG_SQR, L, st, [&] {
      launch_sketch_qr(lv[L], (int)n, s, y, at<void>(ws, p.off_sqr), at<double>(ws, p.off_rs),
                       at<double>(ws, p.off_rst), at<double>(ws, p.off_rinv), ctl, L, st);
    });
    if (autosel && L == 0) {
      float* feat = at<float>(ws, p.off_feat);
      launch(SG_FEATURES, 0, st, [&] { launch_features(at<double>(ws, p.off_rs), (int)n, m, feat, ctl, 0, st); });
      launch(SG_SELECT, 0, st, [&] { launch_mlp_select(feat, ctl, st); });
    }
    enqueue_stage2(p, ws, A, lda, Q, ldq, R, ldr, check, ctl, L, st, fp64p);
  }
  launch(SG_STATS, 0, st, [&] { { ::mrcqr::note_launch(); k_write_stats<<<1, 1, 0, st>>>(ctl, slot); } });
  if (opts && opts->stats_device)
    launch(SG_STATS, 0, st, [&] { { ::mrcqr::note_launch(); k_write_stats<<<1, 1, 0, st>>>(ctl, (mrcqr_stats_t*)opts->stats_device); } });
  cudaFreeAsync(ws, st);
  return finish(st);
}

int mrcqr_factor(int64_t m, int64_t n, const double* A, int64_t lda, double* Q, int64_t ldq, double* R,
                 int sketch_prec, uint64_t seed, mrcqr_stream_t stream) {
  return mrcqr_factor_ex(m, n, A, lda, Q, ldq, R, n, sketch_prec, seed, nullptr, stream);
}

int mrcqr_get_last_status(mrcqr_stream_t stream, mrcqr_stats_t* out) {
  if (!out) return MRCQR_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  mrcqr_stats_t* slot = find_slot(st);
  if (!slot) return MRCQR_ERR_INVALID;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MRCQR_ERR_CUDA;
  if (cudaMemcpy(out, slot, sizeof(mrcqr_stats_t), cudaMemcpyDeviceToHost) != cudaSuccess) return MRCQR_ERR_CUDA;
  return MRCQR_OK;
}

int mrcqr_signs(int64_t m, uint64_t seed, double* d, mrcqr_stream_t stream) {
  if (!d || m < 1 || m >= (int64_t(1) << 31)) return MRCQR_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  launch(SG_PREP, 0, st, [&] { launch_signs(m, seed, d, st); });
  return finish(st);
}

int mrcqr_round(int prec, int64_t count, const double* x, double* y, mrcqr_stream_t stream) {
  if (!x || !y || count < 0 || prec < P_FP16 || prec > P_FP64) return MRCQR_ERR_INVALID;
  if (count == 0) return MRCQR_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  launch(SG_PREP, 0, st, [&] { launch_round(prec, count, x, y, st); });
  return finish(st);
}

int mrcqr_sample_rows(int64_t m, int64_t s, uint64_t seed, uint32_t* idx, mrcqr_stream_t stream) {
  if (!idx || m < 1 || m >= (int64_t(1) << 31) || s < 1 || s > m || s > 8192) return MRCQR_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  launch(SG_SAMPLE, 0, st, [&] { launch_sample(m, (int)s, seed, idx, nullptr, st); });
  return finish(st);
}

int mrcqr_sample_transform_rows(int64_t m, int64_t c, int transform, uint64_t seed, uint32_t* idx,
                                mrcqr_stream_t stream) {
  if (!idx || m < 1 || m >= (int64_t(1) << 31) || sketch_rows(m, c, transform) < 0) return MRCQR_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  launch(SG_SAMPLE, 0, st, [&] { launch_sample(m, (int)c, seed, idx, nullptr, st, transform); });
  return finish(st);
}

int mrcqr_sketch(int64_t m, int64_t n, const double* A, int64_t lda, int64_t s, int sketch_prec, uint64_t seed,
                 double* Y, mrcqr_stream_t stream) {
  return mrcqr_sketch_ex(m, n, A, lda, s, sketch_prec, seed, 0, Y, stream);
}

int mrcqr_sketch_ex(int64_t m, int64_t n, const double* A, int64_t lda, int64_t s, int sketch_prec, uint64_t seed,
                    int variant, double* Y, mrcqr_stream_t stream) {
  return mrcqr_sketch_transform(m, n, A, lda, s, MRCQR_TRANSFORM_DCT, sketch_prec, seed, variant, Y, stream);
}

int mrcqr_sketch_transform(int64_t m, int64_t n, const double* A, int64_t lda, int64_t c, int transform,
                           int sketch_prec, uint64_t seed, int variant, double* Y, mrcqr_stream_t stream) {
  if (!A || !Y || n < 1 || n > kMaxN || m < 1 || m >= (int64_t(1) << 31) || lda < m) return MRCQR_ERR_INVALID;
  const int64_t s = sketch_rows(m, c, transform);
  if (s < 0) return MRCQR_ERR_INVALID;
  if (sketch_prec < P_FP16 || sketch_prec > P_FP64) return MRCQR_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Plan p = make_plan(m, (int)n, (int)s, transform, sketch_prec == P_FP64 && variant != 1 && variant != 3);
  void* ws = nullptr;
  if (cudaMallocAsync(&ws, p.total, st) != cudaSuccess) {
    cudaGetLastError();
    return MRCQR_ERR_ALLOC;
  }
  Ctl* ctl = at<Ctl>(ws, p.off_ctl);
  uint32_t* idx = at<uint32_t>(ws, p.off_idx);
  double* tab = at<double>(ws, p.off_tab);
  launch(SG_INIT, 0, st, [&] { { ::mrcqr::note_launch(); k_init_ctl<<<1, 1, 0, st>>>(ctl, 1, sketch_prec, P_FP64, P_FP64, P_FP64, kDefaultTol); } });
  launch(SG_SAMPLE, 0, st, [&] { launch_sample(m, (int)c, seed, idx, ctl, st, transform); });
  launch(SG_COSTAB, 0, st, [&] { launch_costab(m, tab, st); });
  g_sketch_variant_last = enqueue_sketch(p, ws, sketch_prec, variant, 0, A, lda, seed, Y, ctl, 0, st,
                                         p.planes_bytes ? at<void>(ws, p.off_planes) : nullptr, p.planes_bytes);
  cudaFreeAsync(ws, st);
  return finish(st);
}

int mrcqr_sketch_qr(int64_t n, int64_t s, const double* Y, int prec, double* Rs, mrcqr_stream_t stream) {
  if (!Y || !Rs || n < 1 || n > kMaxN || s < n || s > 8192) return MRCQR_ERR_INVALID;
  if (prec < P_FP16 || prec > P_FP64) return MRCQR_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int npad = (int)((n + 31) / 32 * 32);
  const size_t o_ctl = 0, o_w = align_up(sizeof(Ctl)), o_rst = o_w + align_up(sqr_workspace_bytes((int)n, (int)s)),
               o_rinv = o_rst + align_up(sizeof(double) * n * npad), total = o_rinv + align_up(sizeof(double) * npad);
  void* ws = nullptr;
  if (cudaMallocAsync(&ws, total, st) != cudaSuccess) {
    cudaGetLastError();
    return MRCQR_ERR_ALLOC;
  }
  Ctl* ctl = at<Ctl>(ws, o_ctl);
  launch(SG_INIT, 0, st, [&] { { ::mrcqr::note_launch(); k_init_ctl<<<1, 1, 0, st>>>(ctl, 1, prec, P_FP64, P_FP64, P_FP64, kDefaultTol); } });
  launch(SG_SQR, 0, st, [&] {
    launch_sketch_qr(prec, (int)n, (int)s, Y, at<void>(ws, o_w), Rs, at<double>(ws, o_rst), at<double>(ws, o_rinv),
                     ctl, 0, st);
  });
  cudaFreeAsync(ws, st);
  return finish(st);
}

int mrcqr_cholqr2(int64_t m, int64_t n, const double* A, int64_t lda, double* Q, int64_t ldq, double* R,
                  int64_t ldr, mrcqr_stream_t stream) {
  int rc = validate(m, n, A, lda, Q, ldq, R, ldr, 1);
  if (rc != MRCQR_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Plan p = make_plan(m, (int)n, (int)n);
  mrcqr_stats_t* slot = status_slot(st);
  if (!slot) return MRCQR_ERR_ALLOC;
  void* ws = nullptr;
  if (cudaMallocAsync(&ws, p.total, st) != cudaSuccess) {
    cudaGetLastError();
    return MRCQR_ERR_ALLOC;
  }
  Ctl* ctl = at<Ctl>(ws, p.off_ctl);
  double* Rc = at<double>(ws, p.off_rc);
  double* Rs = at<double>(ws, p.off_rs);
  launch(SG_INIT, 0, st, [&] { { ::mrcqr::note_launch(); k_init_ctl<<<1, 1, 0, st>>>(ctl, 1, P_FP64, P_FP64, P_FP64, P_FP64, kDefaultTol); } });
  // first pass, R only: R_1 = chol(A^T A) (a breakdown ends the call with that status)
  launch(SG_SYRK, 0, st, [&] {
    launch_syrk_oz(p.m, p.n, A, lda, p.oz, at<uint32_t>(ws, p.off_colhi), at<long long>(ws, p.off_ozpart), Rc, ctl, 0, st);
  });
  launch(SG_CHOL, 0, st, [&] { launch_chol(p.n, Rc, ctl, 0, st); });
  // second pass: CholQR of A R_1^{-1} (substitution), R = R_2 R_1, with the orthogonality judge
  cudaMemcpyAsync(Rs, Rc, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, st);
  launch(SG_PREP, 0, st, [&] { launch_rs_prepare((int)n, Rs, at<double>(ws, p.off_rst), at<double>(ws, p.off_rinv), st); });
  enqueue_stage2(p, ws, A, lda, Q, ldq, R, ldr, 1, ctl, 0, st);
  launch(SG_STATS, 0, st, [&] { { ::mrcqr::note_launch(); k_write_stats<<<1, 1, 0, st>>>(ctl, slot); } });
  cudaFreeAsync(ws, st);
  return finish(st);
}

int mrcqr_regime_estimate(int64_t m, int64_t n, const double* A, int64_t lda, int method, uint64_t seed,
                          double* out, mrcqr_stream_t stream) {
  if (!A || !out || n < 1 || n > kMaxN || m < n || m >= (int64_t(1) << 31) || lda < m) return MRCQR_ERR_INVALID;
  if (method != MRCQR_REGIME_CHOLQR_PROBE && method != MRCQR_REGIME_ONENORM) return MRCQR_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Plan p = make_plan(m, (int)n, (int)n);
  const bool probe = method == MRCQR_REGIME_CHOLQR_PROBE;
  const size_t off_w = p.total;   // Q = A R^{-1} of the probe
  const size_t total = off_w + (probe ? align_up(sizeof(double) * (size_t)m * n) : 0);
  void* ws = nullptr;
  if (cudaMallocAsync(&ws, total, st) != cudaSuccess) {
    cudaGetLastError();
    return MRCQR_ERR_ALLOC;
  }
  Ctl* ctl = at<Ctl>(ws, p.off_ctl);
  double* Rc = at<double>(ws, p.off_rc);
  double* E = at<double>(ws, p.off_e);
  double* Rs = at<double>(ws, p.off_rs);
  double* RsT = at<double>(ws, p.off_rst);
  double* rinv = at<double>(ws, p.off_rinv);
  uint32_t* colhi = at<uint32_t>(ws, p.off_colhi);
  long long* part = at<long long>(ws, p.off_ozpart);
  launch(SG_INIT, 0, st, [&] { { ::mrcqr::note_launch(); k_init_ctl<<<1, 1, 0, st>>>(ctl, 1, P_FP64, P_FP64, P_FP64, P_FP64, kDefaultTol); } });
  // G = A^T A (emulated FP64) and its Cholesky factor (a breakdown raises the level status)
  launch(SG_SYRK, 0, st, [&] { launch_syrk_oz(p.m, p.n, A, lda, p.oz, colhi, part, Rc, ctl, 0, st); });
  if (!probe) cudaMemcpyAsync(E, Rc, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, st);
  launch(SG_CHOL, 0, st, [&] { launch_chol(p.n, Rc, ctl, 0, st); });
  cudaMemcpyAsync(Rs, Rc, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, st);
  launch(SG_PREP, 0, st, [&] { launch_rs_prepare((int)n, Rs, RsT, rinv, st); });
  if (probe) {
    // Q = A R^{-1} and E = Q^T Q: the CholQR run whose loss of orthogonality bounds kappa
    double* W = at<double>(ws, off_w);
    launch(SG_TRSM, 0, st, [&] {
      launch_trsm_oz(p.m, p.n, A, lda, RsT, rinv, at<uint32_t>(ws, p.off_tcole), at<unsigned char>(ws, p.off_trd), W,
                     m, ctl, 0, st, colhi);
    });
    launch(SG_CHECK, 0, st, [&] { launch_syrk_oz(p.m, p.n, W, m, p.oz, colhi, part, E, ctl, 0, st, true); });
    launch(SG_JUDGE, 0, st, [&] { launch_probe(p.n, E, ctl, out, st); });
  } else {
    launch(SG_JUDGE, 0, st, [&] { launch_onenorm(p.n, E, Rc, RsT, rinv, seed, ctl, out, st); });
  }
  cudaFreeAsync(ws, st);
  return finish(st);
}

int mrcqr_cholqr_precond(int64_t m, int64_t n, const double* A, int64_t lda, const double* Rs, double* Q,
                         int64_t ldq, double* R, int64_t ldr, mrcqr_stream_t stream) {
  int rc = validate(m, n, A, lda, Q, ldq, R, ldr, 1);
  if (rc != MRCQR_OK) return rc;
  if (!Rs) return MRCQR_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Plan p = make_plan(m, (int)n, (int)n);
  mrcqr_stats_t* slot = status_slot(st);
  if (!slot) return MRCQR_ERR_ALLOC;
  void* ws = nullptr;
  if (cudaMallocAsync(&ws, p.total, st) != cudaSuccess) {
    cudaGetLastError();
    return MRCQR_ERR_ALLOC;
  }
  Ctl* ctl = at<Ctl>(ws, p.off_ctl);
  launch(SG_INIT, 0, st, [&] { { ::mrcqr::note_launch(); k_init_ctl<<<1, 1, 0, st>>>(ctl, 1, P_FP64, P_FP64, P_FP64, P_FP64, kDefaultTol); } });
  cudaMemcpyAsync(at<double>(ws, p.off_rs), Rs, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, st);
  launch(SG_PREP, 0, st, [&] { launch_rs_prepare((int)n, Rs, at<double>(ws, p.off_rst), at<double>(ws, p.off_rinv), st); });
  enqueue_stage2(p, ws, A, lda, Q, ldq, R, ldr, 1, ctl, 0, st);
  launch(SG_STATS, 0, st, [&] { { ::mrcqr::note_launch(); k_write_stats<<<1, 1, 0, st>>>(ctl, slot); } });
  cudaFreeAsync(ws, st);
  return finish(st);
}

int mrcqr_trsm(int64_t m, int64_t n, const double* A, int64_t lda, const double* R, int64_t ldr, double* W,
               int64_t ldw, int fp64_products, mrcqr_stream_t stream) {
  if (!A || !R || !W || n < 1 || n > kMaxN || m < 1 || m >= (int64_t(1) << 31) || lda < m || ldw < m || ldr < n ||
      (fp64_products != 0 && fp64_products != 1))
    return MRCQR_ERR_INVALID;
  const size_t abytes = sizeof(double) * (size_t)((n - 1) * lda + m);
  const size_t wbytes = sizeof(double) * (size_t)((n - 1) * ldw + m);
  const size_t rbytes = sizeof(double) * (size_t)((n - 1) * ldr + n);
  if (overlaps(A, abytes, W, wbytes) || overlaps(R, rbytes, W, wbytes)) return MRCQR_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Plan p = make_plan(m, (int)n, (int)n);
  void* ws = nullptr;
  if (cudaMallocAsync(&ws, p.total, st) != cudaSuccess) {
    cudaGetLastError();
    return MRCQR_ERR_ALLOC;
  }
  Ctl* ctl = at<Ctl>(ws, p.off_ctl);
  double* Rp = at<double>(ws, p.off_rs);
  double* RsT = at<double>(ws, p.off_rst);
  double* rinv = at<double>(ws, p.off_rinv);
  launch(SG_INIT, 0, st, [&] { { ::mrcqr::note_launch(); k_init_ctl<<<1, 1, 0, st>>>(ctl, 1, P_FP64, P_FP64, P_FP64, P_FP64, kDefaultTol); } });
  cudaMemcpy2DAsync(Rp, sizeof(double) * n, R, sizeof(double) * ldr, sizeof(double) * n, n, cudaMemcpyDeviceToDevice, st);
  launch(SG_PREP, 0, st, [&] { launch_rs_prepare((int)n, Rp, RsT, rinv, st); });
  if (fp64_products == 0)
    launch(SG_TRSM, 0, st, [&] {
      launch_trsm_oz(m, (int)n, A, lda, RsT, rinv, at<uint32_t>(ws, p.off_tcole), at<unsigned char>(ws, p.off_trd), W,
                     ldw, ctl, 0, st);
    });
  else
    launch(SG_TRSM, 0, st, [&] { launch_trsm(m, (int)n, A, lda, RsT, rinv, W, ldw, ctl, 0, st); });
  cudaFreeAsync(ws, st);
  return finish(st);
}

int mrcqr_gram(int64_t m, int64_t n, const double* W, int64_t ldw, double* G, int fp64_products,
               mrcqr_stream_t stream) {
  if (!W || !G || n < 1 || n > kMaxN || m < 1 || m >= (int64_t(1) << 31) || ldw < m ||
      (fp64_products != 0 && fp64_products != 1))
    return MRCQR_ERR_INVALID;
  const size_t wbytes = sizeof(double) * (size_t)((n - 1) * ldw + m);
  if (overlaps(W, wbytes, G, sizeof(double) * (size_t)(n * n))) return MRCQR_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Plan p = make_plan(m, (int)n, (int)n);
  void* ws = nullptr;
  if (cudaMallocAsync(&ws, p.total, st) != cudaSuccess) {
    cudaGetLastError();
    return MRCQR_ERR_ALLOC;
  }
  Ctl* ctl = at<Ctl>(ws, p.off_ctl);
  launch(SG_INIT, 0, st, [&] { { ::mrcqr::note_launch(); k_init_ctl<<<1, 1, 0, st>>>(ctl, 1, P_FP64, P_FP64, P_FP64, P_FP64, kDefaultTol); } });
  if (fp64_products == 0) {
    launch(SG_SYRK, 0, st, [&] {
      launch_syrk_oz(m, (int)n, W, ldw, p.oz, at<uint32_t>(ws, p.off_colhi), at<long long>(ws, p.off_ozpart), G, ctl,
                     0, st);
    });
  } else {
    double* Gpart = at<double>(ws, p.off_gpart);
    launch(SG_SYRK, 0, st, [&] { launch_syrk(m, (int)n, W, ldw, p.splits, Gpart, ctl, 0, st); });
    launch(SG_GREDUCE, 0, st, [&] { launch_reduce_partials((int)n, p.splits, Gpart, G, ctl, 0, st); });
  }
  cudaFreeAsync(ws, st);
  return finish(st);
}

int mrcqr_finalize_q(int64_t m, int64_t n, double* Q, int64_t ldq, const double* X, int64_t ldx, int fp64_products,
                     mrcqr_stream_t stream) {
  if (!Q || !X || n < 1 || n > kMaxN || m < 1 || m >= (int64_t(1) << 31) || ldq < m || ldx < n ||
      (fp64_products != 0 && fp64_products != 1))
    return MRCQR_ERR_INVALID;
  const size_t qbytes = sizeof(double) * (size_t)((n - 1) * ldq + m);
  const size_t xbytes = sizeof(double) * (size_t)((n - 1) * ldx + n);
  if (overlaps(Q, qbytes, X, xbytes)) return MRCQR_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Plan p = make_plan(m, (int)n, (int)n);
  void* ws = nullptr;
  if (cudaMallocAsync(&ws, p.total, st) != cudaSuccess) {
    cudaGetLastError();
    return MRCQR_ERR_ALLOC;
  }
  Ctl* ctl = at<Ctl>(ws, p.off_ctl);
  double* XT = at<double>(ws, p.off_xt);
  launch(SG_INIT, 0, st, [&] { { ::mrcqr::note_launch(); k_init_ctl<<<1, 1, 0, st>>>(ctl, 1, P_FP64, P_FP64, P_FP64, P_FP64, kDefaultTol); } });
  launch(SG_PREP, 0, st, [&] { launch_upper_to_xt((int)n, X, ldx, XT, st); });
  if (fp64_products == 1)
    launch(SG_FINALIZE, 0, st, [&] { launch_finalize(m, (int)n, Q, ldq, XT, ctl, 0, st); });
  else
    launch(SG_FINALIZE, 0, st, [&] {
      launch_finalize_oz(m, (int)n, Q, ldq, XT, at<uint32_t>(ws, p.off_oze), at<unsigned char>(ws, p.off_ozx), ctl,
                         0, st);
    });
  cudaFreeAsync(ws, st);
  return finish(st);
}

uint64_t mrcqr_launch_count(void) { return g_kernels.load(); }

int mrcqr_last_sketch_variant(void) { return g_sketch_variant_last; }

const char* mrcqr_stage_name(int stage) {
  return (stage >= 0 && stage < SG_COUNT) ? kStageNames[stage] : "unknown";
}

int mrcqr_profile_begin(void) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  for (auto& r : g_prof.recs) {
    g_prof.pool.push_back(r.a);
    g_prof.pool.push_back(r.b);
  }
  g_prof.recs.clear();
  g_prof.on = true;
  return MRCQR_OK;
}

int mrcqr_profile_end(int max_records, int32_t* stage, int32_t* level, float* ms, int32_t* count) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  g_prof.on = false;
  int k = 0;
  for (auto& r : g_prof.recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return MRCQR_ERR_CUDA;
    if (k < max_records) {
      float t = 0.f;
      cudaEventElapsedTime(&t, r.a, r.b);
      if (stage) stage[k] = r.stage;
      if (level) level[k] = r.level;
      if (ms) ms[k] = t;
    }
    ++k;
    g_prof.pool.push_back(r.a);
    g_prof.pool.push_back(r.b);
  }
  g_prof.recs.clear();
  if (count) *count = k;
  return MRCQR_OK;
}

int mrcqr_selector_num_params(void) { return selector_num_params(); }

int mrcqr_selector_set(const float* params, const float* mu, const float* sd, const float* costs) {
  if (!params || !mu || !sd || !costs) return MRCQR_ERR_INVALID;
  return selector_set(params, mu, sd, costs);
}

int mrcqr_selector_load(const char* path) {
  if (!path) return MRCQR_ERR_INVALID;
  FILE* f = fopen(path, "rb");
  if (!f) return MRCQR_ERR_INVALID;
  char magic[8];
  uint32_t ver = 0, np = 0;
  std::vector<float> aux(35), params;
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "MRCQRSEL", 8) == 0 && fread(&ver, 4, 1, f) == 1 &&
            ver == 1 && fread(&np, 4, 1, f) == 1 && (int)np == selector_num_params() &&
            fread(aux.data(), sizeof(float), 35, f) == 35;
  if (ok) {
    params.resize(np);
    ok = fread(params.data(), sizeof(float), np, f) == np;
  }
  fclose(f);
  if (!ok) return MRCQR_ERR_INVALID;
  return selector_set(params.data(), aux.data(), aux.data() + 16, aux.data() + 32);
}

int mrcqr_selector_features(int64_t m, int64_t n, const double* Rs, float* feat, mrcqr_stream_t stream) {
  if (!Rs || !feat || n < 1 || n > kMaxN || m < 1) return MRCQR_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  launch(SG_FEATURES, 0, st, [&] { launch_features(Rs, (int)n, m, feat, nullptr, 0, st); });
  return finish(st);
}

int mrcqr_mlp_forward(int batch, const float* X, const uint16_t* w_bf16, const float* mu, const float* sd,
                      const float* costs, float* logits, int32_t* choice, mrcqr_stream_t stream) {
  if (batch < 0 || !X || !w_bf16 || !mu || !sd || !costs || !logits) return MRCQR_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  launch(SG_MLP, 0, st, [&] { launch_mlp_forward(w_bf16, mu, sd, costs, batch, X, logits, choice, st); });
  return finish(st);
}

int mrcqr_mlp_train_step(int batch, const float* X, const int32_t* y, const float* class_w, const float* mu,
                         const float* sd, float* master, float* mom, float* var, uint16_t* w_bf16, float lr,
                         float beta1, float beta2, float eps, float wd, int step, int apply, float* grad_out,
                         float* loss_out, mrcqr_stream_t stream) {
  if (batch < 1 || !X || !y || !class_w || !mu || !sd || !w_bf16) return MRCQR_ERR_INVALID;
  if (apply && (!master || !mom || !var || step < 1)) return MRCQR_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int nparts = batch < 128 ? batch : 128;
  void* scratch = nullptr;
  const size_t bytes = sizeof(float) * ((size_t)nparts * selector_num_params() + nparts);
  if (cudaMallocAsync(&scratch, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return MRCQR_ERR_ALLOC;
  }
  float* part = static_cast<float*>(scratch);
  float* lpart = part + (size_t)nparts * selector_num_params();
  launch(SG_MLP, 0, st, [&] { launch_mlp_grad(w_bf16, mu, sd, batch, X, y, class_w, part, lpart, nparts, st); });
  launch(SG_MLP, 0, st, [&] {
    launch_mlp_reduce_adamw(nparts, part, lpart, master, mom, var, w_bf16, lr, beta1, beta2, eps, wd, step, apply,
                            grad_out, loss_out, st);
  });
  cudaFreeAsync(scratch, st);
  return finish(st);
}

int mrcqr_shutdown(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& kv : g_slots) cudaFree(kv.second);
  g_slots.clear();
  return MRCQR_OK;
}

}  // extern "C"
