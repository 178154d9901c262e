// Internal launch interface of the MRCQR kernels (not part of the C ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "common.cuh"

namespace mrcqr {

// Counts one kernel launch (every launch site of the library calls it just
// before its <<<...>>>); read through mrcqr_launch_count.
void note_launch();

struct SyrkOzPlan {     // emulated-FP64 Gram: output tiles (128 x 64) and row slabs
  int ntiles, slabs;
  int64_t rows_per_slab;
  int8_t ti[20], tj[20];       // I block (128 columns), J block (64 columns) of each tile
  int8_t tile_of[4][8];        // (I, J) -> tile, -1 where no tile
};
struct SketchOzPlan {   // emulated-FP64 sketch: 128-column blocks of A x 64-row sample tiles x row slabs
  int mblocks, ntiles, slabs;
  int64_t rows_per_slab;
};

// One problem of a grouped (batched) launch: caller buffers, shape, tuned
// split sizes and its slice of the batch workspace.
struct Prob {
  const double* A;
  double* Q;
  double* R;
  int64_t lda, ldq, ldr;
  int64_t m;
  int n, s, npad, chunks, splits, ntile_syrk, check, nlevels;
  int tf, bins;      // sketch transform (T_DCT, T_RFFT, T_RFFT_REIM) and sampled rows or bins; s = rows of Y
  int lvl_prec[kMaxLevels];
  int64_t rows_per_chunk, rows_per_split;
  uint2 key;
  double tol;
  Ctl* ctl;
  uint32_t* idx;
  double* tab;
  double* ypart;
  double* y;
  void* sqrw;
  double* rs;
  double* rst;
  double* rinv;
  double* gpart;
  double* rc;
  double* xt;
  double* e;
  int32_t* status;   // caller's status entry
  // emulated-FP64 products (grouped heavy phases): plans and this problem's scratch
  SyrkOzPlan oz_sp;
  SketchOzPlan oz_kp;
  uint32_t* oz_colhi;     // column maxima of A, W or Q (high words)
  long long* oz_part;     // Gram / check / FP64-sketch partials
  int* oz_cole;           // TRSM: column exponents of D^-1 R, then e_k (2 x n16 ints)
  unsigned char* oz_rd;   // TRSM: digit panels of D^-1 R
  uint32_t* oz_xe;        // finalize: column exponents of R_c^-1
  unsigned char* oz_xs;   // finalize: digit panels of R_c^-1
  // tensor-core sketch (grouped): TMA maps of A with slabs of 64 rows (FP16/BF16) and 32 rows (FP32);
  // null when A is not eligible (16-byte alignment, even lda)
  const void* tmap64;
  const void* tmap32;
};

// A grouped launch walks a list of work items {problem, a, b, c} with a
// grid-stride loop; every item skips itself unless its problem's control
// block names the launch's escalation level.
struct Group {
  const Prob* probs;
  const int4* items;
  int nitems;
};

void prepare_g_kernels(int max_s);   // kernel attributes; call outside stream capture
void launch_g_init(const Group& g, cudaStream_t st);
void launch_g_sample(const Group& g, int max_s, cudaStream_t st);
void launch_g_costab(const Group& g, cudaStream_t st);
void launch_g_sketch(const Group& g, int prec, int level, cudaStream_t st);
void launch_g_sketch_reduce(const Group& g, int level, cudaStream_t st);
void launch_g_sketch_qr(const Group& g, bool fp64, int level, cudaStream_t st);
void launch_g_trsm(const Group& g, int level, cudaStream_t st);
void launch_g_syrk(const Group& g, int tn, bool check, int level, cudaStream_t st);
void launch_g_reduce(const Group& g, bool check, int level, cudaStream_t st);
void launch_g_chol(const Group& g, int level, cudaStream_t st);
void launch_g_trinv(const Group& g, int level, cudaStream_t st);
void launch_g_rmul(const Group& g, int level, cudaStream_t st);
void launch_g_finalize(const Group& g, int level, cudaStream_t st);
void launch_g_judge(const Group& g, int level, cudaStream_t st);
void launch_g_publish(const Group& g, cudaStream_t st);
// grouped emulated-FP64 heavy phases (ozaki.cu): one persistent launch per kernel over the work list
//   colhi        items {i, column}: column maxima of A (FP64 sketch)
//   sketch_oz    items {i, item of the problem's SketchOzPlan}   sketch_oz_reduce {i, 256-entry block}
//   row_scale    items {i, 8-row block of R_s}                   prep_r {i, column < n16}
//   trsm_oz      items {i, 128-row block}
//   syrk_oz      items {i, item of the problem's SyrkOzPlan}     syrk_oz_reduce {i, 256-entry block}
//   prep_x       items {i, column < n64}                         finalize_oz {i, 128-row block}
void prepare_g_oz_kernels();   // kernel attributes; call outside stream capture
void launch_g_oz_colhi(const Group& g, int level, cudaStream_t st);
void launch_g_oz_sketch(const Group& g, int level, cudaStream_t st);
void launch_g_oz_sketch_reduce(const Group& g, int level, cudaStream_t st);
void launch_g_oz_row_scale(const Group& g, int level, cudaStream_t st);
void launch_g_oz_prep_r(const Group& g, int level, cudaStream_t st);
void launch_g_oz_trsm(const Group& g, int level, cudaStream_t st);
void launch_g_oz_syrk(const Group& g, bool check, int level, cudaStream_t st);
void launch_g_oz_syrk_reduce(const Group& g, bool check, int level, cudaStream_t st);
void launch_g_oz_prep_x(const Group& g, int level, cudaStream_t st);
void launch_g_oz_finalize(const Group& g, int level, cudaStream_t st);

// --- sketch (sketch.cu) ------------------------------------------------------
// tf: the sketch transform (T_DCT, T_RFFT, T_RFFT_REIM of common.cuh); s rows (DCT) or bins (real FFT), written
// to idx[0..s) and, for T_RFFT_REIM, their Im rows to idx[s..2s).
void launch_sample(int64_t m, int s, uint64_t seed, uint32_t* idx, const Ctl* ctl, cudaStream_t st, int tf = 0);
void launch_costab(int64_t m, double* tab, cudaStream_t st);
int sketch_chunks(int64_t m, int n, int s);
// variant: 0 = auto (the faster of the tensor-core variants by the measured choice table, SIMT when
// neither is eligible), 1 = SIMT, 2 = tensor-core dense rows (falls back to SIMT when the TMA
// preconditions fail), 4 = four-step (falls back to 2).  Returns the variant launched (1, 2 or 4) and
// the number of partial-sum chunks written to Ypart in *chunks_used (at most max_chunks).
int launch_sketch(int prec, int variant, const double* A, int64_t lda, int64_t m, int n, int s,
                  const uint32_t* idx, const double* tab, uint64_t seed, int chunks,
                  double* Ypart, Ctl* ctl, int level, cudaStream_t st, int tf = 0, int* chunks_used = nullptr);
// four-step sketch (sketch_fs.cu): DCT, FP16/BF16/FP32, m a multiple of 1024 (<= 2^22), s <= 1024
bool sketch_fs_eligible(int prec, int tf, const double* A, int64_t lda, int64_t m, int n, int s);
int sketch_fs_chunks(int prec, int64_t m, int n);
bool launch_sketch_fs(int prec, const double* A, int64_t lda, int64_t m, int n, int s, const uint32_t* idx,
                      const double* tab, uint64_t seed, int chunks, double* Ypart, Ctl* ctl, int level,
                      cudaStream_t st);
// Partial-sum chunks the sketch of (m, n, s) may write (the larger of the variants' counts).
int sketch_max_chunks(int64_t m, int n, int s);
// tensor-core sketch (sketch_tc.cu): FP16/BF16/FP32, A 16-byte aligned, lda even
bool sketch_tc_eligible(int prec, const double* A, int64_t lda);
// A TMA map of A with slabs of `rows` rows and 64 columns into map_out (host memory of
// sketch_tc_map_bytes(), 64-byte aligned); false when A is not eligible
bool sketch_tc_encode(int rows, const double* A, int64_t lda, int64_t m, int n, void* map_out);
size_t sketch_tc_map_bytes();
void prepare_g_sketch_tc();   // kernel attributes; call outside stream capture
// grouped tensor-core sketch: items {problem, chunk, sample tile of 128 mt rows, 64-column block}
void launch_g_sketch_tc(const Group& g, int prec, int mt, int level, cudaStream_t st);
bool launch_sketch_tc(int prec, const double* A, int64_t lda, int64_t m, int n, int s, const uint32_t* idx,
                      const double* tab, uint64_t seed, int chunks, double* Ypart, Ctl* ctl,
                      int level, cudaStream_t st, int tf = 0);
void launch_sketch_reduce(int64_t m, int n, int s, int chunks, const double* Ypart, const uint32_t* idx,
                          double* Y, Ctl* ctl, int level, cudaStream_t st, int tf = 0);
void launch_round(int prec, int64_t count, const double* x, double* y, cudaStream_t st);
// Signs of rows [0, m) as +-1 doubles (test entry point).
void launch_signs(int64_t m, uint64_t seed, double* out, cudaStream_t st);

// --- sketch QR (sqr.cu) --------------------------------------------------------
size_t sqr_workspace_bytes(int n, int s);
void launch_sketch_qr(int prec, int n, int s, const double* Y, void* work, double* Rs, double* RsT,
                      double* rinv, Ctl* ctl, int level, cudaStream_t st);
void launch_rs_prepare(int n, const double* Rs, double* RsT, double* rinv, cudaStream_t st);

// --- FP64 Cholesky-QR stage (stage2.cu) --------------------------------------
void launch_trsm(int64_t m, int n, const double* A, int64_t lda, const double* RT, const double* rinv,
                 double* W, int64_t ldw, const Ctl* ctl, int level, cudaStream_t st);
int syrk_splits(int64_t m, int n);
int syrk_tile_for(int n);
void launch_syrk(int64_t m, int n, const double* X, int64_t ldx, int splits, double* Gpart, const Ctl* ctl,
                 int level, cudaStream_t st);
void launch_reduce_partials(int n, int splits, const double* part, double* out, const Ctl* ctl, int level,
                            cudaStream_t st);
void launch_chol(int n, double* G, Ctl* ctl, int level, cudaStream_t st);
void launch_trinv(int n, const double* Rc, double* RcinvT, const Ctl* ctl, int level, cudaStream_t st);
void launch_upper_to_xt(int n, const double* X, int64_t ldx, double* XT, cudaStream_t st);
void launch_rmul(int n, const double* Rc, const double* Rs, double* R, int64_t ldr, const Ctl* ctl, int level,
                 cudaStream_t st);
void launch_finalize(int64_t m, int n, double* Q, int64_t ldq, const double* XT, const Ctl* ctl, int level,
                     cudaStream_t st);
void launch_judge(int n, const double* E, int check, Ctl* ctl, int level, cudaStream_t st);

// --- emulated FP64 products on tensor cores (ozaki.cu) ---------------------------
size_t oz_xs_bytes(int n);
// rows_per_slab > 0: that slab height (a tuned value); 0: slabs chosen so tiles x slabs fills the GPU
SyrkOzPlan syrk_oz_plan(int64_t m, int n, int64_t rows_per_slab = 0);
size_t syrk_oz_part_bytes(const SyrkOzPlan& P);
size_t syrk_oz_colhi_bytes(int n);
// colHi holds the column maxima of |W| (high words); colhi_ready: the producer of W
// (launch_trsm_oz / launch_finalize_oz given colHiOut = colHi) already wrote them.
void launch_syrk_oz(int64_t m, int n, const double* W, int64_t ldw, const SyrkOzPlan& P, uint32_t* colHi,
                    long long* part, double* out, Ctl* ctl, int level, cudaStream_t st, bool colhi_ready = false);
SketchOzPlan sketch_oz_plan(int64_t m, int n, int s);
// W = A R^{-1} (k_trsm_oz, 16-column blocks): workspace of the R digit panels and exponents
size_t trsm_oz_rd_bytes(int n);
// columns of the finalize's X digits and exponents (n padded to its tile width)
int oz_x_cols(int n);
size_t trsm_oz_cole_bytes(int n);
void launch_trsm_oz(int64_t m, int n, const double* A, int64_t lda, const double* RT, const double* rinv,
                    uint32_t* colE, unsigned char* Rd, double* W, int64_t ldw, Ctl* ctl, int level, cudaStream_t st,
                    uint32_t* colHiOut = nullptr);
size_t sketch_oz_part_bytes(const SketchOzPlan& P);
void launch_sketch_oz(int64_t m, int n, int s, const double* A, int64_t lda, const uint32_t* idx, const double* tab,
                      uint64_t seed, const SketchOzPlan& P, uint32_t* colHi, long long* part, double* Y, Ctl* ctl,
                      int level, cudaStream_t st, int tf = 0);
void launch_finalize_oz(int64_t m, int n, double* Q, int64_t ldq, const double* XT, uint32_t* colE,
                        unsigned char* Xs, Ctl* ctl, int level, cudaStream_t st, uint32_t* colHiOut = nullptr);
// column maxima of |X| (high words) into colHi, and Y from FP64-sketch partials (P.slabs row slabs)
void launch_oz_col_hi(int64_t m, int n, const double* X, int64_t ldx, uint32_t* colHi, const Ctl* ctl, int level,
                      cudaStream_t st);
void launch_sketch_oz_reduce(int n, int s, const uint32_t* colHi, const uint32_t* idx, const SketchOzPlan& P,
                             const long long* part, double* Y, Ctl* ctl, int level, cudaStream_t st, int tf,
                             int64_t m);

// --- FP64 sketch from digit planes (ozaki_planes.cu) -----------------------------
// The planes of D A (16 bytes per entry) go to `scratch` in row chunks of sketch_ozp_chunk_rows rows
// (0: scratch too small); tabd holds 16 (m + 1) bytes; part must hold sketch_ozp_part_bytes.  False
// (nothing enqueued) when not eligible: scratch not 16-byte aligned or too small, no tensor-map encoder.
int64_t sketch_ozp_chunk_rows(int64_t m, int n, size_t scratch_bytes);
size_t sketch_ozp_part_bytes(int64_t m, int n, int s, size_t scratch_bytes);
bool sketch_ozp_eligible(int64_t m, int n, const void* scratch, size_t scratch_bytes);
bool launch_sketch_ozp(int64_t m, int n, int s, const double* A, int64_t lda, const uint32_t* idx, const double* tab,
                       uint4* tabd, uint64_t seed, uint32_t* colHi, long long* part, size_t part_bytes, double* Y,
                       void* scratch, size_t scratch_bytes, Ctl* ctl, int level, cudaStream_t st, int tf);

// --- regime estimates without learning (regime.cu) -------------------------------
// out (DEVICE double[4]) = {kappa estimate, regime 0/1/2, q, 0} from the Gram E = Q^T Q of a CholQR run,
// or {kappa estimate, regime, ||G||_1, est ||G^-1||_1} from G = A^T A and its Cholesky factor R
// (RT, rinv as launch_rs_prepare writes them).  A raised level status (Cholesky breakdown) gives inf.
void launch_probe(int n, const double* E, const Ctl* ctl, double* out, cudaStream_t st);
void launch_onenorm(int n, const double* G, const double* R, const double* RT, const double* rinv, uint64_t seed,
                    const Ctl* ctl, double* out, cudaStream_t st);

// --- learned selector (selector.cu) --------------------------------------------
int selector_num_params();
bool selector_ready();
int selector_set(const float* params, const float* mu, const float* sd, const float* costs);
void launch_features(const double* Rs, int n, int64_t m, float* out, const Ctl* ctl, int level, cudaStream_t st);
bool launch_mlp_select(const float* feat, Ctl* ctl, cudaStream_t st);
void launch_mlp_forward(const unsigned short* w, const float* mu, const float* sd, const float* costs, int batch,
                        const float* X, float* logits, int32_t* choice, cudaStream_t st);
void launch_mlp_grad(const unsigned short* w, const float* mu, const float* sd, int batch, const float* X,
                     const int32_t* y, const float* class_w, float* part, float* loss_part, int nparts,
                     cudaStream_t st);
void launch_mlp_reduce_adamw(int nparts, const float* part, const float* loss_part, float* master, float* mom,
                             float* var, unsigned short* wbf16, float lr, float beta1, float beta2, float eps,
                             float wd, int step, int apply, float* grad_out, float* loss_out, cudaStream_t st);

}  // namespace mrcqr
