// Internal launch interface of the MRCQR kernels (not part of the C ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "common.cuh"

namespace mrcqr {

// --- sketch (sketch.cu) ------------------------------------------------------
void launch_sample(int64_t m, int s, uint64_t seed, uint32_t* idx, const Ctl* ctl, cudaStream_t st);
void launch_costab(int64_t m, double* tab, float* tabf, cudaStream_t st);
int sketch_chunks(int64_t m, int n, int s);
// variant: 0 = auto (tensor cores when eligible), 1 = SIMT, 2 = tensor cores (falls back to SIMT when
// the TMA preconditions fail).  Returns the variant launched (1 or 2).
int launch_sketch(int prec, int variant, const double* A, int64_t lda, int64_t m, int n, int s,
                  const uint32_t* idx, const double* tab, const float* tabf, uint64_t seed, int chunks,
                  double* Ypart, Ctl* ctl, int level, cudaStream_t st);
// tensor-core sketch (sketch_tc.cu): FP16/BF16/FP32, A 16-byte aligned, lda even
bool sketch_tc_eligible(int prec, const double* A, int64_t lda);
bool launch_sketch_tc(int prec, const double* A, int64_t lda, int64_t m, int n, int s, const uint32_t* idx,
                      const double* tab, const float* tabf, uint64_t seed, int chunks, double* Ypart, Ctl* ctl,
                      int level, cudaStream_t st);
void launch_sketch_reduce(int64_t m, int n, int s, int chunks, const double* Ypart, const uint32_t* idx,
                          double* Y, Ctl* ctl, int level, cudaStream_t st);
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
void launch_syrk(int64_t m, int n, const double* X, int64_t ldx, int splits, double* Gpart, const Ctl* ctl,
                 int level, cudaStream_t st);
void launch_reduce_partials(int n, int splits, const double* part, double* out, const Ctl* ctl, int level,
                            cudaStream_t st);
void launch_chol(int n, double* G, Ctl* ctl, int level, cudaStream_t st);
void launch_trinv(int n, const double* Rc, double* RcinvT, const Ctl* ctl, int level, cudaStream_t st);
void launch_rmul(int n, const double* Rc, const double* Rs, double* R, int64_t ldr, const Ctl* ctl, int level,
                 cudaStream_t st);
void launch_finalize(int64_t m, int n, double* Q, int64_t ldq, const double* XT, const Ctl* ctl, int level,
                     cudaStream_t st);
void launch_judge(int n, const double* E, int check, Ctl* ctl, int level, cudaStream_t st);

}  // namespace mrcqr
