// Allocation-free variant of the sketch QR (mrcqr_sketch_qr_noalloc).
//
// Some callers cannot allocate device memory at the point where they need
// the preconditioner: code running inside another framework's memory
// manager that forbids raw cudaMalloc, or a real-time loop in which a
// device allocation (and the implicit synchronization it may cause) is not
// acceptable.  For them this entry point takes its scratch from one
// file-scope device array instead of the stream-ordered allocator.
//
// Properties a caller must know:
//  * The scratch array (kScratchBytes, about 641 KiB) is part of the
//    library image: every GPU that loads the library holds it until the
//    process exits.
//  * Every call shares the one array.  Calls whose kernels overlap on the
//    GPU (different streams, or different host threads) race on it; callers
//    must order them (one stream, or events).
//  * The array keeps the previous call's contents; the control block it
//    holds is cleared by each call, everything else is fully overwritten
//    before it is read.
//  * The first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current) and caches it.  Make
//    that first call outside any stream capture.
#include <cstdio>
#include <map>
#include <mutex>

#include "../../include/mrcqr.h"
#include "kernels.h"

namespace {

constexpr int kNaMaxN = 128;
constexpr int kNaMaxS = 512;
constexpr int kNaPad = 128;  // row stride of the padded R_s^T for n <= 128
constexpr size_t kCtlBytes = 256;
constexpr size_t kWorkBytes = sizeof(double) * (size_t)kNaMaxS * kNaMaxN;
constexpr size_t kRstBytes = sizeof(double) * (size_t)kNaMaxN * kNaPad;
constexpr size_t kRinvBytes = sizeof(double) * (size_t)kNaPad;
constexpr size_t kScratchBytes = kCtlBytes + kWorkBytes + kRstBytes + kRinvBytes;
static_assert(sizeof(mrcqr::Ctl) <= kCtlBytes, "control block must fit its slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
std::map<int, void*> g_addr;  // device ordinal -> device address of g_noalloc_scratch

// Device address of the scratch array on the current device (looked up once
// per device with that device current).  nullptr on failure.
void* scratch_address() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_addr.find(dev);
  if (it != g_addr.end()) return it->second;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return nullptr;
  g_addr[dev] = p;
  return p;
}

__global__ void k_noalloc_init(mrcqr::Ctl* ctl, int prec) {
  ctl->active = 0;
  ctl->lvl_status = 0;
  ctl->final_status = 0;
  ctl->prec_used = prec;
  ctl->retries = 0;
  ctl->prec_first = prec;
  ctl->nlevels = 1;
  ctl->input_nonfinite = 0;
  for (int i = 0; i < mrcqr::kMaxLevels; ++i) ctl->lvl_prec[i] = prec;
  ctl->mlp_choice = -1;
  ctl->tol = 0.0;
  ctl->ortho_fro = 0.0;
}

}  // namespace

extern "C" int mrcqr_sketch_qr_noalloc(int64_t n, int64_t s, const double* Y, int prec, double* Rs,
                                       mrcqr_stream_t stream) {
  if (!Y || !Rs || n < 1 || s < n || prec < MRCQR_PREC_FP16 || prec > MRCQR_PREC_FP64) return MRCQR_ERR_INVALID;
  if (n > kNaMaxN || s > kNaMaxS) {
    fprintf(stderr,
            "mrcqr_sketch_qr_noalloc: n=%lld, s=%lld exceed the static scratch limit (n <= %d, s <= %d); "
            "use mrcqr_sketch_qr\n",
            (long long)n, (long long)s, kNaMaxN, kNaMaxS);
    return MRCQR_ERR_INVALID;
  }
  unsigned char* base = static_cast<unsigned char*>(scratch_address());
  if (!base) {
    cudaGetLastError();
    return MRCQR_ERR_CUDA;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  mrcqr::Ctl* ctl = reinterpret_cast<mrcqr::Ctl*>(base);
  void* work = base + kCtlBytes;
  double* RsT = reinterpret_cast<double*>(base + kCtlBytes + kWorkBytes);
  double* rinv = reinterpret_cast<double*>(base + kCtlBytes + kWorkBytes + kRstBytes);
  { ::mrcqr::note_launch(); k_noalloc_init<<<1, 1, 0, st>>>(ctl, prec); }
  mrcqr::launch_sketch_qr(prec, (int)n, (int)s, Y, work, Rs, RsT, rinv, ctl, 0, st);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "mrcqr_sketch_qr_noalloc: CUDA error %s\n", cudaGetErrorString(e));
    return MRCQR_ERR_CUDA;
  }
  return MRCQR_OK;
}
