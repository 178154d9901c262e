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
//  * The first call in each CUDA context looks up the array's device address
//    with cudaGetSymbolAddress (with that device current) and caches it under
//    the context's id.  A device reset makes a new context (and reloads the
//    library's device image), so the next call looks the address up again.
//    Make the first call on a device (and the first after a reset) outside
//    any stream capture.
//  * The stream must belong to the current device; a stream of another
//    device is rejected as an invalid argument.
#include <cstdio>
#include <map>
#include <mutex>
#include <utility>

#include <cuda.h>

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
// (device ordinal, context id) -> device address of g_noalloc_scratch
std::map<std::pair<int, unsigned long long>, void*> g_addr;

using PfnCtxGetCurrent = CUresult (*)(CUcontext*);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long*);

// Id of the calling thread's current CUDA context (unique for the life of
// the process, so a context made after a device reset has a new one).
// False when no context is current or the driver lacks the calls.
bool current_context_id(unsigned long long* id) {
  static PfnCtxGetCurrent get_current = nullptr;
  static PfnCtxGetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<PfnCtxGetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<PfnCtxGetId>(f);
    cudaGetLastError();
  });
  if (!get_current || !get_id) return false;
  CUcontext c = nullptr;
  if (get_current(&c) != CUDA_SUCCESS || c == nullptr) return false;
  return get_id(c, id) == CUDA_SUCCESS;
}

// Device address of the scratch array in the current context of device
// `dev` (looked up once per context, with that device current).  nullptr
// on failure.
void* scratch_address(int dev) {
  unsigned long long cid = 0;
  bool have = current_context_id(&cid);
  std::lock_guard<std::mutex> lk(g_mu);
  if (have) {
    auto it = g_addr.find(std::make_pair(dev, cid));
    if (it != g_addr.end()) return it->second;
  }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return nullptr;
  if (!have) have = current_context_id(&cid);   // the lookup made the primary context current
  if (have) g_addr[std::make_pair(dev, cid)] = p;
  return p;
}

// Clears every word of the control block, then sets the fields that do not
// start at zero (the same values the allocating entry point starts from).
__global__ void k_noalloc_init(mrcqr::Ctl* ctl, int prec) {
  int* w = reinterpret_cast<int*>(ctl);
  for (size_t i = 0; i < sizeof(mrcqr::Ctl) / sizeof(int); ++i) w[i] = 0;
  ctl->final_status = mrcqr::ST_OK;
  ctl->prec_used = prec;
  ctl->prec_first = prec;
  ctl->nlevels = 1;
  ctl->lvl_prec[0] = prec;
  for (int i = 1; i < mrcqr::kMaxLevels; ++i) ctl->lvl_prec[i] = mrcqr::P_FP64;
  ctl->mlp_choice = -1;
  ctl->tol = 1e-13;
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
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sdev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaStreamGetDevice(st, &sdev) != cudaSuccess) {
    cudaGetLastError();
    return MRCQR_ERR_CUDA;
  }
  if (sdev != dev) {
    fprintf(stderr, "mrcqr_sketch_qr_noalloc: the stream belongs to device %d, the current device is %d\n", sdev,
            dev);
    return MRCQR_ERR_INVALID;
  }
  unsigned char* base = static_cast<unsigned char*>(scratch_address(dev));
  if (!base) {
    cudaGetLastError();
    return MRCQR_ERR_CUDA;
  }
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
