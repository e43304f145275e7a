// chan_rhs_terms_noalloc: the non-linear terms N_chi, N_omega2 from caller
// buffers, with no device allocation in the call.
//
// Who needs this: code that must not call cudaMalloc at the point where it
// evaluates the terms -- a caller running inside a memory pool it does not
// own (a framework's caching allocator that forbids raw cudaMalloc), a loop
// with a hard latency budget where an allocation's implicit device
// synchronisation is not acceptable, or a caller that has already reserved
// all device memory for its own arena.  Such a caller passes its own input
// and output buffers; the only scratch the kernel needs (the forward sweep
// of the compact first-derivative solve) lives in the fixed array below.
#include <mutex>
#include <string>

#include "chan_internal.cuh"

namespace {

// Scratch for the forward D1 sweep: one double2 per (y, mode) value.  Every
// GPU that loads this library holds these 32 MiB until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
constexpr size_t kNoAllocScratchElems = kNoAllocScratchBytes / sizeof(double2);
static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocScratchElems];

// In host code g_noalloc_scratch names a host-side stand-in, not device
// memory: its device address is looked up once per device (with that device
// current) and cached here.
constexpr int kMaxDevices = 256;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" int chan_rhs_terms_noalloc(chan_t h, const void* H, void* N) {
  if (!h) return CHAN_EINVAL;
  if (!H || !N) {
    h->err = "chan_rhs_terms_noalloc: NULL buffer";
    return CHAN_EINVAL;
  }
  const size_t n = (size_t)h->Ny * h->M;
  if (n > kNoAllocScratchElems) {
    h->err = "chan_rhs_terms_noalloc: Ny*Nz*(Nx/2) = " + std::to_string(n) + " exceeds the " +
             std::to_string(kNoAllocScratchElems) + " complex values (32 MiB) of the built-in scratch";
    return CHAN_EINVAL;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev != h->device || dev < 0 || dev >= kMaxDevices) {
    h->err = "chan_rhs_terms_noalloc: the current device must be the handle's device";
    return CHAN_EINVAL;
  }
  void* scr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      e = cudaGetSymbolAddress(&g_scratch_addr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_scratch_addr[dev] = nullptr;
        h->err = std::string("chan_rhs_terms_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return CHAN_ECUDA;
      }
    }
    scr = g_scratch_addr[dev];
  }
  const double2* Hf = static_cast<const double2*>(H);
  double2* Nf = static_cast<double2*>(N);
  e = launch_nonlin_scratch(h, Hf, Hf + n, Hf + 2 * n, Nf, Nf + n, static_cast<double2*>(scr));
  if (e != cudaSuccess) {
    h->err = std::string("chan_rhs_terms_noalloc: ") + cudaGetErrorString(e);
    return CHAN_ECUDA;
  }
  return CHAN_OK;
}
