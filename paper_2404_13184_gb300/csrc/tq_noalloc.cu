// Allocation-free <Z> readout: the two-pass diagonal reduction with its
// scratch (per-CTA partial sums and the reduced totals) held in a fixed
// file-scope device array instead of memory from cudaMalloc.
//
// Who needs this: a host program whose device memory is entirely owned by
// another allocator (for example a serving process that hands all of HBM to
// PyTorch's caching allocator), or one that must never trigger the
// device-wide synchronisation cudaFree implies, cannot let this library call
// cudaMalloc or cudaFree. It passes its own buffers for rho, the masks and
// the results, and this entry point touches no allocator at all.
#include <mutex>

#include "tq_device.cuh"
#include "tq_internal.h"

namespace {

// Upper bounds of one call: the reduction grid is at most 152 CTAs and a call
// reduces Re tr, Im tr and at most 16 masks (18 quantities).
constexpr int kMaxGrid = 152;
constexpr int kMaxQuant = 18;
constexpr int kMaxMasks = kMaxQuant - 2;
constexpr size_t kPartials = (size_t)kMaxGrid * kMaxQuant;
constexpr size_t kScratchDoubles = kPartials + 32;  // partials, then the totals

// Shared by every call on a device and kept until the process exits
// (kScratchDoubles * 8 = 22,144 bytes per device).
static __device__ __align__(256) double g_readout_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device. The array's
// name is only a host-side stand-in in host code, so its address is looked up
// once per device, with that device current.
tq_status scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TQ_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_readout_scratch) != cudaSuccess || !p) return TQ_ERR_CUDA;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return TQ_OK;
}

}  // namespace

extern "C" tq_status tq_expect_z_noalloc(const void* rho_dev, int n_qubits, int precision,
                                         const uint64_t* masks_dev, int n_masks, double* out_dev,
                                         void* cuda_stream) {
  if (!rho_dev || !masks_dev || !out_dev) return TQ_ERR_ARG;
  if (n_qubits < 1 || n_qubits > tq::kMaxQubits) return TQ_ERR_ARG;
  if (precision != TQ_FP64 && precision != TQ_SPLIT) return TQ_ERR_ARG;
  if (n_masks < 1 || n_masks > kMaxMasks) return TQ_ERR_ARG;  // beyond the scratch array
  if (tq::diag_reduce_grid(n_qubits) > kMaxGrid) return TQ_ERR_ARG;
  double* scratch = nullptr;
  tq_status st = scratch_address(&scratch);
  if (st != TQ_OK) return st;
  // Every partial the final pass reads is written earlier in the same call,
  // so nothing in the array has to start at zero.
  const cudaError_t e = tq::launch_diag_reduce(rho_dev, n_qubits, precision,
                                               reinterpret_cast<const unsigned long long*>(masks_dev), n_masks,
                                               scratch, scratch + kPartials, precision == TQ_SPLIT, out_dev,
                                               static_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? TQ_OK : TQ_ERR_CUDA;
}
