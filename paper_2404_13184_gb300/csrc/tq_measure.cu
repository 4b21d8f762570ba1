// Measurement, readout error and sampling (the measurement gates the paper
// announces in Sec. 3 and for which it describes the readout-error model in
// Sec. 3.5): per-qubit confusion on the outcome probabilities, a fixed-order
// FP64 cumulative distribution, and inverse-CDF sampling of shots.
#include <algorithm>
#include <cmath>

#include "tq_device.cuh"

namespace tq {
namespace {

// Confusion of one qubit q on the 2^n outcome probabilities.
__global__ void k_readout_qubit(double* __restrict__ p, int n, int q, double e10, double e01) {
  const unsigned long long half = 1ull << (n - 1);
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < half;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long x0 = ((t >> q) << (q + 1)) | (t & ((1ull << q) - 1ull));
    const unsigned long long x1 = x0 | (1ull << q);
    const double a = p[x0], b = p[x1];
    p[x0] = (1.0 - e10) * a + e01 * b;
    p[x1] = e10 * a + (1.0 - e01) * b;
  }
}

constexpr int kScanThreads = 1024;

// Inclusive prefix sums in a fixed order: thread t sums its contiguous chunk
// sequentially, thread 0 scans the chunk totals sequentially, then every
// thread writes its chunk's running sums. One CTA; N <= 2^16.
__global__ void __launch_bounds__(kScanThreads) k_cdf(const double* __restrict__ p, unsigned int N,
                                                      double* __restrict__ cdf) {
  __shared__ double part[kScanThreads];
  const unsigned int chunk = (N + kScanThreads - 1) / kScanThreads;
  const unsigned int x0 = threadIdx.x * chunk;
  const unsigned int x1 = min(N, x0 + chunk);
  double s = 0.0;
  for (unsigned int x = x0; x < x1; ++x) s += p[x];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double run = 0.0;
    for (int t = 0; t < kScanThreads; ++t) {
      const double v = part[t];
      part[t] = run;  // exclusive prefix of the chunk totals
      run += v;
    }
  }
  __syncthreads();
  double run = part[threadIdx.x];
  for (unsigned int x = x0; x < x1; ++x) {
    run += p[x];
    cdf[x] = run;
  }
}

// Shot s: the smallest x with u[s] < cdf[x] / cdf[N-1].
__global__ void k_sample(const double* __restrict__ cdf, unsigned int N, const double* __restrict__ u, int shots,
                         unsigned long long* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= shots) return;
  const double total = cdf[N - 1];
  const double v = u[s];
  unsigned int lo = 0, hi = N - 1;  // answer in [lo, hi]
  while (lo < hi) {
    const unsigned int mid = (lo + hi) / 2;
    if (v < cdf[mid] / total)
      hi = mid;
    else
      lo = mid + 1;
  }
  out[s] = lo;
}

}  // namespace

cudaError_t launch_readout(double* p, int n, const double* e10, const double* e01, cudaStream_t st) {
  const unsigned long long half = 1ull << (n - 1);
  const int grid = (int)std::max<unsigned long long>(1, std::min<unsigned long long>(1216, (half + 255) / 256));
  for (int q = 0; q < n; ++q) {
    if (e10[q] == 0.0 && e01[q] == 0.0) continue;
    k_readout_qubit<<<grid, 256, 0, st>>>(p, n, q, e10[q], e01[q]);
  }
  return cudaGetLastError();
}

cudaError_t launch_sample(const double* p, int n, double* cdf, const double* u, int shots, unsigned long long* out,
                          cudaStream_t st) {
  const unsigned int N = 1u << n;
  k_cdf<<<1, kScanThreads, 0, st>>>(p, N, cdf);
  if (shots > 0) k_sample<<<(shots + 255) / 256, 256, 0, st>>>(cdf, N, u, shots, out);
  return cudaGetLastError();
}

}  // namespace tq
