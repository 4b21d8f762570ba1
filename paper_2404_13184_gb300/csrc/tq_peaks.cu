// Issue-rate probes of the arithmetic pipes the apply kernels are bound by:
// the roofline denominators that a copy benchmark and a cuBLAS GEMM do not
// give (the FP64 FMA pipe, the FP64 tensor path, FP32 FMA, and the
// conversions an FP64-accurate tensor-core pass would need).
//
// Each probe is a kernel of independent dependency chains (8 per thread, so
// the pipe, not the latency, is the limit), run on every SM with enough
// warps to fill it, timed with CUDA events on a private stream; the rate is
// work per second of the best of three launches.
#include <algorithm>

#include "tq_device.cuh"
#include "tanq.h"

namespace tq {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(256) k_probe_dfma(double* out, int iters, double seed) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + threadIdx.x + c;
  const double m = 0.999999, k = 1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a[c]) : "d"(m), "d"(k));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.678) out[0] = s;  // keeps the chains alive; never taken in practice
}

__global__ void __launch_bounds__(256) k_probe_ffma(float* out, int iters, float seed) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + threadIdx.x + c;
  const float m = 0.9999f, k = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[c]) : "f"(m), "f"(k));
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.678f) out[0] = s;
}

// FP64 tensor path: mma.sync m8n8k4 (one warp: 8 x 8 x 4 multiply-adds, 512 flops)
__global__ void __launch_bounds__(256) k_probe_dmma(double* out, int iters, double seed) {
  double d[kChains][2];
#pragma unroll
  for (int c = 0; c < kChains; ++c) d[c][0] = d[c][1] = seed + c;
  const double a = 1e-3 * (threadIdx.x & 7), b = 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll / 4; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                     : "+d"(d[c][0]), "+d"(d[c][1])
                     : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += d[c][0] + d[c][1];
  if (s == 12345.678) out[0] = s;
}

// Conversions: 64-bit integer -> FP64 (cvt.rn.f64.s64) and FP32 -> FP64
// (cvt.f64.f32). Each conversion's result feeds the next one of its chain
// (its bit pattern reinterpreted, one integer op), so none can be dropped.
__global__ void __launch_bounds__(256) k_probe_cvt_s64(double* out, int iters, long long seed) {
  long long v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = seed + threadIdx.x * 977 + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        double r;
        asm volatile("cvt.rn.f64.s64 %0, %1;" : "=d"(r) : "l"(v[c]));
        v[c] = __double_as_longlong(r) >> 12;  // a 52-bit integer again
      }
  }
  long long s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  if (s == 12345) out[0] = (double)s;
}

__global__ void __launch_bounds__(256) k_probe_cvt_f32(double* out, int iters, float seed) {
  float v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = seed + threadIdx.x + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        double r;
        asm volatile("cvt.f64.f32 %0, %1;" : "=d"(r) : "f"(v[c]));
        v[c] = __int_as_float(__double2hiint(r) | 0x3f800000);  // a float in [1, 2) again
      }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  if (s == 12345.678f) out[0] = s;
}

}  // namespace
}  // namespace tq

extern "C" tq_status tq_pipe_rate(int pipe, int iters, double* ops_per_s, double* ms_out) {
  using namespace tq;
  if (!ops_per_s || iters < 1 || iters > (1 << 24) || pipe < TQ_PIPE_DFMA || pipe > TQ_PIPE_CVT_F64_F32)
    return TQ_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TQ_ERR_CUDA;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double* sink = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMalloc(&sink, 256);
  const int threads = 256, grid = sms * 4;  // 32 warps per SM
  const double warps = (double)grid * threads / 32.0;
  // work units per thread per outer iteration, and flops (or ops) per unit
  double per_iter = 0.0;
  switch (pipe) {
    case TQ_PIPE_DFMA: per_iter = (double)kUnroll * kChains * 2.0 * threads * grid; break;
    case TQ_PIPE_FFMA: per_iter = (double)kUnroll * kChains * 2.0 * threads * grid; break;
    case TQ_PIPE_DMMA: per_iter = (double)(kUnroll / 4) * kChains * 512.0 * warps; break;
    default: per_iter = (double)kUnroll * kChains * threads * grid; break;
  }
  float best = 0.f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up
    e = cudaEventRecord(e0, st);
    switch (pipe) {
      case TQ_PIPE_DFMA: k_probe_dfma<<<grid, threads, 0, st>>>(sink, iters, 1.0); break;
      case TQ_PIPE_DMMA: k_probe_dmma<<<grid, threads, 0, st>>>(sink, iters, 1.0); break;
      case TQ_PIPE_FFMA: k_probe_ffma<<<grid, threads, 0, st>>>(reinterpret_cast<float*>(sink), iters, 1.f); break;
      case TQ_PIPE_CVT_F64_S64: k_probe_cvt_s64<<<grid, threads, 0, st>>>(sink, iters, 1); break;
      case TQ_PIPE_CVT_F64_F32: k_probe_cvt_f32<<<grid, threads, 0, st>>>(sink, iters, 1.f); break;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (sink) cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (e != cudaSuccess || best <= 0.f) return TQ_ERR_CUDA;
  *ops_per_s = per_iter * iters / (best * 1e-3);
  if (ms_out) *ms_out = best;
  return TQ_OK;
}
