// Split-precision width-2 apply pass on the 5th-generation tensor cores
// (tcgen05, sm_103a), Hermitian mode, for single states. The arithmetic
// (the real-ified 32 x 32 product, (R - I), the three-term BF16 split and
// its six products) is described in tq_tc.cuh.
//
// Tile walk and Hermitian bookkeeping follow the CUDA-core kernel of the
// same pass (tq_apply.cu): 16 x 16 tiles of canonical groups (row rest a <=
// column rest b), one thread per group, a warp covering 8 row rests x 4
// column rests; entries below the diagonal are read as the conjugate of
// their transpose and written back conjugated to it.
//
// Work unit: half of a 16 x 16 tile (16 row rests x 8 column rests, 128
// groups), one CTA of 128 threads, one thread per group, several CTAs per
// SM. Per unit t a thread:
//   - has unit t's 16 entries in registers (loaded during unit t - 1),
//     issues the loads of unit t + 1 into registers, splits unit t's
//     entries into the three BF16 terms and writes its row of the A operand;
//   - after the CTA barrier, one thread issues the 12 MMAs of the unit
//     (M = 128, N = 32, K = 16 each) into the CTA's 32-column tensor-memory
//     accumulator and commits them to an mbarrier;
//   - every thread waits (bounded) for the MMAs, reads its row of D, adds x
//     and stores. Groups are disjoint, so the early loads of unit t + 1
//     never see an entry that unit t writes.
//
// k_batch_tc2 is the same pass over one fusion round of many split states
// (the batch engine's split tile jobs with TQ_ENGINE_TENSOR), from a job
// table (tq_batched.cuh); width-1 blocks there run as S (x) I.
#include <algorithm>
#include <atomic>
#include <mutex>

#include "tq_device.cuh"
#include "tanq.h"
#include "tq_tc.cuh"
#include "tq_batched.cuh"

namespace tq {

namespace {

using namespace tc;

// Waits on the MMA-completion barrier that gave up (a tile's MMAs did not
// complete within the bound); read and cleared by tc_take_timeouts().
__device__ unsigned int g_tc_timeouts;

constexpr int kThreads = 128;
constexpr int kTile = 16;
constexpr uint32_t kATermBytes = 128 * kRowBytes;  // 128 rows (M)
constexpr uint32_t kOffA = 0;
constexpr uint32_t kOffB = kOffA + 3 * kATermBytes;
constexpr uint32_t kOffBar = kOffB + 3 * kBTermBytes;
constexpr uint32_t kOffTmem = kOffBar + 8;
constexpr uint32_t kOffFlag = kOffTmem + 4;
constexpr uint32_t kSmemBytes = kOffFlag + 4;
constexpr uint32_t kTmemCols = 32;
constexpr int kCtasPerSm = 4;
constexpr long long kMaxSpin = 1ll << 22;  // try_wait rounds before a wait gives up (~seconds)

// Failure-path test settings (tq_test_tc_wait_limit), read at each launch.
std::atomic<long long> g_test_max_tries{kMaxSpin};
std::atomic<int> g_test_skip_mma{0};

// This thread's group in a work unit: row and column bases (target bits
// zero), whether it is canonical, whether it is self-conjugate.
struct Group {
  unsigned int rb, cb;
  bool active, self;
};

// max_tries: try_wait rounds before an MMA wait gives up; skip_mma (tests
// of the failure path only): issue neither the MMAs nor their commit, so
// the first wait runs out with nothing in flight.
__global__ void __launch_bounds__(kThreads, kCtasPerSm) k_apply_herm_tc2(float2* rho, const float2* __restrict__ S,
                                                                           const __grid_constant__ ApplyParams p,
                                                                           long long max_tries, int skip_mma) {
  constexpr int D = 16;
  extern __shared__ __align__(1024) unsigned char smem[];
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t bar = sbase + kOffBar;
  volatile uint32_t* s_tmem = reinterpret_cast<volatile uint32_t*>(smem + kOffTmem);
  volatile int* s_abort = reinterpret_cast<volatile int*>(smem + kOffFlag);
  const int tid = threadIdx.x, lane = tid % 32, w = tid / 32;

  int qs[2] = {p.q[0], p.q[1]};
  if (qs[0] > qs[1]) {
    const int t = qs[0];
    qs[0] = qs[1];
    qs[1] = t;
  }
  const unsigned int b0 = 1u << p.q[0], b1 = 1u << p.q[1], N = 1u << p.n;
  build_b(smem + kOffB, S, tid, kThreads);
  if (tid == 0) {
    bar_init(bar, 1);
    *s_abort = 0;
  }
  if (w == 0) tmem_alloc(sbase + kOffTmem, kTmemCols);
  fence_operands();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *s_tmem;

  // a warp covers 8 row rests x 4 column rests of the half tile
  const int i = (lane % 8) + 8 * (w % 2), j0 = (lane / 8) + 4 * (w / 2);
  const unsigned int di = (unsigned int)deposit_zeros(i, qs, 2), dj0 = (unsigned int)deposit_zeros(j0, qs, 2),
                     dj1 = (unsigned int)deposit_zeros(j0 + 8, qs, 2);
  const uint32_t a_row = sbase + kOffA + core_off(tid, 0);
  const uint32_t t_row = tmem + ((uint32_t)(32 * w) << 16);  // this warp's 32 TMEM lanes
  const unsigned long long Mt = (1ull << (p.n - 2)) / kTile;
  const unsigned long long n_units = Mt * (Mt + 1);           // two halves per canonical tile

  auto group_of = [&](unsigned long long u) {
    bool diag = false;
    const unsigned long long tt = canonical_group(u >> 1, 32, &diag);  // (ta, tb) as ta | tb << 32
    const int j = (int)(u & 1ull) * 8 + j0;
    Group g;
    g.active = !(diag && i > j);  // below the diagonal of a diagonal tile: not a canonical group
    g.self = diag && i == j;
    g.rb = (unsigned int)deposit_zeros((tt & 0xffffffffull) * kTile, qs, 2) + di;
    g.cb = (unsigned int)deposit_zeros((tt >> 32) * kTile, qs, 2) + ((u & 1ull) ? dj1 : dj0);
    return g;
  };
  // raw loads of a group's stored entries (conjugation applied at use)
  auto load = [&](const Group& g, float2 x[D]) {
#pragma unroll
    for (int l = 0; l < D; ++l) {
      bool up;
      const unsigned int idx = entry_index(g.rb, g.cb, l, b0, b1, N, &up);
      x[l] = g.active ? rho[idx] : make_float2(0.f, 0.f);
    }
  };

  unsigned long long u = blockIdx.x;
  Group gn{};
  float2 xn[D];
  if (u < n_units) {
    gn = group_of(u);
    load(gn, xn);
  }
  uint32_t phase = 0;
#pragma unroll 1
  for (; u < n_units; u += gridDim.x, phase ^= 1u) {
    const Group g = gn;
    float2 x[D];
#pragma unroll
    for (int l = 0; l < D; ++l) x[l] = xn[l];
    if (u + gridDim.x < n_units) {
      gn = group_of(u + gridDim.x);
      load(gn, xn);
    }
    store_row(x, g.rb, g.cb, b0, b1, N, a_row, kATermBytes);
    fence_operands();
    fence_before_sync();
    __syncthreads();
    if (*s_abort) break;
    if (tid == 0 && !skip_mma) {
      fence_after_sync();
      mma_split3(tmem, sbase + kOffA, kATermBytes, sbase + kOffB, kBTermBytes);
      commit(bar);
    }
    const bool waited = bar_wait(bar, phase, max_tries);
    if (!waited) {
      atomicAdd(&g_tc_timeouts, 1u);
      *s_abort = 1;  // every thread leaves at the next unit's barrier
    }
    // a warp reads the accumulator (tcgen05.ld is warp-collective) only if
    // every lane saw the MMAs complete; otherwise rho keeps this unit's old
    // entries and the timeout is reported by the next readout
    if (!__all_sync(0xffffffffu, waited)) continue;
    fence_after_sync();
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      float dv[16];
      tmem_ld16(t_row + hh * 16, dv);
      if (!g.active) continue;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int o = hh * 8 + q;
        bool up;
        const unsigned int idx = entry_index(g.rb, g.cb, o, b0, b1, N, &up);
        float2 y = make_float2(x[o].x + dv[2 * q], x[o].y + dv[2 * q + 1]);
        if (up) {
          rho[idx] = y;
        } else if (!g.self) {  // a self-conjugate group writes its upper entries only
          y.y = -y.y;
          rho[idx] = y;
        }
      }
    }
    fence_before_sync();
  }
  __syncthreads();
  // after a timeout the unit's MMAs may still be in flight: wait for them
  // (bounded) before the tensor memory is released; the parity was toggled
  // once more after the unit that timed out (in the last unit too)
  if (*s_abort && tid == 0) bar_wait(bar, phase ^ 1u, max_tries);
  __syncthreads();
  if (w == 0) {
    fence_after_sync();
    tmem_free(tmem, kTmemCols);
  }
}

// Batched form of the pass: one fusion round of many independent split
// states (the batch engine's split tile jobs), from a table of (state,
// block) jobs whose units are numbered one after another. Each CTA takes a
// contiguous range of units; where the range crosses into the next job it
// switches to that job's index tables, rebuilds the B operand (the previous
// unit's MMAs completed before any thread left its wait, and the epilogue
// does not read B) and loads the job's first unit without prefetch. The
// per-unit work is the single-state pass's.
__global__ void __launch_bounds__(kThreads, kCtasPerSm) k_batch_tc2(const TcJob* __restrict__ jobs, int n_jobs,
                                                                      unsigned long long n_units_total,
                                                                      unsigned long long chunk, long long max_tries,
                                                                      int skip_mma) {
  constexpr int D = 16;
  extern __shared__ __align__(1024) unsigned char smem[];
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t bar = sbase + kOffBar;
  volatile uint32_t* s_tmem = reinterpret_cast<volatile uint32_t*>(smem + kOffTmem);
  volatile int* s_abort = reinterpret_cast<volatile int*>(smem + kOffFlag);
  const int tid = threadIdx.x, lane = tid % 32, w = tid / 32;
  if (tid == 0) {
    bar_init(bar, 1);
    *s_abort = 0;
  }
  if (w == 0) tmem_alloc(sbase + kOffTmem, kTmemCols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *s_tmem;
  const int i = (lane % 8) + 8 * (w % 2), j0 = (lane / 8) + 4 * (w / 2);
  const uint32_t a_row = sbase + kOffA + core_off(tid, 0);
  const uint32_t t_row = tmem + ((uint32_t)(32 * w) << 16);

  // the current job's tables
  int jn = 0;
  float2* rho = nullptr;
  unsigned int b0 = 0, b1 = 0, N = 0, di = 0, dj0 = 0, dj1 = 0;
  int qs[2] = {0, 0};
  unsigned long long ubase = 0;
  auto set_job = [&](unsigned long long uu) {
    while (jn + 1 < n_jobs && jobs[jn + 1].unit0 <= uu) ++jn;
    const TcJob& J = jobs[jn];
    rho = J.rho;
    qs[0] = min(J.p.q[0], J.p.q[1]);
    qs[1] = max(J.p.q[0], J.p.q[1]);
    b0 = 1u << J.p.q[0];
    b1 = 1u << J.p.q[1];
    N = 1u << J.p.n;
    di = (unsigned int)deposit_zeros(i, qs, 2);
    dj0 = (unsigned int)deposit_zeros(j0, qs, 2);
    dj1 = (unsigned int)deposit_zeros(j0 + 8, qs, 2);
    ubase = J.unit0;
  };
  auto same_job = [&](unsigned long long uu) { return jn + 1 >= n_jobs || jobs[jn + 1].unit0 > uu; };
  auto group_of = [&](unsigned long long uu) {
    const unsigned long long v = uu - ubase;
    bool diag = false;
    const unsigned long long tt = canonical_group(v >> 1, 32, &diag);
    const int j = (int)(v & 1ull) * 8 + j0;
    Group g;
    g.active = !(diag && i > j);
    g.self = diag && i == j;
    g.rb = (unsigned int)deposit_zeros((tt & 0xffffffffull) * kTile, qs, 2) + di;
    g.cb = (unsigned int)deposit_zeros((tt >> 32) * kTile, qs, 2) + ((v & 1ull) ? dj1 : dj0);
    return g;
  };
  auto load = [&](const Group& g, float2 x[D]) {
#pragma unroll
    for (int l = 0; l < D; ++l) {
      bool up;
      const unsigned int idx = entry_index(g.rb, g.cb, l, b0, b1, N, &up);
      x[l] = g.active ? rho[idx] : make_float2(0.f, 0.f);
    }
  };

  unsigned long long u = (unsigned long long)blockIdx.x * chunk;
  const unsigned long long u_end = min(u + chunk, n_units_total);
  Group gn{};
  float2 xn[D];
  bool have = false;
  uint32_t phase = 0;
#pragma unroll 1
  for (; u < u_end; ++u, phase ^= 1u) {
    if (!have) {  // first unit, or the first unit of the next job
      set_job(u);
      build_b(smem + kOffB, jobs[jn].S, tid, kThreads, jobs[jn].embed);
      gn = group_of(u);
      load(gn, xn);
    }
    const Group g = gn;
    float2 x[D];
#pragma unroll
    for (int l = 0; l < D; ++l) x[l] = xn[l];
    have = u + 1 < u_end && same_job(u + 1);
    if (have) {
      gn = group_of(u + 1);
      load(gn, xn);
    }
    store_row(x, g.rb, g.cb, b0, b1, N, a_row, kATermBytes);
    fence_operands();
    fence_before_sync();
    __syncthreads();
    if (*s_abort) break;
    if (tid == 0 && !skip_mma) {
      fence_after_sync();
      mma_split3(tmem, sbase + kOffA, kATermBytes, sbase + kOffB, kBTermBytes);
      commit(bar);
    }
    const bool waited = bar_wait(bar, phase, max_tries);
    if (!waited) {
      atomicAdd(&g_tc_timeouts, 1u);
      *s_abort = 1;
    }
    if (!__all_sync(0xffffffffu, waited)) continue;
    fence_after_sync();
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      float dv[16];
      tmem_ld16(t_row + hh * 16, dv);
      if (!g.active) continue;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int o = hh * 8 + q;
        bool up;
        const unsigned int idx = entry_index(g.rb, g.cb, o, b0, b1, N, &up);
        float2 y = make_float2(x[o].x + dv[2 * q], x[o].y + dv[2 * q + 1]);
        if (up) {
          rho[idx] = y;
        } else if (!g.self) {
          y.y = -y.y;
          rho[idx] = y;
        }
      }
    }
    fence_before_sync();
  }
  __syncthreads();
  if (*s_abort && tid == 0) bar_wait(bar, phase ^ 1u, max_tries);
  __syncthreads();
  if (w == 0) {
    fence_after_sync();
    tmem_free(tmem, kTmemCols);
  }
}

}  // namespace

cudaError_t launch_herm_tc2(float2* rho, const float2* S, const ApplyParams& p, int num_sms, cudaStream_t st) {
  const unsigned long long M = 1ull << (p.n - 2);
  if (p.width != 2 || M < kTile) return cudaErrorInvalidValue;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [&] {
    attr = cudaFuncSetAttribute(k_apply_herm_tc2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  });
  if (attr != cudaSuccess) return attr;
  // persistent grid: kCtasPerSm resident CTAs per SM (registers, shared
  // memory and tensor-memory columns all allow it)
  const unsigned long long Mt = M / kTile, n_units = Mt * (Mt + 1);
  const int grid = (int)std::max<unsigned long long>(
      1, std::min<unsigned long long>(n_units, (unsigned long long)num_sms * kCtasPerSm));
  k_apply_herm_tc2<<<grid, kThreads, kSmemBytes, st>>>(rho, S, p, g_test_max_tries.load(), g_test_skip_mma.load());
  return cudaGetLastError();
}

unsigned long long tc_units(int n) {
  const unsigned long long Mt = (1ull << (n - 2)) / kTile;
  return Mt * (Mt + 1);
}

bool tc_job(float2* rho, const float2* S, const ApplyParams& p, TcJob* out) {
  if ((p.width != 1 && p.width != 2) || p.n - 2 < 4) return false;
  TcJob j{};
  j.rho = rho;
  j.S = S;
  j.p = p;
  if (p.width == 1) {  // S (x) I on (q, q'), q' the highest other qubit
    j.embed = 1;
    j.p.width = 2;
    j.p.q[1] = p.q[0] == p.n - 1 ? p.n - 2 : p.n - 1;
  }
  *out = j;
  return true;
}

cudaError_t launch_batch_tc(const TcJob* jobs, int n_jobs, unsigned long long n_units, int num_sms,
                            cudaStream_t st) {
  if (n_jobs <= 0 || n_units == 0) return cudaSuccess;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [&] {
    attr = cudaFuncSetAttribute(k_batch_tc2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  });
  if (attr != cudaSuccess) return attr;
  const unsigned long long slots = (unsigned long long)num_sms * kCtasPerSm;
  const unsigned long long chunk = (n_units + slots - 1) / slots;
  const int grid = (int)((n_units + chunk - 1) / chunk);
  k_batch_tc2<<<grid, kThreads, kSmemBytes, st>>>(jobs, n_jobs, n_units, chunk, g_test_max_tries.load(),
                                                  g_test_skip_mma.load());
  return cudaGetLastError();
}

void tc_test_limits(long long* max_tries, int* skip_mma) {
  *max_tries = g_test_max_tries.load();
  *skip_mma = g_test_skip_mma.load();
}

cudaError_t tc_take_timeouts(unsigned int* count, cudaStream_t st) {
  unsigned int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(count, g_tc_timeouts, sizeof(unsigned int), 0, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && *count) {
    e = cudaMemcpyToSymbolAsync(g_tc_timeouts, &zero, sizeof(unsigned int), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  return e;
}

}  // namespace tq

extern "C" tq_status tq_test_tc_wait_limit(long long max_tries, int skip_mma) {
  if (max_tries < 0) return TQ_ERR_ARG;
  tq::g_test_max_tries.store(max_tries == 0 ? tq::kMaxSpin : max_tries);
  tq::g_test_skip_mma.store(skip_mma ? 1 : 0);
  return TQ_OK;
}
