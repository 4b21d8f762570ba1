// Split-precision width-2 apply pass on the 5th-generation tensor cores
// (tcgen05, sm_103a), Hermitian mode.
//
// The product y = S x of a width-2 block is a dense 16 x 16 complex
// matrix-vector product per group (TANQ-Sim Sec. 3.1: the C2 update; its
// tensor-core mapping is Sec. 3.2, Listing 1). Real-ified with the entries
// interleaved as (Re x_0, Im x_0, Re x_1, ...), it is a 32 x 32 real matrix R
// times a 32-vector, and over a tile of groups a small GEMM:
//
//     D[m][n] = sum_k X_m[k] (R - I)[n][k],   y_m = x_m + D[m][:]
//
// with M = 128 groups per MMA, N = 32 real outputs, K = 32 real inputs. The
// identity is taken out of R so that the tensor cores only produce the
// change of each entry; the FP32 add of x on the CUDA cores then rounds to
// nearest, and the accumulator's own rounding acts on the (smaller) change.
//
// Operands are complex64 (FP32) values split into three BF16 terms each,
// v = v0 + v1 + v2 (8 significand bits per term; the split is exact to
// ~2^-25 relative). The six products with term orders i + j <= 2 are
// accumulated in FP32 in tensor memory, smallest first; the three dropped
// products are ~2^-24 relative. This is the split FP32/BF16 scheme with
// compensation terms (Sec. 3.2 splits FP64 work over tensor cores in the
// same spirit; here the target is FP32 accuracy).
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
//     entries into the three BF16 terms and writes its row of the A operand
//     (shared memory, K-major, 8 x 16-byte core matrices, no swizzle);
//   - after the CTA barrier, one thread issues the 12 MMAs of the unit
//     (M = 128, N = 32, K = 16 each) into the CTA's 32-column tensor-memory
//     accumulator and commits them to an mbarrier;
//   - every thread waits (bounded) for the MMAs, reads its row of D, adds x
//     and stores. Groups are disjoint, so the early loads of unit t + 1
//     never see an entry that unit t writes.
// Index math is 32-bit (n <= 16, so a vec index fits): a group's rows and
// columns are rb + {0, 2^q0, 2^q1, 2^q0 + 2^q1} and cb + the same.
#include <algorithm>
#include <mutex>

#include "tq_device.cuh"

namespace tq {

namespace {

// Waits on the MMA-completion barrier that gave up (a tile's MMAs did not
// complete within the bound); read and cleared by tc_take_timeouts().
__device__ unsigned int g_tc_timeouts;

constexpr int kThreads = 128;
constexpr int kTile = 16;
constexpr uint32_t kRowBytes = 64;                  // 32 BF16 (K) per operand row
constexpr uint32_t kATermBytes = 128 * kRowBytes;   // 128 rows (M)
constexpr uint32_t kBTermBytes = 32 * kRowBytes;    // 32 output rows (N)
constexpr uint32_t kOffA = 0;
constexpr uint32_t kOffB = kOffA + 3 * kATermBytes;
constexpr uint32_t kOffBar = kOffB + 3 * kBTermBytes;
constexpr uint32_t kOffTmem = kOffBar + 8;
constexpr uint32_t kOffFlag = kOffTmem + 4;
constexpr uint32_t kSmemBytes = kOffFlag + 4;
constexpr uint32_t kTmemCols = 32;
constexpr int kCtasPerSm = 4;
constexpr long long kMaxSpin = 1ll << 22;  // try_wait rounds before a wait gives up (~seconds)

// Byte offset of 16-byte chunk `c` (K elements 8c..8c+7) of operand row `r`
// in the no-swizzle K-major layout: 8-row x 16-byte core matrices of 128
// contiguous bytes, consecutive along K 128 bytes apart (leading byte
// offset), consecutive 8-row groups 512 bytes apart (stride byte offset).
__device__ __forceinline__ uint32_t core_off(uint32_t r, uint32_t c) { return (r >> 3) * 512u + c * 128u + (r & 7u) * 16u; }

// Shared-memory matrix descriptor (tcgen05): start address >> 4 (bits
// 0-13), leading byte offset >> 4 (bits 16-29), stride byte offset >> 4
// (bits 32-45), the fixed 0b001 at bits 46-48, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(512u >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3
// at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

// Three-term BF16 split of the pair (a, b): t[0] + t[1] + t[2] = (a, b) to
// ~2^-25 relative (each remainder is exact in FP32).
__device__ __forceinline__ void split3(float a, float b, uint32_t t[3]) {
  t[0] = pack_bf16x2(a, b);
  a -= bf16_lo(t[0]);
  b -= bf16_hi(t[0]);
  t[1] = pack_bf16x2(a, b);
  a -= bf16_lo(t[1]);
  b -= bf16_hi(t[1]);
  t[2] = pack_bf16x2(a, b);
}

__device__ __forceinline__ void sts128(uint32_t saddr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(saddr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of the barrier; false if it gave up.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < kMaxSpin; ++i)
    if (bar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// This thread's group in a work unit: row and column bases (target bits
// zero), whether it is canonical, whether it is self-conjugate.
struct Group {
  unsigned int rb, cb;
  bool active, self;
};

// Vec index of local entry l of group g (the stored, row <= column, copy:
// entries below the diagonal are held by their transposes), and whether
// entry l is itself on or above the diagonal.
__device__ __forceinline__ unsigned int entry_index(const Group& g, int l, unsigned int b0, unsigned int b1,
                                                    unsigned int N, bool* up) {
  const unsigned int r = g.rb + ((l & 1) ? b0 : 0u) + ((l & 2) ? b1 : 0u);
  const unsigned int c = g.cb + ((l & 4) ? b0 : 0u) + ((l & 8) ? b1 : 0u);
  *up = r <= c;
  return *up ? c * N + r : r * N + c;
}

__global__ void __launch_bounds__(kThreads, kCtasPerSm) k_apply_herm_tc2(float2* rho, const float2* __restrict__ S,
                                                                           const __grid_constant__ ApplyParams p) {
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
  // B operand: (R - I) split into three BF16 terms; item e is the pair
  // (R[n][2l], R[n][2l + 1]) with n = e / 16, l = e % 16.
  for (int e = tid; e < 32 * 16; e += kThreads) {
    const int n = e / 16, l = e % 16, o = n / 2;
    const float2 s = S[o * D + l];
    float a, b;
    if ((n & 1) == 0) {  // Re y_o = Sr x_r - Si x_i
      a = s.x;
      b = -s.y;
    } else {             // Im y_o = Si x_r + Sr x_i
      a = s.y;
      b = s.x;
    }
    if (o == l) {
      if ((n & 1) == 0) a -= 1.0f;
      else b -= 1.0f;
    }
    uint32_t t[3];
    split3(a, b, t);
    const uint32_t off = core_off(n, l / 4) + (l % 4) * 4;
#pragma unroll
    for (int term = 0; term < 3; ++term)
      *reinterpret_cast<uint32_t*>(smem + kOffB + term * kBTermBytes + off) = t[term];
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *s_abort = 0;
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sbase + kOffTmem),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *s_tmem;

  // a warp covers 8 row rests x 4 column rests of the half tile
  const int i = (lane % 8) + 8 * (w % 2), j0 = (lane / 8) + 4 * (w / 2);
  const unsigned int di = (unsigned int)deposit_zeros(i, qs, 2), dj0 = (unsigned int)deposit_zeros(j0, qs, 2),
                     dj1 = (unsigned int)deposit_zeros(j0 + 8, qs, 2);
  const uint32_t a_row = sbase + kOffA;
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
      const unsigned int idx = entry_index(g, l, b0, b1, N, &up);
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
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      uint32_t tw[3][4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int l = 4 * c + e;
        bool up;
        (void)entry_index(g, l, b0, b1, N, &up);
        if (!up) x[l].y = -x[l].y;
        uint32_t tt[3];
        split3(x[l].x, x[l].y, tt);
#pragma unroll
        for (int term = 0; term < 3; ++term) tw[term][e] = tt[term];
      }
#pragma unroll
      for (int term = 0; term < 3; ++term)
        sts128(a_row + term * kATermBytes + core_off(tid, c), tw[term][0], tw[term][1], tw[term][2], tw[term][3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (*s_abort) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // products (A_ta, B_tb), smallest first; two K-halves of 16 each
      const int ta[6] = {2, 1, 0, 1, 0, 0}, tb[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
      for (int q = 0; q < 6; ++q)
#pragma unroll
        for (int kh = 0; kh < 2; ++kh) {
          const uint64_t ad = smem_desc(sbase + kOffA + ta[q] * kATermBytes + kh * 256);
          const uint64_t bd = smem_desc(sbase + kOffB + tb[q] * kBTermBytes + kh * 256);
          mma_bf16(tmem, ad, bd, (q | kh) ? 1u : 0u);
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                   : "memory");
    }
    if (!bar_wait(bar, phase)) {
      atomicAdd(&g_tc_timeouts, 1u);
      *s_abort = 1;  // every thread leaves at the next unit's barrier
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      float dv[16];
      tmem_ld16(t_row + hh * 16, dv);
      if (!g.active) continue;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int o = hh * 8 + q;
        bool up;
        const unsigned int idx = entry_index(g, o, b0, b1, N, &up);
        float2 y = make_float2(x[o].x + dv[2 * q], x[o].y + dv[2 * q + 1]);
        if (up) {
          rho[idx] = y;
        } else if (!g.self) {  // a self-conjugate group writes its upper entries only
          y.y = -y.y;
          rho[idx] = y;
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  // after a timeout the unit's MMAs may still be in flight: wait for them
  // (bounded) before the tensor memory is released; the parity was toggled
  // once more after the unit that timed out (in the last unit too)
  if (*s_abort && tid == 0) bar_wait(bar, phase ^ 1u);
  __syncthreads();
  if (w == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
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
  k_apply_herm_tc2<<<grid, kThreads, kSmemBytes, st>>>(rho, S, p);
  return cudaGetLastError();
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
