// tcgen05 building blocks of the tensor-core apply passes (sm_103a): the
// split-precision width-2 pass (tq_apply_tc.cu) and the FP64-accurate pass
// (tq_apply_oz.cu).
//
// The product y = S x of a width-2 block is a dense 16 x 16 complex
// matrix-vector product per group (TANQ-Sim Sec. 3.1, the C2 update; its
// tensor-core mapping is Sec. 3.2). Real-ified with the entries interleaved
// as (Re x_0, Im x_0, Re x_1, ...), it is a 32 x 32 real matrix R times a
// 32-vector, and over a set of groups (one per operand row) a small GEMM
//
//     D[m][n] = sum_k X_m[k] (R - I)[n][k],   y_m = x_m + D[m][:]
//
// with M = 128 groups per MMA, N = 32 real outputs, K = 32 real inputs
// (two MMAs of K = 16). The identity is taken out of R so that the tensor
// cores produce only the change of each entry; the FP32 add of x on the
// CUDA cores rounds to nearest, and the accumulator's rounding acts on the
// smaller change.
//
// Operands are FP32 values split into three BF16 terms, v = v0 + v1 + v2
// (8 significand bits each; the split is exact to ~2^-25 relative). The six
// products with term orders i + j <= 2 are accumulated in FP32 in tensor
// memory, smallest first; the three dropped products are ~2^-24 relative.
//
// Shared-memory operand layout (both K-major, no swizzle): a row holds 32
// BF16 (64 bytes) as four 16-byte chunks; 8-row x 16-byte core matrices are
// 128 contiguous bytes, consecutive along K 128 bytes apart (leading byte
// offset) and consecutive 8-row groups 512 bytes apart (stride byte offset).
#pragma once

#include <cstdint>

namespace tq {
namespace tc {

constexpr uint32_t kRowBytes = 64;               // 32 BF16 (K) per operand row
constexpr uint32_t kBTermBytes = 32 * kRowBytes;  // B: 32 output rows (N) per term

// Byte offset of 16-byte chunk `c` (K elements 8c..8c+7) of operand row `r`.
__device__ __forceinline__ uint32_t core_off(uint32_t r, uint32_t c) {
  return (r >> 3) * 512u + c * 128u + (r & 7u) * 16u;
}

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading
// byte offset >> 4 (bits 16-29), stride byte offset >> 4 (bits 32-45), the
// fixed 0b001 at bits 46-48, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(512u >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3
// at bits 17-22, M >> 4 at bits 24-28; M = 128, N = 32.
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

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 accumulator,
// M = 128 and N = n (a multiple of 16, 16 .. 256).
__host__ __device__ constexpr uint32_t idesc_m128(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}

// The same with FP16 A and B (type fields 0).
__host__ __device__ constexpr uint32_t idesc_m128_f16(int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}

// kind::f16 MMA with an explicit instruction descriptor: BF16 or FP16
// operands, as the descriptor says (the FP64-accurate pass uses FP16).
__device__ __forceinline__ void mma_bf16_n(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// The 12 MMAs of one set of 128 operand rows: products (A_ta, B_tb) with
// ta + tb <= 2, smallest first, two K-halves of 16 each, into the 32
// accumulator columns at d_tmem. a0 / b0: shared addresses of term 0 of A
// and B; a_term / b_term: bytes between terms.
__device__ __forceinline__ void mma_split3(uint32_t d_tmem, uint32_t a0, uint32_t a_term, uint32_t b0,
                                           uint32_t b_term) {
  const int ta[6] = {2, 1, 0, 1, 0, 0}, tb[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
  for (int q = 0; q < 6; ++q)
#pragma unroll
    for (int kh = 0; kh < 2; ++kh)
      mma_bf16(d_tmem, smem_desc(a0 + ta[q] * a_term + kh * 256), smem_desc(b0 + tb[q] * b_term + kh * 256),
               (q | kh) ? 1u : 0u);
}

__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
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
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, long long max_tries) {
  for (long long i = 0; i < max_tries; ++i)
    if (bar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One warp allocates (and the same warp later frees) `cols` tensor-memory
// columns; the base address lands in shared memory at `slot`.
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t tmem, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the tensor cores
__device__ __forceinline__ void fence_operands() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

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

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}

// Entry (o, l) of the 16 x 16 superoperator a width-2 pass applies: S, or
// S (x) I for a width-1 block S (4 x 4) embedded on local qubit 0 (local
// index l = r0 + 2 r1 + 4 c0 + 8 c1; the identity acts on qubit 1).
__device__ __forceinline__ float2 sop_entry_f(const float2* S, int embed, int o, int l) {
  if (!embed) return S[o * 16 + l];
  if (((o >> 1) & 1) != ((l >> 1) & 1) || ((o >> 3) & 1) != ((l >> 3) & 1)) return make_float2(0.f, 0.f);
  return S[((o & 1) | ((o >> 1) & 2)) * 4 + ((l & 1) | ((l >> 1) & 2))];
}

// B operand of a width-2 block: (R - I) in three BF16 terms at `b` (shared
// memory, kBTermBytes per term) from the 16 x 16 complex superoperator S
// (row-major, any memory space; embed: S is a width-1 block applied as S (x)
// I); items e = tid, tid + nthreads, ... < 512, item e being the pair
// (R[n][2l], R[n][2l + 1]) with n = e / 16, l = e % 16.
__device__ __forceinline__ void build_b(unsigned char* b, const float2* S, int tid, int nthreads, int embed = 0) {
  for (int e = tid; e < 32 * 16; e += nthreads) {
    const int n = e / 16, l = e % 16, o = n / 2;
    const float2 s = sop_entry_f(S, embed, o, l);
    float re, im;
    if ((n & 1) == 0) {  // Re y_o = Sr x_r - Si x_i
      re = s.x;
      im = -s.y;
    } else {  // Im y_o = Si x_r + Sr x_i
      re = s.y;
      im = s.x;
    }
    if (o == l) {
      if ((n & 1) == 0) re -= 1.0f;
      else im -= 1.0f;
    }
    uint32_t t[3];
    split3(re, im, t);
    const uint32_t off = core_off(n, l / 4) + (l % 4) * 4;
#pragma unroll
    for (int term = 0; term < 3; ++term) *reinterpret_cast<uint32_t*>(b + term * kBTermBytes + off) = t[term];
  }
}

// A group's rows and columns are rb + {0, 2^q0, 2^q1, 2^q0 + 2^q1} and cb +
// the same (target bits of local entry l: row bits l & 3, column bits l >> 2).
// Vec index of the stored copy of entry l (row <= column; an entry below
// the diagonal is held by its transpose) in 32 bits (n <= 16), and whether
// entry l is itself on or above the diagonal.
__device__ __forceinline__ unsigned int entry_index(unsigned int rb, unsigned int cb, int l, unsigned int b0,
                                                    unsigned int b1, unsigned int N, bool* up) {
  const unsigned int r = rb + ((l & 1) ? b0 : 0u) + ((l & 2) ? b1 : 0u);
  const unsigned int c = cb + ((l & 4) ? b0 : 0u) + ((l & 8) ? b1 : 0u);
  *up = r <= c;
  return *up ? c * N + r : r * N + c;
}

// Operand row of one group: conjugate the entries that were read from their
// transposes (x is updated in place), split, and store the 3 x 4 chunks.
__device__ __forceinline__ void store_row(float2 x[16], unsigned int rb, unsigned int cb, unsigned int b0,
                                          unsigned int b1, unsigned int N, uint32_t a_row, uint32_t a_term) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    uint32_t tw[3][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int l = 4 * c + e;
      bool up;
      (void)entry_index(rb, cb, l, b0, b1, N, &up);
      if (!up) x[l].y = -x[l].y;
      uint32_t tt[3];
      split3(x[l].x, x[l].y, tt);
#pragma unroll
      for (int term = 0; term < 3; ++term) tw[term][e] = tt[term];
    }
#pragma unroll
    for (int term = 0; term < 3; ++term) sts128(a_row + term * a_term + c * 128u, tw[term][0], tw[term][1], tw[term][2], tw[term][3]);
  }
}

}  // namespace tc
}  // namespace tq
