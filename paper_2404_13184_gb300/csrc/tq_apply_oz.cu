// FP64-accurate width-2 apply pass on the 5th-generation tensor cores
// (tcgen05, sm_103a), Hermitian mode, for single FP64 states: the product
// y = S x of every canonical group (TANQ-Sim Sec. 3.1, the C2 update; the
// paper maps it onto FP64 tensor cores in Sec. 3.2) computed from exact
// integer products on the 16-bit tensor-core path (kind::f16 with FP16
// operands), in the manner of the Ozaki-Ogita-Oishi error-free splitting of
// a dot product.
//
// Real-ified product (as in tq_tc.cuh, without taking out the identity):
// Y[m][n] = sum_k X[m][k] R[n][k], with m one of 128 groups, k one of the
// 32 real inputs (Re, Im of the 16 entries, interleaved) and n one of the 32
// real outputs.
//
// Fixed-point slicing. Every operand value is cut into seven balanced 8-bit
// digits of a fixed-point number aligned to a shared exponent: for group m
// the largest biased exponent E_m of its 32 values, for output row n of R
// the largest biased exponent G_n of the row (both at least 64: a group or
// row whose largest entry is below 2^-959, or is zero, is aligned to 2^-959). With F the value's 53-bit
// significand shifted to that alignment and rounded to nearest (54 bits,
// F < 2^54),
//     |v| ~ F * 2^(E - 1076),   F = sum_i d_i 2^(8 (6 - i)),  -128 <= d_i < 128,
// where the balanced digits come from the bytes of F + 0x0080808080808080
// minus 128 (the added 128s carry exactly where a byte is >= 128; the top
// byte stays below 192, so nothing is lost). A digit is an integer, exact in
// FP16, and enters the tensor cores as such (the value's sign applied to
// all its digits; a conjugated entry's imaginary sign flipped there too, so
// no FP64 instruction touches the operands). Then
//     Y[m][n] ~ 2^(E_m + G_n - 2152) sum_t 2^(8 (12 - t)) P_t,
//     P_t = sum_{i + j = t} sum_k A_i[m][k] B_j[n][k],
// P_t an integer with |P_t| <= 7 * 32 * 128^2 < 2^22: every partial sum is
// an integer below 2^22, so FP32 accumulation in tensor memory is EXACT for
// each order. Orders 0..7 have an accumulator of 32 columns each; orders
// >= 8 (~2^-53 of order 0) are dropped. The B operand holds the digit slabs
// B_0..B_6, and a zero slab B_7, one after another along N, so ONE MMA of A
// digit i against B_0..B_(7-i) (N = 32 (8 - i); digit 0 against all eight,
// which also clears block 7) adds the products of every order i + j to the
// consecutive accumulator blocks i..7: 7 MMAs per K-half.
//
// Recombination without FP64 arithmetic: each accumulator of orders 0..5
// becomes its integer by one FP32 add of 1.5 * 2^23 (the float's low
// mantissa bits then hold P_t); orders 6 and 7 are rounded to units of 2^8
// and 2^16 the same way. The integers are combined into one 64-bit integer
// Z = sum_t P_t 2^(8 (5 - t)) (|Z| < 2^60) with wide integer multiply-adds,
// and Z is converted to FP64 with integer operations only (leading-zero
// count, shift, round to nearest with ties away from zero, exponent placed
// directly): Y = Z * 2^(E_m + G_n - 2096), no FP64 instruction at all. The
// result is FP64-accurate relative to the group's largest entry (rounding of
// the operands at 2^-55 of their alignment, ~2^-53 from the dropped orders
// and the rounding of orders 6 and 7, one final rounding).
//
// Work unit, group walk and Hermitian bookkeeping follow the split
// tensor-core kernel (tq_apply_tc.cu): half of a 16 x 16 tile of canonical
// groups (128 groups), with two threads per group in a CTA of 256 threads,
// each taking 8 of the group's 16 entries and 8 of its 16 outputs. Per unit
// a thread issues the loads of its next group half into registers, slices
// its current half into the seven digit operands (A_0..A_6, 8 KB each in
// shared memory), and after a CTA barrier one thread issues the 14 MMAs (7
// A digits x two K-halves, M = 128, N = 32 (8 - i), K = 16) into the 8
// accumulators of 32 tensor-memory columns and commits them to an mbarrier;
// every thread waits (bounded), reads its part of its row of the
// accumulators and writes its 8 outputs.
//
// Width-1 blocks run through the same kernel as a width-2 block with the
// identity on a second qubit (S (x) I, built while slicing R), which moves
// the same number of bytes as a width-1 Hermitian pass.
//
// k_batch_oz2 is the same pass over one fusion round of many states (the
// batch engine's FP64 tile jobs), from a job table (tq_batched.cuh).
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

// MMA-completion waits of this kernel that gave up; read and cleared by
// oz_take_timeouts().
__device__ unsigned int g_oz_timeouts;

constexpr int kThreads = 256;  // two threads per group of a 128-group unit
constexpr int kTile = 16;
constexpr int kDigits = 7;                          // balanced 8-bit digits per operand value
constexpr int kAccs = 8;                            // one accumulator per order 0..7
constexpr uint32_t kADigitBytes = 128 * kRowBytes;  // 128 groups x 32 FP16
constexpr uint32_t kOffA = 0;
constexpr uint32_t kOffB = kOffA + kDigits * kADigitBytes;
constexpr uint32_t kOffG = kOffB + (kDigits + 1) * kBTermBytes;  // (+ the zero slab B_7) 32 row exponents
constexpr uint32_t kOffE = kOffG + 32 * 4;                // 2 x 128 half maxima
constexpr uint32_t kOffBar = kOffE + 256 * 4;
constexpr uint32_t kOffTmem = kOffBar + 8;
constexpr uint32_t kOffFlag = kOffTmem + 4;
constexpr uint32_t kSmemBytes = kOffFlag + 4;
constexpr uint32_t kTmemCols = 256;
constexpr int kCtasPerSm = 2;

// F + 0x0080808080808080 for v's significand aligned to biased exponent E
// (E >= v's exponent and E >= 64): with M2 the 53-bit significand (implicit
// bit set) times 4 and sh = E - e_v, T = M2 >> sh = floor(M / 2^(sh - 1))
// (PTX clamps shift amounts above 64, giving 0), and F = (T + 1) >> 1 is
// M / 2^sh rounded to nearest with ties away from zero (F < 2^54); the
// offset goes in before the last shift (2 * offset + 1 = 0x0101010101010101).
// Zeros and subnormals (exponent field 0) have sh >= 64 and give F = 0.
// Byte 6 - i of the result, minus 128, is digit i.
__device__ __forceinline__ unsigned long long aligned_offset(uint32_t hi, uint32_t lo, int E) {
  const uint32_t sh = (uint32_t)(E - (int)((hi >> 20) & 0x7ffu));
  const unsigned long long M2 = (((unsigned long long)((hi & 0xfffffu) | 0x100000u) << 32) | lo) << 2;
  unsigned long long T;
  asm("shr.b64 %0, %1, %2;" : "=l"(T) : "l"(M2), "r"(sh));
  return (T + 0x0101010101010101ull) >> 1;
}

__device__ __forceinline__ uint32_t abs_hi(double v) { return (uint32_t)__double2hiint(v) & 0x7fffffffu; }

// FP16x2 word of digit I of a complex entry (low half: Re, high half: Im):
// the two digit bytes are placed in the low mantissa bytes of FP16 1024
// (0x6400), so each half reads 1024 + byte; one FP16 multiply-add by the
// half's sign s (+-1) and -1152 s leaves s (byte - 128) exactly (every
// intermediate is an integer below 2^11).
template <int I>
__device__ __forceinline__ uint32_t digit_pair(unsigned long long fr, unsigned long long fi, uint32_t sgn,
                                               uint32_t nsg) {
  constexpr int k = 6 - I;  // byte of F + offset
  const uint32_t r = k >= 4 ? (uint32_t)(fr >> 32) : (uint32_t)fr;
  const uint32_t i = k >= 4 ? (uint32_t)(fi >> 32) : (uint32_t)fi;
  const uint32_t w = (__byte_perm(r, i, (uint32_t)((k % 4) | ((4 + k % 4) << 8))) & 0x00ff00ffu) | 0x64006400u;
  uint32_t d;
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(w), "r"(sgn), "r"(nsg));
  return d;
}

// The same for two digits of one 32-bit word at once: one byte permute
// gathers (Re, Im) of bytes ka and kb, one more per digit places them under
// the FP16 1024 pattern.
__device__ __forceinline__ void digit_pair2(uint32_t r, uint32_t i, int ka, int kb, uint32_t sgn, uint32_t nsg,
                                            uint32_t& da, uint32_t& db) {
  const uint32_t w = __byte_perm(r, i, (uint32_t)(ka | ((4 + ka) << 4) | (kb << 8) | ((4 + kb) << 12)));
  const uint32_t wa = __byte_perm(w, 0x64646464u, 0x5140u), wb = __byte_perm(w, 0x64646464u, 0x5342u);
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(da) : "r"(wa), "r"(sgn), "r"(nsg));
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(db) : "r"(wb), "r"(sgn), "r"(nsg));
}

// Stores the digit words of 4 consecutive complex entries (one 16-byte chunk
// of every digit operand's row); bit e of conj: entry e is conjugated (its
// imaginary sign flipped in the digits).
__device__ __forceinline__ void store_chunk(const double2 x[4], uint32_t conj, int E, uint32_t row_chunk,
                                            uint32_t digit_bytes) {
  uint32_t w[kDigits][4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const uint32_t rh = (uint32_t)__double2hiint(x[e].x), rl = (uint32_t)__double2loint(x[e].x);
    const uint32_t ih = (uint32_t)__double2hiint(x[e].y), il = (uint32_t)__double2loint(x[e].y);
    const unsigned long long fr = aligned_offset(rh, rl, E), fi = aligned_offset(ih, il, E);
    // FP16 sign bits of both halves
    const uint32_t sign = ((rh & 0x80000000u) >> 16) | ((ih ^ (((conj >> e) & 1u) << 31)) & 0x80000000u);
    const uint32_t sgn = 0x3c003c00u ^ sign, nsg = 0xe480e480u ^ sign;  // FP16 +-1 and -+1152 per half
    const uint32_t rh2 = (uint32_t)(fr >> 32), ih2 = (uint32_t)(fi >> 32), rl2 = (uint32_t)fr, il2 = (uint32_t)fi;
    digit_pair2(rh2, ih2, 2, 1, sgn, nsg, w[0][e], w[1][e]);  // bytes 6, 5
    w[2][e] = digit_pair<2>(fr, fi, sgn, nsg);                // byte 4
    digit_pair2(rl2, il2, 3, 2, sgn, nsg, w[3][e], w[4][e]);  // bytes 3, 2
    digit_pair2(rl2, il2, 1, 0, sgn, nsg, w[5][e], w[6][e]);  // bytes 1, 0
  }
#pragma unroll
  for (int i = 0; i < kDigits; ++i) sts128(row_chunk + i * digit_bytes, w[i][0], w[i][1], w[i][2], w[i][3]);
}

// Entry (i, j) of the 16 x 16 superoperator the pass applies: S itself, or
// S (x) I for a width-1 block S (4 x 4) embedded on local qubit 0 (local
// index l = r0 + 2 r1 + 4 c0 + 8 c1; the identity acts on qubit 1).
__device__ __forceinline__ double2 sop_entry(const double2* S, int embed, int i, int j) {
  if (!embed) return S[i * 16 + j];
  if (((i >> 1) & 1) != ((j >> 1) & 1) || ((i >> 3) & 1) != ((j >> 3) & 1)) return make_double2(0.0, 0.0);
  const int a = (i & 1) | ((i >> 1) & 2), b = (j & 1) | ((j >> 1) & 2);
  return S[a * 4 + b];
}

// B operand: the digits of R (32 x 32 real, row n = 2 o + (0: Re, 1: Im) of
// output o, column k = 2 l + (0: Re, 1: Im) of input l) with per-row
// alignment. Thread t (128 threads) slices row n = t / 4, inputs l = 4 (t %
// 4) .. +3 (one 16-byte chunk of every digit row); s_G[n] receives G_n.
__device__ __forceinline__ void build_b_digits(unsigned char* smem, uint32_t sbase, const double2* S, int embed,
                                               int tid) {
  const int n = tid >> 2, quarter = tid & 3, o = n >> 1;
  double2 r[4];
  uint32_t mx = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const double2 s = sop_entry(S, embed, o, 4 * quarter + e);
    r[e] = (n & 1) ? make_double2(s.y, s.x) : make_double2(s.x, -s.y);  // Im y = Si xr + Sr xi; Re y = Sr xr - Si xi
    mx = max(mx, max(abs_hi(r[e].x), abs_hi(r[e].y)));
  }
  mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
  mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
  const int G = max((int)(mx >> 20), 64);
  if (quarter == 0) reinterpret_cast<int*>(smem + kOffG)[n] = G;
  store_chunk(r, 0u, G, sbase + kOffB + core_off(n, quarter), kBTermBytes);
  // the zero slab B_7: digit 0's MMA reaches it and clears accumulator block 7
  sts128(sbase + kOffB + kDigits * kBTermBytes + core_off(n, quarter), 0u, 0u, 0u, 0u);
}

// 64-bit integer multiply-add of a 32-bit word: c + a * b (unsigned, mod 2^64).
__device__ __forceinline__ unsigned long long mad_wide(uint32_t a, uint32_t b, unsigned long long c) {
  unsigned long long d;
  asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}

// FP32 bit pattern of 1.5 * 2^(23 - u): adding it to a multiple of 2^-u below
// 2^(22 - u) in magnitude leaves that multiple, in units of 2^-u, plus 2^22 in
// the low mantissa bits (exact); for u < 0 the sum is rounded to units of
// 2^-u.
__host__ __device__ constexpr uint32_t magic_bits(int u) { return ((uint32_t)(150 - u) << 23) | 0x400000u; }

// sum over the accumulators of the magic patterns at their weights (mod
// 2^64), subtracted once from the combined raw patterns
__host__ __device__ constexpr unsigned long long magic_offset() {
  return ((unsigned long long)magic_bits(0) << 40) + ((unsigned long long)magic_bits(0) << 32) +
         ((unsigned long long)magic_bits(0) << 24) + ((unsigned long long)magic_bits(0) << 16) +
         ((unsigned long long)magic_bits(0) << 8) + (unsigned long long)magic_bits(0) +
         (unsigned long long)magic_bits(-8) + (unsigned long long)magic_bits(-16);
}

// Real output from its 8 accumulator values (orders 0..7): Z = sum_t P_t
// 2^(8 (5 - t)) (orders 6 and 7 rounded) as the FP64 number Z * 2^scale
// (scale = E + G - 2096), built from Z's bits with integer operations; neg
// (0 or 2^31) flips the result's sign. The magic patterns' sum is taken out
// by starting Z at its negative (mod 2^64).
__device__ __forceinline__ double recombine(const float c[kAccs], int scale, uint32_t neg) {
  constexpr unsigned long long kZ0 = 0ull - magic_offset();
  const float m0 = __uint_as_float(magic_bits(0));
  const uint32_t b0 = __float_as_uint(c[0] + m0);
  const uint32_t b1 = __float_as_uint(c[1] + m0);
  const uint32_t b2 = __float_as_uint(c[2] + m0);
  const uint32_t b3 = __float_as_uint(c[3] + m0);
  const uint32_t b4 = __float_as_uint(c[4] + m0);
  const uint32_t b5 = __float_as_uint(c[5] + m0);
  const uint32_t b6 = __float_as_uint(c[6] + __uint_as_float(magic_bits(-8)));   // rounded to units of 2^8
  const uint32_t b7 = __float_as_uint(c[7] + __uint_as_float(magic_bits(-16)));  // rounded to units of 2^16
  // wraps mod 2^64 like the rest
  unsigned long long Z = ((unsigned long long)(b0 * 256u + b1 + (uint32_t)(kZ0 >> 32)) << 32) | (uint32_t)kZ0;
  Z = mad_wide(b2, 1u << 24, Z);
  Z = mad_wide(b3, 1u << 16, Z);
  Z = mad_wide(b4, 1u << 8, Z);
  Z = mad_wide(b5, 1u, Z);
  Z = mad_wide(b6, 1u, Z);
  Z = mad_wide(b7, 1u, Z);
  // |Z| normalised to bit 63, rounded to 53 bits (a carry into bit 53 lands
  // in the exponent field), placed under the biased exponent 1086 - lz +
  // scale; zero (lz = 64, shifted by 0) and results below the normal range
  // give 0, selected at the end without a branch
  const unsigned long long sm = (unsigned long long)((long long)Z >> 63);
  unsigned long long a = (Z ^ sm) - sm;
  const int lz = __clzll((long long)a);
  const unsigned long long an = a << (lz & 63);
  const unsigned long long mant = (an >> 11) + ((an >> 10) & 1ull);
  const int eb = 1085 - lz + scale;  // biased exponent - 1 (mant carries the leading 1)
  const unsigned long long bits = ((((sm & 0x80000000ull) ^ neg) << 32) + ((unsigned long long)eb << 52) + mant);
  return __longlong_as_double((a == 0ull || eb < 0) ? 0ll : (long long)bits);
}

struct Group {
  unsigned int rb, cb;
  bool active, self;
};

// Accumulator values of this thread's 8 real outputs n0 .. n0 + 7 (columns
// n0.. of each of the 8 accumulators), all loads issued before one wait.
__device__ __forceinline__ void load_accs(uint32_t t_row, int n0, uint32_t r[kAccs][8]) {
#pragma unroll
  for (int a = 0; a < kAccs; ++a)
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[a][0]), "=r"(r[a][1]), "=r"(r[a][2]), "=r"(r[a][3]), "=r"(r[a][4]), "=r"(r[a][5]),
                   "=r"(r[a][6]), "=r"(r[a][7])
                 : "r"(t_row + (uint32_t)(32 * a + n0))
                 : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  // the values are read only after the wait
#pragma unroll
  for (int a = 0; a < kAccs; ++a)
    asm volatile("" : "+r"(r[a][0]), "+r"(r[a][1]), "+r"(r[a][2]), "+r"(r[a][3]), "+r"(r[a][4]), "+r"(r[a][5]),
                 "+r"(r[a][6]), "+r"(r[a][7]));
}

// Two threads per group: thread tid takes group row m = tid % 128 of the unit
// (its A row and TMEM lane) and half h = tid / 128 of the group, the entries
// and outputs 8 h .. 8 h + 7 (A chunks 2 h, 2 h + 1; accumulator columns
// 16 h .. 16 h + 15). The group's alignment exponent is the larger of the two
// halves' maxima, exchanged through shared memory.
// max_tries: try_wait rounds before an MMA wait gives up; skip_mma (tests
// of the failure path only): issue neither the MMAs nor their commit.
__global__ void __launch_bounds__(kThreads, kCtasPerSm) k_apply_herm_oz2(double2* rho, const double2* __restrict__ S,
                                                                           const __grid_constant__ ApplyParams p,
                                                                           int embed, long long max_tries,
                                                                           int skip_mma) {
  constexpr int H = 8;  // entries (and complex outputs) per thread
  extern __shared__ __align__(1024) unsigned char smem[];
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t bar = sbase + kOffBar;
  volatile uint32_t* s_tmem = reinterpret_cast<volatile uint32_t*>(smem + kOffTmem);
  volatile int* s_abort = reinterpret_cast<volatile int*>(smem + kOffFlag);
  const int* s_G = reinterpret_cast<const int*>(smem + kOffG);
  uint32_t* s_E = reinterpret_cast<uint32_t*>(smem + kOffE);  // [2][128] half maxima
  const int tid = threadIdx.x, lane = tid % 32, w = tid / 32;
  const int m = tid & 127, h = tid >> 7, wq = w & 3;

  int qs[2] = {p.q[0], p.q[1]};
  if (qs[0] > qs[1]) {
    const int t = qs[0];
    qs[0] = qs[1];
    qs[1] = t;
  }
  const unsigned int b0 = 1u << p.q[0], b1 = 1u << p.q[1], N = 1u << p.n;
  const unsigned int ch1 = h ? b1 : 0u;  // column target bit of this half's entries (local bit 3)
  if (tid < 128) build_b_digits(smem, sbase, S, embed, tid);
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
  // operand descriptors of A_0 and B_0 (the shared window is below 256 KB, so
  // adding an offset >> 4 to the start-address field never carries out of it)
  const uint64_t a_desc0 = smem_desc(sbase + kOffA), b_desc0 = smem_desc(sbase + kOffB);

  // a warp quarter covers 8 row rests x 4 column rests of the half tile
  const int i = (lane % 8) + 8 * (wq % 2), j0 = (lane / 8) + 4 * (wq / 2);
  const unsigned int di = (unsigned int)deposit_zeros(i, qs, 2), dj0 = (unsigned int)deposit_zeros(j0, qs, 2),
                     dj1 = (unsigned int)deposit_zeros(j0 + 8, qs, 2);
  const uint32_t a_row = sbase + kOffA + core_off(m, 2 * h);
  const uint32_t t_row = tmem + ((uint32_t)(32 * wq) << 16);  // this warp's 32 TMEM lanes
  const unsigned long long Mt = (1ull << (p.n - 2)) / kTile;
  const unsigned long long n_units = Mt * (Mt + 1);

  auto group_of = [&](unsigned long long u) {
    bool diag = false;
    const unsigned long long tt = canonical_group(u >> 1, 32, &diag);
    const int j = (int)(u & 1ull) * 8 + j0;
    Group g;
    g.active = !(diag && i > j);
    g.self = diag && i == j;
    g.rb = (unsigned int)deposit_zeros((tt & 0xffffffffull) * kTile, qs, 2) + di;
    g.cb = (unsigned int)deposit_zeros((tt >> 32) * kTile, qs, 2) + ((u & 1ull) ? dj1 : dj0) + ch1;
    return g;
  };
  // this thread's half of the group: entries 8 h .. 8 h + 7, i.e. local
  // entries l < 8 from a column base that includes bit 3 (stored copies;
  // those read from their transposes are conjugated in the digits). A
  // group below the diagonal of a diagonal tile (not canonical) reads its
  // in-range entries too; its outputs are never written.
  auto load = [&](const Group& g, double2 x[H], uint32_t& conj) {
    conj = 0;
#pragma unroll
    for (int l = 0; l < H; ++l) {
      bool up;
      x[l] = rho[entry_index(g.rb, g.cb, l, b0, b1, N, &up)];
      conj |= (up ? 0u : 1u) << l;
    }
  };

  unsigned long long u = blockIdx.x;
  Group gn{};
  double2 xn[H];
  uint32_t conjn = 0;
  if (u < n_units) {
    gn = group_of(u);
    load(gn, xn, conjn);
  }
  uint32_t phase = 0;
#pragma unroll 1
  for (; u < n_units; u += gridDim.x, phase ^= 1u) {
    const Group g = gn;
    const uint32_t conj = conjn;
    double2 x[H];
#pragma unroll
    for (int l = 0; l < H; ++l) x[l] = xn[l];
    if (u + gridDim.x < n_units) {
      gn = group_of(u + gridDim.x);
      load(gn, xn, conjn);
    }
    uint32_t mx = 0;
#pragma unroll
    for (int l = 0; l < H; ++l) mx = max(mx, max(abs_hi(x[l].x), abs_hi(x[l].y)));
    s_E[tid] = mx;
    __syncthreads();  // both halves' maxima (and the previous unit's TMEM reads are done)
    const int E = max((int)(max(mx, s_E[tid ^ 128]) >> 20), 64);
#pragma unroll
    for (int c = 0; c < 2; ++c) store_chunk(x + 4 * c, conj >> (4 * c), E, a_row + c * 128u, kADigitBytes);
    fence_operands();
    fence_before_sync();
    __syncthreads();
    if (*s_abort) break;
    if (tid == 0 && !skip_mma) {
      fence_after_sync();
      // A digit i against the stacked B_0 .. B_(7-i) (N = 32 (8 - i); B_7 is
      // the zero slab) adds its products of orders i .. 7 to accumulator
      // blocks i .. 7; the first MMA (digit 0, N = 256) overwrites every block
#pragma unroll
      for (int ia = 0; ia < kDigits; ++ia)
#pragma unroll
        for (int kh = 0; kh < 2; ++kh)
          mma_bf16_n(tmem + (uint32_t)(32 * ia), a_desc0 + (uint64_t)((ia * kADigitBytes + kh * 256) >> 4),
                     b_desc0 + (uint64_t)((kh * 256) >> 4), idesc_m128_f16(32 * (8 - ia)),
                     (ia == 0 && kh == 0) ? 0u : 1u);
      commit(bar);
    }
    const bool waited = bar_wait(bar, phase, max_tries);
    if (!waited) {
      atomicAdd(&g_oz_timeouts, 1u);
      *s_abort = 1;  // every thread leaves at the next unit's barrier
    }
    // warp-collective accumulator reads only when every lane saw the MMAs
    // complete; otherwise rho keeps this unit's old entries and the timeout
    // is reported by the next readout
    if (!__all_sync(0xffffffffu, waited)) continue;
    fence_after_sync();
#pragma unroll 1
    for (int ch = 0; ch < 2; ++ch) {  // 8 real outputs (4 entries) per chunk
      uint32_t cv[kAccs][8];
      load_accs(t_row, 16 * h + 8 * ch, cv);
      if (!g.active) continue;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int o = H * h + 4 * ch + e;
        float cr[kAccs], ci[kAccs];
#pragma unroll
        for (int a = 0; a < kAccs; ++a) {
          cr[a] = __uint_as_float(cv[a][2 * e]);
          ci[a] = __uint_as_float(cv[a][2 * e + 1]);
        }
        bool up;
        const unsigned int idx = entry_index(g.rb, g.cb, 4 * ch + e, b0, b1, N, &up);
        double2 y;
        y.x = recombine(cr, E + s_G[2 * o] - 2096, 0u);
        y.y = recombine(ci, E + s_G[2 * o + 1] - 2096, up ? 0u : 0x80000000u);  // conjugated below the diagonal
        if (up || !g.self) rho[idx] = y;  // a self-conjugate group writes its upper entries only
      }
    }
    fence_before_sync();
  }
  __syncthreads();
  // after a timeout the unit's MMAs may still be in flight: wait for them
  // (bounded) before the tensor memory is released
  if (*s_abort && tid == 0) bar_wait(bar, phase ^ 1u, max_tries);
  __syncthreads();
  if (w == 0) {
    fence_after_sync();
    tmem_free(tmem, kTmemCols);
  }
}

// Batched form of the pass: one fusion round of many independent states
// (the batch engine's FP64 tile jobs), from a table of (state, block) jobs
// whose units are numbered one after another. Each CTA takes a contiguous
// range of units, so it crosses few job boundaries. At a boundary it
// switches to the new job's tables, loads that job's first unit without
// prefetch, and rebuilds the superoperator digits after the CTA barrier
// that follows the previous unit's epilogue (every thread is then done with
// the previous digits and row exponents). The per-unit work is the
// single-state pass's.
__global__ void __launch_bounds__(kThreads, kCtasPerSm) k_batch_oz2(const OzJob* __restrict__ jobs, int n_jobs,
                                                                      unsigned long long n_units_total,
                                                                      unsigned long long chunk, long long max_tries,
                                                                      int skip_mma) {
  constexpr int H = 8;  // entries (and complex outputs) per thread
  extern __shared__ __align__(1024) unsigned char smem[];
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t bar = sbase + kOffBar;
  volatile uint32_t* s_tmem = reinterpret_cast<volatile uint32_t*>(smem + kOffTmem);
  volatile int* s_abort = reinterpret_cast<volatile int*>(smem + kOffFlag);
  const int* s_G = reinterpret_cast<const int*>(smem + kOffG);
  uint32_t* s_E = reinterpret_cast<uint32_t*>(smem + kOffE);  // [2][128] half maxima
  const int tid = threadIdx.x, lane = tid % 32, w = tid / 32;
  const int m = tid & 127, h = tid >> 7, wq = w & 3;
  if (tid == 0) {
    bar_init(bar, 1);
    *s_abort = 0;
  }
  if (w == 0) tmem_alloc(sbase + kOffTmem, kTmemCols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *s_tmem;
  const uint64_t a_desc0 = smem_desc(sbase + kOffA), b_desc0 = smem_desc(sbase + kOffB);
  const int i = (lane % 8) + 8 * (wq % 2), j0 = (lane / 8) + 4 * (wq / 2);
  const uint32_t a_row = sbase + kOffA + core_off(m, 2 * h);
  const uint32_t t_row = tmem + ((uint32_t)(32 * wq) << 16);

  // the current job's tables
  int jn = 0;
  double2* rho = nullptr;
  unsigned int b0 = 0, b1 = 0, N = 0, ch1 = 0, di = 0, dj0 = 0, dj1 = 0;
  int qs[2] = {0, 0};
  unsigned long long ubase = 0;
  auto set_job = [&](unsigned long long uu) {
    while (jn + 1 < n_jobs && jobs[jn + 1].unit0 <= uu) ++jn;
    const OzJob& J = jobs[jn];
    rho = J.rho;
    qs[0] = min(J.p.q[0], J.p.q[1]);
    qs[1] = max(J.p.q[0], J.p.q[1]);
    b0 = 1u << J.p.q[0];
    b1 = 1u << J.p.q[1];
    N = 1u << J.p.n;
    ch1 = h ? b1 : 0u;
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
    g.cb = (unsigned int)deposit_zeros((tt >> 32) * kTile, qs, 2) + ((v & 1ull) ? dj1 : dj0) + ch1;
    return g;
  };
  auto load = [&](const Group& g, double2 x[H], uint32_t& conj) {
    conj = 0;
#pragma unroll
    for (int l = 0; l < H; ++l) {
      bool up;
      x[l] = rho[entry_index(g.rb, g.cb, l, b0, b1, N, &up)];
      conj |= (up ? 0u : 1u) << l;
    }
  };

  unsigned long long u = (unsigned long long)blockIdx.x * chunk;
  const unsigned long long u_end = min(u + chunk, n_units_total);
  Group gn{};
  double2 xn[H];
  uint32_t conjn = 0;
  bool have = false, need_b = true;
  uint32_t phase = 0;
#pragma unroll 1
  for (; u < u_end; ++u, phase ^= 1u) {
    if (!have) {  // first unit, or the first unit of the next job
      set_job(u);
      need_b = true;
      gn = group_of(u);
      load(gn, xn, conjn);
    }
    const Group g = gn;
    const uint32_t conj = conjn;
    double2 x[H];
#pragma unroll
    for (int l = 0; l < H; ++l) x[l] = xn[l];
    have = u + 1 < u_end && same_job(u + 1);
    if (have) {
      gn = group_of(u + 1);
      load(gn, xn, conjn);
    }
    uint32_t mx = 0;
#pragma unroll
    for (int l = 0; l < H; ++l) mx = max(mx, max(abs_hi(x[l].x), abs_hi(x[l].y)));
    s_E[tid] = mx;
    __syncthreads();  // both halves' maxima (and the previous unit's TMEM and s_G reads are done)
    const int E = max((int)(max(mx, s_E[tid ^ 128]) >> 20), 64);
    if (need_b) {
      if (tid < 128) build_b_digits(smem, sbase, jobs[jn].S, jobs[jn].embed, tid);
      need_b = false;
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) store_chunk(x + 4 * c, conj >> (4 * c), E, a_row + c * 128u, kADigitBytes);
    fence_operands();
    fence_before_sync();
    __syncthreads();
    if (*s_abort) break;
    if (tid == 0 && !skip_mma) {
      fence_after_sync();
#pragma unroll
      for (int ia = 0; ia < kDigits; ++ia)
#pragma unroll
        for (int kh = 0; kh < 2; ++kh)
          mma_bf16_n(tmem + (uint32_t)(32 * ia), a_desc0 + (uint64_t)((ia * kADigitBytes + kh * 256) >> 4),
                     b_desc0 + (uint64_t)((kh * 256) >> 4), idesc_m128_f16(32 * (8 - ia)),
                     (ia == 0 && kh == 0) ? 0u : 1u);
      commit(bar);
    }
    const bool waited = bar_wait(bar, phase, max_tries);
    if (!waited) {
      atomicAdd(&g_oz_timeouts, 1u);
      *s_abort = 1;
    }
    if (!__all_sync(0xffffffffu, waited)) continue;
    fence_after_sync();
#pragma unroll 1
    for (int ch = 0; ch < 2; ++ch) {
      uint32_t cv[kAccs][8];
      load_accs(t_row, 16 * h + 8 * ch, cv);
      if (!g.active) continue;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int o = H * h + 4 * ch + e;
        float cr[kAccs], ci[kAccs];
#pragma unroll
        for (int a = 0; a < kAccs; ++a) {
          cr[a] = __uint_as_float(cv[a][2 * e]);
          ci[a] = __uint_as_float(cv[a][2 * e + 1]);
        }
        bool up;
        const unsigned int idx = entry_index(g.rb, g.cb, 4 * ch + e, b0, b1, N, &up);
        double2 y;
        y.x = recombine(cr, E + s_G[2 * o] - 2096, 0u);
        y.y = recombine(ci, E + s_G[2 * o + 1] - 2096, up ? 0u : 0x80000000u);
        if (up || !g.self) rho[idx] = y;
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

bool oz_eligible(int n, int width) { return (width == 1 || width == 2) && n - 2 >= 4; }

cudaError_t launch_herm_oz(double2* rho, const double2* S, const ApplyParams& p, int num_sms, cudaStream_t st) {
  if (!oz_eligible(p.n, p.width)) return cudaErrorInvalidValue;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [&] {
    attr = cudaFuncSetAttribute(k_apply_herm_oz2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  });
  if (attr != cudaSuccess) return attr;
  ApplyParams q = p;
  int embed = 0;
  if (p.width == 1) {
    // S (x) I on (q, q'): the second qubit is the highest other qubit
    embed = 1;
    q.width = 2;
    q.q[1] = p.q[0] == p.n - 1 ? p.n - 2 : p.n - 1;
  }
  long long tries = 0;
  int skip = 0;
  tc_test_limits(&tries, &skip);
  const unsigned long long Mt = (1ull << (p.n - 2)) / kTile, n_units = Mt * (Mt + 1);
  const int grid = (int)std::max<unsigned long long>(
      1, std::min<unsigned long long>(n_units, (unsigned long long)num_sms * kCtasPerSm));
  k_apply_herm_oz2<<<grid, kThreads, kSmemBytes, st>>>(rho, S, q, embed, tries, skip);
  return cudaGetLastError();
}

unsigned long long oz_units(int n) {
  const unsigned long long Mt = (1ull << (n - 2)) / kTile;
  return Mt * (Mt + 1);
}

bool oz_job(double2* rho, const double2* S, const ApplyParams& p, OzJob* out) {
  if (!oz_eligible(p.n, p.width)) return false;
  OzJob j{};
  j.rho = rho;
  j.S = S;
  j.p = p;
  if (p.width == 1) {  // S (x) I on (q, q'), q' the highest other qubit (as launch_herm_oz)
    j.embed = 1;
    j.p.width = 2;
    j.p.q[1] = p.q[0] == p.n - 1 ? p.n - 2 : p.n - 1;
  }
  *out = j;
  return true;
}

cudaError_t launch_batch_oz(const OzJob* jobs, int n_jobs, unsigned long long n_units, int num_sms,
                            cudaStream_t st) {
  if (n_jobs <= 0 || n_units == 0) return cudaSuccess;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [&] {
    attr = cudaFuncSetAttribute(k_batch_oz2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  });
  if (attr != cudaSuccess) return attr;
  long long tries = 0;
  int skip = 0;
  tc_test_limits(&tries, &skip);
  // persistent grid, each CTA a contiguous range of units
  const unsigned long long slots = (unsigned long long)num_sms * kCtasPerSm;
  const unsigned long long chunk = (n_units + slots - 1) / slots;
  const int grid = (int)((n_units + chunk - 1) / chunk);
  k_batch_oz2<<<grid, kThreads, kSmemBytes, st>>>(jobs, n_jobs, n_units, chunk, tries, skip);
  return cudaGetLastError();
}

cudaError_t oz_take_timeouts(unsigned int* count, cudaStream_t st) {
  unsigned int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(count, g_oz_timeouts, sizeof(unsigned int), 0, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && *count) {
    e = cudaMemcpyToSymbolAsync(g_oz_timeouts, &zero, sizeof(unsigned int), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  return e;
}

}  // namespace tq
