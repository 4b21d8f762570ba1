// Device side of batched execution, shared by the batch engine (tq_batch.cu)
// and the serving loop (tq_serve.cu).
//
// Work is a list of items in a fixed global order; CTAs take items from a
// ticket counter. An item is either a run of consecutive fused blocks of a
// job whose vec(rho) fits in shared memory ("resident": load rho once, apply
// the blocks with block-wide barriers between them, store once) or a range
// of tiles of one fused block of a larger job. A tile item of block b waits
// until the job's tile counter shows every tile of block b-1 finished.
// Items are ordered round-robin over jobs by block index, so an item only
// ever waits for items with smaller tickets, which are already held by
// running CTAs: the waits always end. Each wait is still bounded; when the
// bound runs out the kernel raises an error flag, skips the remaining work
// and returns, and the host reports TQ_ERR_TIMEOUT.
#pragma once

#include "tq_plan.cuh"

namespace tq {
namespace batch {

constexpr int kThreads = 256;
constexpr int kResidentBytes = 64 * 1024;  // vec(rho) of a resident job
constexpr int kSEntries = 256;             // superoperator cache: widths <= 2
constexpr int kMaxMasks = 16;
constexpr int kResults = 2 + kMaxMasks;    // Re tr, Im tr, masked sums

struct BJob {
  unsigned long long rho_off;  // byte offset of vec(rho) in the arena
  int n;
  int n_blocks;
  int block0;     // first block in the block table
  int tile_log2;  // entries per tile (tile jobs)
  int resident;
  int n_masks;
  int never_ready;  // test hook: this job's waits can never be satisfied
  int herm;         // Hermitian mode: canonical groups only, rows <= columns kept
  int tensor;       // FP64 tile job run by the batched tensor-core pass (not by the batch kernel)
  unsigned long long masks[kMaxMasks];
};

// Pauli-basis row lists of one width-2 block of a tile job (see the Pauli
// section below), built once per run by k_pauli_lists and copied by every
// tile item of the block when it stages the block.
struct PauliRec {
  int on;                     // the block's tile items take these lists
  int nnz;                    // nonzeros of R' kept
  unsigned short rowptr[17];  // row r's nonzeros: rowptr[r] .. rowptr[r + 1] - 1
  unsigned short pad_;
  unsigned char col[256];
  double val[256];            // FP64 jobs: the row lists' values; split jobs: R' as 256 floats,
                              // dense and transposed (entry (a, b) at b * 16 + a)
};
static_assert(sizeof(PauliRec) == 2352, "record layout");

struct BBlk {
  ApplyParams p;
  const void* S;            // fused superoperator, 4^w x 4^w row-major (double2 or float2)
  const PauliRec* pauli;    // width-2 blocks of tile jobs: their Pauli-basis lists; else null
  int tiles;                // tile items of this block (tile jobs)
  int tile_prefix;          // tiles of the job's earlier blocks: the wait target
};

struct BItem {
  int job;
  int block;   // tile item: block index (job-relative); -1: resident item
  int tile0;   // tile item: first tile; resident item: first block
  int ntiles;  // tile item: tiles; resident item: blocks
};

// -v by its sign bit: an integer operation, off the FP64 pipe that bounds
// the FP64 paths
__device__ __forceinline__ double flip_sign(double v) {
  return __hiloint2double(__double2hiint(v) ^ (int)0x80000000, __double2loint(v));
}

template <typename T2>
struct Cx;
template <>
struct Cx<double2> {
  __device__ __forceinline__ static double2 zero() { return make_double2(0.0, 0.0); }
  __device__ __forceinline__ static void fma(double2& acc, double2 a, double2 b) {
    acc.x = ::fma(a.x, b.x, acc.x);
    acc.x = ::fma(-a.y, b.y, acc.x);
    acc.y = ::fma(a.x, b.y, acc.y);
    acc.y = ::fma(a.y, b.x, acc.y);
  }
  __device__ __forceinline__ static double2 ldcg(const double2* p) { return __ldcg(p); }
};
template <>
struct Cx<float2> {
  __device__ __forceinline__ static float2 zero() { return make_float2(0.f, 0.f); }
  __device__ __forceinline__ static void fma(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
  }
  __device__ __forceinline__ static float2 ldcg(const float2* p) { return __ldcg(p); }
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Width-2 products of tile items in the Pauli basis. Every block is a
// Kraus map, so its superoperator S preserves Hermiticity, and in the basis
// of Pauli products (T: per qubit, the entries (r, c) = 00, 10, 01, 11 of
// its 2 x 2 block become I = a00 + a11, X = a01 + a10, Y = i (a01 - a10),
// Z = a00 - a11) it is a REAL 16 x 16 matrix R = T S T^dagger / 4. A
// group's 16 entries (not Hermitian themselves) are mapped by y = T^dagger
// R' T x with R' = R / 4: a real times complex product (2 multiply-adds per
// nonzero instead of 4) between two basis changes (butterflies with
// coefficients +-1, +-i, 128 adds per group). Gates of the circuits here
// (Cliffords, rotations about Pauli axes) and Pauli channels are sparse in
// this basis: the fused width-2 blocks of the 1024-circuit sweep have ~31
// nonzeros of R' against ~120 complex nonzeros of S. R' is computed in FP64
// from the FP64 superoperator; entries at most 2^-47 of its largest are
// rounding residues of structural zeros and are dropped. Slots: the Pauli
// pair (P0, P1) sits where local entry {0, 1, 4, 5}[P0] + {0, 2, 8, 10}[P1]
// sat.
constexpr double kPauliZeroRel = 7.105427357601002e-15;  // 2^-47

template <typename T2>
struct Sc;
template <>
struct Sc<float2> {
  using T = float;
  __device__ __forceinline__ static float2 mk(float a, float b) { return make_float2(a, b); }
};
template <>
struct Sc<double2> {
  using T = double;
  __device__ __forceinline__ static double2 mk(double a, double b) { return make_double2(a, b); }
};

// Butterfly of one qubit on slots b, b + s10 (r = 1), b + s01 (c = 1),
// b + s10 + s01: forward (computational -> Pauli) or inverse (T^dagger).
template <typename T2>
__device__ __forceinline__ void pauli_bfly_fwd(T2& a00, T2& a10, T2& a01, T2& a11) {
  const T2 I = Sc<T2>::mk(a00.x + a11.x, a00.y + a11.y), X = Sc<T2>::mk(a01.x + a10.x, a01.y + a10.y);
  const T2 Y = Sc<T2>::mk(a10.y - a01.y, a01.x - a10.x), Z = Sc<T2>::mk(a00.x - a11.x, a00.y - a11.y);
  a00 = I;
  a10 = X;
  a01 = Y;
  a11 = Z;
}
template <typename T2>
__device__ __forceinline__ void pauli_bfly_inv(T2& I, T2& X, T2& Y, T2& Z) {
  const T2 a00 = Sc<T2>::mk(I.x + Z.x, I.y + Z.y), a11 = Sc<T2>::mk(I.x - Z.x, I.y - Z.y);
  const T2 a10 = Sc<T2>::mk(X.x - Y.y, X.y + Y.x), a01 = Sc<T2>::mk(X.x + Y.y, X.y - Y.x);  // X + i Y, X - i Y
  I = a00;
  X = a10;
  Y = a01;
  Z = a11;
}
// slot bases of the butterflies of qubit q (t < 4) and the slot strides
__host__ __device__ __forceinline__ int pauli_base(int q, int t) { return q == 0 ? (t & 1) * 2 + (t >> 1) * 8 : (t & 1) + (t >> 1) * 4; }
template <typename T2>
__device__ __forceinline__ void pauli_fwd(T2 x[16]) {
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int b = pauli_base(q, t), s10 = q == 0 ? 1 : 2, s01 = q == 0 ? 4 : 8;
      pauli_bfly_fwd(x[b], x[b + s10], x[b + s01], x[b + s10 + s01]);
    }
}
template <typename T2>
__device__ __forceinline__ void pauli_inv(T2 x[16]) {
#pragma unroll
  for (int q = 1; q >= 0; --q)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int b = pauli_base(q, t), s10 = q == 0 ? 1 : 2, s01 = q == 0 ? 4 : 8;
      pauli_bfly_inv(x[b], x[b + s10], x[b + s01], x[b + s10 + s01]);
    }
}

// R'[sa][sb] = Re sum_{l, m} T[sa][l] S[l][m] conj(T[sb][m]) / 16 of a width-2
// superoperator S (FP64): row `slot` of T has 4 nonzeros, the products of
// the two qubits' Pauli coefficients (I: 00 -> 1, 11 -> 1; X: 01, 10 -> 1;
// Y: 01 -> i, 10 -> -i; Z: 00 -> 1, 11 -> -1).
__host__ __device__ __forceinline__ void pauli_row(int slot, int l[4], int cre[4], int cim[4]) {
  const int P[2] = {((slot & 1) ? 1 : 0) | ((slot & 4) ? 2 : 0), ((slot & 2) ? 1 : 0) | ((slot & 8) ? 2 : 0)};
  int r[2][2], c[2][2], fre[2][2], fim[2][2];
  for (int j = 0; j < 2; ++j) {
    const bool diag = P[j] == 0 || P[j] == 3;  // I, Z: entries 00 and 11; X, Y: 01 and 10
    r[j][0] = 0; c[j][0] = diag ? 0 : 1;
    r[j][1] = 1; c[j][1] = diag ? 1 : 0;
    fre[j][0] = P[j] == 2 ? 0 : 1;             fim[j][0] = P[j] == 2 ? 1 : 0;
    fre[j][1] = P[j] == 3 ? -1 : (P[j] == 2 ? 0 : 1);
    fim[j][1] = P[j] == 2 ? -1 : 0;
  }
  for (int u = 0; u < 2; ++u)
    for (int v = 0; v < 2; ++v) {
      l[2 * u + v] = r[0][u] + 2 * r[1][v] + 4 * c[0][u] + 8 * c[1][v];
      cre[2 * u + v] = fre[0][u] * fre[1][v] - fim[0][u] * fim[1][v];
      cim[2 * u + v] = fre[0][u] * fim[1][v] + fim[0][u] * fre[1][v];
    }
}
// Whether a width-2 tile-item block takes the Pauli basis. FP64: when its
// row lists cost fewer FP64 operations per group (2 per nonzero + 128 adds
// against 4 per nonzero of S's row lists). Split: always; it runs R' as a
// dense real 16 x 16 product (512 FFMA + 128 adds per group against 1,024
// FFMA for the complex S), unrolled like the dense split product (the
// row-list loop, a chain of dependent shared-memory loads per nonzero, was
// latency-bound there: 1024-circuit sweep 6,971 against 8,440 circuits/s
// for the dense complex product).
__host__ __device__ __forceinline__ bool pauli_better(int prec, int nnzS, int nnzR) {
  return prec == 0 ? 2 * nnzR + 128 < 4 * nnzS : true;
}

// One CTA of 256 threads per record: R' = T S T^dagger / 16 of the block's
// FP64 fused superoperator in two passes of additions only (T's entries are
// +-1 and +-i): U = T S (thread (a, m)), then R'[a][b] = Re sum_m U[a][m]
// conj(T[b][m]) / 16 (thread (a, b)). Entries at most 2^-47 of the largest
// are dropped; the remaining ones form the row lists (FP64 jobs) or the
// dense transposed R' rounded to FP32 (split jobs), taken when pauli_better
// says so. S's
// nonzeros are counted by bit pattern, as the FP64 staging does.
static __global__ void __launch_bounds__(256) k_pauli_lists(const double2* __restrict__ sb64,
                                                            const unsigned long long* __restrict__ sb_off, int prec,
                                                            PauliRec* __restrict__ out) {
  __shared__ double2 U[256];
  __shared__ double red[8];
  __shared__ unsigned int rowmask[16];
  const int t = threadIdx.x, a = t >> 4, mb = t & 15;
  const double2* S = sb64 + sb_off[blockIdx.x];
  PauliRec& rec = out[blockIdx.x];
  const double2 st = S[t];
  const int nnzS = __syncthreads_count(((__double_as_longlong(st.x) | __double_as_longlong(st.y)) << 1) != 0);
  int l[4], cre[4], cim[4];
  pauli_row(a, l, cre, cim);
  double ur = 0.0, ui = 0.0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    // (cre + i cim)(s.x + i s.y), one of cre, cim zero and the other +-1
    const double2 sv = S[l[u] * 16 + mb];
    const double dx = cim[u] == 0 ? sv.x : sv.y, dy = cim[u] == 0 ? sv.y : sv.x;
    const int sx = cim[u] == 0 ? cre[u] : -cim[u], sy = cim[u] == 0 ? cre[u] : cim[u];
    ur = sx > 0 ? ur + dx : ur - dx;
    ui = sy > 0 ? ui + dy : ui - dy;
  }
  U[t] = make_double2(ur, ui);
  __syncthreads();
  pauli_row(mb, l, cre, cim);  // row b = mb of T
  double r = 0.0;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    // Re (U[a][m] conj(cre + i cim)) = U.x cre + U.y cim
    const double2 uv = U[a * 16 + l[v]];
    const double d = cim[v] == 0 ? uv.x : uv.y;
    const int sg = cim[v] == 0 ? cre[v] : cim[v];
    r = sg > 0 ? r + d : r - d;
  }
  r *= 0.0625;
  double mx = fabs(r);
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((t & 31) == 0) red[t >> 5] = mx;
  __syncthreads();
  mx = red[0];
  for (int w = 1; w < 8; ++w) mx = fmax(mx, red[w]);
  const bool keep = fabs(r) > mx * kPauliZeroRel;
  const unsigned int ball = __ballot_sync(0xffffffffu, keep);
  if ((t & 15) == 0) rowmask[a] = (ball >> (t & 16)) & 0xffffu;
  __syncthreads();
  int off = 0, nnz = 0;
  for (int i = 0; i < 16; ++i) {
    const int c = __popc(rowmask[i]);
    off += i < a ? c : 0;
    nnz += c;
  }
  if (prec == 0) {
    if (keep) {
      const int k = off + __popc(rowmask[a] & ((1u << mb) - 1u));
      rec.col[k] = (unsigned char)mb;
      rec.val[k] = r;
    }
  } else {
    reinterpret_cast<float*>(rec.val)[mb * 16 + a] = keep ? (float)r : 0.f;  // dense, transposed
  }
  if (t <= 16) {
    int o = 0;
    for (int i = 0; i < t; ++i) o += __popc(rowmask[i]);
    rec.rowptr[t] = (unsigned short)o;
  }
  if (t == 0) {
    rec.nnz = nnz;
    rec.on = pauli_better(prec, nnzS, nnz) ? 1 : 0;
  }
}

inline cudaError_t launch_pauli_lists(const double2* sb64, const unsigned long long* sb_off, int n_rec, int prec,
                                      PauliRec* out, cudaStream_t st) {
  if (n_rec <= 0) return cudaSuccess;
  k_pauli_lists<<<n_rec, 256, 0, st>>>(sb64, sb_off, prec, out);
  return cudaGetLastError();
}

// One canonical group of a width-K split block on the shared-memory copy of
// rho (resident items): gather its 4^K entries, multiply by S (shared
// memory), scatter back. t indexes the canonical groups (row rest <= column
// rest); entries below the diagonal are read and written through their
// conjugate transposes, as in the single-state kernels.
template <typename T2, int K>
__device__ __forceinline__ void apply_group(T2* rho, unsigned long long t, const ApplyParams& p, const T2* sS) {
  constexpr int D = 1 << (2 * K);
  bool self = false;
  unsigned long long base = canonical_group(t, p.n - K, &self);
#pragma unroll
  for (int i = 0; i < 2 * K; ++i) {
    const unsigned long long low = base & ((1ull << p.pos[i]) - 1ull);
    base = ((base >> p.pos[i]) << (p.pos[i] + 1)) | low;
  }
  // row / column indices are 32-bit (n <= 16): r = rows of base + row part
  // of off[l], c likewise
  const unsigned int rmask = (1u << p.n) - 1u;
  const unsigned int rb = (unsigned int)(base & rmask), cb = (unsigned int)(base >> p.n);
  T2 x[D];
#pragma unroll
  for (int l = 0; l < D; ++l) {
    const unsigned int r = rb + (unsigned int)(p.off[l] & rmask), c = cb + (unsigned int)(p.off[l] >> p.n);
    const bool conj = r > c;
    T2 v = rho[conj ? ((unsigned long long)c | ((unsigned long long)r << p.n))
                    : ((unsigned long long)r | ((unsigned long long)c << p.n))];
    if (conj) v.y = -v.y;
    x[l] = v;
  }
#pragma unroll
  for (int i = 0; i < D; ++i) {
    T2 acc = Cx<T2>::zero();
#pragma unroll
    for (int j = 0; j < D; ++j) Cx<T2>::fma(acc, sS[i * D + j], x[j]);
    const unsigned int r = rb + (unsigned int)(p.off[i] & rmask), c = cb + (unsigned int)(p.off[i] >> p.n);
    if (r <= c) {
      rho[(unsigned long long)r | ((unsigned long long)c << p.n)] = acc;
    } else if (!self) {  // a self-conjugate group writes its upper entries only
      acc.y = -acc.y;
      rho[(unsigned long long)c | ((unsigned long long)r << p.n)] = acc;
    }
  }
}

// Row lists of an FP64 superoperator in shared memory: the nonzeros of row
// i are val[k], column col[k], for k in [rowptr[i], rowptr[i+1]). FP64
// applies are bound by the FP64 pipe, so only nonzero products are issued;
// the loops run over these lists (a data-dependent trip count, so the
// compiler cannot turn skipped products into predicated ones), and the
// result is that of the dense product (an FMA with a zero product is exact).
struct RowLists {
  int rowptr[17];
  unsigned int mask[16];  // staging: nonzero columns of each row
  unsigned char col[kSEntries];
};
static_assert(16 * kThreads * 16 <= kResidentBytes, "operand columns of a width-2 FP64 tile item");

// Split tile items in Hermitian mode walk the canonical groups in 16 x 16
// tiles of (row rest a, column rest b), one group per thread: thread (i, j)
// takes a = 16 ta + i, b = 16 tb + j. Rows are dep(16 ta) + dep16[i] + rt[l]
// (dep inserts zeros at the target qubits and is additive over disjoint
// bits), columns likewise; a warp covers 8 consecutive a by 4 consecutive
// b, so entries above the diagonal are read and written 8 rows at a time
// and transposed entries below it 4 columns (one 32-byte sector) at a time.
struct Tile16 {
  unsigned dep16[16];
  unsigned rt[16], ct[16];  // row / column target bits of local index l
  int qs[2];                // target qubits ascending
};
static_assert(kThreads == 256, "one 16 x 16 tile of groups per CTA pass");

// Canonical 16 x 16 tiles per work item of a split Hermitian tile job: the
// same entries per item as 2^(tile_log2 - 2w) groups (a tile holds 2^8).
__host__ __device__ inline int tiles16_log2(int tile_log2, int width) {
  const int v = tile_log2 - 2 * width - 8;
  return v > 0 ? v : 0;
}


// FP64 tile items: gather the group's 4^K entries (through L2: other CTAs
// wrote them) into this thread's shared-memory column mine[l * kThreads],
// then each output is a row-list dot product, written back in place.
template <int K, bool HERM>
__device__ __forceinline__ void apply_group_lists_global(double2* rho, unsigned long long t, const ApplyParams& p,
                                                         const double2* val, const RowLists& rl, double2* mine) {
  constexpr int D = 1 << (2 * K);
  bool self = false;
  unsigned long long base = HERM ? canonical_group(t, p.n - K, &self) : t;
#pragma unroll
  for (int i = 0; i < 2 * K; ++i) {
    const unsigned long long low = base & ((1ull << p.pos[i]) - 1ull);
    base = ((base >> p.pos[i]) << (p.pos[i] + 1)) | low;
  }
  const unsigned int rmask = (1u << p.n) - 1u;
  const unsigned int rb = (unsigned int)(base & rmask), cb = (unsigned int)(base >> p.n);
#pragma unroll
  for (int l = 0; l < D; ++l) {
    unsigned long long e;
    bool conj = false;
    if (HERM) {
      const unsigned int r = rb + (unsigned int)(p.off[l] & rmask), c = cb + (unsigned int)(p.off[l] >> p.n);
      conj = r > c;
      e = conj ? ((unsigned long long)c | ((unsigned long long)r << p.n)) : ((unsigned long long)r | ((unsigned long long)c << p.n));
    } else {
      e = base + p.off[l];
    }
    double2 v = __ldcg(&rho[e]);
    if (conj) v.y = flip_sign(v.y);
    mine[l * kThreads] = v;
  }
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double2 acc = make_double2(0.0, 0.0);
    for (int k = rl.rowptr[i]; k < rl.rowptr[i + 1]; ++k) Cx<double2>::fma(acc, val[k], mine[rl.col[k] * kThreads]);
    if (HERM) {
      const unsigned int r = rb + (unsigned int)(p.off[i] & rmask), c = cb + (unsigned int)(p.off[i] >> p.n);
      if (r <= c) {
        rho[(unsigned long long)r | ((unsigned long long)c << p.n)] = acc;
      } else if (!self) {
        acc.y = flip_sign(acc.y);
        rho[(unsigned long long)c | ((unsigned long long)r << p.n)] = acc;
      }
    } else {
      rho[base + p.off[i]] = acc;
    }
  }
}

// FP64 resident items: the operands are read from the shared-memory copy of
// rho as the row lists name them; all 4^K outputs stay in registers until
// the group's last read, then are stored (groups are disjoint, so no other
// thread touches these entries).
template <int K, bool HERM>
__device__ __forceinline__ void apply_group_lists_resident(double2* sR, unsigned int t, const ApplyParams& p,
                                                           const double2* val, const RowLists& rl) {
  constexpr int D = 1 << (2 * K);
  bool self = false;
  unsigned int base = HERM ? (unsigned int)canonical_group(t, p.n - K, &self) : t;
#pragma unroll
  for (int i = 0; i < 2 * K; ++i) {
    const unsigned int low = base & ((1u << p.pos[i]) - 1u);
    base = ((base >> p.pos[i]) << (p.pos[i] + 1)) | low;
  }
  const unsigned int rmask = (1u << p.n) - 1u;
  const unsigned int rb = base & rmask, cb = base >> p.n;
  double2 out[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double2 acc = make_double2(0.0, 0.0);
    for (int k = rl.rowptr[i]; k < rl.rowptr[i + 1]; ++k) {
      const unsigned int off = (unsigned int)p.off[rl.col[k]];
      double2 v;
      if (HERM) {
        const unsigned int r = rb + (off & rmask), c = cb + (off >> p.n);
        v = sR[r <= c ? (r | (c << p.n)) : (c | (r << p.n))];
        if (r > c) v.y = flip_sign(v.y);
      } else {
        v = sR[base + off];
      }
      Cx<double2>::fma(acc, val[k], v);
    }
    out[i] = acc;
  }
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double2 acc = out[i];
    const unsigned int off = (unsigned int)p.off[i];
    if (HERM) {
      const unsigned int r = rb + (off & rmask), c = cb + (off >> p.n);
      if (r <= c) {
        sR[r | (c << p.n)] = acc;
      } else if (!self) {
        acc.y = flip_sign(acc.y);
        sR[c | (r << p.n)] = acc;
      }
    } else {
      sR[base + off] = acc;
    }
  }
}

// One canonical 16 x 16 tile u of a width-K split block (see Tile16).
template <int K>
__device__ __forceinline__ void apply_tile16(float2* rho, unsigned long long u, const ApplyParams& p,
                                             const float2* sS, const Tile16& t) {
  constexpr int D = 1 << (2 * K);
  // a warp covers 8 row rests x 4 column rests (full 32-byte sectors in both
  // orientations)
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
  const int i = (lane % 8) + 8 * (w % 2), j = (lane / 8) + 4 * (w / 2);
  bool diag = false;
  const unsigned long long tt = canonical_group(u, 32, &diag);  // (ta, tb) as ta | tb << 32
  if (diag && i > j) return;  // not a canonical group
  const bool self = diag && i == j;
  const unsigned rbase = (unsigned)deposit_zeros((tt & 0xffffffffull) * 16, t.qs, K) + t.dep16[i];
  const unsigned cbase = (unsigned)deposit_zeros((tt >> 32) * 16, t.qs, K) + t.dep16[j];
  float2 x[D];
#pragma unroll
  for (int l = 0; l < D; ++l) {
    const unsigned r = rbase + t.rt[l], c = cbase + t.ct[l];
    const bool up = r <= c;
    float2 v = __ldcg(&rho[up ? ((unsigned long long)r | ((unsigned long long)c << p.n))
                              : ((unsigned long long)c | ((unsigned long long)r << p.n))]);
    if (!up) v.y = -v.y;
    x[l] = v;
  }
#pragma unroll
  for (int o = 0; o < D; ++o) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int l = 0; l < D; ++l) Cx<float2>::fma(acc, sS[o * D + l], x[l]);
    const unsigned r = rbase + t.rt[o], c = cbase + t.ct[o];
    if (r <= c) {
      rho[(unsigned long long)r | ((unsigned long long)c << p.n)] = acc;
    } else if (!self) {  // a self-conjugate group writes its upper entries only
      acc.y = -acc.y;
      rho[(unsigned long long)c | ((unsigned long long)r << p.n)] = acc;
    }
  }
}

// A cache-global load of one split entry that has L2 fetch 256-byte blocks
// (the PTX prefetch-size qualifier). A tile's reads in one column of rho are
// 128-byte runs, and the neighbouring canonical tile, usually in flight in
// another CTA, reads the other half of the block: 11,465 against 11,406
// circuits/s on the 1024-circuit split sweep, with bitwise-equal results
// (11,525 with the streaming stores of the tile walk below).
__device__ __forceinline__ float2 ld_cg_l2_256(const float2* a) {
  float2 v;
  asm volatile("ld.global.cg.L2::256B.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(a));
  return v;
}

// The same tile walk for a width-2 block in the Pauli basis, over tiles u0 ..
// u1 - 1: a group's entries are transformed in registers, multiplied by R'
// (dense real 16 x 16, stored transposed in shared memory so that column b
// is one run of 16 floats read by warp-uniform broadcast), transformed back
// and stored. The product runs column by column, and each column's register
// pair, once consumed, receives the next tile's entry of the same index: the
// next tile's loads are in flight during this tile's 512 FFMA. Tiles hold
// disjoint canonical groups, so no load of tile u + 1 sees a store of tile u.
__device__ __forceinline__ void apply_tiles16_pauli(float2* rho, unsigned long long u0, unsigned long long u1,
                                                    const ApplyParams& p, const float* Rt, const Tile16& t) {
  constexpr int D = 16;
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
  const int i = (lane % 8) + 8 * (w % 2), j = (lane / 8) + 4 * (w / 2);
  // this thread's group in tile u: row / column bases; canonical (active);
  // self-conjugate
  auto group = [&](unsigned long long u, unsigned& rb, unsigned& cb, bool& act, bool& self) {
    bool diag = false;
    const unsigned long long tt = canonical_group(u, 32, &diag);
    act = !(diag && i > j);
    self = diag && i == j;
    rb = (unsigned)deposit_zeros((tt & 0xffffffffull) * 16, t.qs, 2) + t.dep16[i];
    cb = (unsigned)deposit_zeros((tt >> 32) * 16, t.qs, 2) + t.dep16[j];
  };
  // stored location of entry l (upper triangle; up: read as is)
  auto where = [&](unsigned rb, unsigned cb, int l, bool& up) {
    const unsigned r = rb + t.rt[l], c = cb + t.ct[l];
    up = r <= c;
    return up ? ((unsigned long long)r | ((unsigned long long)c << p.n)) : ((unsigned long long)c | ((unsigned long long)r << p.n));
  };
  if (u0 >= u1) return;
  unsigned rb, cb;
  bool act, self;
  group(u0, rb, cb, act, self);
  float2 x[D];
  unsigned upm = 0;  // bit l: entry l read as is (else conjugated)
#pragma unroll
  for (int l = 0; l < D; ++l) {
    bool up;
    const unsigned long long idx = where(rb, cb, l, up);
    x[l] = act ? ld_cg_l2_256(&rho[idx]) : make_float2(0.f, 0.f);
    upm |= (up ? 1u : 0u) << l;
  }
  for (unsigned long long u = u0; u < u1; ++u) {
#pragma unroll
    for (int l = 0; l < D; ++l)
      if (!((upm >> l) & 1u)) x[l].y = -x[l].y;
    pauli_fwd(x);
    const bool more = u + 1 < u1;
    unsigned rbn = 0, cbn = 0, upn = 0;
    bool actn = false, selfn = false;
    if (more) group(u + 1, rbn, cbn, actn, selfn);
    float2 y[D];
#pragma unroll
    for (int a = 0; a < D; ++a) y[a] = make_float2(0.f, 0.f);
#pragma unroll
    for (int b2 = 0; b2 < D; ++b2) {
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const float v = Rt[b2 * D + a];
        y[a].x = fmaf(v, x[b2].x, y[a].x);
        y[a].y = fmaf(v, x[b2].y, y[a].y);
      }
      bool up;
      const unsigned long long idx = where(rbn, cbn, b2, up);
      if (more && actn) x[b2] = ld_cg_l2_256(&rho[idx]);
      upn |= (up ? 1u : 0u) << b2;
    }
    pauli_inv(y);
    if (act) {
      // streaming stores: the next reader of these entries is the job's next
      // block, usually many items later, so L2 keeps the blocks the
      // neighbouring tiles are still reading instead
#pragma unroll
      for (int o = 0; o < D; ++o) {
        float2 acc = y[o];
        const unsigned r = rb + t.rt[o], c = cb + t.ct[o];
        if (r <= c) {
          __stcs(&rho[(unsigned long long)r | ((unsigned long long)c << p.n)], acc);
        } else if (!self) {
          acc.y = -acc.y;
          __stcs(&rho[(unsigned long long)c | ((unsigned long long)r << p.n)], acc);
        }
      }
    }
    rb = rbn;
    cb = cbn;
    act = actn;
    self = selfn;
    upm = upn;
  }
}

// FP64 tile items of a width-2 block in the Pauli basis: the group's entries
// gathered into this thread's shared-memory column (as the row-list path
// does), transformed there, multiplied by the real R' row lists into
// registers, transformed back and written in place.
__device__ __forceinline__ void apply_group_pauli_global(double2* rho, unsigned long long t, const ApplyParams& p,
                                                         const double* val, const RowLists& rl, double2* mine) {
  constexpr int D = 16;
  bool self = false;
  unsigned long long base = canonical_group(t, p.n - 2, &self);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const unsigned long long low = base & ((1ull << p.pos[i]) - 1ull);
    base = ((base >> p.pos[i]) << (p.pos[i] + 1)) | low;
  }
  const unsigned int rmask = (1u << p.n) - 1u;
  const unsigned int rb = (unsigned int)(base & rmask), cb = (unsigned int)(base >> p.n);
#pragma unroll
  for (int l = 0; l < D; ++l) {
    const unsigned int r = rb + (unsigned int)(p.off[l] & rmask), c = cb + (unsigned int)(p.off[l] >> p.n);
    const bool conj = r > c;
    double2 v = __ldcg(&rho[conj ? ((unsigned long long)c | ((unsigned long long)r << p.n))
                                 : ((unsigned long long)r | ((unsigned long long)c << p.n))]);
    if (conj) v.y = flip_sign(v.y);
    mine[l * kThreads] = v;
  }
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int tb = 0; tb < 4; ++tb) {
      const int b = pauli_base(q, tb), s10 = q == 0 ? 1 : 2, s01 = q == 0 ? 4 : 8;
      double2 a00 = mine[b * kThreads], a10 = mine[(b + s10) * kThreads], a01 = mine[(b + s01) * kThreads],
              a11 = mine[(b + s10 + s01) * kThreads];
      pauli_bfly_fwd(a00, a10, a01, a11);
      mine[b * kThreads] = a00;
      mine[(b + s10) * kThreads] = a10;
      mine[(b + s01) * kThreads] = a01;
      mine[(b + s10 + s01) * kThreads] = a11;
    }
  double2 y[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    double2 acc = make_double2(0.0, 0.0);
    for (int k = rl.rowptr[a]; k < rl.rowptr[a + 1]; ++k) {
      const double v = val[k];
      const double2 xc = mine[rl.col[k] * kThreads];
      acc.x = ::fma(v, xc.x, acc.x);
      acc.y = ::fma(v, xc.y, acc.y);
    }
    y[a] = acc;
  }
  pauli_inv(y);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double2 acc = y[i];
    const unsigned int r = rb + (unsigned int)(p.off[i] & rmask), c = cb + (unsigned int)(p.off[i] >> p.n);
    if (r <= c) {
      rho[(unsigned long long)r | ((unsigned long long)c << p.n)] = acc;
    } else if (!self) {
      acc.y = flip_sign(acc.y);
      rho[(unsigned long long)c | ((unsigned long long)r << p.n)] = acc;
    }
  }
}

// Copy a block's descriptor to shared memory with its superoperator: dense
// (split) or as row lists (FP64; zero tests on the bit patterns, so -0.0
// counts as zero). The row lists take rows in order, each thread i < D
// placing row i after the counts of rows < i.
template <typename T2>
__device__ __forceinline__ void stage_block(const BBlk* blk, BBlk* s_blk, T2* sS, RowLists* rl, Tile16* t16,
                                            int* pauli_on, bool allow_pauli) {
  static_assert(sizeof(BBlk) % 8 == 0 && sizeof(BBlk) / 8 <= kThreads, "descriptor copied one word per thread");
  if (threadIdx.x < sizeof(BBlk) / 8)  // in parallel: one 8-byte word per thread
    reinterpret_cast<unsigned long long*>(s_blk)[threadIdx.x] = reinterpret_cast<const unsigned long long*>(blk)[threadIdx.x];
  __syncthreads();
  const ApplyParams& p = s_blk->p;
  const int K = p.width, D = 1 << (2 * K);
  const T2* S = static_cast<const T2*>(s_blk->S);
  // tile items of width-2 blocks take the Pauli basis when the block's
  // record says so (one word, the same for every thread)
  const PauliRec* pr = allow_pauli ? s_blk->pauli : nullptr;
  const bool pauli = pr != nullptr && pr->on != 0;
  const int e = threadIdx.x;  // one superoperator entry per thread (D * D <= 256)
  if constexpr (sizeof(T2) == 8) {
    if (pauli)
      reinterpret_cast<float*>(sS)[e] = reinterpret_cast<const float*>(pr->val)[e];  // R' dense, transposed
    else if (e < D * D)
      sS[e] = S[e];
    if (threadIdx.x < 16) {
      int qs[2] = {p.q[0], K == 2 ? p.q[1] : 0};
      if (K == 2 && qs[0] > qs[1]) {
        const int t = qs[0];
        qs[0] = qs[1];
        qs[1] = t;
      }
      t16->dep16[threadIdx.x] = (unsigned)deposit_zeros((unsigned long long)threadIdx.x, qs, K);
      if (threadIdx.x < 2) t16->qs[threadIdx.x] = qs[threadIdx.x];
      if (threadIdx.x < D) {
        unsigned rt = 0, ct = 0;
        for (int j = 0; j < K; ++j) {
          rt |= ((threadIdx.x >> j) & 1u) << p.q[j];
          ct |= ((threadIdx.x >> (K + j)) & 1u) << p.q[j];
        }
        t16->rt[threadIdx.x] = rt;
        t16->ct[threadIdx.x] = ct;
      }
    }
  } else if (pauli) {
    // FP64 Pauli row lists as they are
    const int nnz = pr->nnz;
    if (e <= 16) rl->rowptr[e] = pr->rowptr[e];
    for (int k = e; k < nnz; k += blockDim.x) {
      rl->col[k] = pr->col[k];
      reinterpret_cast<double*>(sS)[k] = pr->val[k];
    }
  } else {
    // FP64 row lists of S: nonzero by bit pattern (-0.0 counts as zero), row
    // masks by warp ballot (a row's D entries share a warp), each kept entry
    // placed after the nonzeros of the rows and columns before it
    double2 v = make_double2(0.0, 0.0);
    bool keep = false;
    if (e < D * D) {
      v = S[e];
      keep = ((__double_as_longlong(v.x) | __double_as_longlong(v.y)) << 1) != 0;
    }
    const unsigned ball = __ballot_sync(0xffffffffu, keep);
    const int row = e / D, j = e % D;
    if (e < D * D && j == 0) rl->mask[row] = (ball >> (e & 31)) & ((1u << D) - 1u);
    __syncthreads();
    if (e < D * D) {
      int off = 0;
      for (int r = 0; r < row; ++r) off += __popc(rl->mask[r]);
      if (keep) {
        const int k = off + __popc(rl->mask[row] & ((1u << j) - 1u));
        sS[k] = v;
        rl->col[k] = (unsigned char)j;
      }
      if (j == 0) rl->rowptr[row] = off;
      if (e == D * D - 1) rl->rowptr[D] = off + __popc(rl->mask[row]);
    }
  }
  if (threadIdx.x == 0) *pauli_on = pauli ? 1 : 0;
  __syncthreads();
}

// Every job runs in Hermitian mode (canonical groups; BJob::herm is always
// set by batch_herm). Resident items: FP64 row lists or split dense products
// on the shared-memory copy of rho. Tile items: FP64 row lists over a range
// of canonical groups; split walks a range of canonical 16 x 16 tiles.
template <typename T2>
__global__ void __launch_bounds__(kThreads, 2) k_batch_apply(char* arena, const BJob* __restrict__ jobs,
                                                          const BBlk* __restrict__ blks,
                                                          const BItem* __restrict__ items, int n_items,
                                                          int* counters, int* ticket, int* err, long long max_spin) {
  extern __shared__ __align__(16) unsigned char smem[];
  T2* sS = reinterpret_cast<T2*>(smem);
  T2* sR = sS + kSEntries;
  __shared__ BBlk s_blk;
  __shared__ RowLists s_rl;
  __shared__ Tile16 s_t16;
  __shared__ int s_pauli;  // the staged block's tile items run in the Pauli basis
  __shared__ int s_idx;
  constexpr bool kF64 = sizeof(T2) == 16;
  // thread 0 takes each item's ticket one item ahead, so the atomic's round
  // trip overlaps the current item (tickets are monotone and every wait is
  // on a smaller ticket, so the smallest unfinished item can always run)
  int next = 0;
  if (threadIdx.x == 0) next = atomicAdd(ticket, 1);
  for (;;) {
    if (threadIdx.x == 0) {
      s_idx = next;
      next = atomicAdd(ticket, 1);
    }
    __syncthreads();
    const int idx = s_idx;
    __syncthreads();
    if (idx >= n_items) break;
    const BItem it = items[idx];
    const BJob& jb = jobs[it.job];
    T2* rho = reinterpret_cast<T2*>(arena + jb.rho_off);
    const int n = jb.n;
    if (it.block < 0) {
      // resident job: the whole circuit on a shared-memory copy of rho
      const int N = 1 << (2 * n);
      for (int e = threadIdx.x; e < N; e += blockDim.x) sR[e] = Cx<T2>::ldcg(&rho[e]);
      for (int b = it.tile0; b < it.tile0 + it.ntiles; ++b) {
        stage_block(&blks[jb.block0 + b], &s_blk, sS, &s_rl, &s_t16, &s_pauli, false);
        const ApplyParams& p = s_blk.p;
        for (unsigned long long g = threadIdx.x; g < p.n_canon; g += blockDim.x) {
          if constexpr (kF64) {
            double2* sR64 = reinterpret_cast<double2*>(sR);
            const double2* val = reinterpret_cast<const double2*>(sS);
            if (p.width == 1)
              apply_group_lists_resident<1, true>(sR64, (unsigned int)g, p, val, s_rl);
            else
              apply_group_lists_resident<2, true>(sR64, (unsigned int)g, p, val, s_rl);
          } else {
            if (p.width == 1)
              apply_group<T2, 1>(sR, g, p, sS);
            else
              apply_group<T2, 2>(sR, g, p, sS);
          }
        }
        __syncthreads();
      }
      for (int e = threadIdx.x; e < N; e += blockDim.x) rho[e] = sR[e];
      __syncthreads();
      continue;
    }
    // tile item: stage the block (independent of earlier blocks), then wait
    // until every tile of the previous block of this job is done
    stage_block(&blks[jb.block0 + it.block], &s_blk, sS, &s_rl, &s_t16, &s_pauli, true);
    if (threadIdx.x == 0 && it.block > 0) {
      const int need = jb.never_ready ? 0x7fffffff : s_blk.tile_prefix;
      long long spins = 0;
      while (ld_acquire(&counters[it.job]) < need) {
        if (ld_acquire(err) != 0) break;
        if (++spins > max_spin) {
          atomicExch(err, 1);
          break;
        }
        __nanosleep(128);
      }
    }
    __syncthreads();
    const ApplyParams& p = s_blk.p;
    if (*(volatile int*)err == 0) {
      if constexpr (kF64) {
        // a range of canonical groups; the resident buffer is free in tile
        // items and holds the threads' operand columns (16 x kThreads
        // entries = 64 KiB)
        const unsigned long long gpt = 1ull << (jb.tile_log2 - 2 * p.width);  // groups per tile
        const unsigned long long g0 = (unsigned long long)it.tile0 * gpt;
        const unsigned long long g1 = min(p.n_canon, g0 + (unsigned long long)it.ntiles * gpt);
        double2* mine = reinterpret_cast<double2*>(sR) + threadIdx.x;
        const double2* val = reinterpret_cast<const double2*>(sS);
        double2* rho64 = reinterpret_cast<double2*>(rho);
        for (unsigned long long g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
          if (p.width == 1)
            apply_group_lists_global<1, true>(rho64, g, p, val, s_rl, mine);
          else if (s_pauli)
            apply_group_pauli_global(rho64, g, p, reinterpret_cast<const double*>(sS), s_rl, mine);
          else
            apply_group_lists_global<2, true>(rho64, g, p, val, s_rl, mine);
        }
      } else {
        // a range of canonical 16 x 16 tiles
        const unsigned long long upt = 1ull << tiles16_log2(jb.tile_log2, p.width);
        const unsigned long long Mt = (1ull << (p.n - p.width)) / 16;
        const unsigned long long total = Mt * (Mt + 1) / 2;
        const unsigned long long u0 = (unsigned long long)it.tile0 * upt;
        const unsigned long long u1 = min(total, u0 + (unsigned long long)it.ntiles * upt);
        if (p.width == 2 && s_pauli) {
          apply_tiles16_pauli(rho, u0, u1, p, reinterpret_cast<const float*>(sS), s_t16);
        } else {
          for (unsigned long long u = u0; u < u1; ++u) {
            if (p.width == 1)
              apply_tile16<1>(rho, u, p, sS, s_t16);
            else
              apply_tile16<2>(rho, u, p, sS, s_t16);
          }
        }
      }
    }
    __syncthreads();
    // publish the item's writes (the barrier orders them before this
    // thread's release) and count its tiles
    if (threadIdx.x == 0)
      asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(&counters[it.job]), "r"(it.ntiles) : "memory");
  }
}

static __global__ void k_batch_set_one(char* arena, const BJob* __restrict__ jobs, int n_jobs, int precision) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_jobs) return;
  if (precision == 0)
    reinterpret_cast<double2*>(arena + jobs[j].rho_off)[0] = make_double2(1.0, 0.0);
  else
    reinterpret_cast<float2*>(arena + jobs[j].rho_off)[0] = make_float2(1.f, 0.f);
}

// Per-job FP64 readouts: one CTA per job, fixed thread mapping and tree.
template <typename T2>
__global__ void __launch_bounds__(kThreads) k_batch_reduce(const char* arena, const BJob* __restrict__ jobs,
                                                           int normalize, double* __restrict__ out) {
  __shared__ double red[kResults][kThreads];
  const BJob& jb = jobs[blockIdx.x];
  const T2* rho = reinterpret_cast<const T2*>(arena + jb.rho_off);
  const unsigned long long N = 1ull << jb.n;
  double acc[kResults];
#pragma unroll
  for (int q = 0; q < kResults; ++q) acc[q] = 0.0;
  for (unsigned long long x = threadIdx.x; x < N; x += kThreads) {
    const T2 v = rho[x * (N + 1)];
    const double re = (double)v.x;
    acc[0] += re;
    acc[1] += (double)v.y;
#pragma unroll
    for (int q = 0; q < kMaxMasks; ++q)
      if (q < jb.n_masks) acc[2 + q] += (__popcll(x & jb.masks[q]) & 1) ? -re : re;
  }
#pragma unroll
  for (int q = 0; q < kResults; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int q = 0; q < kResults; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < kResults) {
    double v = red[threadIdx.x][0];
    if (normalize && threadIdx.x >= 2) v /= red[0][0];
    out[blockIdx.x * kResults + threadIdx.x] = v;
  }
}

template <typename T2>
__host__ __device__ constexpr size_t apply_smem() {
  return kSEntries * sizeof(T2) + kResidentBytes;
}

inline bool is_resident(int n, int prec) {
  return (size_t)(prec == 0 ? 16 : 8) << (2 * n) <= (size_t)kResidentBytes;
}

// Hermitian mode in the batch kernel: every job. FP64 and resident split
// jobs take one canonical group per thread; split tile jobs (at least 7
// qubits, so 2^(n-w) >= 32 row rests) walk canonical 16 x 16 tiles.
inline bool batch_herm(int n, int prec) {
  (void)n;
  (void)prec;
  return true;
}

// Fill the per-block tile counts and wait targets of one job's blocks and
// return its total tile count. gpt = 2^(tile_log2 - 2w) groups per tile;
// split tile jobs in Hermitian mode count canonical 16 x 16 tiles instead.
inline long long set_tiles(BBlk* blks, int n_blocks, int tile_log2, bool herm, bool tiled16) {
  long long prefix = 0;
  for (int b = 0; b < n_blocks; ++b) {
    ApplyParams& p = blks[b].p;
    const unsigned long long M = 1ull << (p.n - p.width);
    p.herm = herm ? 1 : 0;
    p.n_canon = M * (M + 1) / 2;
    unsigned long long total, per;
    if (herm && tiled16) {
      const unsigned long long Mt = M / 16;
      total = Mt * (Mt + 1) / 2;
      per = 1ull << tiles16_log2(tile_log2, p.width);
    } else {
      total = herm ? p.n_canon : p.n_groups;
      per = 1ull << (tile_log2 - 2 * p.width);
    }
    blks[b].tiles = (int)((total + per - 1) / per);
    blks[b].tile_prefix = (int)prefix;
    prefix += blks[b].tiles;
  }
  return prefix;
}

// Split tile jobs walk canonical 16 x 16 tiles (needs 2^(n-w) >= 16).
inline bool tiled16_job(int n, int prec) { return prec != 0 && !is_resident(n, prec); }

}  // namespace batch
}  // namespace tq
