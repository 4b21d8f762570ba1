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
  unsigned long long masks[kMaxMasks];
};

struct BBlk {
  ApplyParams p;
  const void* S;       // fused superoperator, 4^w x 4^w row-major (double2 or float2)
  const double2* S64;  // the same in FP64 (the fused product; FP64 jobs build their Pauli-basis lists from it)
  int tiles;           // tile items of this block (tile jobs)
  int tile_prefix;     // tiles of the job's earlier blocks: the wait target
};

struct BItem {
  int job;
  int block;   // tile item: block index (job-relative); -1: resident item
  int tile0;   // tile item: first tile; resident item: first block
  int ntiles;  // tile item: tiles; resident item: blocks
};

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

// Width-2 products of FP64 tile items in the Pauli basis. Every block is a
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
__host__ __device__ __forceinline__ double pauli_entry(const double2* S, int sa, int sb) {
  int la[4], lb[4], ar[4], ai[4], br[4], bi[4];
  pauli_row(sa, la, ar, ai);
  pauli_row(sb, lb, br, bi);
  double acc = 0.0;
  for (int u = 0; u < 4; ++u)
    for (int v = 0; v < 4; ++v) {
      const double2 sv = S[la[u] * 16 + lb[v]];
      const double tr = ar[u] * sv.x - ai[u] * sv.y, ti = ar[u] * sv.y + ai[u] * sv.x;  // T[sa][l] S[l][m]
      acc += tr * br[v] + ti * bi[v];                                                // Re (t conj(T[sb][m]))
    }
  return acc * (1.0 / 16.0);
}
// Whether an FP64 width-2 tile-item block takes the Pauli row lists: when
// they cost fewer FP64 operations per group (2 per nonzero + 128 adds against
// 4 per nonzero of S's row lists). Split blocks keep the dense product: their
// tile items are HBM-bound, and building R' (FP64, at staging) cost more than
// it saved (1024-circuit sweep: 4,584 against 8,311 circuits/s).
__host__ __device__ __forceinline__ bool pauli_better(int nnzS, int nnzR) { return 2 * nnzR + 128 < 4 * nnzS; }

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
    if (conj) v.y = -v.y;
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
        acc.y = -acc.y;
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
        if (r > c) v.y = -v.y;
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
        acc.y = -acc.y;
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
    if (conj) v.y = -v.y;
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
      acc.y = -acc.y;
      rho[(unsigned long long)c | ((unsigned long long)r << p.n)] = acc;
    }
  }
}

// Copy a block's descriptor to shared memory with its superoperator: dense
// (split) or as row lists (FP64; zero tests on the bit patterns, so -0.0
// counts as zero). The row lists take rows in order, each thread i < D
// placing row i after the counts of rows < i.
// Shared state of the Pauli-basis decision of a staged block.
struct PauliStage {
  double R[256];       // R' of a width-2 block, FP64
  double thr;          // structural-zero threshold
  unsigned short mask[16];
  int on;              // the staged block takes the Pauli row lists
};

template <typename T2>
__device__ __forceinline__ void stage_block(const BBlk* blk, BBlk* s_blk, T2* sS, RowLists* rl, Tile16* t16,
                                            PauliStage* ps, bool allow_pauli) {
  static_assert(sizeof(BBlk) % 8 == 0 && sizeof(BBlk) / 8 <= kThreads, "descriptor copied one word per thread");
  if (threadIdx.x < sizeof(BBlk) / 8)  // in parallel: one 8-byte word per thread
    reinterpret_cast<unsigned long long*>(s_blk)[threadIdx.x] = reinterpret_cast<const unsigned long long*>(blk)[threadIdx.x];
  __syncthreads();
  const int D = 1 << (2 * s_blk->p.width);
  const T2* S = static_cast<const T2*>(s_blk->S);
  if (sizeof(T2) == 8) {
    for (int e = threadIdx.x; e < D * D; e += blockDim.x) sS[e] = S[e];
    const ApplyParams& p = s_blk->p;
    const int K = p.width;
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
  } else {
    const unsigned long long* bits = reinterpret_cast<const unsigned long long*>(S);
    unsigned int m = 0;
    if (threadIdx.x < D)
      for (int j = 0; j < D; ++j) {
        const int e = threadIdx.x * D + j;
        if (((bits[2 * e] | bits[2 * e + 1]) << 1) != 0ull) m |= 1u << j;
      }
    if (threadIdx.x < D) rl->rowptr[threadIdx.x + 1] = __popc(m);
    if (threadIdx.x == 0) rl->rowptr[0] = 0;
    __syncthreads();
    if (threadIdx.x == 0)
      for (int i = 1; i <= D; ++i) rl->rowptr[i] += rl->rowptr[i - 1];
    __syncthreads();
    if (threadIdx.x < D) {
      int k = rl->rowptr[threadIdx.x];
      for (int j = 0; j < D; ++j)
        if ((m >> j) & 1u) {
          sS[k] = S[threadIdx.x * D + j];
          rl->col[k] = (unsigned char)j;
          ++k;
        }
    }
  }
  if (threadIdx.x == 0) ps->on = 0;
  __syncthreads();
  if (!allow_pauli || sizeof(T2) == 8 || s_blk->p.width != 2) return;
  // tile items of width-2 blocks: R' in FP64, structural zeros dropped, and
  // the Pauli row lists replace S's when they cost less (pauli_better)
  ps->R[threadIdx.x] = pauli_entry(s_blk->S64, threadIdx.x / 16, threadIdx.x % 16);
  __syncthreads();
  if (threadIdx.x < 32) {
    double mx = 0.0;
    for (int e = threadIdx.x; e < 256; e += 32) mx = fmax(mx, fabs(ps->R[e]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0) ps->thr = mx * kPauliZeroRel;
  }
  __syncthreads();
  if (threadIdx.x < 16) {
    unsigned m = 0;
    for (int j = 0; j < 16; ++j)
      if (fabs(ps->R[threadIdx.x * 16 + j]) > ps->thr) m |= 1u << j;
    ps->mask[threadIdx.x] = (unsigned short)m;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int nnzR = 0;
    for (int i = 0; i < 16; ++i) nnzR += __popc(ps->mask[i]);
    ps->on = pauli_better(rl->rowptr[16], nnzR) ? 1 : 0;
    if (ps->on) {
      rl->rowptr[0] = 0;
      for (int i = 0; i < 16; ++i) rl->rowptr[i + 1] = rl->rowptr[i] + __popc(ps->mask[i]);
    }
  }
  __syncthreads();
  if (ps->on && threadIdx.x < 16) {
    int k = rl->rowptr[threadIdx.x];
    for (int j = 0; j < 16; ++j)
      if ((ps->mask[threadIdx.x] >> j) & 1u) {
        reinterpret_cast<double*>(sS)[k] = ps->R[threadIdx.x * 16 + j];
        rl->col[k] = (unsigned char)j;
        ++k;
      }
  }
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
  __shared__ PauliStage s_ps;  // Pauli-basis decision and R' of the staged block
  __shared__ int s_idx;
  constexpr bool kF64 = sizeof(T2) == 16;
  for (;;) {
    if (threadIdx.x == 0) s_idx = atomicAdd(ticket, 1);
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
        stage_block(&blks[jb.block0 + b], &s_blk, sS, &s_rl, &s_t16, &s_ps, false);
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
    stage_block(&blks[jb.block0 + it.block], &s_blk, sS, &s_rl, &s_t16, &s_ps, true);
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
          else if (s_ps.on)
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
        for (unsigned long long u = u0; u < u1; ++u) {
          if (p.width == 1)
            apply_tile16<1>(rho, u, p, sS, s_t16);
          else
            apply_tile16<2>(rho, u, p, sS, s_t16);
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&counters[it.job], it.ntiles);
    }
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
