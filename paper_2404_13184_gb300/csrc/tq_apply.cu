// Apply kernels: one pass of a fused width-K superoperator over vec(rho)
// (TANQ-Sim Sec. 3.1, the C1/C2 update generalised to K <= 4).
//
// Hermitian mode (FP64 states): every op is a Kraus map, which keeps
// rho = rho^dagger. Writing a group's rest bits as (a, b) = (row rest,
// column rest), group (b, a) holds the conjugate transposes of group (a, b),
// so only the canonical groups a <= b are computed and only entries with
// row <= column are kept current: an input below the diagonal is read as
// the conjugate of its transpose, an output below the diagonal is written,
// conjugated, to its transpose. The diagonal (all readouts) is always
// current; tq_get_rho fills the lower triangle before copying out.
//
// vec(rho) has 4^n entries; a width-K block on qubits q_0..q_{K-1} splits the
// 2n index bits into 2K target bits (q_j and q_j + n) and 2n - 2K group bits.
// Group g's base index is g with zeros inserted at the target bits; its 4^K
// entries sit at base + off[l], where bit j of l selects row bit q_j and bit
// K + j selects column bit q_j + n. Each group is replaced by S x (x = its
// 4^K entries). Groups are disjoint, so the update runs in place: every
// entry is read once and written once, by the CTA that owns its group.
#include <algorithm>
#include <mutex>

#include "tq_device.cuh"

namespace tq {

namespace {

template <typename T2>
struct CplxOps;

template <>
struct CplxOps<double2> {
  __device__ __forceinline__ static double2 zero() { return make_double2(0.0, 0.0); }
  // Shared-memory load kept inside the loop (volatile): S stays in shared
  // memory instead of being hoisted into (and spilled from) registers.
  __device__ __forceinline__ static double2 lds(const double2* p) {
    double2 v;
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];"
                 : "=d"(v.x), "=d"(v.y)
                 : "r"((unsigned)__cvta_generic_to_shared(p)));
    return v;
  }
  __device__ __forceinline__ static void fma(double2& acc, double2 a, double2 b) {
    acc.x = ::fma(a.x, b.x, acc.x);
    acc.x = ::fma(-a.y, b.y, acc.x);
    acc.y = ::fma(a.x, b.y, acc.y);
    acc.y = ::fma(a.y, b.x, acc.y);
  }
};

template <>
struct CplxOps<float2> {
  __device__ __forceinline__ static float2 zero() { return make_float2(0.f, 0.f); }
  __device__ __forceinline__ static float2 lds(const float2* p) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];"
                 : "=f"(v.x), "=f"(v.y)
                 : "r"((unsigned)__cvta_generic_to_shared(p)));
    return v;
  }
  __device__ __forceinline__ static void fma(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
  }
};

// Widths 1 and 2: one thread per group, the group's 4^K entries in
// registers. S (16 or 256 complex) is staged in shared memory; for width 1
// the compiler keeps it in registers across the group loop, for width 2 it is
// re-read from shared memory (warp-uniform broadcast) for every group.
// Grid-stride over groups; consecutive threads take consecutive groups, so a
// warp's loads of one local index are contiguous whenever the low index bits
// are group bits.
template <typename T2, int K, bool HERM>
__device__ __forceinline__ void apply_direct_body(T2* rho, const T2* __restrict__ S, const ApplyParams& p) {
  constexpr int D = 1 << (2 * K);
  __shared__ T2 sS[D * D];
  for (int i = threadIdx.x; i < D * D; i += blockDim.x) sS[i] = S[i];
  __syncthreads();
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long total = HERM ? p.n_canon : p.n_groups;
  const unsigned long long rmask = (1ull << p.n) - 1ull;
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < total; t += stride) {
    bool self = false;
    unsigned long long base = HERM ? canonical_group(t, p.n - K, &self) : t;
#pragma unroll
    for (int i = 0; i < 2 * K; ++i) {
      const unsigned long long low = base & ((1ull << p.pos[i]) - 1ull);
      base = ((base >> p.pos[i]) << (p.pos[i] + 1)) | low;
    }
    T2 x[D];
    if (!HERM) {
#pragma unroll
      for (int l = 0; l < D; ++l) x[l] = rho[base + p.off[l]];
    } else {
      // entries below the diagonal are read as the conjugate of their transpose
#pragma unroll
      for (int l = 0; l < D; ++l) {
        const unsigned long long e = base + p.off[l], r = e & rmask, c = e >> p.n;
        const bool up = r <= c;
        T2 v = rho[up ? e : (c | (r << p.n))];
        if (!up) v.y = -v.y;
        x[l] = v;
      }
    }
#pragma unroll
    for (int i = 0; i < D; ++i) {
      T2 acc = CplxOps<T2>::zero();
#pragma unroll
      for (int j = 0; j < D; ++j)
        CplxOps<T2>::fma(acc, K == 1 ? sS[i * D + j] : CplxOps<T2>::lds(&sS[i * D + j]), x[j]);
      if (!HERM) {
        rho[base + p.off[i]] = acc;
      } else {
        // outputs below the diagonal go, conjugated, to their transpose (which
        // lies in the skipped partner group; in a self-conjugate group the
        // transpose is written directly by its own row)
        const unsigned long long e = base + p.off[i], r = e & rmask, c = e >> p.n;
        if (r <= c) {
          rho[e] = acc;
        } else if (!self) {
          acc.y = -acc.y;
          rho[c | (r << p.n)] = acc;
        }
      }
    }
  }
}

template <typename T2, int K>
__global__ void __launch_bounds__(256) k_apply_direct(T2* rho, const T2* __restrict__ S,
                                                      const __grid_constant__ ApplyParams p) {
  apply_direct_body<T2, K, false>(rho, S, p);
}

// Hermitian variant (FP64): the DFMA pipe needs few warps, so the extra
// address registers of this path (one CTA per SM at width 2) cost nothing.
template <typename T2, int K>
__global__ void __launch_bounds__(256) k_apply_direct_herm(T2* rho, const T2* __restrict__ S,
                                                              const __grid_constant__ ApplyParams p) {
  apply_direct_body<T2, K, true>(rho, S, p);
}

// Sparse FP64 blocks (width <= 2): the row lists sit in shared memory and a
// thread's group entries in its own shared-memory column (slot l at
// sX[l * 256 + thread]), so a row costs one broadcast entry load, one
// conflict-free slot load and four DFMA per nonzero.
template <int K, bool HERM>
__global__ void __launch_bounds__(256) k_apply_sparse(double2* rho, const SparseBlock* __restrict__ sp,
                                                      const __grid_constant__ ApplyParams p) {
  constexpr int D = 1 << (2 * K);
  __shared__ int s_rowptr[D + 1];
  __shared__ double2 s_v[D * D];
  __shared__ int s_col[D * D];
  extern __shared__ __align__(16) double2 sX[];
  if (threadIdx.x <= D) s_rowptr[threadIdx.x] = sp->rowptr[threadIdx.x];
  __syncthreads();
  for (int k = threadIdx.x; k < s_rowptr[D]; k += blockDim.x) {
    s_v[k] = sp->e[k].v;
    s_col[k] = sp->e[k].col;
  }
  __syncthreads();
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long total = HERM ? p.n_canon : p.n_groups;
  const unsigned long long rmask = (1ull << p.n) - 1ull;
  double2* mine = sX + threadIdx.x;
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < total; t += stride) {
    bool self = false;
    unsigned long long base = HERM ? canonical_group(t, p.n - K, &self) : t;
#pragma unroll
    for (int i = 0; i < 2 * K; ++i) {
      const unsigned long long low = base & ((1ull << p.pos[i]) - 1ull);
      base = ((base >> p.pos[i]) << (p.pos[i] + 1)) | low;
    }
#pragma unroll
    for (int l = 0; l < D; ++l) {
      const unsigned long long e = base + p.off[l];
      double2 v;
      if (!HERM) {
        v = rho[e];
      } else {
        const unsigned long long r = e & rmask, c = e >> p.n;
        v = rho[r <= c ? e : (c | (r << p.n))];
        if (r > c) v.y = -v.y;
      }
      mine[l * 256] = v;
    }
#pragma unroll
    for (int i = 0; i < D; ++i) {
      double2 acc = make_double2(0.0, 0.0);
      for (int k = s_rowptr[i]; k < s_rowptr[i + 1]; ++k)
        CplxOps<double2>::fma(acc, s_v[k], mine[s_col[k] * 256]);
      const unsigned long long e = base + p.off[i];
      if (!HERM) {
        rho[e] = acc;
      } else {
        const unsigned long long r = e & rmask, c = e >> p.n;
        if (r <= c) {
          rho[e] = acc;
        } else if (!self) {
          acc.y = -acc.y;
          rho[c | (r << p.n)] = acc;
        }
      }
    }
  }
}

template <int K, bool HERM>
cudaError_t run_sparse(double2* rho, const SparseBlock* sp, const ApplyParams& p, int num_sms, cudaStream_t st) {
  constexpr int D = 1 << (2 * K);
  const size_t smem = (size_t)D * 256 * sizeof(double2);
  static std::once_flag once;
  std::call_once(once, [&] {
    cudaFuncSetAttribute(k_apply_sparse<K, HERM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  const unsigned long long blocks = ((HERM ? p.n_canon : p.n_groups) + 255) / 256;
  const int grid = (int)std::max<unsigned long long>(1, std::min<unsigned long long>(blocks, (unsigned long long)num_sms * 8));
  k_apply_sparse<K, HERM><<<grid, 256, smem, st>>>(rho, sp, p);
  return cudaGetLastError();
}

// Hermitian mode for split states on the CUDA cores: width 1 (width-2 blocks
// run on the tensor cores, tq_apply_tc.cu; the template still covers K = 2,
// with the same tile walk as the tensor-core kernel). The pass is HBM-bound, so
// the canonical groups are walked in T x T tiles: row-rest a in
// [ta T, ta T + T), column-rest b in [tb T, tb T + T), ta <= tb, one thread
// per group; a warp covers 8 consecutive a by 4 consecutive b. Entries on or
// above the diagonal are read and written in place (8 consecutive rows of a
// column); entries below it are held by their transposes, whose 4
// consecutive columns of a row fill one 32-byte sector. Diagonal tiles
// (ta == tb) compute the groups with a <= b.
//
// Row index r = dep(a) + rt[l], column index c = dep(b) + ct[l], vec index
// r + c 2^n; dep() inserts zeros at the target qubits (the same positions for
// rows and columns) and is additive over disjoint bits, so dep(a0 + i) =
// dep(a0) + dep(i) for a tile base a0 (a multiple of T): the index math is
// table lookups and adds.
template <int K, int T>
__global__ void __launch_bounds__(T * T) k_apply_herm_tiled(float2* rho, const float2* __restrict__ S,
                                                            const __grid_constant__ ApplyParams p) {
  constexpr int D = 1 << (2 * K);
  __shared__ float2 sS[D * D];
  __shared__ unsigned int s_dep[T];          // deposit of i < T into the non-target positions
  __shared__ unsigned int s_rt[D], s_ct[D];  // row / column target bits of local index l
  int qs[K];
#pragma unroll
  for (int j = 0; j < K; ++j) qs[j] = p.q[j];
#pragma unroll
  for (int x = 0; x < K; ++x)  // sort the target qubits ascending
#pragma unroll
    for (int y = 0; y + 1 < K; ++y)
      if (qs[y] > qs[y + 1]) {
        const int t = qs[y];
        qs[y] = qs[y + 1];
        qs[y + 1] = t;
      }
  for (int i = threadIdx.x; i < D * D; i += blockDim.x) sS[i] = S[i];
  if (threadIdx.x < T) s_dep[threadIdx.x] = (unsigned int)deposit_zeros(threadIdx.x, qs, K);
  if (threadIdx.x < D) {
    unsigned int rt = 0, ct = 0;
    for (int j = 0; j < K; ++j) {
      rt |= ((threadIdx.x >> j) & 1u) << p.q[j];
      ct |= ((threadIdx.x >> (K + j)) & 1u) << p.q[j];
    }
    s_rt[threadIdx.x] = rt;
    s_ct[threadIdx.x] = ct;
  }
  __syncthreads();
  const unsigned int* rt = s_rt;  // warp-uniform reads (broadcast)
  const unsigned int* ct = s_ct;
  // a warp covers 8 row rests x 4 column rests: 8 consecutive rows of one
  // column above the diagonal (64 B), 4 consecutive columns of one row
  // below it (one full 32-byte sector)
  static_assert(T == 16, "warp layout of a 16 x 16 tile");
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
  const int i = (lane % 8) + 8 * (w % 2), j = (lane / 8) + 4 * (w / 2);
  const unsigned int di = s_dep[i], dj = s_dep[j];
  const unsigned long long Mt = (1ull << (p.n - K)) / T;
  const unsigned long long n_tiles = Mt * (Mt + 1) / 2;
  for (unsigned long long u = blockIdx.x; u < n_tiles; u += gridDim.x) {
    bool diag = false;
    const unsigned long long tt = canonical_group(u, 32, &diag);  // (ta, tb) as ta | tb << 32
    if (diag && i > j) continue;  // not a canonical group
    const bool self = diag && i == j;
    const unsigned int rbase = (unsigned int)deposit_zeros((tt & 0xffffffffull) * T, qs, K) + di;
    const unsigned int cbase = (unsigned int)deposit_zeros((tt >> 32) * T, qs, K) + dj;
    float2 x[D];
#pragma unroll
    for (int l = 0; l < D; ++l) {
      const unsigned int r = rbase + rt[l], c = cbase + ct[l];
      const bool up = r <= c;
      float2 v = rho[up ? ((unsigned long long)r | ((unsigned long long)c << p.n))
                        : ((unsigned long long)c | ((unsigned long long)r << p.n))];
      if (!up) v.y = -v.y;
      x[l] = v;
    }
#pragma unroll
    for (int o = 0; o < D; ++o) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int l = 0; l < D; ++l)
        CplxOps<float2>::fma(acc, K == 1 ? sS[o * D + l] : CplxOps<float2>::lds(&sS[o * D + l]), x[l]);
      const unsigned int r = rbase + rt[o], c = cbase + ct[o];
      if (r <= c) {
        rho[(unsigned long long)r | ((unsigned long long)c << p.n)] = acc;
      } else if (!self) {  // a self-conjugate group writes its upper entries only
        acc.y = -acc.y;
        rho[(unsigned long long)c | ((unsigned long long)r << p.n)] = acc;
      }
    }
  }
}

template <int K>
cudaError_t run_herm_tiled_split(float2* rho, const float2* S, const ApplyParams& p, int num_sms, cudaStream_t st) {
  constexpr int T = 16;
  const unsigned long long M = 1ull << (p.n - K);
  if (M < T) return cudaErrorInvalidValue;  // the caller uses full updates for tiny registers
  const unsigned long long Mt = M / T, n_tiles = Mt * (Mt + 1) / 2;
  const int grid = (int)std::max<unsigned long long>(1, std::min<unsigned long long>(n_tiles, (unsigned long long)num_sms * 8));
  k_apply_herm_tiled<K, T><<<grid, T * T, 0, st>>>(rho, S, p);
  return cudaGetLastError();
}

// Widths 3 and 4: a CTA stages the entries of G consecutive groups (4^K x G)
// in shared memory, then thread (rowset, gi) computes rows i = rowset +
// (256/G) r of group gi and writes them straight back to global memory (the
// tile's entries were all read before the first write). S sits in shared
// memory when it fits (K = 3) and is read through L1/L2 otherwise (K = 4).
template <typename T2, int K, int G, bool S_SMEM, bool HERM>
__global__ void __launch_bounds__(256) k_apply_tiled(T2* rho, const T2* __restrict__ S,
                                                     const __grid_constant__ ApplyParams p) {
  constexpr int D = 1 << (2 * K);
  constexpr int ROWSETS = 256 / G;
  constexpr int ROWS = D / ROWSETS;  // rows per thread
  constexpr int CH = 8;              // rows per accumulation chunk
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned long long* sOff = reinterpret_cast<unsigned long long*>(smem_raw);
  T2* sX = reinterpret_cast<T2*>(sOff + D);
  T2* sS = sX + D * G;
  for (int l = threadIdx.x; l < D; l += blockDim.x) {
    unsigned long long v = 0;
    for (int j = 0; j < K; ++j) {
      if ((l >> j) & 1) v |= 1ull << p.q[j];
      if ((l >> (K + j)) & 1) v |= 1ull << (p.q[j] + p.n);
    }
    sOff[l] = v;
  }
  if (S_SMEM)
    for (int e = threadIdx.x; e < D * D; e += blockDim.x) sS[e] = S[e];
  __syncthreads();
  const int gi = threadIdx.x % G;
  const int rowset = threadIdx.x / G;
  const unsigned long long total = HERM ? p.n_canon : p.n_groups;
  const unsigned long long rmask = (1ull << p.n) - 1ull;
  const unsigned long long n_tiles = (total + G - 1) / G;
  for (unsigned long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const unsigned long long g0 = tile * G;
    for (int e = threadIdx.x; e < D * G; e += blockDim.x) {
      const int l = e / G, gg = e % G;
      const unsigned long long t = g0 + gg;
      if (t < total) {
        bool self = false;
        const unsigned long long g = HERM ? canonical_group(t, p.n - K, &self) : t;
        const unsigned long long idx = deposit_zeros(g, p.pos, 2 * K) + sOff[l];
        if (!HERM) {
          sX[e] = rho[idx];
        } else {
          const unsigned long long r = idx & rmask, c = idx >> p.n;
          T2 v = rho[r <= c ? idx : (c | (r << p.n))];
          if (r > c) v.y = -v.y;
          sX[e] = v;
        }
      }
    }
    __syncthreads();
    const unsigned long long t = g0 + gi;
    if (t < total) {
      bool self = false;
      const unsigned long long g = HERM ? canonical_group(t, p.n - K, &self) : t;
      const unsigned long long base = deposit_zeros(g, p.pos, 2 * K);
#pragma unroll 1
      for (int r0 = 0; r0 < ROWS; r0 += CH) {
        T2 acc[CH];
#pragma unroll
        for (int r = 0; r < CH; ++r) acc[r] = CplxOps<T2>::zero();
#pragma unroll 4
        for (int j = 0; j < D; ++j) {
          const T2 xj = sX[j * G + gi];
#pragma unroll
          for (int r = 0; r < CH; ++r) {
            const int i = rowset + ROWSETS * (r0 + r);
            const T2 s = S_SMEM ? sS[i * D + j] : __ldg(&S[i * D + j]);
            CplxOps<T2>::fma(acc[r], s, xj);
          }
        }
#pragma unroll
        for (int r = 0; r < CH; ++r) {
          const int i = rowset + ROWSETS * (r0 + r);
          const unsigned long long idx = base + sOff[i];
          if (!HERM) {
            rho[idx] = acc[r];
          } else {
            const unsigned long long rr = idx & rmask, cc = idx >> p.n;
            if (rr <= cc) {
              rho[idx] = acc[r];
            } else if (!self) {
              T2 v = acc[r];
              v.y = -v.y;
              rho[cc | (rr << p.n)] = v;
            }
          }
        }
      }
    }
    __syncthreads();
  }
}

template <typename T2, int K, int G, bool S_SMEM>
size_t tiled_smem_bytes() {
  constexpr int D = 1 << (2 * K);
  return D * sizeof(unsigned long long) + (size_t)D * G * sizeof(T2) + (S_SMEM ? (size_t)D * D * sizeof(T2) : 0);
}

template <typename T2, int K, int G, bool S_SMEM, bool HERM>
cudaError_t run_tiled(T2* rho, const T2* S, const ApplyParams& p, int num_sms, cudaStream_t st) {
  static std::once_flag once;
  static int per_sm = 1;
  const size_t smem = tiled_smem_bytes<T2, K, G, S_SMEM>();
  std::call_once(once, [&] {
    cudaFuncSetAttribute(k_apply_tiled<T2, K, G, S_SMEM, HERM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_apply_tiled<T2, K, G, S_SMEM, HERM>, 256, smem) == cudaSuccess && b > 0)
      per_sm = b;
  });
  const unsigned long long n_tiles = ((p.herm ? p.n_canon : p.n_groups) + G - 1) / G;
  const int grid = (int)std::max<unsigned long long>(1, std::min<unsigned long long>(n_tiles, (unsigned long long)num_sms * per_sm));
  k_apply_tiled<T2, K, G, S_SMEM, HERM><<<grid, 256, smem, st>>>(rho, S, p);
  return cudaGetLastError();
}

template <typename T2, int K, bool HERM>
cudaError_t run_direct(T2* rho, const T2* S, const ApplyParams& p, int num_sms, cudaStream_t st) {
  const unsigned long long blocks = ((p.herm ? p.n_canon : p.n_groups) + 255) / 256;
  const int grid = (int)std::max<unsigned long long>(1, std::min<unsigned long long>(blocks, (unsigned long long)num_sms * 8));
  if (HERM)
    k_apply_direct_herm<T2, K><<<grid, 256, 0, st>>>(rho, S, p);
  else
    k_apply_direct<T2, K><<<grid, 256, 0, st>>>(rho, S, p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_apply(void* rho, int precision, const void* S, const ApplyParams& p, int num_sms,
                         cudaStream_t st, const SparseBlock* sparse) {
  if (precision == 0) {
    double2* r = static_cast<double2*>(rho);
    const double2* s = static_cast<const double2*>(S);
    if (p.sparse && sparse && p.width <= 2) {
      if (p.herm)
        return p.width == 1 ? run_sparse<1, true>(r, sparse, p, num_sms, st) : run_sparse<2, true>(r, sparse, p, num_sms, st);
      return p.width == 1 ? run_sparse<1, false>(r, sparse, p, num_sms, st) : run_sparse<2, false>(r, sparse, p, num_sms, st);
    }
    if (p.herm) {
      switch (p.width) {
        case 1: return run_direct<double2, 1, true>(r, s, p, num_sms, st);
        case 2: return run_direct<double2, 2, true>(r, s, p, num_sms, st);
        case 3: return run_tiled<double2, 3, 32, true, true>(r, s, p, num_sms, st);
        case 4: return run_tiled<double2, 4, 16, false, true>(r, s, p, num_sms, st);
      }
    } else {
      switch (p.width) {
        case 1: return run_direct<double2, 1, false>(r, s, p, num_sms, st);
        case 2: return run_direct<double2, 2, false>(r, s, p, num_sms, st);
        case 3: return run_tiled<double2, 3, 32, true, false>(r, s, p, num_sms, st);
        case 4: return run_tiled<double2, 4, 16, false, false>(r, s, p, num_sms, st);
      }
    }
  } else {
    float2* r = static_cast<float2*>(rho);
    const float2* s = static_cast<const float2*>(S);
    if (p.herm) {
      if (p.width == 1) return run_herm_tiled_split<1>(r, s, p, num_sms, st);
      if (p.width == 2) return launch_herm_tc2(r, s, p, num_sms, st);
      return cudaErrorInvalidValue;  // split Hermitian mode covers widths 1 and 2
    }
    switch (p.width) {
      case 1: return run_direct<float2, 1, false>(r, s, p, num_sms, st);
      case 2: return run_direct<float2, 2, false>(r, s, p, num_sms, st);
      case 3: return run_tiled<float2, 3, 32, true, false>(r, s, p, num_sms, st);
      case 4: return run_tiled<float2, 4, 32, false, false>(r, s, p, num_sms, st);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace tq
