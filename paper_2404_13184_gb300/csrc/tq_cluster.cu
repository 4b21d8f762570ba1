// Small registers: a program's whole sequence of fused blocks (Sec. 3.1
// apply step, one pass per block) as ONE kernel on a thread-block cluster,
// with vec(rho) held in the cluster's distributed shared memory. Each of the
// C CTAs keeps a C-th of vec(rho) (entries [rank N/C, (rank+1) N/C)) in its
// own shared memory; every CTA applies a C-th of each block's canonical
// groups (Hermitian mode), reading and writing the entries wherever they
// live through the cluster shared-memory window, and a hardware cluster
// barrier with release/acquire semantics separates consecutive blocks. rho
// is loaded from and stored back to global memory once per run, so a pass
// costs on-chip traffic and a barrier instead of a kernel launch and L2
// round trips. The per-group arithmetic follows the batch engine's (FP64
// row lists, split dense products).
#include <algorithm>
#include <mutex>
#include <vector>

#include "tq_batch_kernels.cuh"

namespace tq {
namespace {

using namespace tq::batch;

constexpr int kClusterLog2 = 3;
constexpr int kClusterCtas = 1 << kClusterLog2;  // portable cluster size

// Staging next to the slice: the superoperator (or its row-list values)
// and one operand slot per thread.
template <typename T2>
__host__ __device__ constexpr size_t cluster_smem() {
  return (kSEntries + kThreads) * sizeof(T2);
}

// Largest slice of vec(rho) per CTA next to the staging buffers.
template <typename T2>
constexpr size_t max_slice_bytes() {
  return 227 * 1024 - cluster_smem<T2>() - 4096;
}

__device__ __forceinline__ unsigned mapa(unsigned local, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Accessors of vec(rho) in the cluster window: entry e lives in CTA
// e >> slice_log2 at local index e & (slice - 1); base[c] is the window
// address of CTA c's slice.
struct Dsm {
  const unsigned* base;
  int slice_log2;
  __device__ __forceinline__ unsigned addr(unsigned long long e, unsigned esz) const {
    return base[e >> slice_log2] + (unsigned)(e & ((1ull << slice_log2) - 1ull)) * esz;
  }
};

__device__ __forceinline__ double2 dsm_ld(unsigned a, double2*) {
  double2 v;
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ float2 dsm_ld(unsigned a, float2*) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void dsm_st(unsigned a, double2 v) {
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v.x), "d"(v.y) : "memory");
}
__device__ __forceinline__ void dsm_st(unsigned a, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}

// One canonical group of a width-K block, entries in the cluster window,
// spread over D = 4^K consecutive lanes of a warp: lane l of the group loads
// entry l (conjugating one read through its transpose) into its slot of
// sX, and after a warp barrier over the group's lanes computes output row l
// from the group's slots (FP64: over the row list of nonzeros; split:
// dense), then stores it; a second warp barrier keeps the slots until every
// lane of the group has read them. Every load of a group precedes its
// stores. A self-conjugate group stores its upper entries only.
template <typename T2, int K>
__device__ __forceinline__ void cluster_group_row(const Dsm& rho, unsigned long long t, int l, unsigned gmask,
                                                  const ApplyParams& p, const T2* sS, const RowLists& rl, T2* sX) {
  constexpr int D = 1 << (2 * K);
  constexpr bool kF64 = sizeof(T2) == 16;
  bool self = false;
  unsigned long long base = canonical_group(t, p.n - K, &self);
#pragma unroll
  for (int i = 0; i < 2 * K; ++i) {
    const unsigned long long low = base & ((1ull << p.pos[i]) - 1ull);
    base = ((base >> p.pos[i]) << (p.pos[i] + 1)) | low;
  }
  const unsigned rmask = (1u << p.n) - 1u;
  const unsigned rb = (unsigned)(base & rmask), cb = (unsigned)(base >> p.n);
  const unsigned r = rb + (unsigned)(p.off[l] & rmask), c = cb + (unsigned)(p.off[l] >> p.n);
  const bool cj = r > c;
  const unsigned a = rho.addr(cj ? ((unsigned long long)c | ((unsigned long long)r << p.n))
                                 : ((unsigned long long)r | ((unsigned long long)c << p.n)),
                              sizeof(T2));
  T2 xv = dsm_ld(a, (T2*)nullptr);
  if (cj) xv.y = -xv.y;
  sX[threadIdx.x] = xv;
  __syncwarp(gmask);
  const T2* gx = sX + (threadIdx.x & ~(D - 1));  // the group's entries
  T2 acc;
  acc.x = 0;
  acc.y = 0;
  if constexpr (kF64) {
    for (int k = rl.rowptr[l]; k < rl.rowptr[l + 1]; ++k) Cx<double2>::fma(acc, sS[k], gx[rl.col[k]]);
  } else {
#pragma unroll
    for (int j = 0; j < D; ++j) Cx<T2>::fma(acc, sS[l * D + j], gx[j]);
  }
  __syncwarp(gmask);
  if (cj) {
    if (self) return;
    acc.y = -acc.y;
  }
  dsm_st(a, acc);
}

// A block as the cluster kernel sees it: width and qubits packed in wq
// (width | q0 << 8 | q1 << 16) and the offset of its superoperator in the
// fused table (entries). The per-group offsets are derived on the device.
struct CBlk {
  unsigned wq;
  unsigned pad;
  unsigned long long s_off;
};

// Fill the apply parameters of a width-w block on qubits (q0, q1) of an
// n-qubit register in Hermitian mode (as apply_params on the host).
__device__ __forceinline__ void cluster_params(unsigned wq, int n, ApplyParams* p) {
  const int w = wq & 0xff, q[2] = {(int)((wq >> 8) & 0xff), (int)((wq >> 16) & 0xff)};
  const int D = 1 << (2 * w);
  if (threadIdx.x < D) {
    unsigned long long v = 0;
    for (int j = 0; j < w; ++j) {
      if ((threadIdx.x >> j) & 1) v |= 1ull << q[j];
      if ((threadIdx.x >> (w + j)) & 1) v |= 1ull << (q[j] + n);
    }
    p->off[threadIdx.x] = v;
  }
  if (threadIdx.x == 0) {
    int pos[4];
    for (int j = 0; j < w; ++j) {
      p->q[j] = q[j];
      pos[2 * j] = q[j];
      pos[2 * j + 1] = q[j] + n;
    }
    for (int a = 0; a < 2 * w; ++a)  // ascending
      for (int b = 0; b + 1 < 2 * w; ++b)
        if (pos[b] > pos[b + 1]) {
          const int t = pos[b];
          pos[b] = pos[b + 1];
          pos[b + 1] = t;
        }
    for (int a = 0; a < 2 * w; ++a) p->pos[a] = pos[a];
    p->n = n;
    p->width = w;
    p->npos = 2 * w;
    p->n_groups = 1ull << (2 * (n - w));
    const unsigned long long M = 1ull << (n - w);
    p->herm = 1;
    p->n_canon = M * (M + 1) / 2;
  }
}

template <typename T2>
__global__ void __launch_bounds__(kThreads, 1) k_cluster_program(T2* rho, const T2* __restrict__ sb,
                                                                 const CBlk* __restrict__ tab, int n_blocks, int n) {
  extern __shared__ __align__(16) unsigned char smem[];
  T2* sS = reinterpret_cast<T2*>(smem);
  T2* sX = sS + kSEntries;                                      // one operand slot per thread
  T2* sRho = reinterpret_cast<T2*>(smem + cluster_smem<T2>());  // this CTA's slice of vec(rho)
  __shared__ ApplyParams s_p;
  __shared__ RowLists s_rl;
  __shared__ int s_cnt[16];
  __shared__ unsigned s_base[kClusterCtas];
  constexpr bool kF64 = sizeof(T2) == 16;
  const int tid = threadIdx.x;
  const unsigned rank = cluster_rank();
  const int slice_log2 = 2 * n - kClusterLog2;
  const unsigned long long slice = 1ull << slice_log2;
  if (tid < kClusterCtas) s_base[tid] = mapa((unsigned)__cvta_generic_to_shared(sRho), tid);
  for (unsigned long long e = tid; e < slice; e += kThreads) sRho[e] = __ldcg(&rho[rank * slice + e]);
  // two-stage prefetch: the table entry two blocks ahead and this thread's
  // superoperator entry one block ahead, loaded while a block computes
  CBlk cur = tab[0], nxt = n_blocks > 1 ? tab[1] : CBlk{};
  T2 sv;
  sv.x = 0;
  sv.y = 0;
  if (tid < (1 << (4 * (cur.wq & 0xff)))) sv = sb[cur.s_off + tid];
  cluster_sync();  // every slice loaded before any CTA reads another's
  const Dsm win{s_base, slice_log2};
  for (int b = 0; b < n_blocks; ++b) {
    // stage block b from registers: parameters, superoperator (FP64: row lists)
    const int w = cur.wq & 0xff, D = 1 << (2 * w);
    cluster_params(cur.wq, n, &s_p);
    if constexpr (kF64) {
      // entry tid = (row i, column j) of S; a row's nonzero mask by ballot
      const bool in = tid < D * D;
      const unsigned long long* bits = reinterpret_cast<const unsigned long long*>(&sv);
      const bool nz = in && ((bits[0] | bits[1]) << 1) != 0ull;
      const unsigned ball = __ballot_sync(0xffffffffu, nz);
      const int i = in ? tid / D : 0, j = in ? tid % D : 0;
      const unsigned row_mask = (ball >> ((tid & 31) & ~(D - 1))) & ((1u << D) - 1u);  // D divides 32
      if (in && j == 0) s_cnt[i] = __popc(row_mask);
      __syncthreads();
      if (tid == 0) {
        int run = 0;
        for (int r = 0; r < D; ++r) {
          s_rl.rowptr[r] = run;
          run += s_cnt[r];
        }
        s_rl.rowptr[D] = run;
      }
      __syncthreads();
      if (nz) {
        const int k = s_rl.rowptr[i] + __popc(row_mask & ((1u << j) - 1u));
        sS[k] = sv;
        s_rl.col[k] = (unsigned char)j;
      }
    } else {
      if (tid < D * D) sS[tid] = sv;
    }
    __syncthreads();
    // prefetch: superoperator of block b+1, table entry of block b+2
    T2 sv_next;
    sv_next.x = 0;
    sv_next.y = 0;
    CBlk nxt2 = nxt;
    if (b + 1 < n_blocks && tid < (1 << (4 * (nxt.wq & 0xff)))) sv_next = sb[nxt.s_off + tid];
    if (b + 2 < n_blocks) nxt2 = tab[b + 2];
    const unsigned long long total = s_p.n_canon;
    const unsigned long long g0 = total * rank / kClusterCtas, g1 = total * (rank + 1) / kClusterCtas;
    // D lanes per group, 256 / D groups per pass over the CTA's threads; all
    // lanes of a group take the same groups, so the warp barriers match
    const int l = tid & (D - 1), lane0 = (tid & 31) & ~(D - 1);
    const unsigned gmask = ((1u << D) - 1u) << lane0;
    for (unsigned long long g = g0 + (unsigned long long)(tid >> (2 * w)); g < g1; g += kThreads >> (2 * w)) {
      if (w == 1)
        cluster_group_row<T2, 1>(win, g, l, gmask, s_p, sS, s_rl, sX);
      else
        cluster_group_row<T2, 2>(win, g, l, gmask, s_p, sS, s_rl, sX);
    }
    cluster_sync();  // every group of block b is written before block b+1 reads
    cur = nxt;
    nxt = nxt2;
    sv = sv_next;
  }
  for (unsigned long long e = tid; e < slice; e += kThreads) rho[rank * slice + e] = sRho[e];
  cluster_sync();  // no CTA leaves while others may still read its slice
}

template <typename T2>
cudaError_t launch(T2* rho, const T2* sb, const CBlk* tab, int n_blocks, int n, cudaStream_t st) {
  const size_t slice_bytes = sizeof(T2) << (2 * n - kClusterLog2);
  if (slice_bytes > max_slice_bytes<T2>()) return cudaErrorInvalidValue;
  const size_t smem = cluster_smem<T2>() + slice_bytes;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(k_cluster_program<T2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(cluster_smem<T2>() + max_slice_bytes<T2>()));
  });
  if (attr_err != cudaSuccess) return attr_err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kClusterCtas);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterCtas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_cluster_program<T2>, rho, sb, tab, n_blocks, n);
}

}  // namespace

bool cluster_program_eligible(int n, int max_width, size_t n_blocks) {
  // vec(rho) fits the cluster's shared memory (8 qubits: 1 MiB in FP64, an
  // eighth per CTA), every block of width <= 2 has a Hermitian per-group
  // form, and there is more than one pass to save
  return n >= 2 && n <= 8 && max_width <= 2 && n_blocks >= 2;
}

void cluster_block_table(const std::vector<ApplyParams>& params, const std::vector<long long>& sb_off,
                         std::vector<unsigned char>* out) {
  std::vector<CBlk> tab(params.size());
  for (size_t b = 0; b < params.size(); ++b) {
    const ApplyParams& p = params[b];
    tab[b].wq = (unsigned)p.width | ((unsigned)p.q[0] << 8) | ((unsigned)(p.width > 1 ? p.q[1] : 0) << 16);
    tab[b].pad = 0;
    tab[b].s_off = (unsigned long long)sb_off[b];
  }
  out->assign(reinterpret_cast<const unsigned char*>(tab.data()),
              reinterpret_cast<const unsigned char*>(tab.data()) + tab.size() * sizeof(CBlk));
}

cudaError_t launch_cluster_program(void* rho, int precision, int n, const void* sb, const void* tab, int n_blocks,
                                   cudaStream_t st) {
  if (precision == 0)
    return launch<double2>(static_cast<double2*>(rho), static_cast<const double2*>(sb), static_cast<const CBlk*>(tab),
                           n_blocks, n, st);
  return launch<float2>(static_cast<float2*>(rho), static_cast<const float2*>(sb), static_cast<const CBlk*>(tab),
                        n_blocks, n, st);
}

}  // namespace tq
