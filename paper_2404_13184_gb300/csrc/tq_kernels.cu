// Superoperator construction, fusion, readout reductions and small utility
// kernels (sm_103a). Everything here runs in FP64.
#include <algorithm>

#include "tq_device.cuh"

namespace tq {

namespace {

__device__ __forceinline__ double2 cmul_conj_a(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

// S = sum_t conj(K_t) (x) K_t (Sec. 3.1): with local index l = r + d*c (d =
// 2^k), S[r' + d c'][r + d c] = sum_t conj(K_t[c'][c]) * K_t[r'][r].
__global__ void __launch_bounds__(256) k_build_superops(const double2* __restrict__ kraus,
                                                        const OpDesc* __restrict__ ops, int op0,
                                                        double2* __restrict__ sops) {
  const OpDesc od = ops[op0 + blockIdx.y];
  const int d = 1 << od.k;
  const int D = d * d;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= D * D) return;
  const int i = e / D, j = e % D;
  const int rp = i % d, cp = i / d, r = j % d, c = j / d;
  double2 acc = make_double2(0.0, 0.0);
  const double2* K = kraus + od.kraus_off;
  for (int t = 0; t < od.m; ++t) {
    const double2 a = K[(long long)t * d * d + cp * d + c];
    const double2 b = K[(long long)t * d * d + rp * d + r];
    const double2 p = cmul_conj_a(a, b);
    acc.x += p.x;
    acc.y += p.y;
  }
  sops[od.sop_off + e] = acc;
}

constexpr int kFuseEntries = 1024;  // complex entries per ping-pong buffer

// Fusion (Sec. 3.3, generalised): S_block = S_last ... S_first, each member
// superoperator embedded at its qubits' block-local positions. Columns of
// S_block are independent: column l starts as the unit vector e_l and every
// member is applied to it in circuit order, out of place between two shared
// memory buffers. One CTA owns C columns of one block.
__global__ void __launch_bounds__(256) k_fuse(const double2* __restrict__ sops,
                                              const OpDesc* __restrict__ ops,
                                              const BlockDesc* __restrict__ blocks,
                                              const MemberDesc* __restrict__ members,
                                              const FuseWork* __restrict__ work,
                                              double2* __restrict__ sb64, float2* __restrict__ sb32) {
  __shared__ double2 buf0[kFuseEntries];
  __shared__ double2 buf1[kFuseEntries];
  __shared__ int dep[256];
  const FuseWork w = work[blockIdx.x];
  const BlockDesc b = blocks[w.block];
  const int W = b.width;
  const int D = 1 << (2 * W);
  const int C = min(D, kFuseEntries / D);
  const int ncols = min(C, D - w.col0);
  double2* A = buf0;
  double2* B = buf1;
  for (int e = threadIdx.x; e < ncols * D; e += blockDim.x) {
    const int c = e / D, i = e % D;
    A[e] = make_double2(i == w.col0 + c ? 1.0 : 0.0, 0.0);
  }
  for (int mi = 0; mi < b.n_members; ++mi) {
    const MemberDesc md = members[b.member_off + mi];
    const OpDesc od = ops[md.op];
    const int k = md.k;
    const int Dp = 1 << (2 * k);
    unsigned mask = 0;
    for (int j = 0; j < k; ++j) mask |= (1u << md.pos[j]) | (1u << (md.pos[j] + W));
    // block-index offset of every op-local index
    for (int l = threadIdx.x; l < Dp; l += blockDim.x) {
      int v = 0;
      for (int j = 0; j < k; ++j) {
        if ((l >> j) & 1) v |= 1 << md.pos[j];
        if ((l >> (k + j)) & 1) v |= 1 << (md.pos[j] + W);
      }
      dep[l] = v;
    }
    __syncthreads();
    const double2* S = sops + od.sop_off;
    for (int e = threadIdx.x; e < ncols * D; e += blockDim.x) {
      const int c = e / D, i = e % D;
      int lout = 0;
      for (int j = 0; j < k; ++j) {
        lout |= ((i >> md.pos[j]) & 1) << j;
        lout |= ((i >> (md.pos[j] + W)) & 1) << (k + j);
      }
      const int base = i & ~(int)mask;
      double2 acc = make_double2(0.0, 0.0);
      const double2* Srow = S + (long long)lout * Dp;
      for (int lin = 0; lin < Dp; ++lin) cfma(acc, __ldg(&Srow[lin]), A[c * D + (base | dep[lin])]);
      B[e] = acc;
    }
    __syncthreads();
    double2* t = A;
    A = B;
    B = t;
  }
  for (int e = threadIdx.x; e < ncols * D; e += blockDim.x) {
    const int c = e / D, i = e % D;
    const long long o = b.sb_off + (long long)i * D + w.col0 + c;
    sb64[o] = A[e];
    if (sb32) sb32[o] = make_float2((float)A[e].x, (float)A[e].y);
  }
}

// One CTA per sparse block: row i's nonzeros (exactly zero entries of the
// fused FP64 superoperator are dropped) in column order.
__global__ void k_compress_sparse(const double2* __restrict__ sb64, const BlockDesc* __restrict__ blocks,
                                  const SparseWork* __restrict__ work, SparseBlock* __restrict__ out) {
  __shared__ int cnt[16];
  const SparseWork w = work[blockIdx.x];
  const BlockDesc b = blocks[w.block];
  const int D = 1 << (2 * b.width);
  const double2* S = sb64 + b.sb_off;
  SparseBlock* o = out + w.slot;
  const int i = threadIdx.x;
  if (i < D) {
    int c = 0;
    for (int j = 0; j < D; ++j) {
      const double2 v = S[i * D + j];
      c += (v.x != 0.0 || v.y != 0.0) ? 1 : 0;
    }
    cnt[i] = c;
  }
  __syncthreads();
  if (i == 0) {
    int acc = 0;
    for (int r = 0; r < D; ++r) {
      o->rowptr[r] = acc;
      acc += cnt[r];
    }
    o->rowptr[D] = acc;
  }
  __syncthreads();
  if (i < D) {
    int k = o->rowptr[i];
    for (int j = 0; j < D; ++j) {
      const double2 v = S[i * D + j];
      if (v.x != 0.0 || v.y != 0.0) {
        o->e[k].v = v;
        o->e[k].col = j;
        ++k;
      }
    }
  }
}

__global__ void k_set_one(void* rho, int precision) {
  if (precision == 0)
    reinterpret_cast<double2*>(rho)[0] = make_double2(1.0, 0.0);
  else
    reinterpret_cast<float2*>(rho)[0] = make_float2(1.0f, 0.0f);
}

constexpr int kRedThreads = 256;
constexpr int kMaxQuant = 18;  // Re tr, Im tr and up to 16 masks per launch

// Per-CTA partial sums over a fixed contiguous range of diagonal indices x
// (vec index x (2^n + 1)), each thread in a fixed stride order, then a fixed
// shared-memory tree: the result depends only on n and the grid size.
template <typename T2>
__global__ void __launch_bounds__(kRedThreads) k_diag_partial(const T2* __restrict__ rho, int n,
                                                              const unsigned long long* __restrict__ masks,
                                                              int n_masks, double* __restrict__ partials) {
  __shared__ double red[kMaxQuant][kRedThreads];
  __shared__ unsigned long long s_masks[16];
  if (threadIdx.x < n_masks) s_masks[threadIdx.x] = masks[threadIdx.x];
  __syncthreads();
  const unsigned long long N = 1ull << n;
  const unsigned long long chunk = (N + gridDim.x - 1) / gridDim.x;
  const unsigned long long x0 = blockIdx.x * chunk;
  const unsigned long long x1 = min(N, x0 + chunk);
  double acc[kMaxQuant];
#pragma unroll
  for (int q = 0; q < kMaxQuant; ++q) acc[q] = 0.0;
  for (unsigned long long x = x0 + threadIdx.x; x < x1; x += kRedThreads) {
    const T2 v = rho[x * (N + 1)];
    const double re = (double)v.x, im = (double)v.y;
    acc[0] += re;
    acc[1] += im;
#pragma unroll
    for (int q = 0; q < 16; ++q)
      if (q < n_masks) acc[2 + q] += (__popcll(x & s_masks[q]) & 1) ? -re : re;
  }
  const int nq = 2 + n_masks;
#pragma unroll
  for (int q = 0; q < kMaxQuant; ++q)
    if (q < nq) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int q = 0; q < nq; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < nq) partials[blockIdx.x * nq + threadIdx.x] = red[threadIdx.x][0];
}

// Sums the per-CTA partials in CTA order. With `normalize`, the masked sums
// are divided by Re Tr(rho) (FP64 trace renormalisation of split states).
// `masked_out` (optional) receives the masked sums alone.
__global__ void k_reduce_final(const double* __restrict__ partials, int nblocks, int nq, int normalize,
                               double* __restrict__ out, double* __restrict__ masked_out) {
  __shared__ double tot[kMaxQuant];
  const int q = threadIdx.x;
  if (q < nq) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[b * nq + q];
    tot[q] = s;
  }
  __syncthreads();
  if (q < nq) {
    const double v = (normalize && q >= 2) ? tot[q] / tot[0] : tot[q];
    out[q] = v;
    if (masked_out && q >= 2) masked_out[q - 2] = v;
  }
}

template <typename T2>
__global__ void k_diag_probs(const T2* __restrict__ rho, int n, const double* __restrict__ trace,
                             double* __restrict__ out) {
  const unsigned long long N = 1ull << n;
  const double scale = trace ? 1.0 / trace[0] : 1.0;
  for (unsigned long long x = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; x < N;
       x += (unsigned long long)gridDim.x * blockDim.x)
    out[x] = (double)rho[x * (N + 1)].x * scale;
}

template <typename T2>
__global__ void k_mirror_lower(T2* rho, int n) {
  const unsigned long long N = 1ull << n, total = N * N;
  for (unsigned long long e = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; e < total;
       e += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long r = e & (N - 1), c = e >> n;
    if (r > c) {
      T2 v = rho[c | (r << n)];
      v.y = -v.y;
      rho[e] = v;
    }
  }
}

template <typename T2>
__global__ void __launch_bounds__(256) k_hermiticity(const T2* __restrict__ rho, int n, double* out) {
  __shared__ double s_d[256], s_m[256];
  const unsigned long long N = 1ull << n, total = N * N;
  double d = 0.0, m = 0.0;
  for (unsigned long long e = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; e < total;
       e += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long r = e & (N - 1), c = e >> n;
    const T2 v = rho[e];
    m = fmax(m, fmax(fabs((double)v.x), fabs((double)v.y)));
    if (r < c) {
      const T2 w = rho[c | (r << n)];
      d = fmax(d, fmax(fabs((double)v.x - (double)w.x), fabs((double)v.y + (double)w.y)));
    } else if (r == c) {
      d = fmax(d, fabs((double)v.y));
    }
  }
  s_d[threadIdx.x] = d;
  s_m[threadIdx.x] = m;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      s_d[threadIdx.x] = fmax(s_d[threadIdx.x], s_d[threadIdx.x + s]);
      s_m[threadIdx.x] = fmax(s_m[threadIdx.x], s_m[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(s_d[0]));
    atomicMax(reinterpret_cast<unsigned long long*>(out + 1), (unsigned long long)__double_as_longlong(s_m[0]));
  }
}

__global__ void k_f64_to_f32(const double* __restrict__ in, float* __restrict__ out, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
__global__ void k_f32_to_f64(const float* __restrict__ in, double* __restrict__ out, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

}  // namespace

cudaError_t launch_build_superops(const double2* kraus, const OpDesc* ops, int n_ops, int max_dim2,
                                  double2* sops, cudaStream_t st) {
  const int gx = (max_dim2 + 255) / 256;
  for (int op0 = 0; op0 < n_ops; op0 += 65535) {
    const int cnt = std::min(65535, n_ops - op0);
    k_build_superops<<<dim3(gx, cnt), 256, 0, st>>>(kraus, ops, op0, sops);
  }
  return cudaGetLastError();
}

cudaError_t launch_fuse(const double2* sops, const OpDesc* ops, const BlockDesc* blocks,
                        const MemberDesc* members, const FuseWork* work, int n_work, double2* sb64,
                        float2* sb32, cudaStream_t st) {
  if (n_work <= 0) return cudaSuccess;
  k_fuse<<<n_work, 256, 0, st>>>(sops, ops, blocks, members, work, sb64, sb32);
  return cudaGetLastError();
}

cudaError_t launch_compress_sparse(const double2* sb64, const BlockDesc* blocks, const SparseWork* work, int n_work,
                                   SparseBlock* out, cudaStream_t st) {
  if (n_work <= 0) return cudaSuccess;
  k_compress_sparse<<<n_work, 32, 0, st>>>(sb64, blocks, work, out);
  return cudaGetLastError();
}

cudaError_t launch_init_zero_state(void* rho, int n, int precision, cudaStream_t st) {
  const size_t bytes = (size_t)(precision == 0 ? 16 : 8) << (2 * n);
  cudaError_t e = cudaMemsetAsync(rho, 0, bytes, st);
  if (e != cudaSuccess) return e;
  k_set_one<<<1, 1, 0, st>>>(rho, precision);
  return cudaGetLastError();
}

int build_superops_launches(int n_ops) { return (n_ops + 65534) / 65535; }

int diag_reduce_grid(int n) {
  const long long N = 1ll << n;
  return (int)std::max(1ll, std::min(152ll, N / 512));
}

cudaError_t launch_diag_reduce(const void* rho, int n, int precision, const unsigned long long* masks,
                               int n_masks, double* partials, double* out, bool normalize, double* masked_out,
                               cudaStream_t st) {
  if (n_masks < 0 || n_masks > 16) return cudaErrorInvalidValue;
  const int grid = diag_reduce_grid(n);
  if (precision == 0)
    k_diag_partial<double2><<<grid, kRedThreads, 0, st>>>((const double2*)rho, n, masks, n_masks, partials);
  else
    k_diag_partial<float2><<<grid, kRedThreads, 0, st>>>((const float2*)rho, n, masks, n_masks, partials);
  k_reduce_final<<<1, 32, 0, st>>>(partials, grid, 2 + n_masks, normalize ? 1 : 0, out, masked_out);
  return cudaGetLastError();
}

cudaError_t launch_diag_probs(const void* rho, int n, int precision, const double* trace_or_null,
                              double* out, cudaStream_t st) {
  const long long N = 1ll << n;
  const int grid = (int)std::min<long long>(1216, (N + 255) / 256);
  if (precision == 0)
    k_diag_probs<double2><<<grid, 256, 0, st>>>((const double2*)rho, n, trace_or_null, out);
  else
    k_diag_probs<float2><<<grid, 256, 0, st>>>((const float2*)rho, n, trace_or_null, out);
  return cudaGetLastError();
}

cudaError_t launch_mirror_lower(void* rho, int n, int precision, cudaStream_t st) {
  const unsigned long long total = 1ull << (2 * n);
  const int grid = (int)std::min<unsigned long long>(152 * 16, (total + 255) / 256);
  if (precision == 0)
    k_mirror_lower<double2><<<grid, 256, 0, st>>>(static_cast<double2*>(rho), n);
  else
    k_mirror_lower<float2><<<grid, 256, 0, st>>>(static_cast<float2*>(rho), n);
  return cudaGetLastError();
}

cudaError_t launch_hermiticity(const void* rho, int n, int precision, double* out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  const unsigned long long total = 1ull << (2 * n);
  const int grid = (int)std::min<unsigned long long>(152 * 8, (total + 255) / 256);
  if (precision == 0)
    k_hermiticity<double2><<<grid, 256, 0, st>>>(static_cast<const double2*>(rho), n, out);
  else
    k_hermiticity<float2><<<grid, 256, 0, st>>>(static_cast<const float2*>(rho), n, out);
  return cudaGetLastError();
}

cudaError_t launch_convert_f64_to_f32(const double* in, float* out, size_t count, cudaStream_t st) {
  if (!count) return cudaSuccess;
  const int grid = (int)std::min<size_t>(4864, (count + 255) / 256);
  k_f64_to_f32<<<grid, 256, 0, st>>>(in, out, count);
  return cudaGetLastError();
}

cudaError_t launch_convert_f32_to_f64(const float* in, double* out, size_t count, cudaStream_t st) {
  if (!count) return cudaSuccess;
  const int grid = (int)std::min<size_t>(4864, (count + 255) / 256);
  k_f32_to_f64<<<grid, 256, 0, st>>>(in, out, count);
  return cudaGetLastError();
}

}  // namespace tq
