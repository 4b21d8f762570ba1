// Device-side types and kernel entry points shared by the library's CUDA
// translation units (sm_103a).
#pragma once

#include <vector>

#include <cuda_runtime.h>
#include <cstdint>

namespace tq {

// One op after resolution: k qubits, m Kraus matrices at kraus_off (complex
// units) in the uploaded Kraus blob, its superoperator at sop_off.
struct OpDesc {
  int k;
  int m;
  long long kraus_off;
  long long sop_off;
};

// One fused block: `width` qubits, members [member_off, member_off +
// n_members) in the member table, fused superoperator at sb_off (complex
// units; D x D row-major with D = 4^width).
struct BlockDesc {
  int width;
  int n_members;
  int member_off;
  int pad;
  long long sb_off;
};

// A member op of a block: which op, and the block-local position of each of
// its qubits (op local bit j sits at block local bit pos[j]).
struct MemberDesc {
  int op;
  int k;
  int pos[4];
};

// Work item of the fusion kernel: block index and first column.
struct FuseWork {
  int block;
  int col0;
};

// Launch parameters of one apply pass of a width-K block over vec(rho).
// pos: the 2K target bit positions, ascending (for the group-base deposit).
// off: vec offset of every local index l < 4^K (direct kernels, K <= 2).
// q:   block qubits in local order (row bits; column bits are q + n).
struct ApplyParams {
  unsigned long long n_groups;
  int n;
  int width;
  int npos;
  int pos[8];
  int q[4];
  unsigned long long off[16];
  // Hermitian mode: rho = rho^dagger is kept exactly by computing only the
  // canonical groups (row rest a <= column rest b, n_canon of them) and
  // storing only entries with row <= column (see tq_apply.cu).
  int herm;
  int sparse;  // FP64 blocks of width <= 2: apply from the block's row lists
  unsigned long long n_canon;
};

// Row lists of a sparse FP64 superoperator (width <= 2, D <= 16): the
// nonzeros of row i are e[rowptr[i] .. rowptr[i+1]).
struct SparseEntry {
  double2 v;
  int col;
  int pad[3];
};
struct SparseBlock {
  int rowptr[17];
  int pad[15];
  SparseEntry e[256];
};

// Work item of the sparse compression: block index and its row-list slot.
struct SparseWork {
  int block;
  int slot;
};

// Group index of the t-th canonical group (a <= b, enumerated column by
// column: t = b (b + 1) / 2 + a); rest_bits = n - width.
__host__ __device__ __forceinline__ unsigned long long canonical_group(unsigned long long t, int rest_bits,
                                                                       bool* self) {
  // FP32 estimate (off by at most one for t < 2^31), corrected exactly in
  // integers; the FP64 pipe stays free for the apply arithmetic. Below 2^30
  // (every register up to 16 qubits) the conversions and the correction are
  // 32-bit: 64-bit integer <-> float conversions run on the FP64 pipe.
  if (t < (1ull << 30)) {
    const unsigned int t32 = (unsigned int)t;
    const float est = (sqrtf(8.0f * (float)t32 + 1.0f) - 1.0f) * 0.5f;
    unsigned int b = est > 0.0f ? (unsigned int)est : 0u;  // b < 46341: (b + 1) (b + 2) < 2^31
    while (b * (b + 1) / 2 > t32) --b;
    while ((b + 1) * (b + 2) / 2 <= t32) ++b;
    const unsigned int a = t32 - b * (b + 1) / 2;
    *self = a == b;
    return (unsigned long long)a | ((unsigned long long)b << rest_bits);
  }
  const float est = (sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f;
  unsigned long long b = est > 0.0f ? (unsigned long long)est : 0ull;
  while (b * (b + 1) / 2 > t) --b;
  while ((b + 1) * (b + 2) / 2 <= t) ++b;
  const unsigned long long a = t - b * (b + 1) / 2;
  *self = a == b;
  return a | (b << rest_bits);
}

// Insert a zero bit at each of the first `npos` positions of `pos`
// (ascending): the base index of group g (Sec. 3.1, index s_i, generalised).
__host__ __device__ __forceinline__ unsigned long long deposit_zeros(unsigned long long g,
                                                                    const int* pos, int npos) {
  for (int i = 0; i < npos; ++i) {
    const unsigned long long low = g & ((1ull << pos[i]) - 1ull);
    g = ((g >> pos[i]) << (pos[i] + 1)) | low;
  }
  return g;
}

// --- kernel launchers (tq_kernels.cu) -------------------------------------
cudaError_t launch_build_superops(const double2* kraus, const OpDesc* ops, int n_ops,
                                  int max_dim2, double2* sops, cudaStream_t st);
cudaError_t launch_fuse(const double2* sops, const OpDesc* ops, const BlockDesc* blocks,
                        const MemberDesc* members, const FuseWork* work, int n_work,
                        double2* sb64, float2* sb32, cudaStream_t st);
cudaError_t launch_init_zero_state(void* rho, int n, int precision, cudaStream_t st);
// Row lists (exact zeros dropped) of the fused FP64 superoperators of the
// listed blocks.
cudaError_t launch_compress_sparse(const double2* sb64, const BlockDesc* blocks, const SparseWork* work, int n_work,
                                   SparseBlock* out, cudaStream_t st);
// Reductions over the diagonal: quantities [Re tr, Im tr, Re Tr(rho Z_mask_i)...]
// partials: gridDim x nq doubles of scratch; out: nq doubles (device).
int diag_reduce_grid(int n);
int build_superops_launches(int n_ops);
cudaError_t launch_diag_reduce(const void* rho, int n, int precision, const unsigned long long* masks,
                               int n_masks, double* partials, double* out, bool normalize, double* masked_out,
                               cudaStream_t st);
cudaError_t launch_diag_probs(const void* rho, int n, int precision, const double* trace_or_null,
                              double* out, cudaStream_t st);
cudaError_t launch_convert_f64_to_f32(const double* in, float* out, size_t count, cudaStream_t st);
cudaError_t launch_convert_f32_to_f64(const float* in, double* out, size_t count, cudaStream_t st);
// Hermitian mode helpers: fill every entry with row > column from the
// conjugate of its transpose; and measure max |rho - rho^dagger| and max
// |rho| (two doubles at out, as non-negative bit patterns via atomicMax).
cudaError_t launch_mirror_lower(void* rho, int n, int precision, cudaStream_t st);
cudaError_t launch_hermiticity(const void* rho, int n, int precision, double* out, cudaStream_t st);

// --- measurement (tq_measure.cu) -------------------------------------------
// Per-qubit readout confusion on 2^n outcome probabilities (host arrays of
// n rates); fixed-order CDF and inverse-CDF sampling of `shots` uniforms.
cudaError_t launch_readout(double* p, int n, const double* e10, const double* e01, cudaStream_t st);
cudaError_t launch_sample(const double* p, int n, double* cdf, const double* u, int shots, unsigned long long* out,
                          cudaStream_t st);

// --- apply kernels (tq_apply.cu) ------------------------------------------
// One pass of a fused block over vec(rho). S: 4^K x 4^K superoperator,
// row-major (double2 for FP64 states, float2 for split states).
// Small registers: all blocks of a program as one kernel on a thread-block
// cluster with vec(rho) in distributed shared memory (tq_cluster.cu).
// eligible: n <= 8, widths <= 2, >= 2 blocks. cluster_block_table: the
// device table of blocks (bytes, to upload): width, qubits and superoperator
// offset in the fused table `sb` (FP64 or FP32 by precision).
bool cluster_program_eligible(int n, int max_width, size_t n_blocks);
void cluster_block_table(const std::vector<ApplyParams>& params, const std::vector<long long>& sb_off,
                         std::vector<unsigned char>* out);
cudaError_t launch_cluster_program(void* rho, int precision, int n, const void* sb, const void* tab, int n_blocks,
                                   cudaStream_t st);
cudaError_t launch_apply(void* rho, int precision, const void* S, const ApplyParams& p,
                         int num_sms, cudaStream_t st, const SparseBlock* sparse = nullptr);
// Split states, width 2, Hermitian mode: the pass on the tcgen05 tensor
// cores (tq_apply_tc.cu); needs n - 2 >= 4.
cudaError_t launch_herm_tc2(float2* rho, const float2* S, const ApplyParams& p, int num_sms, cudaStream_t st);
// Bounded tensor-core waits that gave up since the last call (any state on
// the current device); clears the count. Synchronises `st`.
cudaError_t tc_take_timeouts(unsigned int* count, cudaStream_t st);
// Failure-path test settings of the tensor-core passes (tq_test_tc_wait_limit).
void tc_test_limits(long long* max_tries, int* skip_mma);
// FP64 states, widths 1-2, Hermitian mode: the FP64-accurate pass on the
// tcgen05 tensor cores (tq_apply_oz.cu; a width-1 block runs as S (x) I);
// needs n - 2 >= 4. S: the block's FP64 superoperator (4^w x 4^w).
bool oz_eligible(int n, int width);
// Whether an FP64 engine setting (tq_fp64_engine) means the tensor cores
// (TQ_ENGINE_TENSOR, or TQ_ENGINE_AUTO where the library chooses them).
bool fp64_engine_is_tensor(int engine);
cudaError_t launch_herm_oz(double2* rho, const double2* S, const ApplyParams& p, int num_sms, cudaStream_t st);
cudaError_t oz_take_timeouts(unsigned int* count, cudaStream_t st);

}  // namespace tq
