// Planning structures shared by the single-state path and the batch engine
// (CUDA translation units only).
#pragma once

#include <vector>

#include "tq_device.cuh"
#include "tq_internal.h"

namespace tq {

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct DevBuf {
  void* ptr = nullptr;
  size_t cap = 0;
};

struct PinBuf {
  void* ptr = nullptr;
  size_t cap = 0;
};


// Host tables of one planned circuit, packed into a single upload.
struct HostTables {
  std::vector<double2> kraus;
  std::vector<OpDesc> ops;
  std::vector<BlockDesc> blocks;
  std::vector<MemberDesc> members;
  std::vector<FuseWork> work;
  std::vector<SparseWork> spw;  // blocks applied from row lists (FP64)
  long long sop_entries = 0;
  long long sb_entries = 0;
};


}  // namespace tq

// A planned circuit: host-side launch parameters plus device tables.
struct tq_program {
  int n = 0;
  int prec = 0;
  size_t n_ops = 0;   // ops of the circuit
  size_t n_uops = 0;  // distinct op descriptors (superoperators built): identical named ops share one
  int max_width = 0;
  int max_dim2 = 0;
  int n_work = 0;
  std::vector<tq::ApplyParams> params;  // per block
  std::vector<long long> sb_off;    // per block, complex entries
  std::vector<int> sp_slot;         // per block: row-list slot, or -1 (dense)
  std::vector<int> nnz;             // per block: structural nonzeros (D*D if dense)
  int n_sparse = 0;
  // device tables (one blob: Kraus sets, op/block/member/work tables)
  tq::DevBuf blob, sops, sb64, sb32, sps;
  size_t o_kraus = 0, o_ops = 0, o_blk = 0, o_mem = 0, o_work = 0, o_spw = 0, blob_bytes = 0;
  bool owns = true;  // standalone programs own their buffers
  // tq_program_run replays the program's whole launch sequence as a CUDA
  // graph, captured once per (rho, Hermitian-mode entry flags): the graph
  // bakes in the state's buffer and the per-block Hermitian decisions
  mutable cudaGraphExec_t g_exec = nullptr;
  mutable cudaStream_t g_capture = nullptr;  // private stream the graph is captured on
  mutable const void* g_rho = nullptr;
  mutable int g_key = -1;                    // herm allowed | lower stale on entry << 1
  mutable bool g_lower_after = false;
  mutable unsigned long long g_launches = 0;
  // device table of the blocks for the cluster path (small registers)
  mutable tq::DevBuf g_blk;
  mutable bool g_blk_ready = false;
};


namespace tq {

ApplyParams apply_params(int n, const Block& B);

// Validate, resolve and plan `ops` into P's host fields and `t`. f64_tensor:
// plan FP64 blocks for the tensor-core engine (its cost model).
tq_status plan_program(int n, int prec, const tq_op* ops, size_t n_ops, int width, tq_program* P, HostTables* t,
                       bool f64_tensor = false);

void pack_blob(const tq_program& P, const HostTables& t, char* h);

}  // namespace tq
