// Internal declarations shared by the library's translation units.
#pragma once

#include <complex>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/tanq.h"

namespace tq {

using cplx = std::complex<double>;

constexpr int kMaxQubits = 16;   // 16 * 4^16 B = 64 GiB in FP64
constexpr int kMaxWidth = 4;     // widest fused superoperator (256 x 256)

// An op resolved to an explicit Kraus set (a unitary is a set of one).
struct ResolvedOp {
  int k = 0;
  int qubits[4] = {0, 0, 0, 0};
  std::vector<cplx> kraus;  // m matrices of 2^k x 2^k, row-major
  int m = 0;
};

// Structural nonzero pattern of a superoperator on at most 2 qubits
// (D = 4^width <= 16 local indices): bit j of row[i] is set when S[i][j]
// may be nonzero. Used only for planning and kernel choice.
struct Pattern {
  int width = 0;
  uint16_t row[16] = {};
};

// One fused block: an ordered qubit list (local bit j = qubits[j]) and the
// ops it composes, in circuit order. has_pat: pat is the block's pattern
// (blocks of at most 2 qubits whose ops all have patterns).
struct Block {
  int width = 0;
  int qubits[4] = {0, 0, 0, 0};
  std::vector<int> ops;
  bool has_pat = false;
  Pattern pat;
};

// An op as the planner sees it.
struct PlanOp {
  std::vector<int> qubits;
  bool has_pat = false;
  Pattern pat;
};

// Structural pattern of an op's superoperator S = sum conj(K) (x) K (ops on
// at most 2 qubits; false otherwise). Depolarising channels use their exact
// pattern (the X and Y Pauli terms cancel on coherence-to-coherence entries).
bool op_pattern(const tq_op& op, const ResolvedOp& r, Pattern* out);
int pattern_nnz(const Pattern& p);
// Sparse apply kernels are used for FP64 blocks of width <= 2 whose pattern
// has at most this fraction of nonzeros.
constexpr double kSparseFraction = 0.75;
bool block_is_sparse(const Block& b, int precision);

// Validate an op against n qubits (qubit range, distinctness, k, m, mats).
tq_status validate_op(int n, const tq_op& op);

// Resolve a (validated) op into its Kraus set, in FP64.
tq_status resolve_op(const tq_op& op, ResolvedOp* out);

// Planning-only precision code: FP64 states whose blocks of width <= 2 run
// on the tensor cores (TQ_ENGINE_TENSOR); their passes are bound by HBM, not
// by the FP64 pipe, so merging ops into blocks of up to 2 qubits is free.
constexpr int kPlanF64Tensor = 16;
// Relative pass time of the tensor-core FP64 engine against an HBM-bound
// pass at the copy bandwidth, in the cost model's units (measured on GB300:
// a 15-qubit width-2 pass takes 5.46 ms against 18.05 ms for the DFMA
// row-list pass of the same 80-nonzero block, which the model prices at 40
// flops per entry at the DFMA rate: 0.302 x (40 / 1.2e12) / (32 / 6.8e12)).
constexpr double kTensorF64PassFactor = 2.14;

// Per-precision cost (arbitrary units per 4^n entries) of one apply pass of
// a block of the given width; nnz < 0 means dense. Used by the automatic
// fusion planner; precision is TQ_FP64, TQ_SPLIT or kPlanF64Tensor.
double block_cost(int width, int precision, int nnz = -1);

// Greedy fusion planner (Sec. 3.3, generalised to blocks of <= max_width
// qubits). max_width 0: one block per op; -1: automatic (cost model).
tq_status plan_fusion(int n, const std::vector<PlanOp>& ops, int max_width, int precision,
                      std::vector<Block>* blocks);

}  // namespace tq
