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

// One fused block: an ordered qubit list (local bit j = qubits[j]) and the
// ops it composes, in circuit order.
struct Block {
  int width = 0;
  int qubits[4] = {0, 0, 0, 0};
  std::vector<int> ops;
};

// Validate an op against n qubits (qubit range, distinctness, k, m, mats).
tq_status validate_op(int n, const tq_op& op);

// Resolve a (validated) op into its Kraus set, in FP64.
tq_status resolve_op(const tq_op& op, ResolvedOp* out);

// Per-precision cost (arbitrary units per 4^n entries) of one apply pass of
// a block of the given width; used by the automatic fusion planner.
double block_cost(int width, int precision);

// Greedy fusion planner (Sec. 3.3, generalised to blocks of <= max_width
// qubits). max_width 0: one block per op; -1: automatic (cost model).
tq_status plan_fusion(int n, const std::vector<std::vector<int>>& op_qubits, int max_width,
                      int precision, std::vector<Block>* blocks);

}  // namespace tq
