// Host-side FP64 pieces of the library: the named gate and channel library
// (Kraus sets, TANQ-Sim Sec. 3.5), op validation, the fusion planner
// (Sec. 3.3) and small helpers. No GPU work happens in this file.
#include <algorithm>
#include <map>
#include <array>
#include <cmath>
#include <cstring>

#include "tq_internal.h"

namespace tq {

namespace {

const double kInvSqrt2 = 0.70710678118654752440;

void put(double* out, int d, int i, int j, cplx v) {
  out[2 * (i * d + j)] = v.real();
  out[2 * (i * d + j) + 1] = v.imag();
}

// Pauli matrices I, X, Y, Z.
const cplx kPauli[4][2][2] = {
    {{1.0, 0.0}, {0.0, 1.0}},
    {{0.0, 1.0}, {1.0, 0.0}},
    {{0.0, cplx(0, -1)}, {cplx(0, 1), 0.0}},
    {{1.0, 0.0}, {0.0, -1.0}},
};

bool finite_all(const double* p, int cnt) {
  for (int i = 0; i < cnt; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

}  // namespace

tq_status validate_op(int n, const tq_op& op) {
  if (op.k < 1 || op.k > kMaxWidth) return TQ_ERR_ARG;
  for (int j = 0; j < op.k; ++j) {
    if (op.qubits[j] < 0 || op.qubits[j] >= n) return TQ_ERR_QUBIT;
    for (int i = 0; i < j; ++i)
      if (op.qubits[i] == op.qubits[j]) return TQ_ERR_QUBIT;
  }
  switch (op.kind) {
    case TQ_OP_UNITARY:
      if (!op.mats) return TQ_ERR_ARG;
      return finite_all(op.mats, 2 << (2 * op.k)) ? TQ_OK : TQ_ERR_ARG;
    case TQ_OP_KRAUS:
      if (!op.mats || op.m < 1 || op.m > 4096) return TQ_ERR_ARG;
      return finite_all(op.mats, op.m * (2 << (2 * op.k))) ? TQ_OK : TQ_ERR_ARG;
    case TQ_OP_GATE:
    case TQ_OP_CHANNEL: {
      ResolvedOp tmp;
      return resolve_op(op, &tmp);
    }
    default:
      return TQ_ERR_ARG;
  }
}

tq_status resolve_op(const tq_op& op, ResolvedOp* out) {
  out->k = op.k;
  for (int j = 0; j < 4; ++j) out->qubits[j] = j < op.k ? op.qubits[j] : 0;
  const int d = 1 << op.k;
  if (op.kind == TQ_OP_UNITARY || op.kind == TQ_OP_KRAUS) {
    out->m = op.kind == TQ_OP_UNITARY ? 1 : op.m;
    out->kraus.resize((size_t)out->m * d * d);
    for (size_t i = 0; i < out->kraus.size(); ++i)
      out->kraus[i] = cplx(op.mats[2 * i], op.mats[2 * i + 1]);
    return TQ_OK;
  }
  if (op.kind == TQ_OP_GATE) {
    double U[32];
    int k = 0;
    tq_status st = tq_gate_matrix(op.name, op.params, &k, U);
    if (st != TQ_OK) return st;
    if (k != op.k) return TQ_ERR_ARG;
    out->m = 1;
    out->kraus.resize(d * d);
    for (int i = 0; i < d * d; ++i) out->kraus[i] = cplx(U[2 * i], U[2 * i + 1]);
    return TQ_OK;
  }
  if (op.kind == TQ_OP_CHANNEL) {
    int m = 0;
    tq_status st = tq_channel_kraus(op.name, op.k, op.params, 0, &m, nullptr);
    if (st != TQ_OK) return st;
    if (m <= 0) return TQ_ERR_ARG;
    std::vector<double> buf((size_t)m * d * d * 2);
    st = tq_channel_kraus(op.name, op.k, op.params, m, &m, buf.data());
    if (st != TQ_OK) return st;
    out->m = m;
    out->kraus.resize((size_t)m * d * d);
    for (size_t i = 0; i < out->kraus.size(); ++i) out->kraus[i] = cplx(buf[2 * i], buf[2 * i + 1]);
    return TQ_OK;
  }
  return TQ_ERR_ARG;
}

namespace {

// Index helpers for patterns: local index l = r + d c (d = 2^w), with bit j
// of r and of c for local qubit j.
int op_index(int i, const int* pos, int k, int W) {
  int r = 0, c = 0;
  for (int j = 0; j < k; ++j) {
    r |= ((i >> pos[j]) & 1) << j;
    c |= ((i >> (pos[j] + W)) & 1) << j;
  }
  return r | (c << k);
}

int rest_of(int i, const int* pos, int k, int W) {
  int m = 0;
  for (int j = 0; j < k; ++j) m |= (1 << pos[j]) | (1 << (pos[j] + W));
  return i & ~m;
}

// Pattern p (width k) placed at block positions pos[0..k-1] of a width-W block.
Pattern embed(const Pattern& p, const int* pos, int W) {
  bool identity = p.width == W;
  for (int j = 0; j < p.width && identity; ++j) identity = pos[j] == j;
  if (identity) return p;
  Pattern o;
  o.width = W;
  const int D = 1 << (2 * W);
  int rest[16], idx[16];
  for (int i = 0; i < D; ++i) {
    rest[i] = rest_of(i, pos, p.width, W);
    idx[i] = op_index(i, pos, p.width, W);
  }
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j)
      if (rest[i] == rest[j] && ((p.row[idx[i]] >> idx[j]) & 1)) o.row[i] |= (uint16_t)(1u << j);
  return o;
}

// later x earlier (both of the same width)
Pattern compose(const Pattern& later, const Pattern& earlier) {
  Pattern o;
  o.width = later.width;
  const int D = 1 << (2 * later.width);
  for (int i = 0; i < D; ++i)
    for (int m = 0; m < D; ++m)
      if ((later.row[i] >> m) & 1) o.row[i] |= earlier.row[m];
  return o;
}

}  // namespace

int pattern_nnz(const Pattern& p) {
  int c = 0;
  for (int i = 0; i < (1 << (2 * p.width)); ++i) c += __builtin_popcount(p.row[i]);
  return c;
}

bool op_pattern(const tq_op& op, const ResolvedOp& r, Pattern* out) {
  if (r.k > 2) return false;
  Pattern p;
  p.width = r.k;
  const int d = 1 << r.k, D = d * d;
  const bool depol = op.kind == TQ_OP_CHANNEL && op.name == TQ_CH_DEPOLARIZING;
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      const int rp = i % d, cp = i / d, rr = j % d, cc = j / d;
      bool nz = false;
      if (depol) {
        nz = (rp == cp && rr == cc) || (rp == rr && cp == cc);
      } else {
        for (int t = 0; t < r.m && !nz; ++t) {
          const cplx* K = r.kraus.data() + (size_t)t * d * d;
          nz = K[rp * d + rr] != cplx(0.0, 0.0) && K[cp * d + cc] != cplx(0.0, 0.0);
        }
      }
      if (nz) p.row[i] |= (uint16_t)(1u << j);
    }
  *out = p;
  return true;
}

bool block_is_sparse(const Block& b, int precision) {
  if ((precision != TQ_FP64 && precision != kPlanF64Tensor) || !b.has_pat || b.width > 2) return false;
  const int D = 1 << (2 * b.width);
  return pattern_nnz(b.pat) <= kSparseFraction * D * D;
}

double block_cost(int width, int precision, int nnz) {
  // Time of one pass over all 4^n entries, relative units, from the measured
  // GB300 rates: HBM ~6.8 TB/s, DFMA ~1.2 TFLOP/s, FFMA ~74 TFLOP/s.
  // A width-k pass moves 2*B bytes per entry and does 8*4^k flops per entry
  // (dense), or 8 * nnz / 4^k with a sparse FP64 superoperator.
  const double hbm = 6.8e12, dfma = 1.2e12, ffma = 74e12;
  if (precision == kPlanF64Tensor) {
    if (width <= 2) return kTensorF64PassFactor * 32.0 / hbm * 1e12;  // any width <= 2: one HBM-bound pass
    precision = TQ_FP64;                                               // wider blocks: the DFMA kernels
  }
  const double bytes = precision == TQ_FP64 ? 32.0 : 16.0;
  const int D = 1 << (2 * width);
  const bool sparse = precision == TQ_FP64 && width <= 2 && nnz >= 0 && nnz <= kSparseFraction * D * D;
  const double flops = sparse ? 8.0 * nnz / D : 8.0 * D;
  const double pipe = precision == TQ_FP64 ? dfma : ffma;
  return std::max(bytes / hbm, flops / pipe) * 1e12;
}

namespace {

double cost_of(const Block& b, int precision) {
  return block_cost(b.width, precision, b.has_pat ? pattern_nnz(b.pat) : -1);
}

// The block B extended by op: its qubit list and (if both have patterns and
// the result is at most 2 wide) its pattern.
Block extended(const Block& B, const PlanOp& op) {
  Block X;
  X.width = B.width;
  for (int j = 0; j < B.width; ++j) X.qubits[j] = B.qubits[j];
  for (int v : op.qubits)
    if (std::find(X.qubits, X.qubits + X.width, v) == X.qubits + X.width) {
      if (X.width < 4) X.qubits[X.width] = v;
      ++X.width;
    }
  X.has_pat = X.width <= 2 && op.has_pat && (B.has_pat || B.ops.empty());
  if (X.has_pat) {
    int pos_b[2] = {0, 1}, pos_o[2] = {0, 0};
    for (size_t j = 0; j < op.qubits.size(); ++j)
      pos_o[j] = (int)(std::find(X.qubits, X.qubits + X.width, op.qubits[j]) - X.qubits);
    const Pattern po = embed(op.pat, pos_o, X.width);
    X.pat = B.ops.empty() ? po : compose(po, embed(B.pat, pos_b, X.width));
  }
  return X;
}

}  // namespace

tq_status plan_fusion(int n, const std::vector<PlanOp>& ops, int max_width, int precision,
                      std::vector<Block>* blocks) {
  blocks->clear();
  if (max_width < -1 || max_width > kMaxWidth) return TQ_ERR_ARG;
  const bool automatic = max_width == -1;
  const int cap = automatic ? kMaxWidth : max_width;
  // last block index that touched each qubit
  std::vector<int> last(n, -1);
  for (size_t i = 0; i < ops.size(); ++i) {
    const std::vector<int>& q = ops[i].qubits;
    const int k = (int)q.size();
    int chosen = -1;
    Block chosen_ext;
    if (max_width != 0 && k <= cap) {
      int barrier = -1;
      for (int v : q) barrier = std::max(barrier, last[v]);
      // Candidates: the barrier block (the latest one sharing a qubit with the
      // op) and every later block, which is disjoint from the op, so the op
      // commutes past the blocks between. Pick the smallest growth (width, or
      // cost in automatic mode); ties go to the latest block.
      const int lo = barrier >= 0 ? barrier : std::max(0, (int)blocks->size() - 8);
      double best_delta = 1e300;
      for (int b = (int)blocks->size() - 1; b >= lo; --b) {
        const Block& B = (*blocks)[b];
        Block X = extended(B, ops[i]);
        if (X.width > cap) continue;
        const double delta = automatic ? cost_of(X, precision) - cost_of(B, precision) : (double)(X.width - B.width);
        if (delta < best_delta - 1e-9) {
          best_delta = delta;
          chosen = b;
          chosen_ext = X;
        }
      }
      // automatic mode merges only when that is no dearer than a pass of its own
      if (automatic && chosen >= 0) {
        Block alone = extended(Block(), ops[i]);
        if (best_delta > cost_of(alone, precision) * (1 + 1e-9)) chosen = -1;
      }
    }
    if (chosen < 0) {
      blocks->push_back(extended(Block(), ops[i]));
      chosen = (int)blocks->size() - 1;
    } else {
      Block& B = (*blocks)[chosen];
      B.width = chosen_ext.width;
      for (int j = 0; j < 4; ++j) B.qubits[j] = chosen_ext.qubits[j];
      B.has_pat = chosen_ext.has_pat;
      B.pat = chosen_ext.pat;
    }
    Block& B = (*blocks)[chosen];
    for (int v : q) last[v] = std::max(last[v], chosen);
    B.ops.push_back((int)i);
  }
  return TQ_OK;
}

}  // namespace tq

using namespace tq;

extern "C" {

tq_status tq_gate_matrix(int gate, const double* params, int* k_out, double* U) {
  if (!k_out || !U) return TQ_ERR_ARG;
  const bool needs_angle = gate == TQ_GATE_RX || gate == TQ_GATE_RY || gate == TQ_GATE_RZ ||
                           gate == TQ_GATE_RZZ || gate == TQ_GATE_SU2;
  if (needs_angle && !params) return TQ_ERR_ARG;
  if (needs_angle && !finite_all(params, gate == TQ_GATE_SU2 ? 4 : 1)) return TQ_ERR_ARG;
  cplx m[4][4] = {};
  int k = 1;
  const cplx I(0, 1);
  switch (gate) {
    case TQ_GATE_ID: m[0][0] = m[1][1] = 1; break;
    case TQ_GATE_H:
      m[0][0] = m[0][1] = m[1][0] = kInvSqrt2;
      m[1][1] = -kInvSqrt2;
      break;
    case TQ_GATE_X: m[0][1] = m[1][0] = 1; break;
    case TQ_GATE_Y: m[0][1] = -I; m[1][0] = I; break;
    case TQ_GATE_Z: m[0][0] = 1; m[1][1] = -1; break;
    case TQ_GATE_S: m[0][0] = 1; m[1][1] = I; break;
    case TQ_GATE_SDG: m[0][0] = 1; m[1][1] = -I; break;
    case TQ_GATE_T: m[0][0] = 1; m[1][1] = std::polar(1.0, M_PI / 4); break;
    case TQ_GATE_TDG: m[0][0] = 1; m[1][1] = std::polar(1.0, -M_PI / 4); break;
    case TQ_GATE_SX:
      m[0][0] = m[1][1] = cplx(0.5, 0.5);
      m[0][1] = m[1][0] = cplx(0.5, -0.5);
      break;
    case TQ_GATE_RX: {
      const double c = std::cos(params[0] / 2), s = std::sin(params[0] / 2);
      m[0][0] = m[1][1] = c;
      m[0][1] = m[1][0] = cplx(0, -s);
      break;
    }
    case TQ_GATE_RY: {
      const double c = std::cos(params[0] / 2), s = std::sin(params[0] / 2);
      m[0][0] = m[1][1] = c;
      m[0][1] = -s;
      m[1][0] = s;
      break;
    }
    case TQ_GATE_RZ:
      m[0][0] = std::polar(1.0, -params[0] / 2);
      m[1][1] = std::polar(1.0, params[0] / 2);
      break;
    case TQ_GATE_SU2: {
      double a = params[0], b = params[1], c = params[2], d = params[3];
      const double nrm = std::sqrt(a * a + b * b + c * c + d * d);
      if (!(nrm > 0)) return TQ_ERR_ARG;
      a /= nrm; b /= nrm; c /= nrm; d /= nrm;
      m[0][0] = cplx(a, b);
      m[0][1] = cplx(c, d);
      m[1][0] = cplx(-c, d);
      m[1][1] = cplx(a, -b);
      break;
    }
    case TQ_GATE_CX:  // local index b0 + 2 b1, b0 = control
      k = 2;
      for (int b0 = 0; b0 < 2; ++b0)
        for (int b1 = 0; b1 < 2; ++b1) m[b0 + 2 * (b1 ^ b0)][b0 + 2 * b1] = 1;
      break;
    case TQ_GATE_CZ:
      k = 2;
      m[0][0] = m[1][1] = m[2][2] = 1;
      m[3][3] = -1;
      break;
    case TQ_GATE_SWAP:
      k = 2;
      for (int b0 = 0; b0 < 2; ++b0)
        for (int b1 = 0; b1 < 2; ++b1) m[b1 + 2 * b0][b0 + 2 * b1] = 1;
      break;
    case TQ_GATE_RZZ:
      k = 2;
      for (int i = 0; i < 4; ++i) {
        const int zz = ((i & 1) == (i >> 1)) ? 1 : -1;  // eigenvalue of Z(x)Z
        m[i][i] = std::polar(1.0, -0.5 * params[0] * zz);
      }
      break;
    default:
      return TQ_ERR_ARG;
  }
  const int d = 1 << k;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) put(U, d, i, j, m[i][j]);
  *k_out = k;
  return TQ_OK;
}

tq_status tq_channel_kraus(int channel, int k, const double* params, int capacity, int* m_out,
                           double* K) {
  if (!m_out || !params) return TQ_ERR_ARG;
  *m_out = 0;
  const int d = 1 << k;
  std::vector<std::vector<cplx>> ks;  // each d*d row-major
  auto add = [&](const std::vector<cplx>& mat) { ks.push_back(mat); };
  switch (channel) {
    case TQ_CH_DEPOLARIZING: {
      if (k < 1 || k > 2) return TQ_ERR_ARG;
      const double p = params[0];
      const double n4 = std::pow(4.0, k);
      if (!std::isfinite(p) || p < 0 || p > n4 / (n4 - 1)) return TQ_ERR_ARG;
      for (int idx = 0; idx < (int)n4; ++idx) {
        const double w = idx == 0 ? 1.0 - p * (n4 - 1) / n4 : p / n4;
        const double sw = std::sqrt(std::max(w, 0.0));
        std::vector<cplx> mat(d * d);
        // local bit j carries Pauli digit (idx >> 2j) & 3
        for (int r = 0; r < d; ++r)
          for (int c = 0; c < d; ++c) {
            cplx v = sw;
            for (int j = 0; j < k; ++j) v *= kPauli[(idx >> (2 * j)) & 3][(r >> j) & 1][(c >> j) & 1];
            mat[r * d + c] = v;
          }
        add(mat);
      }
      break;
    }
    case TQ_CH_AMPLITUDE_DAMPING:
    case TQ_CH_PHASE_DAMPING: {
      if (k != 1) return TQ_ERR_ARG;
      const double g = params[0];
      if (!std::isfinite(g) || g < 0 || g > 1) return TQ_ERR_ARG;
      std::vector<cplx> k0 = {1.0, 0.0, 0.0, std::sqrt(1 - g)};
      std::vector<cplx> k1 = channel == TQ_CH_AMPLITUDE_DAMPING
                                 ? std::vector<cplx>{0.0, std::sqrt(g), 0.0, 0.0}
                                 : std::vector<cplx>{0.0, 0.0, 0.0, std::sqrt(g)};
      add(k0);
      add(k1);
      break;
    }
    case TQ_CH_RESET: {
      if (k != 1) return TQ_ERR_ARG;
      add(std::vector<cplx>{1.0, 0.0, 0.0, 0.0});  // |0><0|
      add(std::vector<cplx>{0.0, 1.0, 0.0, 0.0});  // |0><1|
      break;
    }
    case TQ_CH_THERMAL: {
      if (k < 1 || k > 2) return TQ_ERR_ARG;
      const double t = params[0], t1 = params[1], t2 = params[2];
      if (!std::isfinite(t) || !std::isfinite(t1) || !std::isfinite(t2) || t < 0 || t1 <= 0 ||
          t2 <= 0 || t2 > 2 * t1)
        return TQ_ERR_ARG;
      // Per qubit: amplitude damping gamma = 1 - e^{-t/T1}, then phase damping
      // lambda with (1 - lambda) = e^{-2t/T2} / e^{-t/T1}, so coherences decay
      // by sqrt(1-gamma) sqrt(1-lambda) = e^{-t/T2}. Kraus set of the product:
      // {P_b A_a}, a, b in {0, 1}.
      const double gam = 1 - std::exp(-t / t1);
      const double lam = std::min(1.0, std::max(0.0, 1 - std::exp(-2 * t / t2 + t / t1)));
      const cplx A[2][2][2] = {{{1, 0}, {0, std::sqrt(1 - gam)}}, {{0, std::sqrt(gam)}, {0, 0}}};
      const cplx P[2][2][2] = {{{1, 0}, {0, std::sqrt(1 - lam)}}, {{0, 0}, {0, std::sqrt(lam)}}};
      std::vector<std::vector<cplx>> one;  // 2x2 Kraus set for one qubit
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          std::vector<cplx> mat(4, 0.0);
          for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c)
              for (int x = 0; x < 2; ++x) mat[r * 2 + c] += P[b][r][x] * A[a][x][c];
          one.push_back(mat);
        }
      if (k == 1) {
        for (auto& mat : one) add(mat);
      } else {  // independently on both qubits: tensor products (local bit 0 = first qubit)
        for (auto& hi : one)
          for (auto& lo : one) {
            std::vector<cplx> mat(16);
            for (int r = 0; r < 4; ++r)
              for (int c = 0; c < 4; ++c)
                mat[r * 4 + c] = lo[(r & 1) * 2 + (c & 1)] * hi[(r >> 1) * 2 + (c >> 1)];
            add(mat);
          }
      }
      break;
    }
    default:
      return TQ_ERR_ARG;
  }
  *m_out = (int)ks.size();
  if (!K) return TQ_OK;  // count query
  if (capacity < (int)ks.size()) return TQ_ERR_ARG;
  for (size_t i = 0; i < ks.size(); ++i)
    for (int e = 0; e < d * d; ++e) {
      K[2 * (i * d * d + e)] = ks[i][e].real();
      K[2 * (i * d * d + e) + 1] = ks[i][e].imag();
    }
  return TQ_OK;
}

tq_status tq_plan_fusion(int n, const tq_op* ops, size_t n_ops, int max_width, int precision,
                         int* block_of_op, int* block_width, size_t* n_blocks_out) {
  if (n < 1 || n > kMaxQubits || (!ops && n_ops) || !n_blocks_out) return TQ_ERR_ARG;
  if (precision != TQ_FP64 && precision != TQ_SPLIT) return TQ_ERR_ARG;
  std::vector<PlanOp> pops(n_ops);
  // named gates and channels with equal parameters share one pattern
  std::map<std::array<uint64_t, 7>, size_t> seen;
  for (size_t i = 0; i < n_ops; ++i) {
    tq_status st = validate_op(n, ops[i]);
    if (st != TQ_OK) return st;
    pops[i].qubits.assign(ops[i].qubits, ops[i].qubits + ops[i].k);
    const bool named = ops[i].kind == TQ_OP_GATE || ops[i].kind == TQ_OP_CHANNEL;
    std::array<uint64_t, 7> key{(uint64_t)ops[i].kind, (uint64_t)ops[i].name, (uint64_t)ops[i].k, 0, 0, 0, 0};
    std::memcpy(&key[3], ops[i].params, 4 * sizeof(double));
    auto it = named ? seen.find(key) : seen.end();
    if (it != seen.end()) {
      pops[i].has_pat = pops[it->second].has_pat;
      pops[i].pat = pops[it->second].pat;
      continue;
    }
    ResolvedOp r;
    if ((st = resolve_op(ops[i], &r)) != TQ_OK) return st;
    pops[i].has_pat = op_pattern(ops[i], r, &pops[i].pat);
    if (named) seen.emplace(key, i);
  }
  std::vector<Block> blocks;
  tq_status st = plan_fusion(n, pops, max_width, precision, &blocks);
  if (st != TQ_OK) return st;
  for (size_t b = 0; b < blocks.size(); ++b) {
    for (int i : blocks[b].ops)
      if (block_of_op) block_of_op[i] = (int)b;
    if (block_width) block_width[b] = blocks[b].width;
  }
  *n_blocks_out = blocks.size();
  return TQ_OK;
}

tq_status tq_op_pattern(const tq_op* op, int* width_out, int* nnz_out, uint16_t* rows_out) {
  if (!op || !width_out || !nnz_out) return TQ_ERR_ARG;
  tq_status st = validate_op(kMaxQubits, *op);
  if (st != TQ_OK) return st;
  ResolvedOp r;
  if ((st = resolve_op(*op, &r)) != TQ_OK) return st;
  Pattern p;
  if (!op_pattern(*op, r, &p)) return TQ_ERR_UNSUPPORTED;
  *width_out = p.width;
  *nnz_out = pattern_nnz(p);
  if (rows_out)
    for (int i = 0; i < (1 << (2 * p.width)); ++i) rows_out[i] = p.row[i];
  return TQ_OK;
}

uint64_t tq_group_base(uint64_t g, const int* positions, int n_positions) {
  int p[8];
  const int cnt = n_positions < 0 ? 0 : (n_positions > 8 ? 8 : n_positions);
  for (int i = 0; i < cnt; ++i) {  // insertion sort, ascending
    int v = positions[i], j = i;
    for (; j > 0 && p[j - 1] > v; --j) p[j] = p[j - 1];
    p[j] = v;
  }
  for (int i = 0; i < cnt; ++i) {
    const uint64_t low = g & ((1ull << p[i]) - 1);
    g = ((g >> p[i]) << (p[i] + 1)) | low;
  }
  return g;
}

const char* tq_status_string(int status) {
  switch (status) {
    case TQ_OK: return "ok";
    case TQ_ERR_ARG: return "invalid argument";
    case TQ_ERR_QUBIT: return "qubit index out of range or repeated";
    case TQ_ERR_OOM: return "out of memory";
    case TQ_ERR_CUDA: return "CUDA error (state poisoned)";
    case TQ_ERR_TIMEOUT: return "bounded device wait timed out";
    case TQ_ERR_STATE: return "state poisoned by an earlier CUDA error";
    case TQ_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

const char* tq_version(void) { return "tanq-gb300 0.1 (sm_103a)"; }

}  // extern "C"
