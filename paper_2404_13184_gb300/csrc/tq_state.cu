// States, programs, circuit runs and readouts: the C-ABI entry points that
// do GPU work. Host code here validates ops, plans fusion, packs tables and
// enqueues kernels; every arithmetic step of the simulation runs on the
// device (superoperator build and fusion in FP64, apply passes, reductions).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <unordered_map>
#include <vector>

#include "tq_device.cuh"
#include "tq_internal.h"
#include "tq_plan.cuh"

using namespace tq;

namespace {


// Kernel kinds for launch counting and event profiling.
enum Kind {
  K_BUILD = 0, K_FUSE, K_REDUCE, K_APPLY64 /* +w-1 */, K_APPLY32 = K_APPLY64 + 4, K_PACK = K_APPLY32 + 4,
  K_SPARSE64 /* +w-1 */, K_TC64 = K_SPARSE64 + 2 /* +w-1 */, K_NKINDS = K_TC64 + 2
};
const char* kKindName[K_NKINDS] = {"superop_build", "fuse",         "reduce",        "apply_f64_w1",
                                   "apply_f64_w2",  "apply_f64_w3", "apply_f64_w4",  "apply_f32_w1",
                                   "apply_f32_w2",  "apply_f32_w3", "apply_f32_w4",  "sparse_pack",
                                   "apply_f64_sparse_w1", "apply_f64_sparse_w2", "apply_f64tc_w1",
                                   "apply_f64tc_w2"};

// Whether FP64 passes of widths <= 2 run on the tensor cores when the
// engine is TQ_ENGINE_AUTO.
constexpr bool kAutoTensor = true;

struct Pending {
  int kind;
  cudaEvent_t e0, e1;
};

// Algorithmic flops of a row-list launch, resolved once the row lists it
// applied have been copied back: 8 flops per applied nonzero per group.
struct PendingFlops {
  int kind;
  double groups;
  const int* rowptr;  // pinned host copy of the block's rowptr[0..16]
  int dim;            // rowptr[dim] = nonzeros of the block
};

// Pinned host memory for the row-list counts of profiled launches, in chunks
// that are never reallocated (pending copies keep pointing into them).
struct CountArena {
  static constexpr size_t kChunkInts = 1 << 14;
  std::vector<int*> chunks;
  size_t used = 0;  // ints used in the last chunk
  int* take(size_t ints) {
    if (ints > kChunkInts) return nullptr;
    if (chunks.empty() || used + ints > kChunkInts) {
      void* p = nullptr;
      if (cudaHostAlloc(&p, kChunkInts * sizeof(int), cudaHostAllocDefault) != cudaSuccess) return nullptr;
      chunks.push_back(static_cast<int*>(p));
      used = 0;
    }
    int* out = chunks.back() + used;
    used += ints;
    return out;
  }
  void reset() {
    for (size_t i = 1; i < chunks.size(); ++i) cudaFreeHost(chunks[i]);
    if (chunks.size() > 1) chunks.resize(1);
    used = 0;
  }
  void release() {
    for (int* c : chunks) cudaFreeHost(c);
    chunks.clear();
    used = 0;
  }
};

}  // namespace

struct tq_state {
  int n = 0;
  int prec = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 152;
  void* rho = nullptr;
  size_t rho_bytes = 0;
  bool owns_rho = false;
  bool poisoned = false;
  DevBuf red, probs, staging, shots;
  PinBuf pin, pin_small;
  cudaEvent_t pin_free = nullptr;  // recorded after the last upload from `pin`
  tq_program scratch;              // plan of the last tq_run_circuit call
  // Hermitian mode (FP64): half of the groups, entries with row <= column kept
  bool herm_mode = true;     // allowed by the caller
  bool herm_ok = true;       // rho is known to be Hermitian
  bool lower_stale = false;  // entries with row > column are out of date
  bool tc_used = false;      // a tensor-core pass (bounded waits) was enqueued
  int fp64_engine = TQ_ENGINE_AUTO;  // products of FP64 passes (tq_set_fp64_engine)
  uint64_t launches = 0;
  bool prof_on = false;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  uint64_t prof_launches[K_NKINDS] = {};
  double prof_ms[K_NKINDS] = {};
  double prof_flops[K_NKINDS] = {};  // summed over launches
  double prof_bytes[K_NKINDS] = {};  // summed over launches
  std::vector<PendingFlops> pending_flops;
  CountArena counts;
};

namespace {

tq_status cuda_fail(tq_state* s, cudaError_t e) {
  if (e == cudaSuccess) return TQ_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();  // not sticky: clear it, keep the state usable
    return TQ_ERR_OOM;
  }
  if (s) s->poisoned = true;
  return TQ_ERR_CUDA;
}

// Grow a device buffer (contents not kept). With a stream, waits for it
// first because queued kernels may still read the old buffer.
cudaError_t grow(DevBuf& b, size_t bytes, cudaStream_t wait_on, bool sync) {
  if (b.cap >= bytes) return cudaSuccess;
  if (sync) {
    cudaError_t e = cudaStreamSynchronize(wait_on);
    if (e != cudaSuccess) return e;
  }
  if (b.ptr) cudaFree(b.ptr);
  b.ptr = nullptr;
  b.cap = 0;
  const size_t want = align_up(std::max<size_t>(bytes, 4096), 4096);
  cudaError_t e = cudaMalloc(&b.ptr, want);
  if (e != cudaSuccess) {
    b.ptr = nullptr;
    return e;
  }
  b.cap = want;
  return cudaSuccess;
}

tq_status ensure(tq_state* s, DevBuf& b, size_t bytes) { return cuda_fail(s, grow(b, bytes, s->stream, true)); }

tq_status ensure_pinned(tq_state* s, PinBuf& b, size_t bytes) {
  if (b.cap >= bytes) return TQ_OK;
  if (b.ptr) cudaFreeHost(b.ptr);
  b.ptr = nullptr;
  b.cap = 0;
  const size_t want = align_up(std::max<size_t>(bytes, 4096), 4096);
  cudaError_t e = cudaHostAlloc(&b.ptr, want, cudaHostAllocDefault);
  if (e != cudaSuccess) {
    b.ptr = nullptr;
    return cuda_fail(s, e);
  }
  b.cap = want;
  return TQ_OK;
}

void free_buf(DevBuf& b) {
  if (b.ptr) cudaFree(b.ptr);
  b.ptr = nullptr;
  b.cap = 0;
}

size_t entry_bytes(int prec) { return prec == TQ_FP64 ? 16 : 8; }

bool fp64_on_tensor(const tq_state* s) { return fp64_engine_is_tensor(s->fp64_engine); }

tq_status check_state(tq_state* s) {
  if (!s) return TQ_ERR_ARG;
  if (s->poisoned) return TQ_ERR_STATE;
  return TQ_OK;
}

// End of a synchronising readout: CUDA errors poison the state, and so does
// a tensor-core pass whose bounded wait gave up (its results are not valid).
tq_status readout_done(tq_state* s, cudaError_t e) {
  if (e != cudaSuccess) return cuda_fail(s, e);
  if (!s->tc_used) return TQ_OK;
  unsigned int timeouts = 0, oz = 0;
  e = tc_take_timeouts(&timeouts, s->stream);
  if (e == cudaSuccess) e = oz_take_timeouts(&oz, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e);
  if (timeouts || oz) {
    s->poisoned = true;
    return TQ_ERR_TIMEOUT;
  }
  return TQ_OK;
}

// ---- launch accounting -------------------------------------------------

// Run `launch` (which enqueues `count` kernels of one kind on s->stream),
// bracketed by events when profiling is on.
template <typename F>
cudaError_t timed(tq_state* s, int kind, int count, F launch) {
  Pending pd{kind, nullptr, nullptr};
  if (s->prof_on) {
    for (cudaEvent_t* ev : {&pd.e0, &pd.e1}) {
      if (!s->event_pool.empty()) {
        *ev = s->event_pool.back();
        s->event_pool.pop_back();
      } else {
        cudaError_t e = cudaEventCreate(ev);
        if (e != cudaSuccess) return e;
      }
    }
    cudaEventRecord(pd.e0, s->stream);
  }
  cudaError_t e = launch();
  s->launches += count;
  if (s->prof_on) {
    cudaEventRecord(pd.e1, s->stream);
    s->pending.push_back(pd);
    s->prof_launches[kind] += count;
  }
  return e;
}

// Fold finished launches into the statistics (the stream has been
// synchronised, so the row-list counts have landed in host memory).
void fold_pending(tq_state* s) {
  for (const Pending& pd : s->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pd.e0, pd.e1) == cudaSuccess) s->prof_ms[pd.kind] += ms;
    s->event_pool.push_back(pd.e0);
    s->event_pool.push_back(pd.e1);
  }
  s->pending.clear();
  for (const PendingFlops& pf : s->pending_flops) s->prof_flops[pf.kind] += 8.0 * pf.groups * (double)pf.rowptr[pf.dim];
  s->pending_flops.clear();
  s->counts.reset();
}

// ---- planning ------------------------------------------------------------

}  // namespace

namespace tq {

bool fp64_engine_is_tensor(int engine) {
  return engine == TQ_ENGINE_TENSOR || (engine == TQ_ENGINE_AUTO && kAutoTensor);
}

ApplyParams apply_params(int n, const Block& B) {
  ApplyParams p{};
  p.n = n;
  p.width = B.width;
  p.npos = 2 * B.width;
  p.n_groups = 1ull << (2 * (n - B.width));
  int pos[8];
  for (int j = 0; j < B.width; ++j) {
    p.q[j] = B.qubits[j];
    pos[2 * j] = B.qubits[j];
    pos[2 * j + 1] = B.qubits[j] + n;
  }
  std::sort(pos, pos + p.npos);
  for (int i = 0; i < p.npos; ++i) p.pos[i] = pos[i];
  if (B.width <= 2) {
    const int D = 1 << (2 * B.width);
    for (int l = 0; l < D; ++l) {
      unsigned long long v = 0;
      for (int j = 0; j < B.width; ++j) {
        if ((l >> j) & 1) v |= 1ull << B.qubits[j];
        if ((l >> (B.width + j)) & 1) v |= 1ull << (B.qubits[j] + n);
      }
      p.off[l] = v;
    }
  }
  return p;
}

// Validate, resolve and plan `ops` into P's host fields and `t`.
// Identity of a named gate or channel: its superoperator depends on nothing
// else (not on the qubits it acts on).
struct OpKey {
  int kind, name, k;
  uint64_t p[4];
  bool operator==(const OpKey& o) const {
    return kind == o.kind && name == o.name && k == o.k && p[0] == o.p[0] && p[1] == o.p[1] && p[2] == o.p[2] &&
           p[3] == o.p[3];
  }
};
struct OpKeyHash {
  size_t operator()(const OpKey& key) const {
    uint64_t h = (uint64_t)key.kind * 0x9E3779B97F4A7C15ull ^ (uint64_t)key.name * 0xC2B2AE3D27D4EB4Full ^ (uint64_t)key.k;
    for (uint64_t v : key.p) h = (h ^ v) * 0x100000001B3ull;
    return (size_t)h;
  }
};

tq_status plan_program(int n, int prec, const tq_op* ops, size_t n_ops, int width, tq_program* P, HostTables* t,
                       bool f64_tensor) {
  if (width < -1 || width > kMaxWidth) return TQ_ERR_ARG;
  std::vector<PlanOp> qs(n_ops);
  std::vector<int> uop(n_ops);  // op -> its descriptor (identical named ops share one)
  std::vector<Pattern> upat;
  std::vector<char> uhas;
  std::unordered_map<OpKey, int, OpKeyHash> seen;
  t->ops.clear();
  P->max_dim2 = 0;
  for (size_t i = 0; i < n_ops; ++i) {
    tq_status st = validate_op(n, ops[i]);
    if (st != TQ_OK) return st;
    const bool named = ops[i].kind == TQ_OP_GATE || ops[i].kind == TQ_OP_CHANNEL;
    OpKey key{ops[i].kind, ops[i].name, ops[i].k, {0, 0, 0, 0}};
    std::memcpy(key.p, ops[i].params, sizeof(key.p));
    auto it = named ? seen.find(key) : seen.end();
    if (it != seen.end()) {
      uop[i] = it->second;
    } else {
      ResolvedOp r;
      st = resolve_op(ops[i], &r);
      if (st != TQ_OK) return st;
      uop[i] = (int)t->ops.size();
      upat.emplace_back();
      uhas.push_back(op_pattern(ops[i], r, &upat.back()) ? 1 : 0);
      OpDesc od{};
      od.k = r.k;
      od.m = r.m;
      od.kraus_off = (long long)t->kraus.size();
      od.sop_off = t->sop_entries;
      for (const cplx& v : r.kraus) t->kraus.push_back(make_double2(v.real(), v.imag()));
      const long long d2 = 1ll << (2 * r.k);
      t->sop_entries += d2 * d2;
      P->max_dim2 = std::max<int>(P->max_dim2, (int)(d2 * d2));
      t->ops.push_back(od);
      if (named) seen.emplace(key, uop[i]);
    }
    qs[i].qubits.assign(ops[i].qubits, ops[i].qubits + ops[i].k);
    qs[i].has_pat = uhas[uop[i]] != 0;
    qs[i].pat = upat[uop[i]];
  }
  std::vector<Block> plan;
  const int plan_prec = prec == TQ_FP64 && f64_tensor && oz_eligible(n, 2) ? kPlanF64Tensor : prec;
  tq_status st = plan_fusion(n, qs, width, plan_prec, &plan);
  if (st != TQ_OK) return st;
  P->n = n;
  P->prec = prec;
  P->n_ops = n_ops;
  P->n_uops = t->ops.size();
  P->max_width = 0;
  P->params.clear();
  P->sb_off.clear();
  P->sp_slot.clear();
  P->nnz.clear();
  P->n_sparse = 0;
  for (size_t b = 0; b < plan.size(); ++b) {
    const Block& B = plan[b];
    BlockDesc bd{};
    bd.width = B.width;
    bd.n_members = (int)B.ops.size();
    bd.member_off = (int)t->members.size();
    bd.sb_off = t->sb_entries;
    const int D = 1 << (2 * B.width);
    t->sb_entries += (long long)D * D;
    for (int oi : B.ops) {
      MemberDesc md{};
      md.op = uop[oi];
      md.k = ops[oi].k;
      for (int j = 0; j < md.k; ++j)
        md.pos[j] = (int)(std::find(B.qubits, B.qubits + B.width, ops[oi].qubits[j]) - B.qubits);
      t->members.push_back(md);
    }
    t->blocks.push_back(bd);
    const int C = std::min(D, 1024 / D);
    for (int c0 = 0; c0 < D; c0 += C) t->work.push_back(FuseWork{(int)b, c0});
    ApplyParams ap = apply_params(n, B);
    P->nnz.push_back(B.has_pat ? pattern_nnz(B.pat) : D * D);
    if (block_is_sparse(B, prec)) {
      ap.sparse = 1;
      t->spw.push_back(SparseWork{(int)b, P->n_sparse});
      P->sp_slot.push_back(P->n_sparse++);
    } else {
      P->sp_slot.push_back(-1);
    }
    P->params.push_back(ap);
    P->sb_off.push_back(bd.sb_off);
    P->max_width = std::max(P->max_width, B.width);
  }
  P->n_work = (int)t->work.size();
  size_t off = 0;
  P->o_kraus = off; off = align_up(off + t->kraus.size() * sizeof(double2), 256);
  P->o_ops = off;   off = align_up(off + t->ops.size() * sizeof(OpDesc), 256);
  P->o_blk = off;   off = align_up(off + t->blocks.size() * sizeof(BlockDesc), 256);
  P->o_mem = off;   off = align_up(off + t->members.size() * sizeof(MemberDesc), 256);
  P->o_work = off;  off = align_up(off + t->work.size() * sizeof(FuseWork), 256);
  P->o_spw = off;   off = align_up(off + t->spw.size() * sizeof(SparseWork), 256);
  P->blob_bytes = std::max<size_t>(off, 256);
  return TQ_OK;
}

void pack_blob(const tq_program& P, const HostTables& t, char* h) {
  std::memcpy(h + P.o_kraus, t.kraus.data(), t.kraus.size() * sizeof(double2));
  std::memcpy(h + P.o_ops, t.ops.data(), t.ops.size() * sizeof(OpDesc));
  std::memcpy(h + P.o_blk, t.blocks.data(), t.blocks.size() * sizeof(BlockDesc));
  std::memcpy(h + P.o_mem, t.members.data(), t.members.size() * sizeof(MemberDesc));
  std::memcpy(h + P.o_work, t.work.data(), t.work.size() * sizeof(FuseWork));
  if (!t.spw.empty()) std::memcpy(h + P.o_spw, t.spw.data(), t.spw.size() * sizeof(SparseWork));
}

}  // namespace tq

namespace {

// Enqueue superoperator build, fusion and every apply pass of P on s.
tq_status enqueue_program(tq_state* s, const tq_program& P) {
  if (P.n_uops == 0) return TQ_OK;
  char* d = static_cast<char*>(P.blob.ptr);
  const double2* d_kraus = reinterpret_cast<const double2*>(d + P.o_kraus);
  const OpDesc* d_ops = reinterpret_cast<const OpDesc*>(d + P.o_ops);
  const BlockDesc* d_blk = reinterpret_cast<const BlockDesc*>(d + P.o_blk);
  const MemberDesc* d_mem = reinterpret_cast<const MemberDesc*>(d + P.o_mem);
  const FuseWork* d_work = reinterpret_cast<const FuseWork*>(d + P.o_work);
  double2* sops = static_cast<double2*>(P.sops.ptr);
  double2* sb64 = static_cast<double2*>(P.sb64.ptr);
  float2* sb32 = P.prec == TQ_SPLIT ? static_cast<float2*>(P.sb32.ptr) : nullptr;
  cudaError_t e = timed(s, K_BUILD, build_superops_launches((int)P.n_uops), [&] {
    return launch_build_superops(d_kraus, d_ops, (int)P.n_uops, P.max_dim2, sops, s->stream);
  });
  if (e == cudaSuccess)
    e = timed(s, K_FUSE, 1, [&] { return launch_fuse(sops, d_ops, d_blk, d_mem, d_work, P.n_work, sb64, sb32, s->stream); });
  if (e == cudaSuccess && s->herm_mode && s->herm_ok && !s->prof_on && P.g_blk_ready) {
    // small register: every block in one cluster kernel (Hermitian mode; the
    // kernel builds its own row lists, so no compression pass)
    s->launches += 1;
    s->lower_stale = true;
    e = launch_cluster_program(s->rho, s->prec, s->n, s->prec == TQ_FP64 ? (const void*)sb64 : (const void*)sb32,
                               P.g_blk.ptr, (int)P.params.size(), s->stream);
    return cuda_fail(s, e);
  }
  SparseBlock* sps = static_cast<SparseBlock*>(P.sps.ptr);
  // row lists serve the DFMA kernels only: none are needed when every block
  // of width <= 2 runs on the tensor-core FP64 engine
  const bool rows_unused = s->prec == TQ_FP64 && s->herm_mode && s->herm_ok && fp64_on_tensor(s) && oz_eligible(s->n, 2);
  if (e == cudaSuccess && P.n_sparse > 0 && !rows_unused)
    e = timed(s, K_PACK, 1, [&] {
      return launch_compress_sparse(sb64, d_blk, reinterpret_cast<const SparseWork*>(d + P.o_spw), P.n_sparse, sps,
                                    s->stream);
    });
  // profiling: copy every row list's rowptr back, so that the flops of a
  // row-list launch count the nonzeros it actually applied
  const int* counts = nullptr;
  if (e == cudaSuccess && s->prof_on && P.n_sparse > 0 && !rows_unused) {
    constexpr size_t kRow = sizeof(SparseBlock::rowptr);
    int* h = s->counts.take((size_t)P.n_sparse * (kRow / sizeof(int)));
    if (!h) return TQ_ERR_OOM;
    e = cudaMemcpy2DAsync(h, kRow, sps, sizeof(SparseBlock), kRow, (size_t)P.n_sparse, cudaMemcpyDeviceToHost,
                          s->stream);
    counts = h;
  }
  const double entries = (double)(1ull << (2 * s->n));
  const bool herm_state = s->herm_mode && s->herm_ok;
  for (size_t b = 0; b < P.params.size() && e == cudaSuccess; ++b) {
    ApplyParams p = P.params[b];
    double groups = (double)p.n_groups;
    // FP64 kernels all have a Hermitian path; split ones for widths 1-2 on
    // registers with at least 16 row-rest values (tiles of 16 x 16 groups)
    const bool herm = herm_state && (s->prec == TQ_FP64 || (p.width <= 2 && s->n - p.width >= 4));
    if (herm) {
      const unsigned long long M = 1ull << (s->n - p.width);
      p.herm = 1;
      p.n_canon = M * (M + 1) / 2;
      groups = (double)p.n_canon;
      s->lower_stale = true;
    } else if (s->lower_stale) {  // a full update needs every entry current
      s->launches += 1;
      e = launch_mirror_lower(s->rho, s->n, s->prec, s->stream);
      s->lower_stale = false;
      if (e != cudaSuccess) break;
    }
    const void* S = s->prec == TQ_FP64 ? (const void*)(sb64 + P.sb_off[b]) : (const void*)(sb32 + P.sb_off[b]);
    // FP64 blocks of widths <= 2 on the tensor cores (FP64-accurate slicing)
    const bool oz = herm && s->prec == TQ_FP64 && fp64_on_tensor(s) && oz_eligible(s->n, p.width);
    const bool sparse = !oz && p.sparse && s->prec == TQ_FP64 && P.sp_slot[b] >= 0;
    if (!sparse) p.sparse = 0;
    const int kind = oz ? K_TC64 + p.width - 1
                        : sparse ? K_SPARSE64 + p.width - 1 : (s->prec == TQ_FP64 ? K_APPLY64 : K_APPLY32) + p.width - 1;
    const SparseBlock* spb = sparse ? sps + P.sp_slot[b] : nullptr;
    if (herm && ((s->prec == TQ_SPLIT && p.width == 2) || oz)) s->tc_used = true;
    if (oz)
      e = timed(s, kind, 1, [&] {
        return launch_herm_oz(static_cast<double2*>(s->rho), static_cast<const double2*>(S), p, s->num_sms, s->stream);
      });
    else
      e = timed(s, kind, 1, [&] { return launch_apply(s->rho, s->prec, S, p, s->num_sms, s->stream, spb); });
    if (s->prof_on) {  // per launch: the groups computed x (8 * 16^w flops, 2 * B * 4^w bytes) each
      const int per = 1 << (2 * p.width);
      if (sparse)  // 8 flops per nonzero of the row lists the kernel applied
        s->pending_flops.push_back(PendingFlops{kind, groups, counts + (size_t)P.sp_slot[b] * 17, per});
      else
        s->prof_flops[kind] += 8.0 * groups * (double)per * (double)per;
      s->prof_bytes[kind] += 2.0 * groups * (double)per * (double)entry_bytes(s->prec);
    }
    (void)entries;
  }
  return cuda_fail(s, e);
}

tq_status create_impl(int n, int precision, void* stream, void* ext, size_t ext_bytes, tq_state** out) {
  if (!out) return TQ_ERR_ARG;
  *out = nullptr;
  if (n < 1 || n > kMaxQubits) return TQ_ERR_ARG;
  if (precision != TQ_FP64 && precision != TQ_SPLIT) return TQ_ERR_ARG;
  tq_state* s = new (std::nothrow) tq_state();
  if (!s) return TQ_ERR_OOM;
  s->n = n;
  s->prec = precision;
  s->stream = static_cast<cudaStream_t>(stream);
  s->rho_bytes = entry_bytes(precision) << (2 * n);
  s->scratch.owns = false;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    delete s;
    return TQ_ERR_CUDA;
  }
  if (ext) {
    if (ext_bytes < s->rho_bytes || (reinterpret_cast<uintptr_t>(ext) & 255)) {
      delete s;
      return TQ_ERR_ARG;
    }
    s->rho = ext;
    s->owns_rho = false;
  } else {
    e = cudaMalloc(&s->rho, s->rho_bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete s;
      return e == cudaErrorMemoryAllocation ? TQ_ERR_OOM : TQ_ERR_CUDA;
    }
    s->owns_rho = true;
  }
  e = cudaEventCreateWithFlags(&s->pin_free, cudaEventDisableTiming);
  if (e == cudaSuccess) e = launch_init_zero_state(s->rho, n, precision, s->stream);
  s->launches += 1;
  if (e != cudaSuccess) {
    tq_free(s);
    return TQ_ERR_CUDA;
  }
  *out = s;
  return TQ_OK;
}

tq_status run_impl(tq_state* s, const tq_op* ops, size_t n_ops, int width, size_t* n_blocks_out) {
  tq_status st = check_state(s);
  if (st != TQ_OK) return st;
  if (!ops && n_ops) return TQ_ERR_ARG;
  if (n_blocks_out) *n_blocks_out = 0;
  if (n_ops == 0) return TQ_OK;
  tq_program plan;
  HostTables t;
  st = plan_program(s->n, s->prec, ops, n_ops, width, &plan, &t, fp64_on_tensor(s));
  if (st != TQ_OK) return st;
  // reuse the state's scratch buffers for this plan
  tq_program& P = s->scratch;
  P.n = plan.n;
  P.prec = plan.prec;
  P.n_ops = plan.n_ops;
  P.n_uops = plan.n_uops;
  P.max_width = plan.max_width;
  P.max_dim2 = plan.max_dim2;
  P.n_work = plan.n_work;
  P.params.swap(plan.params);
  P.sb_off.swap(plan.sb_off);
  P.sp_slot.swap(plan.sp_slot);
  P.nnz.swap(plan.nnz);
  P.n_sparse = plan.n_sparse;
  P.o_kraus = plan.o_kraus; P.o_ops = plan.o_ops; P.o_blk = plan.o_blk; P.o_mem = plan.o_mem;
  P.o_work = plan.o_work; P.o_spw = plan.o_spw; P.blob_bytes = plan.blob_bytes;
  if (P.n_sparse > 0 && (st = ensure(s, P.sps, (size_t)P.n_sparse * sizeof(SparseBlock))) != TQ_OK) return st;
  if ((st = ensure(s, P.blob, P.blob_bytes)) != TQ_OK) return st;
  if ((st = ensure(s, P.sops, t.sop_entries * sizeof(double2))) != TQ_OK) return st;
  if ((st = ensure(s, P.sb64, t.sb_entries * sizeof(double2))) != TQ_OK) return st;
  if (s->prec == TQ_SPLIT && (st = ensure(s, P.sb32, t.sb_entries * sizeof(float2))) != TQ_OK) return st;
  // the pinned staging buffer is reused: wait until its last upload finished
  cudaError_t e = cudaEventSynchronize(s->pin_free);
  if (e != cudaSuccess) return cuda_fail(s, e);
  if ((st = ensure_pinned(s, s->pin, P.blob_bytes)) != TQ_OK) return st;
  pack_blob(P, t, static_cast<char*>(s->pin.ptr));
  e = cudaMemcpyAsync(P.blob.ptr, s->pin.ptr, P.blob_bytes, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaEventRecord(s->pin_free, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e);
  st = enqueue_program(s, P);
  if (st == TQ_OK && n_blocks_out) *n_blocks_out = P.params.size();
  return st;
}

// Reduction scratch: [16 masks][18 outputs][grid x 18 partials]
constexpr size_t kRedMasks = 0, kRedOut = 256, kRedPartials = 512;
constexpr size_t kRedBytes = kRedPartials + 152 * 18 * sizeof(double);

tq_status reduce_device(tq_state* s, const unsigned long long* masks_dev, int n_masks, bool normalize,
                        double* masked_out_dev) {
  tq_status st = ensure(s, s->red, kRedBytes);
  if (st != TQ_OK) return st;
  char* d = static_cast<char*>(s->red.ptr);
  cudaError_t e = timed(s, K_REDUCE, 2, [&] {
    return launch_diag_reduce(s->rho, s->n, s->prec, masks_dev, n_masks, reinterpret_cast<double*>(d + kRedPartials),
                              reinterpret_cast<double*>(d + kRedOut), normalize, masked_out_dev, s->stream);
  });
  return cuda_fail(s, e);
}

tq_status reduce_impl(tq_state* s, const unsigned long long* masks, int n_masks, bool normalize, double* host_out) {
  tq_status st = ensure(s, s->red, kRedBytes);
  if (st != TQ_OK) return st;
  if ((st = ensure_pinned(s, s->pin_small, 4096)) != TQ_OK) return st;
  char* d = static_cast<char*>(s->red.ptr);
  unsigned long long* hm = static_cast<unsigned long long*>(s->pin_small.ptr);
  double* hout = reinterpret_cast<double*>(hm + 32);
  cudaError_t e = cudaSuccess;
  if (n_masks > 0) {
    std::memcpy(hm, masks, n_masks * sizeof(unsigned long long));
    e = cudaMemcpyAsync(d + kRedMasks, hm, n_masks * sizeof(unsigned long long), cudaMemcpyHostToDevice, s->stream);
  }
  if (e != cudaSuccess) return cuda_fail(s, e);
  st = reduce_device(s, reinterpret_cast<unsigned long long*>(d + kRedMasks), n_masks, normalize, nullptr);
  if (st != TQ_OK) return st;
  e = cudaMemcpyAsync(hout, d + kRedOut, (2 + n_masks) * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if ((st = readout_done(s, e)) != TQ_OK) return st;
  std::memcpy(host_out, hout, (2 + n_masks) * sizeof(double));
  return TQ_OK;
}

// After tq_set_rho: Hermitian mode stays on only if the new rho is Hermitian
// to rounding (max |rho - rho^dagger| <= 4 eps max |rho|, checked on the GPU).
tq_status check_hermitian(tq_state* s) {
  tq_status st = ensure(s, s->red, kRedBytes);
  if (st != TQ_OK) return st;
  if ((st = ensure_pinned(s, s->pin_small, 4096)) != TQ_OK) return st;
  double* dres = reinterpret_cast<double*>(static_cast<char*>(s->red.ptr) + kRedOut);
  double* hres = static_cast<double*>(s->pin_small.ptr) + 64;
  cudaError_t e = launch_hermiticity(s->rho, s->n, s->prec, dres, s->stream);
  s->launches += 1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(hres, dres, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e);
  const double eps = s->prec == TQ_FP64 ? 2.220446049250313e-16 : 1.1920928955078125e-07;
  s->herm_ok = hres[0] <= 4.0 * eps * hres[1];
  s->lower_stale = false;
  return TQ_OK;
}

}  // namespace

extern "C" {

tq_status tq_create(int n_qubits, int precision, void* cuda_stream, tq_state** out) {
  return create_impl(n_qubits, precision, cuda_stream, nullptr, 0, out);
}

tq_status tq_create_on(int n_qubits, int precision, void* cuda_stream, void* rho_dev, size_t bytes,
                       tq_state** out) {
  if (!rho_dev) return TQ_ERR_ARG;
  return create_impl(n_qubits, precision, cuda_stream, rho_dev, bytes, out);
}

void tq_free(tq_state* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  if (s->owns_rho && s->rho) cudaFree(s->rho);
  for (DevBuf* b : {&s->red, &s->probs, &s->staging, &s->shots, &s->scratch.blob, &s->scratch.sops, &s->scratch.sb64,
                    &s->scratch.sb32, &s->scratch.sps})
    free_buf(*b);
  for (PinBuf* b : {&s->pin, &s->pin_small})
    if (b->ptr) cudaFreeHost(b->ptr);
  if (s->pin_free) cudaEventDestroy(s->pin_free);
  for (const Pending& pd : s->pending) {
    cudaEventDestroy(pd.e0);
    cudaEventDestroy(pd.e1);
  }
  for (cudaEvent_t ev : s->event_pool) cudaEventDestroy(ev);
  s->counts.release();
  delete s;
}

tq_status tq_info(const tq_state* s, int* n_qubits, int* precision) {
  if (!s) return TQ_ERR_ARG;
  if (n_qubits) *n_qubits = s->n;
  if (precision) *precision = s->prec;
  return TQ_OK;
}

tq_status tq_reset(tq_state* s) {
  tq_status st = check_state(s);
  if (st != TQ_OK) return st;
  s->launches += 1;
  s->herm_ok = true;
  s->lower_stale = false;
  return cuda_fail(s, launch_init_zero_state(s->rho, s->n, s->prec, s->stream));
}

tq_status tq_rho_device_ptr(tq_state* s, void** out) {
  if (!s || !out) return TQ_ERR_ARG;
  if (s->lower_stale && !s->poisoned) {
    s->launches += 1;
    tq_status st = cuda_fail(s, launch_mirror_lower(s->rho, s->n, s->prec, s->stream));
    if (st != TQ_OK) return st;
    s->lower_stale = false;
  }
  *out = s->rho;
  return TQ_OK;
}

tq_status tq_set_fp64_engine(tq_state* s, int engine) {
  if (!s || engine < TQ_ENGINE_AUTO || engine > TQ_ENGINE_TENSOR) return TQ_ERR_ARG;
  s->fp64_engine = engine;
  return TQ_OK;
}

tq_status tq_fp64_on_tensor(const tq_state* s, int* on_tensor) {
  if (!s || !on_tensor) return TQ_ERR_ARG;
  *on_tensor = fp64_on_tensor(s) ? 1 : 0;
  return TQ_OK;
}

tq_status tq_set_hermitian(tq_state* s, int on) {
  tq_status st = check_state(s);
  if (st != TQ_OK) return st;
  if (!on && s->lower_stale) {
    s->launches += 1;
    st = cuda_fail(s, launch_mirror_lower(s->rho, s->n, s->prec, s->stream));
    if (st != TQ_OK) return st;
    s->lower_stale = false;
  }
  s->herm_mode = on != 0;
  return TQ_OK;
}

tq_status tq_is_hermitian_mode(const tq_state* s, int* active) {
  if (!s || !active) return TQ_ERR_ARG;
  *active = (s->herm_mode && s->herm_ok) ? 1 : 0;
  return TQ_OK;
}

tq_status tq_get_rho(tq_state* s, double* out) {
  tq_status st = check_state(s);
  if (st != TQ_OK) return st;
  if (!out) return TQ_ERR_ARG;
  const size_t entries = 1ull << (2 * s->n);
  cudaError_t e;
  if (s->prec == TQ_FP64) {
    void* full = nullptr;
    if ((st = tq_rho_device_ptr(s, &full)) != TQ_OK) return st;  // fills the lower triangle if needed
    e = cudaMemcpyAsync(out, s->rho, entries * 16, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return readout_done(s, e);
  }
  const size_t chunk = std::min<size_t>(entries, 1ull << 22);  // complex entries per pass
  if ((st = ensure(s, s->staging, chunk * 16)) != TQ_OK) return st;
  void* full = nullptr;
  if ((st = tq_rho_device_ptr(s, &full)) != TQ_OK) return st;  // fills the lower triangle if needed
  for (size_t c0 = 0; c0 < entries; c0 += chunk) {
    const size_t cnt = std::min(chunk, entries - c0);
    e = launch_convert_f32_to_f64(static_cast<const float*>(s->rho) + 2 * c0, static_cast<double*>(s->staging.ptr),
                                  2 * cnt, s->stream);
    s->launches += 1;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out + 2 * c0, s->staging.ptr, cnt * 16, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e);
  }
  return readout_done(s, cudaSuccess);
}

tq_status tq_set_rho(tq_state* s, const double* in) {
  tq_status st = check_state(s);
  if (st != TQ_OK) return st;
  if (!in) return TQ_ERR_ARG;
  const size_t entries = 1ull << (2 * s->n);
  cudaError_t e;
  if (s->prec == TQ_FP64) {
    e = cudaMemcpyAsync(s->rho, in, entries * 16, cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e);
    return check_hermitian(s);
  }
  const size_t chunk = std::min<size_t>(entries, 1ull << 22);
  if ((st = ensure(s, s->staging, chunk * 16)) != TQ_OK) return st;
  for (size_t c0 = 0; c0 < entries; c0 += chunk) {
    const size_t cnt = std::min(chunk, entries - c0);
    e = cudaMemcpyAsync(s->staging.ptr, in + 2 * c0, cnt * 16, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
      e = launch_convert_f64_to_f32(static_cast<const double*>(s->staging.ptr), static_cast<float*>(s->rho) + 2 * c0,
                                    2 * cnt, s->stream);
    s->launches += 1;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e);
  }
  return check_hermitian(s);
}

tq_status tq_apply_gate(tq_state* s, const int* qubits, int k, const double* U) {
  if (!qubits || !U || k < 1 || k > kMaxWidth) return TQ_ERR_ARG;
  tq_op op{};
  op.kind = TQ_OP_UNITARY;
  op.k = k;
  for (int j = 0; j < k; ++j) op.qubits[j] = qubits[j];
  op.m = 1;
  op.mats = U;
  return run_impl(s, &op, 1, 0, nullptr);
}

tq_status tq_apply_kraus(tq_state* s, const int* qubits, int k, int m, const double* K) {
  if (!qubits || !K || k < 1 || k > kMaxWidth || m < 1) return TQ_ERR_ARG;
  tq_op op{};
  op.kind = TQ_OP_KRAUS;
  op.k = k;
  for (int j = 0; j < k; ++j) op.qubits[j] = qubits[j];
  op.m = m;
  op.mats = K;
  return run_impl(s, &op, 1, 0, nullptr);
}

tq_status tq_run_circuit(tq_state* s, const tq_op* ops, size_t n_ops, int max_fuse_width, size_t* n_blocks_out) {
  return run_impl(s, ops, n_ops, max_fuse_width, n_blocks_out);
}

tq_status tq_program_create(int n, int precision, const tq_op* ops, size_t n_ops, int max_fuse_width,
                            tq_program** out) {
  if (!out) return TQ_ERR_ARG;
  *out = nullptr;
  if (n < 1 || n > kMaxQubits || (precision != TQ_FP64 && precision != TQ_SPLIT) || (!ops && n_ops))
    return TQ_ERR_ARG;
  tq_program* P = new (std::nothrow) tq_program();
  if (!P) return TQ_ERR_OOM;
  HostTables t;
  tq_status st = plan_program(n, precision, ops, n_ops, max_fuse_width, P, &t, kAutoTensor);
  if (st != TQ_OK) {
    delete P;
    return st;
  }
  cudaError_t e = grow(P->blob, P->blob_bytes, nullptr, false);
  if (e == cudaSuccess) e = grow(P->sops, t.sop_entries * sizeof(double2) + 16, nullptr, false);
  if (e == cudaSuccess) e = grow(P->sb64, t.sb_entries * sizeof(double2) + 16, nullptr, false);
  if (e == cudaSuccess && precision == TQ_SPLIT) e = grow(P->sb32, t.sb_entries * sizeof(float2) + 16, nullptr, false);
  if (e == cudaSuccess && P->n_sparse > 0) e = grow(P->sps, (size_t)P->n_sparse * sizeof(SparseBlock), nullptr, false);
  if (e == cudaSuccess) {
    std::vector<char> h(P->blob_bytes);
    pack_blob(*P, t, h.data());
    e = cudaMemcpy(P->blob.ptr, h.data(), P->blob_bytes, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    tq_program_free(P);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      return TQ_ERR_OOM;
    }
    return TQ_ERR_CUDA;
  }
  *out = P;
  return TQ_OK;
}

tq_status tq_program_run(tq_state* s, const tq_program* p) {
  tq_status st = check_state(s);
  if (st != TQ_OK) return st;
  if (!p || p->n != s->n || p->prec != s->prec) return TQ_ERR_ARG;
  if (s->prof_on) return enqueue_program(s, *p);  // per-launch events: launch directly
  if (!p->g_blk_ready && cluster_program_eligible(p->n, p->max_width, p->params.size())) {
    std::vector<unsigned char> tab;
    cluster_block_table(p->params, p->sb_off, &tab);
    cudaError_t e = grow(p->g_blk, tab.size(), nullptr, false);
    if (e == cudaSuccess) e = cudaMemcpy(p->g_blk.ptr, tab.data(), tab.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(s, e);
    p->g_blk_ready = true;
  }
  const int key = (s->herm_mode && s->herm_ok ? 1 : 0) | (s->lower_stale ? 2 : 0) | (fp64_on_tensor(s) ? 4 : 0);
  if (!(p->g_exec && p->g_rho == s->rho && p->g_key == key)) {
    // (re)capture the launch sequence on a private stream; the state's flags
    // and launch count advance as if it ran, which is what the graph does
    if (p->g_exec) {  // an earlier launch may still run on any stream (rare path)
      cudaDeviceSynchronize();
      cudaGraphExecDestroy(p->g_exec);
    }
    p->g_exec = nullptr;
    if (!p->g_capture && cudaStreamCreateWithFlags(&p->g_capture, cudaStreamNonBlocking) != cudaSuccess) {
      p->g_capture = nullptr;
      return enqueue_program(s, *p);
    }
    const bool lower0 = s->lower_stale;
    const uint64_t l0 = s->launches;
    cudaStream_t real = s->stream;
    s->stream = p->g_capture;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(p->g_capture, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      st = enqueue_program(s, *p);
      e = cudaStreamEndCapture(p->g_capture, &g);
    }
    s->stream = real;
    if (e == cudaSuccess && st == TQ_OK) e = cudaGraphInstantiate(&p->g_exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess || st != TQ_OK || !p->g_exec) {  // not capturable here: run directly
      cudaGetLastError();
      p->g_exec = nullptr;
      s->lower_stale = lower0;
      s->launches = l0;
      s->poisoned = false;
      return enqueue_program(s, *p);
    }
    p->g_rho = s->rho;
    p->g_key = key;
    p->g_lower_after = s->lower_stale;
    p->g_launches = s->launches - l0;
  } else {
    s->lower_stale = p->g_lower_after;
    s->launches += p->g_launches;
  }
  return cuda_fail(s, cudaGraphLaunch(p->g_exec, s->stream));
}

tq_status tq_program_info(const tq_program* p, size_t* n_ops, size_t* n_blocks, int* max_width,
                          size_t* table_bytes) {
  if (!p) return TQ_ERR_ARG;
  if (table_bytes) *table_bytes = p->blob_bytes;
  if (n_ops) *n_ops = p->n_ops;
  if (n_blocks) *n_blocks = p->params.size();
  if (max_width) *max_width = p->max_width;
  return TQ_OK;
}

void tq_program_free(tq_program* p) {
  if (!p) return;
  if (p->g_exec) {
    cudaDeviceSynchronize();  // its launches may still run on any stream
    cudaGraphExecDestroy(p->g_exec);
  }
  if (p->g_capture) {
    cudaStreamSynchronize(p->g_capture);
    cudaStreamDestroy(p->g_capture);
  }
  for (DevBuf* b : {&p->blob, &p->sops, &p->sb64, &p->sb32, &p->sps, &p->g_blk}) free_buf(*b);
  delete p;
}

tq_status tq_trace(tq_state* s, double* re, double* im) {
  tq_status st = check_state(s);
  if (st != TQ_OK) return st;
  double out[2];
  if ((st = reduce_impl(s, nullptr, 0, false, out)) != TQ_OK) return st;
  if (re) *re = out[0];
  if (im) *im = out[1];
  return TQ_OK;
}

tq_status tq_expect_z(tq_state* s, const uint64_t* masks, int n_masks, double* out) {
  tq_status st = check_state(s);
  if (st != TQ_OK) return st;
  if (n_masks < 0 || (n_masks > 0 && (!masks || !out))) return TQ_ERR_ARG;
  double buf[18];
  for (int m0 = 0; m0 < n_masks; m0 += 16) {
    const int cnt = std::min(16, n_masks - m0);
    if ((st = reduce_impl(s, reinterpret_cast<const unsigned long long*>(masks + m0), cnt, s->prec == TQ_SPLIT, buf)) != TQ_OK)
      return st;
    for (int i = 0; i < cnt; ++i) out[m0 + i] = buf[2 + i];
  }
  return TQ_OK;
}

tq_status tq_expect_z_device(tq_state* s, const uint64_t* masks_dev, int n_masks, double* out_dev) {
  tq_status st = check_state(s);
  if (st != TQ_OK) return st;
  if (n_masks < 1 || n_masks > 16 || !masks_dev || !out_dev) return TQ_ERR_ARG;
  return reduce_device(s, reinterpret_cast<const unsigned long long*>(masks_dev), n_masks, s->prec == TQ_SPLIT, out_dev);
}

}  // extern "C"

namespace {

// Outcome probabilities (renormalised for split states) into s->probs on
// the device, then the optional per-qubit readout confusion.
tq_status probs_device(tq_state* s, const double* e10, const double* e01) {
  const size_t N = 1ull << s->n;
  tq_status st = ensure(s, s->probs, 2 * N * sizeof(double));  // probabilities, then the CDF
  if (st != TQ_OK) return st;
  const double* tr = nullptr;
  if (s->prec == TQ_SPLIT) {
    double tmp[2];
    if ((st = reduce_impl(s, nullptr, 0, false, tmp)) != TQ_OK) return st;
    tr = reinterpret_cast<const double*>(static_cast<char*>(s->red.ptr) + kRedOut);
  }
  cudaError_t e = launch_diag_probs(s->rho, s->n, s->prec, tr, static_cast<double*>(s->probs.ptr), s->stream);
  s->launches += 1;
  if (e == cudaSuccess && e10 && e01) {
    e = launch_readout(static_cast<double*>(s->probs.ptr), s->n, e10, e01, s->stream);
    s->launches += s->n;
  }
  return cuda_fail(s, e);
}

bool rates_ok(const double* e, int n) {
  for (int q = 0; q < n; ++q)
    if (!(e[q] >= 0.0 && e[q] <= 1.0)) return false;
  return true;
}

}  // namespace

extern "C" {

tq_status tq_probs(tq_state* s, double* out) {
  tq_status st = check_state(s);
  if (st != TQ_OK) return st;
  if (!out) return TQ_ERR_ARG;
  if ((st = probs_device(s, nullptr, nullptr)) != TQ_OK) return st;
  const size_t N = 1ull << s->n;
  cudaError_t e = cudaMemcpyAsync(out, s->probs.ptr, N * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return readout_done(s, e);
}

tq_status tq_probs_readout(tq_state* s, const double* e10, const double* e01, double* out) {
  tq_status st = check_state(s);
  if (st != TQ_OK) return st;
  if (!out || !e10 || !e01 || !rates_ok(e10, s->n) || !rates_ok(e01, s->n)) return TQ_ERR_ARG;
  if ((st = probs_device(s, e10, e01)) != TQ_OK) return st;
  const size_t N = 1ull << s->n;
  cudaError_t e = cudaMemcpyAsync(out, s->probs.ptr, N * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return readout_done(s, e);
}

tq_status tq_sample(tq_state* s, const double* u, int shots, const double* e10, const double* e01,
                    uint64_t* outcomes) {
  tq_status st = check_state(s);
  if (st != TQ_OK) return st;
  if (shots < 0 || (shots > 0 && (!u || !outcomes)) || (!e10) != (!e01)) return TQ_ERR_ARG;
  if (e10 && (!rates_ok(e10, s->n) || !rates_ok(e01, s->n))) return TQ_ERR_ARG;
  for (int i = 0; i < shots; ++i)
    if (!(u[i] >= 0.0 && u[i] < 1.0)) return TQ_ERR_ARG;
  if (shots == 0) return TQ_OK;
  if ((st = probs_device(s, e10, e01)) != TQ_OK) return st;
  const size_t N = 1ull << s->n;
  const size_t bytes = (size_t)shots * 16;
  if ((st = ensure(s, s->shots, bytes)) != TQ_OK) return st;
  if ((st = ensure_pinned(s, s->pin, bytes)) != TQ_OK) return st;
  cudaError_t e = cudaEventSynchronize(s->pin_free);  // the staging buffer is shared with uploads
  if (e != cudaSuccess) return cuda_fail(s, e);
  std::memcpy(s->pin.ptr, u, (size_t)shots * sizeof(double));
  double* du = static_cast<double*>(s->shots.ptr);
  unsigned long long* dout = reinterpret_cast<unsigned long long*>(du + shots);
  e = cudaMemcpyAsync(du, s->pin.ptr, (size_t)shots * sizeof(double), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess)
    e = launch_sample(static_cast<const double*>(s->probs.ptr), s->n, static_cast<double*>(s->probs.ptr) + N, du,
                      shots, dout, s->stream);
  s->launches += 2;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->pin.ptr, dout, (size_t)shots * sizeof(uint64_t), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if ((st = readout_done(s, e)) != TQ_OK) return st;
  std::memcpy(outcomes, s->pin.ptr, (size_t)shots * sizeof(uint64_t));
  return TQ_OK;
}

tq_status tq_measure(tq_state* s, int qubit, double u, int* outcome, double* probability) {
  tq_status st = check_state(s);
  if (st != TQ_OK) return st;
  if (qubit < 0 || qubit >= s->n) return TQ_ERR_QUBIT;
  if (!outcome || !(u >= 0.0 && u < 1.0)) return TQ_ERR_ARG;
  const unsigned long long mask = 1ull << qubit;
  double red[3];
  if ((st = reduce_impl(s, &mask, 1, false, red)) != TQ_OK) return st;  // Re tr, Im tr, Re Tr(rho Z_q)
  const double tr = red[0];
  const double p0 = 0.5 * (tr + red[2]);
  if (!(tr > 0.0)) return TQ_ERR_ARG;
  const int m = u < p0 / tr ? 0 : 1;
  const double pm = m == 0 ? p0 : tr - p0;
  if (!(pm > 0.0)) return TQ_ERR_ARG;
  // project with |m><m| and renormalise: one Kraus matrix |m><m| / sqrt(p_m)
  double K[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  K[m == 0 ? 0 : 6] = 1.0 / std::sqrt(pm);
  tq_op op{};
  op.kind = TQ_OP_KRAUS;
  op.k = 1;
  op.qubits[0] = qubit;
  op.m = 1;
  op.mats = K;
  if ((st = run_impl(s, &op, 1, 0, nullptr)) != TQ_OK) return st;
  *outcome = m;
  if (probability) *probability = pm / tr;
  return TQ_OK;
}

tq_status tq_profile_enable(tq_state* s, int on) {
  if (!s) return TQ_ERR_ARG;
  if (on) {
    cudaStreamSynchronize(s->stream);
    fold_pending(s);
    s->counts.release();
    for (int k = 0; k < K_NKINDS; ++k) {
      s->prof_launches[k] = 0;
      s->prof_ms[k] = s->prof_flops[k] = s->prof_bytes[k] = 0.0;
    }
  }
  s->prof_on = on != 0;
  return TQ_OK;
}

tq_status tq_profile_read(tq_state* s, tq_kernel_stat* out, int capacity, int* count) {
  if (!s || !count || (capacity > 0 && !out)) return TQ_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e);
  fold_pending(s);
  int c = 0;
  for (int k = 0; k < K_NKINDS; ++k) {
    if (!s->prof_launches[k]) continue;
    if (c < capacity) {
      tq_kernel_stat& o = out[c];
      std::memset(&o, 0, sizeof(o));
      std::strncpy(o.name, kKindName[k], sizeof(o.name) - 1);
      o.launches = s->prof_launches[k];
      o.total_ms = s->prof_ms[k];
      o.flops = s->prof_flops[k] / (double)s->prof_launches[k];
      o.bytes = s->prof_bytes[k] / (double)s->prof_launches[k];
    }
    ++c;
  }
  *count = c;
  return TQ_OK;
}

tq_status tq_launch_count(const tq_state* s, uint64_t* out) {
  if (!s || !out) return TQ_ERR_ARG;
  *out = s->launches;
  return TQ_OK;
}

}  // extern "C"
