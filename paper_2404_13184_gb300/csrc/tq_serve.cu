// Continuous-batching serving loop for noisy-circuit requests.
//
// Requests wait in a FIFO queue and are admitted, in order, while their
// density matrix (16 * 4^n bytes in FP64, 8 * 4^n in split) fits the HBM
// budget of the rho arena and a live slot is free. Admission uploads the
// request's Kraus sets and plan, builds and fuses its superoperators (FP64,
// on the GPU) and resets its rho; rho then stays resident until the request
// finishes. Every tick launches ONE persistent batch kernel (the work-item
// scheme of tq_batch_kernels.cuh) that advances every live request by a
// quantum of fused blocks, so requests that arrive while others run join the
// next tick. Finished requests are reduced (trace, <Z_mask>), their memory
// returns to the arenas, and the next queued requests are admitted.
#include <algorithm>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <unordered_map>
#include <vector>

#include "tq_batch_kernels.cuh"

using namespace tq;
using namespace tq::batch;

namespace {

// First-fit allocator over one device range (offsets; host bookkeeping).
class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align_up(std::max<size_t>(bytes, 256), 256);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rem = it->second - bytes;
        const size_t noff = it->first + bytes;
        free_.erase(it);
        if (rem) free_[noff] = rem;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(std::max<size_t>(bytes, 256), 256);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<size_t, size_t> free_;
};

// Requests of at least this many qubits advance through the single-state
// apply kernels, one launch per fused block, instead of the persistent
// batch kernel: their passes are long (>= ~40 us) next to a launch, and the
// single-state kernels run on the tensor cores (split width 2; FP64 widths
// <= 2 with the tensor-core engine), closer to the HBM bound than the batch
// kernel's CUDA-core tiles.
constexpr int kDirectQubits = 12;

struct Req {
  int n = 0;
  std::vector<unsigned long long> masks;
  tq_program prog;
  HostTables t;
  size_t rho_off = 0, rho_bytes = 0;
  size_t tab_off = 0, tab_bytes = 0;
  size_t o_sops = 0, o_sb = 0, o_sb64 = 0;  // within the table allocation
  size_t o_pwork = 0, o_pauli = 0;          // Pauli-basis records and their sb64 offsets
  std::vector<long long> blk_rec;           // per block: its Pauli record, or -1
  std::vector<unsigned long long> rec_sb;   // per record: its block's sb64 offset
  int next_block = 0;
  int state = 0;  // 0 queued, 1 live, 2 done
  double result[2 + 16] = {};
};

}  // namespace

struct tq_server {
  int prec = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 152;
  int per_sm = 1;
  int max_live = 64;
  long long max_spin = 20000000;
  size_t rho_budget = 0, tab_budget = 0;
  DevBuf rho_mem, tab_mem, djobs, dblks, ditems, counters, ctl, results;
  // pinned staging, one buffer per use so that nothing in a tick waits for
  // the tick's own copies: admission blobs, tick tables, readout results
  // (all free again once the previous tick has been collected)
  PinBuf pin, pin_tick, pin_res;
  Arena rho_arena, tab_arena;
  std::unordered_map<int, Req> reqs;
  std::deque<int> queue;
  std::vector<int> live;
  int next_id = 0;
  size_t rho_live_bytes = 0;
  unsigned long long ticks = 0, blocks_applied = 0;
  // the launched, not yet collected tick: requests it finishes (results land
  // in `pin` at res_off), whether it ran items (error flag at err_off)
  bool pending = false;
  std::vector<int> pend_done;
  bool pend_items = false;
  size_t res_off = 0, err_off = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // GPU time of the pending tick
  double gpu_ms = 0.0;
  int fp64_engine = TQ_ENGINE_AUTO;  // tq_server_set_fp64_engine
  bool pend_direct_tc = false;       // the pending tick launched tensor-core passes
};

namespace {

// Whether a live request of n qubits advances through single-state launches.
bool direct_request(const tq_server* s, int n) {
  if (n < kDirectQubits) return false;
  if (s->prec == TQ_SPLIT) return true;
  return fp64_engine_is_tensor(s->fp64_engine) && oz_eligible(n, 2);
}

tq_status st_of(cudaError_t e) {
  if (e == cudaSuccess) return TQ_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return TQ_ERR_OOM;
  }
  return TQ_ERR_CUDA;
}

cudaError_t grow_dev(DevBuf& b, size_t bytes) {
  if (b.cap >= bytes && b.ptr) return cudaSuccess;
  if (b.ptr) cudaFree(b.ptr);
  b.ptr = nullptr;
  b.cap = 0;
  const size_t want = align_up(std::max<size_t>(bytes, 4096) * 2, 4096);
  cudaError_t e = cudaMalloc(&b.ptr, want);
  if (e == cudaSuccess) b.cap = want;
  return e;
}

cudaError_t grow_pin(PinBuf& b, size_t bytes) {
  if (b.cap >= bytes && b.ptr) return cudaSuccess;
  if (b.ptr) cudaFreeHost(b.ptr);
  b.ptr = nullptr;
  b.cap = 0;
  const size_t want = align_up(std::max<size_t>(bytes, 4096) * 2, 4096);
  cudaError_t e = cudaHostAlloc(&b.ptr, want, cudaHostAllocDefault);
  if (e == cudaSuccess) b.cap = want;
  return e;
}

size_t entry_size(int prec) { return prec == TQ_FP64 ? 16 : 8; }


// Blocks a live request advances per tick: about 8 passes of a 12-qubit
// register's worth of entries, at least one block.
int quantum(int n) {
  const int shift = 2 * (12 - n);
  if (shift <= 0) return std::max(1, 8 >> std::min(30, -shift));
  return (int)std::min<long long>(1 << 20, 8ll << std::min(shift, 24));
}

// Layout of a request's table allocation: the uploaded blob, the per-op
// superoperators, the fused FP64 superoperators, (split) their FP32 copies,
// and the Pauli-basis records of its width-2 blocks with their sb64
// offsets. Sets r.o_sops, r.o_sb, r.o_pwork, r.o_pauli and r.tab_bytes;
// returns the FP64 fused table's offset.
size_t table_layout(int prec, Req& r) {
  size_t off = align_up(r.prog.blob_bytes, 256);
  r.o_sops = off;
  off = align_up(off + r.t.sop_entries * sizeof(double2), 256);
  const size_t o_sb64 = off;
  r.o_sb64 = o_sb64;
  off = align_up(off + r.t.sb_entries * sizeof(double2), 256);
  r.o_sb = prec == TQ_FP64 ? o_sb64 : off;
  if (prec == TQ_SPLIT) off = align_up(off + r.t.sb_entries * sizeof(float2), 256);
  r.o_pwork = off;
  off = align_up(off + r.rec_sb.size() * sizeof(unsigned long long), 256);
  r.o_pauli = off;
  off = align_up(off + r.rec_sb.size() * sizeof(PauliRec), 256);
  r.tab_bytes = off;
  return o_sb64;
}

// Pauli-basis records for the width-2 blocks of a request that runs as a
// tile job of the batch kernel (not resident in shared memory, not direct).
void plan_pauli(const tq_server* s, Req& r) {
  r.blk_rec.assign(r.prog.params.size(), -1);
  r.rec_sb.clear();
  if (is_resident(r.n, s->prec) || direct_request(s, r.n)) return;
  for (size_t k = 0; k < r.prog.params.size(); ++k)
    if (r.prog.params[k].width == 2) {
      r.blk_rec[k] = (long long)r.rec_sb.size();
      r.rec_sb.push_back((unsigned long long)r.prog.sb_off[k]);
    }
}

// Admit the request: allocate, upload its tables, build + fuse, reset rho.
tq_status admit(tq_server* s, Req& r, char* stage, size_t* stage_used) {
  const size_t esz = entry_size(s->prec);
  r.rho_bytes = esz << (2 * r.n);
  if (!s->rho_arena.alloc(r.rho_bytes, &r.rho_off)) return TQ_ERR_OOM;
  const tq_program& P = r.prog;
  const size_t o_sb64 = table_layout(s->prec, r);
  if (!s->tab_arena.alloc(r.tab_bytes, &r.tab_off)) {
    s->rho_arena.release(r.rho_off, r.rho_bytes);
    return TQ_ERR_OOM;
  }
  char* tab = static_cast<char*>(s->tab_mem.ptr) + r.tab_off;
  char* h = stage + *stage_used;
  pack_blob(P, r.t, h);
  *stage_used = align_up(*stage_used + P.blob_bytes, 256);
  cudaError_t e = cudaMemcpyAsync(tab, h, P.blob_bytes, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess && !r.rec_sb.empty()) {
    char* hw = stage + *stage_used;
    const size_t bytes = r.rec_sb.size() * sizeof(unsigned long long);
    std::memcpy(hw, r.rec_sb.data(), bytes);
    *stage_used = align_up(*stage_used + bytes, 256);
    e = cudaMemcpyAsync(tab + r.o_pwork, hw, bytes, cudaMemcpyHostToDevice, s->stream);
  }
  if (e == cudaSuccess && P.n_uops > 0) {
    e = launch_build_superops(reinterpret_cast<const double2*>(tab + P.o_kraus), reinterpret_cast<const OpDesc*>(tab + P.o_ops),
                              (int)P.n_uops, P.max_dim2, reinterpret_cast<double2*>(tab + r.o_sops), s->stream);
    if (e == cudaSuccess)
      e = launch_fuse(reinterpret_cast<const double2*>(tab + r.o_sops), reinterpret_cast<const OpDesc*>(tab + P.o_ops),
                      reinterpret_cast<const BlockDesc*>(tab + P.o_blk), reinterpret_cast<const MemberDesc*>(tab + P.o_mem),
                      reinterpret_cast<const FuseWork*>(tab + P.o_work), P.n_work, reinterpret_cast<double2*>(tab + o_sb64),
                      s->prec == TQ_SPLIT ? reinterpret_cast<float2*>(tab + r.o_sb) : nullptr, s->stream);
    if (e == cudaSuccess)
      e = launch_pauli_lists(reinterpret_cast<const double2*>(tab + o_sb64),
                             reinterpret_cast<const unsigned long long*>(tab + r.o_pwork), (int)r.rec_sb.size(),
                             s->prec == TQ_FP64 ? 0 : 1, reinterpret_cast<PauliRec*>(tab + r.o_pauli), s->stream);
  }
  if (e == cudaSuccess)
    e = launch_init_zero_state(static_cast<char*>(s->rho_mem.ptr) + r.rho_off, r.n, s->prec, s->stream);
  if (e != cudaSuccess) return st_of(e);
  r.state = 1;
  r.next_block = 0;
  s->rho_live_bytes += r.rho_bytes;
  return TQ_OK;
}

void retire(tq_server* s, Req& r) {
  s->rho_arena.release(r.rho_off, r.rho_bytes);
  s->tab_arena.release(r.tab_off, r.tab_bytes);
  s->rho_live_bytes -= r.rho_bytes;
  r.state = 2;
  r.prog.params.clear();
  r.prog.params.shrink_to_fit();
  r.t = HostTables();
}

}  // namespace

extern "C" {

tq_status tq_server_create(int precision, void* cuda_stream, size_t rho_budget_bytes, size_t table_budget_bytes,
                           int max_live, tq_server** out) {
  if (!out || (precision != TQ_FP64 && precision != TQ_SPLIT) || rho_budget_bytes < 256 || table_budget_bytes < 4096 ||
      max_live < 1)
    return TQ_ERR_ARG;
  *out = nullptr;
  tq_server* s = new (std::nothrow) tq_server();
  if (!s) return TQ_ERR_OOM;
  s->prec = precision;
  s->stream = static_cast<cudaStream_t>(cuda_stream);
  s->max_live = max_live;
  s->rho_budget = align_up(rho_budget_bytes, 256);
  s->tab_budget = align_up(table_budget_bytes, 256);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaMalloc(&s->rho_mem.ptr, s->rho_budget);
  if (e == cudaSuccess) {
    s->rho_mem.cap = s->rho_budget;
    e = cudaMalloc(&s->tab_mem.ptr, s->tab_budget);
  }
  if (e == cudaSuccess) {
    s->tab_mem.cap = s->tab_budget;
    const size_t smem = precision == TQ_FP64 ? apply_smem<double2>() : apply_smem<float2>();
    if (precision == TQ_FP64) {
      e = cudaFuncSetAttribute(k_batch_apply<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s->per_sm, k_batch_apply<double2>, kThreads, smem);
    } else {
      e = cudaFuncSetAttribute(k_batch_apply<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s->per_sm, k_batch_apply<float2>, kThreads, smem);
    }
  }
  if (e == cudaSuccess) e = cudaEventCreate(&s->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&s->ev1);
  if (e != cudaSuccess) {
    tq_server_free(s);
    return st_of(e);
  }
  s->per_sm = std::max(1, s->per_sm);
  s->rho_arena.reset(s->rho_budget);
  s->tab_arena.reset(s->tab_budget);
  *out = s;
  return TQ_OK;
}

tq_status tq_server_submit(tq_server* s, int n_qubits, const tq_op* ops, size_t n_ops, int max_fuse_width,
                           const uint64_t* masks, int n_masks, int* request_id) {
  if (!s || (!ops && n_ops) || n_masks < 0 || n_masks > kMaxMasks || (n_masks && !masks)) return TQ_ERR_ARG;
  if (n_qubits < 1 || n_qubits > kMaxQubits) return TQ_ERR_ARG;
  if (max_fuse_width > 2) return TQ_ERR_UNSUPPORTED;
  if (entry_size(s->prec) << (2 * n_qubits) > s->rho_budget) return TQ_ERR_OOM;  // can never be admitted
  Req r;
  r.n = n_qubits;
  tq_status st = plan_program(n_qubits, s->prec, ops, n_ops, max_fuse_width, &r.prog, &r.t);
  if (st == TQ_OK && r.prog.max_width > 2) {
    r = Req();
    r.n = n_qubits;
    st = plan_program(n_qubits, s->prec, ops, n_ops, 2, &r.prog, &r.t);
    if (st == TQ_OK && r.prog.max_width > 2) st = TQ_ERR_UNSUPPORTED;
  }
  if (st != TQ_OK) return st;
  // its tables must fit the table arena on their own, or it would block the
  // FIFO head forever
  plan_pauli(s, r);
  table_layout(s->prec, r);
  if (align_up(r.tab_bytes, 256) > s->tab_budget) return TQ_ERR_OOM;
  for (int m = 0; m < n_masks; ++m) r.masks.push_back(masks[m]);
  const int id = s->next_id++;
  s->reqs.emplace(id, std::move(r));
  s->queue.push_back(id);
  if (request_id) *request_id = id;
  return TQ_OK;
}

}  // extern "C"

namespace {

// Collect the pending tick: wait for it, hand the finished requests their
// readouts and release their memory. *n_finished: requests it finished.
tq_status collect_tick(tq_server* s, int* n_finished) {
  if (n_finished) *n_finished = 0;
  if (!s->pending) return TQ_OK;
  s->pending = false;
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return st_of(e);
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, s->ev0, s->ev1) == cudaSuccess) s->gpu_ms += ms;
  const char* h = static_cast<const char*>(s->pin_res.ptr);
  int err_flag = 0;
  if (s->pend_items) std::memcpy(&err_flag, h + s->err_off, sizeof(int));
  if (s->pend_direct_tc) {  // bounded waits of the tick's tensor-core passes
    unsigned int a = 0, b = 0;
    e = tc_take_timeouts(&a, s->stream);
    if (e == cudaSuccess) e = oz_take_timeouts(&b, s->stream);
    if (e != cudaSuccess) return st_of(e);
    if (a || b) err_flag = 1;
    s->pend_direct_tc = false;
  }
  if (!s->pend_done.empty()) {
    const double* res = reinterpret_cast<const double*>(h + s->res_off);
    for (size_t k = 0; k < s->pend_done.size(); ++k) {
      Req& r = s->reqs[s->pend_done[k]];
      std::memcpy(r.result, res + k * kResults, kResults * sizeof(double));
      retire(s, r);
    }
    std::vector<int> still;
    for (int id : s->live)
      if (s->reqs[id].state == 1) still.push_back(id);
    s->live.swap(still);
  }
  if (n_finished) *n_finished = (int)s->pend_done.size();
  s->pend_done.clear();
  return err_flag ? TQ_ERR_TIMEOUT : TQ_OK;
}

// Admit and launch one tick without waiting for it. The previous tick must
// have been collected (which waited for the stream), so every staging buffer
// is free; each is written once per tick, so no step below waits for the GPU.
tq_status launch_tick(tq_server* s, int* n_live, int* n_queued) {
  cudaEventRecord(s->ev0, s->stream);
  // 1. admission, FIFO by HBM footprint: stop at the first request that does not fit
  size_t stage_need = 0;
  std::vector<int> admit_ids;
  {
    size_t probe_live = s->live.size();
    for (int id : s->queue) {
      if ((int)probe_live >= s->max_live) break;
      const Req& q = s->reqs[id];
      stage_need += align_up(q.prog.blob_bytes, 256) + align_up(q.rec_sb.size() * sizeof(unsigned long long), 256);
      admit_ids.push_back(id);
      ++probe_live;
    }
  }
  // tick tables size (upper bound, computed after admission)
  cudaError_t e = grow_pin(s->pin, stage_need + 4096);
  if (e != cudaSuccess) return st_of(e);
  size_t used = 0;
  int admitted = 0;
  for (int id : admit_ids) {
    Req& r = s->reqs[id];
    tq_status st = admit(s, r, static_cast<char*>(s->pin.ptr), &used);
    if (st == TQ_ERR_OOM) break;  // does not fit yet: wait for memory to free up
    if (st != TQ_OK) return st;
    s->queue.pop_front();
    s->live.push_back(id);
    ++admitted;
  }
  // 2. this tick's work: every live request advances by its quantum
  std::vector<BJob> jobs;
  std::vector<BBlk> blks;
  std::vector<BItem> items;
  std::vector<int> job_req;
  std::vector<int> finishing;
  int max_cnt = 0;
  std::vector<int> cnts, is_direct;
  for (int id : s->live) {
    Req& r = s->reqs[id];
    const int nb = (int)r.prog.params.size();
    const int cnt = std::min(nb - r.next_block, quantum(r.n));
    BJob j;
    std::memset(&j, 0, sizeof(j));
    j.rho_off = r.rho_off;
    j.n = r.n;
    j.n_blocks = cnt;
    j.block0 = (int)blks.size();
    j.tile_log2 = std::min(std::max({std::min(2 * r.n, 16), 4, 2 * r.n - 16}), 2 * r.n);
    j.resident = is_resident(r.n, s->prec) ? 1 : 0;
    j.herm = batch_herm(r.n, s->prec) ? 1 : 0;
    j.n_masks = (int)r.masks.size();
    for (size_t m = 0; m < r.masks.size(); ++m) j.masks[m] = r.masks[m];
    const size_t esz = s->prec == TQ_FP64 ? sizeof(double2) : sizeof(float2);
    const char* sb = static_cast<const char*>(s->tab_mem.ptr) + r.tab_off + r.o_sb;
    const PauliRec* recs =
        reinterpret_cast<const PauliRec*>(static_cast<const char*>(s->tab_mem.ptr) + r.tab_off + r.o_pauli);
    for (int b = r.next_block; b < r.next_block + cnt; ++b) {
      BBlk bb;
      std::memset(&bb, 0, sizeof(bb));
      bb.p = r.prog.params[b];
      bb.S = sb + (size_t)r.prog.sb_off[b] * esz;
      bb.pauli = r.blk_rec[b] < 0 ? nullptr : recs + r.blk_rec[b];
      blks.push_back(bb);
    }
    set_tiles(blks.data() + j.block0, cnt, j.tile_log2, j.herm != 0, tiled16_job(r.n, s->prec));
    const bool direct = direct_request(s, r.n);
    if (cnt > 0 && j.resident && !direct) items.push_back(BItem{(int)jobs.size(), -1, 0, cnt});
    job_req.push_back(id);
    cnts.push_back(cnt);
    is_direct.push_back(direct ? 1 : 0);
    if (!j.resident && !direct) max_cnt = std::max(max_cnt, cnt);
    jobs.push_back(j);
  }
  for (int k = 0; k < max_cnt; ++k)
    for (size_t j = 0; j < jobs.size(); ++j) {
      if (jobs[j].resident || is_direct[j] || k >= cnts[j]) continue;
      const int tiles = blks[jobs[j].block0 + k].tiles;
      for (int t = 0; t < tiles; ++t) items.push_back(BItem{(int)j, k, t, 1});
    }
  if (!items.empty()) {
    const size_t bj = jobs.size() * sizeof(BJob), bb = blks.size() * sizeof(BBlk), bi = items.size() * sizeof(BItem);
    e = grow_dev(s->djobs, bj);
    if (e == cudaSuccess) e = grow_dev(s->dblks, bb);
    if (e == cudaSuccess) e = grow_dev(s->ditems, bi);
    if (e == cudaSuccess) e = grow_dev(s->counters, jobs.size() * sizeof(int));
    if (e == cudaSuccess) e = grow_dev(s->ctl, 256);
    if (e == cudaSuccess) e = grow_pin(s->pin_tick, bj + bb + bi + 1024);
    if (e != cudaSuccess) return st_of(e);
    char* h = static_cast<char*>(s->pin_tick.ptr);
    std::memcpy(h, jobs.data(), bj);
    std::memcpy(h + align_up(bj, 256), blks.data(), bb);
    std::memcpy(h + align_up(bj, 256) + align_up(bb, 256), items.data(), bi);
    e = cudaMemcpyAsync(s->djobs.ptr, h, bj, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->dblks.ptr, h + align_up(bj, 256), bb, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->ditems.ptr, h + align_up(bj, 256) + align_up(bb, 256), bi, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->counters.ptr, 0, jobs.size() * sizeof(int), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->ctl.ptr, 0, 256, s->stream);
    if (e != cudaSuccess) return st_of(e);
    int* ticket = static_cast<int*>(s->ctl.ptr);
    const int grid = (int)std::max<size_t>(1, std::min<size_t>(items.size(), (size_t)s->num_sms * s->per_sm));
    if (s->prec == TQ_FP64)
      k_batch_apply<double2><<<grid, kThreads, apply_smem<double2>(), s->stream>>>(
          static_cast<char*>(s->rho_mem.ptr), static_cast<const BJob*>(s->djobs.ptr), static_cast<const BBlk*>(s->dblks.ptr),
          static_cast<const BItem*>(s->ditems.ptr), (int)items.size(), static_cast<int*>(s->counters.ptr), ticket,
          ticket + 32, s->max_spin);
    else
      k_batch_apply<float2><<<grid, kThreads, apply_smem<float2>(), s->stream>>>(
          static_cast<char*>(s->rho_mem.ptr), static_cast<const BJob*>(s->djobs.ptr), static_cast<const BBlk*>(s->dblks.ptr),
          static_cast<const BItem*>(s->ditems.ptr), (int)items.size(), static_cast<int*>(s->counters.ptr), ticket,
          ticket + 32, s->max_spin);
    e = cudaGetLastError();
    if (e != cudaSuccess) return st_of(e);
  }
  // 2b. large requests: their blocks as single-state launches (Hermitian
  // mode, as in the batch kernel), after the batch kernel on the same stream
  for (size_t j = 0; j < jobs.size(); ++j) {
    if (!is_direct[j]) continue;
    char* rho = static_cast<char*>(s->rho_mem.ptr) + jobs[j].rho_off;
    for (int k = 0; k < cnts[j]; ++k) {
      const BBlk& bb = blks[jobs[j].block0 + k];
      ApplyParams p = bb.p;
      p.sparse = 0;
      if (s->prec == TQ_FP64) {
        e = launch_herm_oz(reinterpret_cast<double2*>(rho), static_cast<const double2*>(bb.S), p, s->num_sms,
                           s->stream);
        s->pend_direct_tc = true;
      } else if (p.width == 2) {
        e = launch_herm_tc2(reinterpret_cast<float2*>(rho), static_cast<const float2*>(bb.S), p, s->num_sms,
                            s->stream);
        s->pend_direct_tc = true;
      } else {
        e = launch_apply(rho, TQ_SPLIT, bb.S, p, s->num_sms, s->stream);
      }
      if (e != cudaSuccess) return st_of(e);
    }
  }
  // 3. progress; readouts of the requests this tick finishes are reduced and
  // copied to the staging buffer behind the tick (collected later)
  std::vector<BJob> done_jobs;
  std::vector<int> done_ids;
  for (size_t j = 0; j < jobs.size(); ++j) {
    Req& r = s->reqs[job_req[j]];
    r.next_block += cnts[j];
    s->blocks_applied += cnts[j];
    if (r.next_block >= (int)r.prog.params.size()) {
      done_jobs.push_back(jobs[j]);
      done_ids.push_back(job_req[j]);
    }
  }
  const size_t bj = done_jobs.size() * sizeof(BJob);
  const size_t br = done_jobs.size() * kResults * sizeof(double);
  e = grow_pin(s->pin_res, align_up(bj, 256) + br + 256);
  if (e != cudaSuccess) return st_of(e);
  char* h = static_cast<char*>(s->pin_res.ptr);
  s->res_off = align_up(bj, 256);
  s->err_off = s->res_off + br;
  if (!done_jobs.empty()) {
    e = grow_dev(s->results, br + bj);
    if (e != cudaSuccess) return st_of(e);
    std::memcpy(h, done_jobs.data(), bj);
    char* dres = static_cast<char*>(s->results.ptr);
    e = cudaMemcpyAsync(dres + br, h, bj, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) {
      if (s->prec == TQ_FP64)
        k_batch_reduce<double2><<<(int)done_jobs.size(), kThreads, 0, s->stream>>>(
            static_cast<const char*>(s->rho_mem.ptr), reinterpret_cast<const BJob*>(dres + br), 0,
            reinterpret_cast<double*>(dres));
      else
        k_batch_reduce<float2><<<(int)done_jobs.size(), kThreads, 0, s->stream>>>(
            static_cast<const char*>(s->rho_mem.ptr), reinterpret_cast<const BJob*>(dres + br), 1,
            reinterpret_cast<double*>(dres));
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h + s->res_off, dres, br, cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return st_of(e);
  }
  if (!items.empty()) {
    e = cudaMemcpyAsync(h + s->err_off, static_cast<int*>(s->ctl.ptr) + 32, sizeof(int), cudaMemcpyDeviceToHost,
                        s->stream);
    if (e != cudaSuccess) return st_of(e);
  }
  cudaEventRecord(s->ev1, s->stream);
  s->pending = true;
  s->pend_done.swap(done_ids);
  s->pend_items = !items.empty();
  ++s->ticks;
  if (n_live) *n_live = (int)(s->live.size() - s->pend_done.size());
  if (n_queued) *n_queued = (int)s->queue.size();
  (void)admitted;
  return TQ_OK;
}

}  // namespace

extern "C" {

tq_status tq_server_step(tq_server* s, int* n_live, int* n_queued, int* n_finished) {
  if (!s) return TQ_ERR_ARG;
  if (n_finished) *n_finished = 0;
  tq_status st = collect_tick(s, nullptr);  // a tick launched by tq_server_step_async
  if (st != TQ_OK) return st;
  if ((st = launch_tick(s, n_live, n_queued)) != TQ_OK) return st;
  return collect_tick(s, n_finished);
}

tq_status tq_server_step_async(tq_server* s, int* n_live, int* n_queued, int* n_finished) {
  if (!s) return TQ_ERR_ARG;
  tq_status st = collect_tick(s, n_finished);
  if (st != TQ_OK) return st;
  return launch_tick(s, n_live, n_queued);
}

tq_status tq_server_set_fp64_engine(tq_server* s, int engine) {
  if (!s || engine < TQ_ENGINE_AUTO || engine > TQ_ENGINE_TENSOR) return TQ_ERR_ARG;
  s->fp64_engine = engine;
  return TQ_OK;
}

tq_status tq_server_gpu_ms(const tq_server* s, double* ms) {
  if (!s || !ms) return TQ_ERR_ARG;
  *ms = s->gpu_ms;
  return TQ_OK;
}

tq_status tq_server_poll(tq_server* s, int request_id, int* state, double* out) {
  if (!s || !state) return TQ_ERR_ARG;
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return TQ_ERR_ARG;
  *state = it->second.state;
  if (it->second.state == 2 && out)
    std::memcpy(out, it->second.result, (2 + it->second.masks.size()) * sizeof(double));
  return TQ_OK;
}

tq_status tq_server_info(const tq_server* s, size_t* rho_live_bytes, unsigned long long* ticks,
                         unsigned long long* blocks_applied) {
  if (!s) return TQ_ERR_ARG;
  if (rho_live_bytes) *rho_live_bytes = s->rho_live_bytes;
  if (ticks) *ticks = s->ticks;
  if (blocks_applied) *blocks_applied = s->blocks_applied;
  return TQ_OK;
}

void tq_server_free(tq_server* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  for (DevBuf* d : {&s->rho_mem, &s->tab_mem, &s->djobs, &s->dblks, &s->ditems, &s->counters, &s->ctl, &s->results})
    if (d->ptr) cudaFree(d->ptr);
  for (PinBuf* b : {&s->pin, &s->pin_tick, &s->pin_res})
    if (b->ptr) cudaFreeHost(b->ptr);
  for (cudaEvent_t ev : {s->ev0, s->ev1})
    if (ev) cudaEventDestroy(ev);
  delete s;
}

}  // extern "C"
