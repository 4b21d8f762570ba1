// Batched execution of many independent noisy circuits in one persistent
// kernel launch, captured in a CUDA graph (the single-kernel execution idea
// of TANQ-Sim Sec. 3.4 / Listing 2, applied across jobs instead of across
// GPUs).
//
// The persistent kernel and its work-item scheme are in tq_batch_kernels.cuh.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "tq_batch_kernels.cuh"
#include "tq_batched.cuh"

using namespace tq;
using namespace tq::batch;

struct BatchJob {
  int n = 0;
  std::vector<unsigned long long> masks;
  tq_program prog;
  HostTables t;
};

struct tq_batch {
  int prec = 0;
  cudaStream_t stream = nullptr;   // where the graph is launched (the caller's)
  cudaStream_t capture = nullptr;  // private stream the graph is captured on
  cudaStream_t capture2 = nullptr;  // second branch of the graph: the tensor-core rounds
  cudaEvent_t fork = nullptr, join = nullptr;
  int num_sms = 152;
  int per_sm = 1;
  std::vector<BatchJob> jobs;
  int tile_log2_for_n[kMaxQubits + 1] = {};
  long long max_spin = 20000000;  // ~ seconds with 128 ns sleeps
  int never_ready_job = -1;       // test hook
  // device
  DevBuf arena, blob, sops, sb64, sb32, djobs, dblks, ditems, counters, ctl, results;
  DevBuf pauli, pwork;  // Pauli-basis records of width-2 tile-job blocks and their sb64 offsets
  int n_pauli = 0;
  // tile jobs on the batched tensor-core pass of their precision: one
  // launch per fusion round over every such job's block of that round
  int fp64_engine = TQ_ENGINE_AUTO;
  struct PassRound {
    size_t off;
    int count;
    unsigned long long units;
  };
  DevBuf pass_jobs;
  std::vector<PassRound> rounds;
  size_t n_tensor_jobs = 0;
  PinBuf host_out;  // results + error flag
  size_t n_items = 0;
  size_t arena_bytes = 0;
  bool ready = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<unsigned long long> rho_off;
};

namespace tq {

// Whether a batch's tile jobs take the batched tensor-core pass. FP64: with
// the tensor-core engine (the default; 3,536 against 1,781 circuits/s on the
// 1024-circuit sweep). Split: only when TQ_ENGINE_TENSOR is asked for; the
// default keeps the persistent kernel, measured faster on the same sweep
// (11,381 against 10,900 circuits/s; its rounds cannot share SMs with the
// persistent kernel, and small registers have few units per round).
bool batch_tensor_engine(int precision, int engine) {
  return precision == TQ_FP64 ? fp64_engine_is_tensor(engine) : engine == TQ_ENGINE_TENSOR;
}

}  // namespace tq

namespace {

tq_status to_status(cudaError_t e) {
  if (e == cudaSuccess) return TQ_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return TQ_ERR_OOM;
  }
  return TQ_ERR_CUDA;
}

cudaError_t alloc(DevBuf& b, size_t bytes) {
  if (b.cap >= bytes && b.ptr) return cudaSuccess;
  if (b.ptr) cudaFree(b.ptr);
  b.ptr = nullptr;
  b.cap = 0;
  const size_t want = align_up(std::max<size_t>(bytes, 256), 256);
  cudaError_t e = cudaMalloc(&b.ptr, want);
  if (e == cudaSuccess) b.cap = want;
  return e;
}

int default_tile_log2(int n, int prec) {
  (void)prec;
  return std::min(2 * n, 16);
}


// Algorithmic flops and HBM bytes of one run (see tq_batch_work): one CTA
// per job, threads over its blocks; FP64 counts the nonzeros of S by their
// bit patterns, as the row-list staging does; width-2 blocks of tile jobs
// whose Pauli-basis record is taken count the Pauli-basis product.
__global__ void k_batch_work(const BJob* __restrict__ jobs, const BBlk* __restrict__ blks, int prec,
                             unsigned long long* __restrict__ out) {
  const BJob& jb = jobs[blockIdx.x];
  const unsigned long long esz = prec == 0 ? 16 : 8;
  const unsigned long long N = 1ull << (2 * jb.n), R = 1ull << jb.n;
  unsigned long long fl = 0, by = 0;
  for (int b = threadIdx.x; b < jb.n_blocks; b += blockDim.x) {
    const BBlk& bk = blks[jb.block0 + b];
    const int D = 1 << (2 * bk.p.width);
    unsigned long long nnz = (unsigned long long)D * D;
    if (prec == 0) {
      const unsigned long long* bits = static_cast<const unsigned long long*>(bk.S);
      nnz = 0;
      for (int e = 0; e < D * D; ++e) nnz += ((bits[2 * e] | bits[2 * e + 1]) << 1) != 0ull;
    }
    // flops per group: 8 per complex multiply-add of S (its nonzeros, or all
    // of them), or in the Pauli basis 4 per real-times-complex multiply-add
    // (FP64: the nonzeros of R'; split: all 256) plus the 128 adds of the two
    // basis changes
    unsigned long long per = 8ull * nnz;
    if (bk.pauli && bk.pauli->on) per = 4ull * (prec == 0 ? (unsigned long long)bk.pauli->nnz : 256ull) + 128;
    if (jb.tensor) per = 8ull * D * D;  // the tensor-core pass: the dense product's algorithmic count
    const unsigned long long groups = jb.herm ? bk.p.n_canon : bk.p.n_groups;
    fl += per * groups;
    if (!jb.resident) by += (jb.herm ? N + R : 2 * N) * esz;
  }
  if (jb.resident && threadIdx.x == 0 && jb.n_blocks > 0) by += 2 * N * esz;
  atomicAdd(&out[0], fl);
  atomicAdd(&out[1], by);
}

void drop_graph(tq_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// Concatenate every job's tables, allocate device memory, upload, build the
// work-item order and capture the run into a CUDA graph.
tq_status finalize(tq_batch* b) {
  drop_graph(b);
  HostTables all;
  std::vector<BJob> hjobs(b->jobs.size());
  std::vector<BBlk> hblks;
  std::vector<long long> blk_rec;          // per block: its Pauli record, or -1
  std::vector<unsigned long long> rec_sb;  // per record: its block's sb64 offset
  size_t arena = 0;
  b->rho_off.assign(b->jobs.size(), 0);
  int max_dim2 = 1;
  for (size_t j = 0; j < b->jobs.size(); ++j) {
    BatchJob& J = b->jobs[j];
    const long long kbase = (long long)all.kraus.size(), sbase = all.sop_entries, bbase = (long long)all.blocks.size();
    const long long mbase = (long long)all.members.size(), obase = (long long)all.ops.size(), sbb = all.sb_entries;
    all.kraus.insert(all.kraus.end(), J.t.kraus.begin(), J.t.kraus.end());
    for (OpDesc od : J.t.ops) {
      od.kraus_off += kbase;
      od.sop_off += sbase;
      all.ops.push_back(od);
    }
    for (BlockDesc bd : J.t.blocks) {
      bd.member_off += (int)mbase;
      bd.sb_off += sbb;
      all.blocks.push_back(bd);
    }
    for (MemberDesc md : J.t.members) {
      md.op += (int)obase;
      all.members.push_back(md);
    }
    for (FuseWork w : J.t.work) {
      w.block += (int)bbase;
      all.work.push_back(w);
    }
    all.sop_entries += J.t.sop_entries;
    all.sb_entries += J.t.sb_entries;
    max_dim2 = std::max(max_dim2, J.prog.max_dim2);
    BJob& hj = hjobs[j];
    std::memset(&hj, 0, sizeof(hj));
    hj.rho_off = arena;
    b->rho_off[j] = arena;
    hj.n = J.n;
    hj.n_blocks = (int)J.prog.params.size();
    hj.block0 = (int)hblks.size();
    hj.resident = is_resident(J.n, b->prec) ? 1 : 0;
    const int tl = b->tile_log2_for_n[J.n] ? b->tile_log2_for_n[J.n] : default_tile_log2(J.n, b->prec);
    // at least 16 groups' worth of entries per tile, at most 2^16 tiles per block
    hj.tile_log2 = std::min(std::max({tl, 4, 2 * J.n - 16}), 2 * J.n);
    hj.herm = batch_herm(J.n, b->prec) ? 1 : 0;
    // tile jobs whose blocks are all eligible run on the batched tensor-core
    // pass of their precision when batch_tensor_engine says so (a job under
    // the never-ready test hook stays on the batch kernel, whose waits it
    // tests)
    hj.tensor = 0;
    if (batch_tensor_engine(b->prec, b->fp64_engine) && !hj.resident && (int)j != b->never_ready_job) {
      bool all = !J.prog.params.empty();
      for (const ApplyParams& pp : J.prog.params) all = all && oz_eligible(pp.n, pp.width);
      hj.tensor = all ? 1 : 0;
    }
    hj.n_masks = (int)J.masks.size();
    hj.never_ready = (int)j == b->never_ready_job ? 1 : 0;
    for (size_t m = 0; m < J.masks.size(); ++m) hj.masks[m] = J.masks[m];
    for (size_t k = 0; k < J.prog.params.size(); ++k) {
      BBlk bb;
      std::memset(&bb, 0, sizeof(bb));
      bb.p = J.prog.params[k];
      bb.S = reinterpret_cast<const void*>(J.prog.sb_off[k] + sbb);  // offset; made absolute below
      if (!hj.resident && !hj.tensor && bb.p.width == 2) {
        blk_rec.push_back((long long)rec_sb.size());
        rec_sb.push_back((unsigned long long)(J.prog.sb_off[k] + sbb));
      } else {
        blk_rec.push_back(-1);
      }
      hblks.push_back(bb);
    }
    if (set_tiles(hblks.data() + hj.block0, hj.n_blocks, hj.tile_log2, hj.herm != 0, tiled16_job(J.n, b->prec)) >= (1ll << 31))
      return TQ_ERR_UNSUPPORTED;
    arena = align_up(arena + ((size_t)(b->prec == TQ_FP64 ? 16 : 8) << (2 * J.n)), 256);
  }
  b->arena_bytes = arena;
  // work items: resident jobs first (independent), then tile items round-robin by block
  std::vector<BItem> items;
  int max_blocks = 0;
  for (size_t j = 0; j < hjobs.size(); ++j) {
    if (hjobs[j].resident) {
      if (hjobs[j].n_blocks > 0) items.push_back(BItem{(int)j, -1, 0, hjobs[j].n_blocks});
    } else {
      max_blocks = std::max(max_blocks, hjobs[j].n_blocks);
    }
  }
  for (int r = 0; r < max_blocks; ++r)
    for (size_t j = 0; j < hjobs.size(); ++j) {
      const BJob& hj = hjobs[j];
      if (hj.resident || hj.tensor || r >= hj.n_blocks) continue;
      const int tiles = hblks[hj.block0 + r].tiles;
      for (int t = 0; t < tiles; ++t) items.push_back(BItem{(int)j, r, t, 1});
    }
  b->n_items = items.size();

  tq_program P;  // layout of the concatenated upload
  P.n_ops = all.ops.size();
  P.n_uops = all.ops.size();
  size_t off = 0;
  P.o_kraus = off; off = align_up(off + all.kraus.size() * sizeof(double2), 256);
  P.o_ops = off;   off = align_up(off + all.ops.size() * sizeof(OpDesc), 256);
  P.o_blk = off;   off = align_up(off + all.blocks.size() * sizeof(BlockDesc), 256);
  P.o_mem = off;   off = align_up(off + all.members.size() * sizeof(MemberDesc), 256);
  P.o_work = off;  off = align_up(off + all.work.size() * sizeof(FuseWork), 256);
  P.blob_bytes = std::max<size_t>(off, 256);
  std::vector<char> h(P.blob_bytes);
  pack_blob(P, all, h.data());

  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess) e = alloc(b->arena, arena);
  if (e == cudaSuccess) e = alloc(b->blob, P.blob_bytes);
  if (e == cudaSuccess) e = alloc(b->sops, all.sop_entries * sizeof(double2) + 16);
  if (e == cudaSuccess) e = alloc(b->sb64, all.sb_entries * sizeof(double2) + 16);
  if (e == cudaSuccess && b->prec == TQ_SPLIT) e = alloc(b->sb32, all.sb_entries * sizeof(float2) + 16);
  if (e == cudaSuccess) e = alloc(b->djobs, hjobs.size() * sizeof(BJob));
  if (e == cudaSuccess) e = alloc(b->dblks, std::max<size_t>(1, hblks.size()) * sizeof(BBlk));
  if (e == cudaSuccess) e = alloc(b->ditems, std::max<size_t>(1, items.size()) * sizeof(BItem));
  if (e == cudaSuccess) e = alloc(b->counters, hjobs.size() * sizeof(int));
  if (e == cudaSuccess) e = alloc(b->ctl, 256);
  if (e == cudaSuccess) e = alloc(b->results, hjobs.size() * kResults * sizeof(double));
  b->n_pauli = (int)rec_sb.size();
  if (e == cudaSuccess) e = alloc(b->pauli, std::max<size_t>(1, rec_sb.size()) * sizeof(PauliRec));
  if (e == cudaSuccess) e = alloc(b->pwork, std::max<size_t>(1, rec_sb.size()) * sizeof(unsigned long long));
  if (e != cudaSuccess) return to_status(e);
  if (b->host_out.cap < hjobs.size() * kResults * sizeof(double) + 64) {
    if (b->host_out.ptr) cudaFreeHost(b->host_out.ptr);
    b->host_out.cap = 0;
    e = cudaHostAlloc(&b->host_out.ptr, hjobs.size() * kResults * sizeof(double) + 64, cudaHostAllocDefault);
    if (e != cudaSuccess) return to_status(e);
    b->host_out.cap = hjobs.size() * kResults * sizeof(double) + 64;
  }
  {
    const size_t esz = b->prec == TQ_FP64 ? sizeof(double2) : sizeof(float2);
    char* sbase = static_cast<char*>(b->prec == TQ_FP64 ? b->sb64.ptr : b->sb32.ptr);
    for (size_t k = 0; k < hblks.size(); ++k) {
      BBlk& bb = hblks[k];
      bb.S = sbase + reinterpret_cast<size_t>(bb.S) * esz;
      bb.pauli = blk_rec[k] < 0 ? nullptr : static_cast<const PauliRec*>(b->pauli.ptr) + blk_rec[k];
    }
  }
  e = cudaMemcpy(b->blob.ptr, h.data(), P.blob_bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->djobs.ptr, hjobs.data(), hjobs.size() * sizeof(BJob), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !hblks.empty())
    e = cudaMemcpy(b->dblks.ptr, hblks.data(), hblks.size() * sizeof(BBlk), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpy(b->ditems.ptr, items.data(), items.size() * sizeof(BItem), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !rec_sb.empty())
    e = cudaMemcpy(b->pwork.ptr, rec_sb.data(), rec_sb.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice);
  // the tensor-core rounds: round r holds block r of every tensor job that has one
  b->rounds.clear();
  b->n_tensor_jobs = 0;
  {
    std::vector<OzJob> oz;
    std::vector<TcJob> tc;
    int rounds = 0;
    for (const BJob& hj : hjobs)
      if (hj.tensor) {
        ++b->n_tensor_jobs;
        rounds = std::max(rounds, hj.n_blocks);
      }
    for (int r = 0; r < rounds; ++r) {
      tq_batch::PassRound rd{b->prec == TQ_FP64 ? oz.size() : tc.size(), 0, 0};
      for (size_t j = 0; j < hjobs.size(); ++j) {
        const BJob& hj = hjobs[j];
        if (!hj.tensor || r >= hj.n_blocks) continue;
        const BBlk& bb = hblks[hj.block0 + r];
        char* rho = static_cast<char*>(b->arena.ptr) + hj.rho_off;
        if (b->prec == TQ_FP64) {
          OzJob oj{};
          oz_job(reinterpret_cast<double2*>(rho), static_cast<const double2*>(bb.S), bb.p, &oj);
          oj.unit0 = rd.units;
          oz.push_back(oj);
        } else {
          TcJob tj{};
          tc_job(reinterpret_cast<float2*>(rho), static_cast<const float2*>(bb.S), bb.p, &tj);
          tj.unit0 = rd.units;
          tc.push_back(tj);
        }
        rd.units += oz_units(hj.n);
        ++rd.count;
      }
      b->rounds.push_back(rd);
    }
    const size_t bytes = b->prec == TQ_FP64 ? oz.size() * sizeof(OzJob) : tc.size() * sizeof(TcJob);
    if (e == cudaSuccess) e = alloc(b->pass_jobs, std::max<size_t>(16, bytes));
    if (e == cudaSuccess && bytes)
      e = cudaMemcpy(b->pass_jobs.ptr, b->prec == TQ_FP64 ? (const void*)oz.data() : (const void*)tc.data(), bytes,
                     cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return to_status(e);

  const size_t smem = b->prec == TQ_FP64 ? apply_smem<double2>() : apply_smem<float2>();
  if (b->prec == TQ_FP64) {
    e = cudaFuncSetAttribute(k_batch_apply<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->per_sm, k_batch_apply<double2>, kThreads, smem);
  } else {
    e = cudaFuncSetAttribute(k_batch_apply<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->per_sm, k_batch_apply<float2>, kThreads, smem);
  }
  if (e != cudaSuccess) return to_status(e);
  b->per_sm = std::max(1, b->per_sm);

  // capture: reset every rho, build + fuse every job's superoperators, run
  // all items, reduce per job, copy results and the error flag to the host
  char* d = static_cast<char*>(b->blob.ptr);
  const int n_jobs = (int)hjobs.size();
  int* counters = static_cast<int*>(b->counters.ptr);
  int* ticket = static_cast<int*>(b->ctl.ptr);
  int* err = ticket + 32;
  cudaStream_t st = b->capture;
  e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return to_status(e);
  cudaMemsetAsync(b->arena.ptr, 0, arena, st);
  k_batch_set_one<<<(n_jobs + 255) / 256, 256, 0, st>>>(static_cast<char*>(b->arena.ptr),
                                                        static_cast<const BJob*>(b->djobs.ptr), n_jobs, b->prec);
  if (P.n_uops > 0) {
    launch_build_superops(reinterpret_cast<const double2*>(d + P.o_kraus), reinterpret_cast<const OpDesc*>(d + P.o_ops),
                          (int)P.n_uops, max_dim2, static_cast<double2*>(b->sops.ptr), st);
    launch_fuse(static_cast<const double2*>(b->sops.ptr), reinterpret_cast<const OpDesc*>(d + P.o_ops),
                reinterpret_cast<const BlockDesc*>(d + P.o_blk), reinterpret_cast<const MemberDesc*>(d + P.o_mem),
                reinterpret_cast<const FuseWork*>(d + P.o_work), (int)all.work.size(),
                static_cast<double2*>(b->sb64.ptr),
                b->prec == TQ_SPLIT ? static_cast<float2*>(b->sb32.ptr) : nullptr, st);
    launch_pauli_lists(static_cast<const double2*>(b->sb64.ptr), static_cast<const unsigned long long*>(b->pwork.ptr),
                       b->n_pauli, b->prec == TQ_FP64 ? 0 : 1, static_cast<PauliRec*>(b->pauli.ptr), st);
  }
  cudaMemsetAsync(b->counters.ptr, 0, n_jobs * sizeof(int), st);
  cudaMemsetAsync(b->ctl.ptr, 0, 256, st);
  // the tensor-core rounds are a second branch of the graph, beside the
  // persistent kernel (they hold other jobs): CTAs of the rounds take the SMs
  // that the persistent kernel's CTAs leave when its items run out
  const bool branch = !b->rounds.empty();
  if (branch) {
    cudaEventRecord(b->fork, st);
    cudaStreamWaitEvent(b->capture2, b->fork, 0);
  }
  const int grid = (int)std::max<size_t>(1, std::min<size_t>(b->n_items, (size_t)b->num_sms * b->per_sm));
  if (b->n_items > 0) {
    if (b->prec == TQ_FP64)
      k_batch_apply<double2><<<grid, kThreads, smem, st>>>(
          static_cast<char*>(b->arena.ptr), static_cast<const BJob*>(b->djobs.ptr),
          static_cast<const BBlk*>(b->dblks.ptr), static_cast<const BItem*>(b->ditems.ptr), (int)b->n_items,
          counters, ticket, err, b->max_spin);
    else
      k_batch_apply<float2><<<grid, kThreads, smem, st>>>(
          static_cast<char*>(b->arena.ptr), static_cast<const BJob*>(b->djobs.ptr),
          static_cast<const BBlk*>(b->dblks.ptr), static_cast<const BItem*>(b->ditems.ptr), (int)b->n_items,
          counters, ticket, err, b->max_spin);
  }
  for (const tq_batch::PassRound& rd : b->rounds) {
    if (b->prec == TQ_FP64)
      launch_batch_oz(static_cast<const OzJob*>(b->pass_jobs.ptr) + rd.off, rd.count, rd.units, b->num_sms, b->capture2);
    else
      launch_batch_tc(static_cast<const TcJob*>(b->pass_jobs.ptr) + rd.off, rd.count, rd.units, b->num_sms, b->capture2);
  }
  if (branch) {
    cudaEventRecord(b->join, b->capture2);
    cudaStreamWaitEvent(st, b->join, 0);
  }
  if (b->prec == TQ_FP64)
    k_batch_reduce<double2><<<n_jobs, kThreads, 0, st>>>(static_cast<const char*>(b->arena.ptr),
                                                         static_cast<const BJob*>(b->djobs.ptr), 0,
                                                         static_cast<double*>(b->results.ptr));
  else
    k_batch_reduce<float2><<<n_jobs, kThreads, 0, st>>>(static_cast<const char*>(b->arena.ptr),
                                                        static_cast<const BJob*>(b->djobs.ptr), 1,
                                                        static_cast<double*>(b->results.ptr));
  cudaMemcpyAsync(b->host_out.ptr, b->results.ptr, n_jobs * kResults * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(static_cast<char*>(b->host_out.ptr) + n_jobs * kResults * sizeof(double), err, sizeof(int),
                  cudaMemcpyDeviceToHost, st);
  e = cudaStreamEndCapture(st, &b->graph);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) {
    drop_graph(b);
    return to_status(e);
  }
  b->ready = true;
  return TQ_OK;
}

}  // namespace

extern "C" {

tq_status tq_batch_create(int precision, void* cuda_stream, tq_batch** out) {
  if (!out || (precision != TQ_FP64 && precision != TQ_SPLIT)) return TQ_ERR_ARG;
  *out = nullptr;
  tq_batch* b = new (std::nothrow) tq_batch();
  if (!b) return TQ_ERR_OOM;
  b->prec = precision;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->capture2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) != cudaSuccess) {
    if (b->capture) cudaStreamDestroy(b->capture);
    if (b->capture2) cudaStreamDestroy(b->capture2);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    delete b;
    return TQ_ERR_CUDA;
  }
  *out = b;
  return TQ_OK;
}

tq_status tq_batch_add(tq_batch* b, int n_qubits, const tq_op* ops, size_t n_ops, int max_fuse_width,
                       const uint64_t* masks, int n_masks, int* job_out) {
  if (!b || (!ops && n_ops) || n_masks < 0 || n_masks > kMaxMasks || (n_masks && !masks)) return TQ_ERR_ARG;
  if (n_qubits < 1 || n_qubits > kMaxQubits) return TQ_ERR_ARG;
  if (max_fuse_width > 2) return TQ_ERR_UNSUPPORTED;  // the batch kernel applies blocks of <= 2 qubits
  BatchJob J;
  J.n = n_qubits;
  tq_status st = plan_program(n_qubits, b->prec, ops, n_ops, max_fuse_width == -1 ? -1 : max_fuse_width, &J.prog, &J.t);
  if (st != TQ_OK) return st;
  if (J.prog.max_width > 2) {
    // automatic planning may pick wider blocks; cap at 2 for the batch kernel
    J = BatchJob();
    J.n = n_qubits;
    st = plan_program(n_qubits, b->prec, ops, n_ops, 2, &J.prog, &J.t);
    if (st != TQ_OK) return st;
    if (J.prog.max_width > 2) return TQ_ERR_UNSUPPORTED;  // an op on more than 2 qubits
  }
  for (int m = 0; m < n_masks; ++m) J.masks.push_back(masks[m]);
  b->jobs.push_back(std::move(J));
  b->ready = false;
  if (job_out) *job_out = (int)b->jobs.size() - 1;
  return TQ_OK;
}

tq_status tq_batch_set_tile(tq_batch* b, int n_qubits, int tile_log2) {
  if (!b || n_qubits < 1 || n_qubits > kMaxQubits || tile_log2 < 4 || tile_log2 > 2 * kMaxQubits) return TQ_ERR_ARG;
  b->tile_log2_for_n[n_qubits] = tile_log2;
  b->ready = false;
  return TQ_OK;
}

tq_status tq_batch_set_fp64_engine(tq_batch* b, int engine) {
  if (!b || engine < TQ_ENGINE_AUTO || engine > TQ_ENGINE_TENSOR) return TQ_ERR_ARG;
  b->fp64_engine = engine;
  b->ready = false;
  return TQ_OK;
}

tq_status tq_batch_tensor_jobs(const tq_batch* b, size_t* n_jobs) {
  if (!b || !n_jobs) return TQ_ERR_ARG;
  *n_jobs = b->ready ? b->n_tensor_jobs : 0;
  return TQ_OK;
}

tq_status tq_batch_test_wait_limit(tq_batch* b, long long max_spin, int never_ready_job) {
  if (!b || max_spin < 1 || never_ready_job < -1 || never_ready_job >= (int)b->jobs.size()) return TQ_ERR_ARG;
  b->max_spin = max_spin;
  b->never_ready_job = never_ready_job;
  b->ready = false;
  return TQ_OK;
}

tq_status tq_batch_run(tq_batch* b) {
  if (!b) return TQ_ERR_ARG;
  if (b->jobs.empty()) return TQ_OK;
  if (!b->ready) {
    tq_status st = finalize(b);
    if (st != TQ_OK) return st;
  }
  return to_status(cudaGraphLaunch(b->exec, b->stream));
}

tq_status tq_batch_wait(tq_batch* b) {
  if (!b) return TQ_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return TQ_ERR_CUDA;
  if (!b->ready) return TQ_OK;
  const int err = *reinterpret_cast<const int*>(static_cast<const char*>(b->host_out.ptr) +
                                                b->jobs.size() * kResults * sizeof(double));
  unsigned int tc_timeouts = 0;
  if (b->n_tensor_jobs && (b->prec == TQ_FP64 ? oz_take_timeouts(&tc_timeouts, b->stream)
                                              : tc_take_timeouts(&tc_timeouts, b->stream)) != cudaSuccess)
    return TQ_ERR_CUDA;
  return err || tc_timeouts ? TQ_ERR_TIMEOUT : TQ_OK;
}

tq_status tq_batch_result(tq_batch* b, int job, double* out) {
  if (!b || !out || job < 0 || job >= (int)b->jobs.size() || !b->ready) return TQ_ERR_ARG;
  tq_status st = tq_batch_wait(b);
  if (st != TQ_OK) return st;
  const double* r = static_cast<const double*>(b->host_out.ptr) + (size_t)job * kResults;
  std::memcpy(out, r, (2 + b->jobs[job].masks.size()) * sizeof(double));
  return TQ_OK;
}

tq_status tq_batch_get_rho(tq_batch* b, int job, double* out) {
  if (!b || !out || job < 0 || job >= (int)b->jobs.size() || !b->ready) return TQ_ERR_ARG;
  tq_status st = tq_batch_wait(b);
  if (st != TQ_OK) return st;
  const int n = b->jobs[job].n;
  const size_t entries = 1ull << (2 * n);
  char* src = static_cast<char*>(b->arena.ptr) + b->rho_off[job];
  if (batch_herm(n, b->prec)) {  // Hermitian mode kept rows <= columns only: fill the rest
    cudaError_t em = launch_mirror_lower(src, n, b->prec, b->stream);
    if (em == cudaSuccess) em = cudaStreamSynchronize(b->stream);
    if (em != cudaSuccess) return to_status(em);
  }
  if (b->prec == TQ_FP64) return to_status(cudaMemcpy(out, src, entries * 16, cudaMemcpyDeviceToHost));
  std::vector<float> tmp(2 * entries);
  cudaError_t e = cudaMemcpy(tmp.data(), src, entries * 8, cudaMemcpyDeviceToHost);
  for (size_t i = 0; i < 2 * entries; ++i) out[i] = tmp[i];  // widen complex64 to the complex128 layout
  return to_status(e);
}

tq_status tq_batch_info(const tq_batch* b, size_t* n_jobs, size_t* n_items, size_t* rho_bytes) {
  if (!b) return TQ_ERR_ARG;
  if (n_jobs) *n_jobs = b->jobs.size();
  if (n_items) *n_items = b->n_items;
  if (rho_bytes) *rho_bytes = b->arena_bytes;
  return TQ_OK;
}

tq_status tq_batch_work(tq_batch* b, double* flops, double* bytes) {
  if (!b) return TQ_ERR_ARG;
  if (!b->ready) return TQ_ERR_STATE;
  tq_status st = tq_batch_wait(b);
  if (st != TQ_OK) return st;
  unsigned long long h[2] = {0, 0};
  DevBuf tmp;
  cudaError_t e = alloc(tmp, sizeof(h));
  if (e == cudaSuccess) e = cudaMemsetAsync(tmp.ptr, 0, sizeof(h), b->stream);
  if (e == cudaSuccess) {
    k_batch_work<<<(unsigned)b->jobs.size(), 256, 0, b->stream>>>(static_cast<const BJob*>(b->djobs.ptr),
                                                                  static_cast<const BBlk*>(b->dblks.ptr), b->prec,
                                                                  static_cast<unsigned long long*>(tmp.ptr));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, tmp.ptr, sizeof(h), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (tmp.ptr) cudaFree(tmp.ptr);
  if (e != cudaSuccess) return to_status(e);
  if (flops) *flops = (double)h[0];
  if (bytes) *bytes = (double)h[1];
  return TQ_OK;
}

void tq_batch_free(tq_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  for (DevBuf* d : {&b->arena, &b->blob, &b->sops, &b->sb64, &b->sb32, &b->djobs, &b->dblks, &b->ditems, &b->pauli, &b->pwork, &b->pass_jobs,
                    &b->counters, &b->ctl, &b->results})
    if (d->ptr) cudaFree(d->ptr);
  if (b->host_out.ptr) cudaFreeHost(b->host_out.ptr);
  if (b->capture) cudaStreamDestroy(b->capture);
  if (b->capture2) cudaStreamDestroy(b->capture2);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  delete b;
}

}  // extern "C"
