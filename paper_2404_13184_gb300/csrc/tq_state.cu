// States, circuit runs and readouts: the C-ABI entry points that do GPU
// work. Host code here validates, plans fusion, packs tables and enqueues
// kernels; every arithmetic step of the simulation runs on the device.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "tq_device.cuh"
#include "tq_internal.h"

using namespace tq;

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct DevBuf {
  void* ptr = nullptr;
  size_t cap = 0;
};

struct PinBuf {
  void* ptr = nullptr;
  size_t cap = 0;
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
  DevBuf upload, sops, sb64, sb32, red, probs, staging;
  PinBuf pin, pin_small;
  cudaEvent_t pin_free = nullptr;  // recorded after the last upload from `pin`
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

// Grow a device buffer; the old contents are not kept. Waits for the stream
// first because queued kernels may still read the old buffer.
tq_status ensure(tq_state* s, DevBuf& b, size_t bytes) {
  if (b.cap >= bytes) return TQ_OK;
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e);
  if (b.ptr) cudaFree(b.ptr);
  b.ptr = nullptr;
  b.cap = 0;
  const size_t want = align_up(std::max<size_t>(bytes, 4096), 4096);
  e = cudaMalloc(&b.ptr, want);
  if (e != cudaSuccess) {
    b.ptr = nullptr;
    return cuda_fail(s, e);
  }
  b.cap = want;
  return TQ_OK;
}

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

size_t entry_bytes(int prec) { return prec == TQ_FP64 ? 16 : 8; }

tq_status check_state(tq_state* s) {
  if (!s) return TQ_ERR_ARG;
  if (s->poisoned) return TQ_ERR_STATE;
  return TQ_OK;
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
  if (e != cudaSuccess) {
    tq_free(s);
    return TQ_ERR_CUDA;
  }
  *out = s;
  return TQ_OK;
}

// Host tables of one circuit run, packed into a single upload.
struct RunPlan {
  std::vector<double2> kraus;
  std::vector<OpDesc> ops;
  std::vector<BlockDesc> blocks;
  std::vector<MemberDesc> members;
  std::vector<FuseWork> work;
  std::vector<Block> plan;
  long long sop_entries = 0;
  long long sb_entries = 0;
  int max_dim2 = 0;
};

tq_status build_plan(int n, int prec, const tq_op* ops, size_t n_ops, int width, RunPlan* rp) {
  std::vector<std::vector<int>> qs(n_ops);
  rp->ops.resize(n_ops);
  for (size_t i = 0; i < n_ops; ++i) {
    tq_status st = validate_op(n, ops[i]);
    if (st != TQ_OK) return st;
    ResolvedOp r;
    st = resolve_op(ops[i], &r);
    if (st != TQ_OK) return st;
    qs[i].assign(ops[i].qubits, ops[i].qubits + ops[i].k);
    OpDesc& od = rp->ops[i];
    od.k = r.k;
    od.m = r.m;
    od.kraus_off = (long long)rp->kraus.size();
    od.sop_off = rp->sop_entries;
    for (const cplx& v : r.kraus) rp->kraus.push_back(make_double2(v.real(), v.imag()));
    const long long d2 = 1ll << (2 * r.k);
    rp->sop_entries += d2 * d2;
    rp->max_dim2 = std::max<int>(rp->max_dim2, (int)(d2 * d2));
  }
  tq_status st = plan_fusion(n, qs, width, prec, &rp->plan);
  if (st != TQ_OK) return st;
  for (size_t b = 0; b < rp->plan.size(); ++b) {
    const Block& B = rp->plan[b];
    BlockDesc bd{};
    bd.width = B.width;
    bd.n_members = (int)B.ops.size();
    bd.member_off = (int)rp->members.size();
    bd.sb_off = rp->sb_entries;
    const int D = 1 << (2 * B.width);
    rp->sb_entries += (long long)D * D;
    for (int oi : B.ops) {
      MemberDesc md{};
      md.op = oi;
      md.k = ops[oi].k;
      for (int j = 0; j < md.k; ++j)
        md.pos[j] = (int)(std::find(B.qubits, B.qubits + B.width, ops[oi].qubits[j]) - B.qubits);
      rp->members.push_back(md);
    }
    rp->blocks.push_back(bd);
    const int C = std::min(D, 1024 / D);
    for (int c0 = 0; c0 < D; c0 += C) rp->work.push_back(FuseWork{(int)b, c0});
  }
  return TQ_OK;
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

template <typename T>
T* section(char* base, size_t& off, size_t count) {
  T* p = reinterpret_cast<T*>(base + off);
  off = align_up(off + count * sizeof(T), 256);
  return p;
}

tq_status run_impl(tq_state* s, const tq_op* ops, size_t n_ops, int width, size_t* n_blocks_out) {
  tq_status st = check_state(s);
  if (st != TQ_OK) return st;
  if (!ops && n_ops) return TQ_ERR_ARG;
  if (width < -1 || width > kMaxWidth) return TQ_ERR_ARG;
  if (n_blocks_out) *n_blocks_out = 0;
  if (n_ops == 0) return TQ_OK;
  RunPlan rp;
  st = build_plan(s->n, s->prec, ops, n_ops, width, &rp);
  if (st != TQ_OK) return st;

  // layout of the upload blob (byte offsets; 256-byte aligned sections)
  size_t off = 0;
  const size_t o_kraus = off; off = align_up(off + rp.kraus.size() * sizeof(double2), 256);
  const size_t o_ops = off;   off = align_up(off + rp.ops.size() * sizeof(OpDesc), 256);
  const size_t o_blk = off;   off = align_up(off + rp.blocks.size() * sizeof(BlockDesc), 256);
  const size_t o_mem = off;   off = align_up(off + rp.members.size() * sizeof(MemberDesc), 256);
  const size_t o_work = off;  off = align_up(off + rp.work.size() * sizeof(FuseWork), 256);
  const size_t blob = off;

  if ((st = ensure(s, s->upload, blob)) != TQ_OK) return st;
  if ((st = ensure(s, s->sops, rp.sop_entries * sizeof(double2))) != TQ_OK) return st;
  if ((st = ensure(s, s->sb64, rp.sb_entries * sizeof(double2))) != TQ_OK) return st;
  if (s->prec == TQ_SPLIT && (st = ensure(s, s->sb32, rp.sb_entries * sizeof(float2))) != TQ_OK) return st;

  // the pinned staging buffer is reused: wait until its last upload finished
  cudaError_t e = cudaEventSynchronize(s->pin_free);
  if (e != cudaSuccess) return cuda_fail(s, e);
  if ((st = ensure_pinned(s, s->pin, blob)) != TQ_OK) return st;
  char* h = static_cast<char*>(s->pin.ptr);
  std::memcpy(h + o_kraus, rp.kraus.data(), rp.kraus.size() * sizeof(double2));
  std::memcpy(h + o_ops, rp.ops.data(), rp.ops.size() * sizeof(OpDesc));
  std::memcpy(h + o_blk, rp.blocks.data(), rp.blocks.size() * sizeof(BlockDesc));
  std::memcpy(h + o_mem, rp.members.data(), rp.members.size() * sizeof(MemberDesc));
  std::memcpy(h + o_work, rp.work.data(), rp.work.size() * sizeof(FuseWork));
  e = cudaMemcpyAsync(s->upload.ptr, h, blob, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaEventRecord(s->pin_free, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e);

  char* d = static_cast<char*>(s->upload.ptr);
  const double2* d_kraus = reinterpret_cast<const double2*>(d + o_kraus);
  const OpDesc* d_ops = reinterpret_cast<const OpDesc*>(d + o_ops);
  const BlockDesc* d_blk = reinterpret_cast<const BlockDesc*>(d + o_blk);
  const MemberDesc* d_mem = reinterpret_cast<const MemberDesc*>(d + o_mem);
  const FuseWork* d_work = reinterpret_cast<const FuseWork*>(d + o_work);
  double2* sops = static_cast<double2*>(s->sops.ptr);
  double2* sb64 = static_cast<double2*>(s->sb64.ptr);
  float2* sb32 = s->prec == TQ_SPLIT ? static_cast<float2*>(s->sb32.ptr) : nullptr;

  e = launch_build_superops(d_kraus, d_ops, (int)rp.ops.size(), rp.max_dim2, sops, s->stream);
  if (e == cudaSuccess)
    e = launch_fuse(sops, d_ops, d_blk, d_mem, d_work, (int)rp.work.size(), sb64, sb32, s->stream);
  for (size_t b = 0; b < rp.plan.size() && e == cudaSuccess; ++b) {
    const ApplyParams p = apply_params(s->n, rp.plan[b]);
    const void* S = s->prec == TQ_FP64 ? (const void*)(sb64 + rp.blocks[b].sb_off)
                                       : (const void*)(sb32 + rp.blocks[b].sb_off);
    e = launch_apply(s->rho, s->prec, S, p, s->num_sms, s->stream);
  }
  if (e != cudaSuccess) return cuda_fail(s, e);
  if (n_blocks_out) *n_blocks_out = rp.plan.size();
  return TQ_OK;
}

// Reduction scratch: [16 masks][18 outputs][grid x 18 partials]
constexpr size_t kRedMasks = 0, kRedOut = 256, kRedPartials = 512;

tq_status reduce_impl(tq_state* s, const unsigned long long* masks, int n_masks, bool normalize, double* host_out) {
  tq_status st = ensure(s, s->red, kRedPartials + 152 * 18 * sizeof(double) + 256);
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
  if (e == cudaSuccess)
    e = launch_diag_reduce(s->rho, s->n, s->prec, reinterpret_cast<unsigned long long*>(d + kRedMasks), n_masks,
                           reinterpret_cast<double*>(d + kRedPartials), reinterpret_cast<double*>(d + kRedOut),
                           normalize, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hout, d + kRedOut, (2 + n_masks) * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e);
  std::memcpy(host_out, hout, (2 + n_masks) * sizeof(double));
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
  for (DevBuf* b : {&s->upload, &s->sops, &s->sb64, &s->sb32, &s->red, &s->probs, &s->staging})
    if (b->ptr) cudaFree(b->ptr);
  for (PinBuf* b : {&s->pin, &s->pin_small})
    if (b->ptr) cudaFreeHost(b->ptr);
  if (s->pin_free) cudaEventDestroy(s->pin_free);
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
  return cuda_fail(s, launch_init_zero_state(s->rho, s->n, s->prec, s->stream));
}

tq_status tq_rho_device_ptr(tq_state* s, void** out) {
  if (!s || !out) return TQ_ERR_ARG;
  *out = s->rho;
  return TQ_OK;
}

tq_status tq_get_rho(tq_state* s, double* out) {
  tq_status st = check_state(s);
  if (st != TQ_OK) return st;
  if (!out) return TQ_ERR_ARG;
  const size_t entries = 1ull << (2 * s->n);
  cudaError_t e;
  if (s->prec == TQ_FP64) {
    e = cudaMemcpyAsync(out, s->rho, entries * 16, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return cuda_fail(s, e);
  }
  const size_t chunk = std::min<size_t>(entries, 1ull << 22);  // complex entries per pass
  if ((st = ensure(s, s->staging, chunk * 16)) != TQ_OK) return st;
  for (size_t c0 = 0; c0 < entries; c0 += chunk) {
    const size_t cnt = std::min(chunk, entries - c0);
    e = launch_convert_f32_to_f64(static_cast<const float*>(s->rho) + 2 * c0, static_cast<double*>(s->staging.ptr),
                                  2 * cnt, s->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out + 2 * c0, s->staging.ptr, cnt * 16, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e);
  }
  return TQ_OK;
}

tq_status tq_set_rho(tq_state* s, const double* in) {
  tq_status st = check_state(s);
  if (st != TQ_OK) return st;
  if (!in) return TQ_ERR_ARG;
  const size_t entries = 1ull << (2 * s->n);
  cudaError_t e;
  if (s->prec == TQ_FP64) {
    e = cudaMemcpyAsync(s->rho, in, entries * 16, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return cuda_fail(s, e);
  }
  const size_t chunk = std::min<size_t>(entries, 1ull << 22);
  if ((st = ensure(s, s->staging, chunk * 16)) != TQ_OK) return st;
  for (size_t c0 = 0; c0 < entries; c0 += chunk) {
    const size_t cnt = std::min(chunk, entries - c0);
    e = cudaMemcpyAsync(s->staging.ptr, in + 2 * c0, cnt * 16, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
      e = launch_convert_f64_to_f32(static_cast<const double*>(s->staging.ptr), static_cast<float*>(s->rho) + 2 * c0,
                                    2 * cnt, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e);
  }
  return TQ_OK;
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

tq_status tq_probs(tq_state* s, double* out) {
  tq_status st = check_state(s);
  if (st != TQ_OK) return st;
  if (!out) return TQ_ERR_ARG;
  const size_t N = 1ull << s->n;
  if ((st = ensure(s, s->probs, N * sizeof(double))) != TQ_OK) return st;
  const double* tr = nullptr;
  if (s->prec == TQ_SPLIT) {
    double tmp[2];
    if ((st = reduce_impl(s, nullptr, 0, false, tmp)) != TQ_OK) return st;
    tr = reinterpret_cast<const double*>(static_cast<char*>(s->red.ptr) + kRedOut);
  }
  cudaError_t e = launch_diag_probs(s->rho, s->n, s->prec, tr, static_cast<double*>(s->probs.ptr), s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, s->probs.ptr, N * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return cuda_fail(s, e);
}

}  // extern "C"
