// Autotuner for the batch engine: for one register size and precision it
// times every candidate (fusion width, tile size) on a synthetic batch that
// fills the GPU, keeps the fastest, and remembers it in a plain-text cache
// keyed by GPU name, precision and register size.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <iomanip>
#include <sstream>
#include <string>
#include <vector>

#include "tq_internal.h"
#include <cuda_runtime.h>

namespace tq {
bool batch_tensor_engine(int precision, int engine);  // tq_batch.cu
}

namespace {

// splitmix64: the tuner's own workload generator (not a parity input)
struct Rng {
  unsigned long long s;
  unsigned long long next() {
    unsigned long long z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (next() >> 11) * (1.0 / 9007199254740992.0); }
  int below(int m) { return (int)(next() % (unsigned long long)m); }
};

// A random noisy circuit over {H, RZ, RX, CX} with depolarising noise.
std::vector<tq_op> synth_circuit(int n, int depth, Rng& rng) {
  std::vector<tq_op> ops;
  for (int i = 0; i < depth; ++i) {
    tq_op g{};
    tq_op ch{};
    g.kind = TQ_OP_GATE;
    ch.kind = TQ_OP_CHANNEL;
    ch.name = TQ_CH_DEPOLARIZING;
    ch.params[0] = 1e-3;
    const int which = rng.below(4);
    if (which == 3 && n >= 2) {
      g.name = TQ_GATE_CX;
      g.k = 2;
      g.qubits[0] = rng.below(n);
      do g.qubits[1] = rng.below(n); while (g.qubits[1] == g.qubits[0]);
      ch.k = 2;
      ch.qubits[0] = g.qubits[0];
      ch.qubits[1] = g.qubits[1];
    } else {
      g.name = which == 0 ? TQ_GATE_H : (which == 1 ? TQ_GATE_RZ : TQ_GATE_RX);
      g.k = 1;
      g.qubits[0] = rng.below(n);
      g.params[0] = 6.283185307179586 * rng.uniform();
      ch.k = 1;
      ch.qubits[0] = g.qubits[0];
    }
    ops.push_back(g);
    ops.push_back(ch);
  }
  return ops;
}

std::string cache_key(int precision, int tensor, int n) {
  cudaDeviceProp prop;
  int dev = 0;
  std::string name = "unknown";
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
  for (char& c : name)
    if (c == ' ') c = '_';
  std::ostringstream os;
  os << name << " " << (precision == TQ_FP64 ? (tensor ? "fp64" : "fp64-dfma") : (tensor ? "split-tc" : "split")) << " "
     << n;
  return os.str();
}

bool cache_lookup(const char* path, const std::string& key, int* tile, int* width, double* ms) {
  if (!path) return false;
  std::ifstream f(path);
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    if (line.compare(0, key.size(), key) != 0 || line.size() <= key.size() || line[key.size()] != ' ') continue;
    std::istringstream is(line.substr(key.size()));
    int t, w;
    double m;
    if (is >> t >> w >> m) {
      *tile = t;
      *width = w;
      *ms = m;
      found = true;  // the last entry wins
    }
  }
  return found;
}

}  // namespace

extern "C" tq_status tq_autotune_engine(int precision, int fp64_engine, int n_qubits, const char* cache_path,
                                        int* tile_log2_out, int* width_out, double* ms_out) {
  if ((precision != TQ_FP64 && precision != TQ_SPLIT) || n_qubits < 2 || n_qubits > 14 || !tile_log2_out ||
      !width_out || fp64_engine < TQ_ENGINE_AUTO || fp64_engine > TQ_ENGINE_TENSOR)
    return TQ_ERR_ARG;
  // batches tune on the engine they will run with (the tile size only
  // matters on the persistent kernel)
  const int tensor = tq::batch_tensor_engine(precision, fp64_engine) ? 1 : 0;
  const std::string key = cache_key(precision, tensor, n_qubits);
  int tile = 0, width = 0;
  double best_ms = 0;
  if (cache_lookup(cache_path, key, &tile, &width, &best_ms)) {
    *tile_log2_out = tile;
    *width_out = width;
    if (ms_out) *ms_out = best_ms;
    return TQ_OK;
  }
  // a synthetic batch of about 2^24 density-matrix entries in total, and at
  // least enough jobs that the largest tile candidate (2^16 entries) still
  // gives ~8 work items per SM and fusion round (two resident CTAs each, four
  // items apiece); otherwise large registers would be tuned on a batch that
  // leaves most of the GPU idle at large tiles
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TQ_ERR_CUDA;
  const long long tiles_per_block = std::max(1ll, (1ll << (2 * n_qubits - 1)) >> 16);  // canonical half / 2^16
  const long long by_items = (8ll * sms + tiles_per_block - 1) / tiles_per_block;
  const int jobs = (int)std::max(1ll, std::min(256ll, std::max((1ll << 24) >> (2 * n_qubits), by_items)));
  Rng rng{0x243F6A8885A308D3ull ^ (unsigned long long)(n_qubits * 131 + precision)};
  std::vector<std::vector<tq_op>> circuits;
  for (int j = 0; j < jobs; ++j) circuits.push_back(synth_circuit(n_qubits, 64, rng));
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return TQ_ERR_CUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  best_ms = 1e300;
  tq_status result = TQ_OK;
  std::vector<int> tiles = {2 * n_qubits};
  for (int t : {16, 14, 12, 10})
    if (t < 2 * n_qubits && t >= 4) tiles.push_back(t);
  for (int w : {1, 2}) {
    for (int t : tiles) {
      tq_batch* b = nullptr;
      tq_status s = tq_batch_create(precision, st, &b);
      if (s == TQ_OK) s = tq_batch_set_fp64_engine(b, fp64_engine);
      for (int j = 0; j < jobs && s == TQ_OK; ++j)
        s = tq_batch_add(b, n_qubits, circuits[j].data(), circuits[j].size(), w, nullptr, 0, nullptr);
      if (s == TQ_OK) s = tq_batch_set_tile(b, n_qubits, t);
      if (s == TQ_OK) s = tq_batch_run(b);  // plans, captures the graph, first run
      if (s == TQ_OK) s = tq_batch_wait(b);
      float ms = 0.f;
      if (s == TQ_OK) {
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && s == TQ_OK; ++r) s = tq_batch_run(b);
        cudaEventRecord(e1, st);
        if (s == TQ_OK) s = tq_batch_wait(b);
        if (s == TQ_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) s = TQ_ERR_CUDA;
      }
      tq_batch_free(b);
      if (s != TQ_OK) {
        result = s;
        break;
      }
      if (ms / 3 < best_ms) {
        best_ms = ms / 3;
        tile = t;
        width = w;
      }
    }
    if (result != TQ_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (result != TQ_OK) return result;
  *tile_log2_out = tile;
  *width_out = width;
  if (ms_out) *ms_out = best_ms;
  if (cache_path) {
    std::ofstream f(cache_path, std::ios::app);
    f << key << " " << tile << " " << width << " " << std::setprecision(17) << best_ms << "\n";
  }
  return TQ_OK;
}

extern "C" tq_status tq_autotune(int precision, int n_qubits, const char* cache_path, int* tile_log2_out,
                                 int* width_out, double* ms_out) {
  return tq_autotune_engine(precision, TQ_ENGINE_AUTO, n_qubits, cache_path, tile_log2_out, width_out, ms_out);
}
