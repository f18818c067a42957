// Feature-dimension sweep (§II-D: the kernel matrices for every qubit count n of a study)
// as one native call: every item's symmetric Gram through dk_gram_tile and, for complex64
// FP32 / split-BF16 items, its refinement pass (dk_gram_refine, tau = DK_REFINE_TAU), in
// order, on the caller's stream, optionally recorded once into a CUDA graph that the context keeps and
// replays, so a sweep of many Gram launches of uneven size costs one graph launch.
//
// Graph cache: keyed by the exact bytes of the item list and the call's parameters (the
// pointers included, so a replay reads and writes the same buffers); at most kMaxGraphs
// entries, the oldest evicted. The first call with a new key runs the items eagerly (so the
// one-time set-up of every kernel happens outside any capture), then records them without
// executing and instantiates the graph; later calls with the same key launch the graph.
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace dk {
namespace {

constexpr size_t kMaxGraphs = 16;

struct GraphEntry {
  std::vector<unsigned char> key;
  cudaGraphExec_t exec;
};

struct GraphCache {
  std::mutex mu;
  std::vector<GraphEntry> entries;  // oldest first
};

std::vector<unsigned char> make_key(const dk_sweep_item* items, int n_items, int chi_max, dk_dtype dtype,
                                    dk_precision prec, float w, const void* ws, size_t ws_bytes) {
  const size_t head = sizeof(dk_sweep_item) * size_t(n_items);
  std::vector<unsigned char> key(head + 4 * sizeof(int) + sizeof(ws) + sizeof(ws_bytes));
  memcpy(key.data(), items, head);
  int tail[4] = {chi_max, int(dtype), int(prec), 0};
  memcpy(&tail[3], &w, sizeof(float));
  memcpy(key.data() + head, tail, sizeof(tail));
  memcpy(key.data() + head + sizeof(tail), &ws, sizeof(ws));
  memcpy(key.data() + head + sizeof(tail) + sizeof(ws), &ws_bytes, sizeof(ws_bytes));
  return key;
}

dk_status run_items(dk_ctx* ctx, const dk_sweep_item* items, int n_items, int chi_max, dk_dtype dtype,
                    dk_precision prec, float w, void* ws, size_t ws_bytes, cudaStream_t st) {
  const int saved = ctx->gram_config;
  dk_status s = DK_OK;
  for (int t = 0; t < n_items && s == DK_OK; ++t) {
    const dk_sweep_item& it = items[t];
    ctx->gram_config = it.tile_shape;
    s = dk_gram_tile(ctx, it.mps, it.m, it.mps, it.m, it.n, chi_max, dtype, 0, it.m, 0, it.m, it.log_norm,
                     it.log_norm, it.x, it.x, 1.0f / float(it.n), w, prec, it.k, it.kq, it.kc, it.logkq, it.ld, 1,
                     st);
    const bool refinable = dtype == DK_C64 && (chi_max == 4 || chi_max == 8 || chi_max == 32) &&
                           (prec == DK_PREC_F32 || prec == DK_PREC_BF16X3) && (it.kq || it.logkq);
    if (s == DK_OK && refinable)
      s = dk_gram_refine(ctx, it.mps, it.m, it.mps, it.m, it.n, chi_max, dtype, 0, it.m, 0, it.m, it.x, it.x,
                         1.0f / float(it.n), w, DK_REFINE_TAU, it.k, it.kq, it.kc, it.logkq, it.ld, 1, ws, ws_bytes,
                         st);
  }
  ctx->gram_config = saved;
  return s;
}

}  // namespace

void sweep_cache_free(dk_ctx* ctx) {
  GraphCache* c = static_cast<GraphCache*>(ctx->graphs);
  if (!c) return;
  for (GraphEntry& e : c->entries) cudaGraphExecDestroy(e.exec);
  delete c;
  ctx->graphs = nullptr;
}

}  // namespace dk

DK_API dk_status dk_gram_sweep(dk_ctx* ctx, const dk_sweep_item* items, int n_items, int chi_max, dk_dtype dtype,
                               dk_precision prec, float w, int graph, void* ws, size_t ws_bytes, void* stream) {
  using namespace dk;
  if (!ctx || !items || n_items < 1) return DK_ERR_ARG;
  if (dtype == DK_SPLIT_BF16) return DK_ERR_UNSUPPORTED;  // the refinement needs the complex64 tensors
  for (int t = 0; t < n_items; ++t) {
    const dk_sweep_item& it = items[t];
    if (!it.mps || !it.log_norm || it.m < 1 || it.n < 1) return DK_ERR_ARG;
    if (!it.k && !it.kq && !it.kc && !it.logkq) return DK_ERR_ARG;
    if (it.ld < it.m) return DK_ERR_ARG;
    if (it.tile_shape < 0 || it.tile_shape > dk_gram_config_count(dtype, chi_max)) return DK_ERR_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!graph) return run_items(ctx, items, n_items, chi_max, dtype, prec, w, ws, ws_bytes, st);
  if (st == nullptr) return DK_ERR_ARG;  // the legacy default stream cannot be captured

  std::vector<unsigned char> key = make_key(items, n_items, chi_max, dtype, prec, w, ws, ws_bytes);
  if (!ctx->graphs) ctx->graphs = new GraphCache();
  GraphCache* cache = static_cast<GraphCache*>(ctx->graphs);
  std::lock_guard<std::mutex> lock(cache->mu);
  for (GraphEntry& e : cache->entries)
    if (e.key == key) return cudaGraphLaunch(e.exec, st) == cudaSuccess ? DK_OK : DK_ERR_CUDA;

  // new key: run eagerly, then record the same launches without executing them
  dk_status s = run_items(ctx, items, n_items, chi_max, dtype, prec, w, ws, ws_bytes, st);
  if (s != DK_OK) return s;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return DK_ERR_CUDA;
  }
  s = run_items(ctx, items, n_items, chi_max, dtype, prec, w, ws, ws_bytes, st);
  cudaGraph_t g = nullptr;
  const cudaError_t end = cudaStreamEndCapture(st, &g);
  if (s != DK_OK || end != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return s != DK_OK ? s : DK_ERR_CUDA;
  }
  cudaGraphExec_t exec = nullptr;
  const cudaError_t inst = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  if (inst != cudaSuccess || !exec) {
    cudaGetLastError();
    return DK_ERR_CUDA;
  }
  if (cache->entries.size() >= kMaxGraphs) {
    cudaGraphExecDestroy(cache->entries.front().exec);
    cache->entries.erase(cache->entries.begin());
  }
  cache->entries.push_back(GraphEntry{std::move(key), exec});
  return DK_OK;
}
