// Step scheduling of a domain (Algorithm 1) and the small host utilities around it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "runtime.h"

using namespace lbm;

namespace lbm {
struct GraphCache {
  // graphs[p] advances the single-block domain by `chunk` steps starting from level p
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  int chunk = 0;
};
}  // namespace lbm

void lbm_domain::pick_tiles(int b) {
  Block& B = blocks[b];
  // x-contiguous tiles of 256 threads; narrow blocks use a 32-wide tile with more rows
  B.bx = B.nx >= 128 ? 128 : B.nx >= 64 ? 64 : 32;
  B.by = 256 / B.bx;
  B.tuned = false;
  if (const char* env = std::getenv("LBM_TILE")) {  // "bx,by" forces a tile shape
    int bx = 0, by = 0;
    if (std::sscanf(env, "%d,%d", &bx, &by) == 2 && bx > 0 && by > 0 && bx * by <= 256 &&
        bx % 32 == 0) {
      B.bx = bx;
      B.by = by;
      B.tuned = true;
    }
  }
}

// Times candidate tile shapes of the collide-stream launch on the block's current state and
// keeps the fastest.  Candidates read the current level and write the next one without
// advancing the clock, so tuning changes no result (every shape computes the same values).
lbm_status lbm_domain::autotune_tiles(int b) {
  Block& B = blocks[b];
  if (B.tuned) return LBM_OK;
  B.tuned = true;
  if (B.N < (size_t)1 << 18 || B.lv.size() < 2) return LBM_OK;
  const int cand[][2] = {{32, 8}, {64, 4}, {128, 2}, {256, 1}, {32, 4}, {64, 2}, {128, 1}};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(cudaGetLastError(), "event");
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(cudaGetLastError(), "event"); }
  const int to = (B.cur + 1) % (int)B.lv.size();
  float best = 1e30f;
  int bx = B.bx, by = B.by;
  for (const auto& c : cand) {
    if (c[0] > 32 && c[0] > B.nx + 31) continue;
    const BlockView v = view(b, B.cur, to);
    cudaError_t e = launch_step(v, desc.storage, c[0], c[1], stream);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, stream);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_step(v, desc.storage, c[0], c[1], stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0); cudaEventDestroy(e1);
      return cuda_fail(e, "tile autotuning");
    }
    if (ms < best) { best = ms; bx = c[0]; by = c[1]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  B.bx = bx;
  B.by = by;
  return LBM_OK;
}

void lbm_domain::invalidate_graphs() {
  if (!graphs) return;
  for (int p = 0; p < 2; ++p)
    if (graphs->exec[p]) cudaGraphExecDestroy(graphs->exec[p]);
  delete graphs;
  graphs = nullptr;
}

void release_tape(lbm_domain* dom);        // adjoint.cu
void release_batch_plan(lbm_domain* dom);  // batch.cu

void lbm_domain::release_extras() {
  invalidate_graphs();
  release_batch_plan(this);
  release_tape(this);
  if (small_host) cudaFreeHost(small_host);
  small_host = nullptr;
  if (small_done) cudaEventDestroy(small_done);
  small_done = nullptr;
}

// Small host arrays (inflow records) go through a pinned bounce buffer so the copy is
// asynchronous and the caller can reuse its array on return.
const void* lbm_domain::upload_small(const void* src, size_t bytes, lbm_status* st) {
  *st = LBM_OK;
  if (bytes > small_bytes) {
    if (small_done) cudaEventSynchronize(small_done);
    if (small_host) cudaFreeHost(small_host);
    small_host = nullptr;
    dev_free(small_dev);
    small_dev = nullptr;
    size_t cap = std::max<size_t>(bytes, 4096);
    if (cudaMallocHost(&small_host, cap) != cudaSuccess) {
      small_host = nullptr;
      *st = fail(LBM_ERR_OOM, "pinned allocation failed");
      return nullptr;
    }
    small_dev = dev_alloc(cap);
    if (!small_dev) { *st = fail(LBM_ERR_OOM, "device allocation failed"); return nullptr; }
    small_bytes = cap;
  }
  if (!small_done) {
    if (cudaEventCreateWithFlags(&small_done, cudaEventDisableTiming) != cudaSuccess) {
      *st = fail(LBM_ERR_CUDA, "cudaEventCreate");
      return nullptr;
    }
  } else {
    cudaEventSynchronize(small_done);  // previous upload has left the bounce buffer
  }
  std::memcpy(small_host, src, bytes);
  cudaError_t e = cudaMemcpyAsync(small_dev, small_host, bytes, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaEventRecord(small_done, stream);
  if (e != cudaSuccess) { *st = cuda_fail(e, "small upload"); return nullptr; }
  return small_dev;
}

void lbm_domain::on_state_reset(int b) {
  (void)b;
  steps = 0;
  invalidate_graphs();
  release_tape(this);
}

lbm_status tape_before_step(lbm_domain* dom);  // adjoint.cu
lbm_status multiscale_step(lbm_domain* dom);  // coupling.cu

// n reference steps launched one kernel at a time.
lbm_status lbm_domain::advance_direct(int n) {
  for (int i = 0; i < n; ++i) {
    lbm_status st = tape_before_step(this);
    if (st != LBM_OK) return st;
    if (blocks.size() == 1) {
      Block& B = blocks[0];
      const int nxt = B.cur ^ 1;
      cudaError_t e = launch_step(view(0, B.cur, nxt), desc.storage, B.bx, B.by, stream);
      if (e != cudaSuccess) return cuda_fail(e, "collide-stream launch");
      B.cur = nxt;
    } else {
      st = multiscale_step(this);
      if (st != LBM_OK) return st;
    }
    ++steps;
  }
  return LBM_OK;
}

// Single-block domains without a tape replay a captured graph of `chunk` steps; the rest
// (and multi-block domains) launch directly.
lbm_status lbm_domain::advance(int n) {
  const int chunk = 16;
  if (n > 0) {
    for (size_t b = 0; b < blocks.size(); ++b) {
      const bool was = blocks[b].tuned;
      lbm_status st = autotune_tiles((int)b);
      if (st != LBM_OK) return st;
      if (!was) invalidate_graphs();
    }
  }
  if (blocks.size() != 1 || tape != nullptr || n < 2 * chunk) return advance_direct(n);
  Block& B = blocks[0];
  if (!graphs) {
    graphs = new GraphCache();
    graphs->chunk = chunk;
  }
  int done = 0;
  while (n - done >= chunk) {
    const int p = B.cur;
    if (!graphs->exec[p]) {
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
      int cur = p;
      for (int i = 0; i < chunk && e == cudaSuccess; ++i) {
        e = launch_step(view(0, cur, cur ^ 1), desc.storage, B.bx, B.by, stream);
        cur ^= 1;
      }
      cudaError_t e2 = cudaStreamEndCapture(stream, &g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(e != cudaSuccess ? e : e2, "step graph capture");
      }
      e = cudaGraphInstantiate(&graphs->exec[p], g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) { graphs->exec[p] = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
    }
    cudaError_t e = cudaGraphLaunch(graphs->exec[p], stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    if (chunk % 2) B.cur ^= 1;
    steps += chunk;
    done += chunk;
  }
  return advance_direct(n - done);
}
