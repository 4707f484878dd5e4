// Step scheduling of a domain (Algorithm 1) and the small host utilities around it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "runtime.h"

using namespace lbm;

namespace lbm {
// Captured step graphs, one per starting assignment of time levels (the `cur` level of every
// block).  Each graph advances `chunk` reference steps, a multiple of the period after which
// the level assignment repeats, so it ends in the assignment it started from.
struct GraphCache {
  std::vector<std::pair<std::vector<int>, cudaGraphExec_t>> exec;     // chunk-step graphs
  std::vector<std::pair<std::vector<int>, cudaGraphExec_t>> single;   // one-step graphs
  int chunk = 0;
};

// Level assignment after one reference step (mirrors the schedule of multiscale_step).
static std::vector<int> next_levels(const std::vector<lbm::Block>& blocks, std::vector<int> cur) {
  cur[0] ^= 1;
  for (size_t b = 1; b < blocks.size(); ++b) {
    if (blocks[b].far) {     // far-field blocks ping-pong like the reference block
      cur[b] ^= 1;
      continue;
    }
    const int L = cur[b], A = (L + 1) % 3, B = (L + 2) % 3;
    int c = L;
    for (int j = 1; j <= blocks[b].substeps; ++j) c = (j == 1) ? A : (c == A ? B : A);
    cur[b] = c;
  }
  return cur;
}
}  // namespace lbm

void lbm_domain::pick_tiles(int b) {
  Block& B = blocks[b];
  // x-contiguous tiles of 256 threads; narrow blocks use a 32-wide tile with more rows
  B.bx = B.nx >= 128 ? 128 : B.nx >= 64 ? 64 : 32;
  B.by = 256 / B.bx;
  B.tuned = false;
  B.minb = 3;
  if (const char* env = std::getenv("LBM_TILE")) {  // "bx,by[,minb]" forces a launch shape
    int bx = 0, by = 0, mb = 3;
    const int n = std::sscanf(env, "%d,%d,%d", &bx, &by, &mb);
    const bool mb_ok = mb == 3 || mb == 4 || (mb >= STEP_PAIR + 4 && mb <= STEP_PAIR + 6);
    if (n >= 2 && bx > 0 && by > 0 && bx * by <= 256 && bx % 32 == 0 && mb_ok) {
      B.bx = bx;
      B.by = by;
      B.minb = mb;
      B.tuned = true;
    }
  }
}

// Times candidate launch shapes of the collide-stream kernel (tile shape x register bound) on
// the block's current state and keeps the fastest.  Candidates read the current level and write the next one without
// advancing the clock, so tuning changes no result (every shape computes the same values).
lbm_status lbm_domain::autotune_tiles(int b) {
  Block& B = blocks[b];
  if (B.tuned) return LBM_OK;
  B.tuned = true;
  if (B.N < (size_t)1 << 18 || B.lv.size() < 2) return LBM_OK;
  const int nx_class = B.nx >= 256 ? 3 : B.nx >= 128 ? 2 : B.nx >= 64 ? 1 : 0;
  const int n_class = B.N < ((size_t)1 << 20) ? 0 : B.N < ((size_t)1 << 23) ? 1 : 2;
  for (const TunedShape& t : tuned_shapes)
    if (t.nx_class == nx_class && t.n_class == n_class) {
      B.bx = t.bx;
      B.by = t.by;
      B.minb = t.minb;
      return LBM_OK;
    }
  const int cand[][2] = {{32, 8}, {64, 4}, {128, 2}, {256, 1}, {32, 4}, {64, 2}, {128, 1}};
  // bound codes: one-node kernel at 3 or 4 CTAs of the tile per SM, then (even nx) the
  // two-node kernel at 4, 5 or 6 CTAs of half the threads, on tiles of at least 64 x-nodes
  const int bounds[] = {3, 4, STEP_PAIR + 4, STEP_PAIR + 5, STEP_PAIR + 6};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(cudaGetLastError(), "event");
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(cudaGetLastError(), "event"); }
  const int to = (B.cur + 1) % (int)B.lv.size();
  float best = 1e30f;
  int bx = B.bx, by = B.by, minb = B.minb;
  for (const int mb : bounds)
  for (const auto& c : cand) {
    if (c[0] > 32 && c[0] > B.nx + 31) continue;
    if (step_is_pair(mb) && (B.nx % 2 != 0 || c[0] < 64 || c[0] > B.nx + 63)) continue;
    const BlockView v = view(b, B.cur, to);
    cudaError_t e = launch_step(v, desc.storage, c[0], c[1], stream, mb);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, stream);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_step(v, desc.storage, c[0], c[1], stream, mb);
    if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0); cudaEventDestroy(e1);
      return cuda_fail(e, "tile autotuning");
    }
    if (ms < best) { best = ms; bx = c[0]; by = c[1]; minb = mb; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  B.bx = bx;
  B.by = by;
  B.minb = minb;
  tuned_shapes.push_back({nx_class, n_class, bx, by, minb});
  return LBM_OK;
}

void lbm_domain::invalidate_graphs() {
  if (!graphs) return;
  for (auto& kv : graphs->exec)
    if (kv.second) cudaGraphExecDestroy(kv.second);
  for (auto& kv : graphs->single)
    if (kv.second) cudaGraphExecDestroy(kv.second);
  delete graphs;
  graphs = nullptr;
}

void release_tape(lbm_domain* dom);        // adjoint.cu
void release_batch_plan(lbm_domain* dom);  // batch.cu

lbm_status lbm_domain::aux(cudaStream_t* out) {
  if (!aux_stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&aux_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { aux_stream = nullptr; return cuda_fail(e, "cudaStreamCreate"); }
  }
  *out = aux_stream;
  return LBM_OK;
}

cudaEvent_t lbm_domain::event(int i) {
  while ((int)events.size() <= i) {
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    events.push_back(ev);
  }
  return events[i];
}

cudaStream_t lbm_domain::post_stream(int k) {
  while ((int)post_streams.size() <= k) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    post_streams.push_back(st);
  }
  return post_streams[k];
}

void lbm_domain::release_extras() {
  invalidate_graphs();
  release_batch_plan(this);
  if (rb_dev) dev_free(rb_dev);
  rb_dev = nullptr;
  rb_dev_bytes = 0;
  if (rb_host) cudaFreeHost(rb_host);
  rb_host = nullptr;
  rb_host_bytes = 0;
  if (ib_done) cudaEventSynchronize(ib_done);
  if (ib_dev) dev_free(ib_dev);
  ib_dev = nullptr;
  ib_dev_bytes = 0;
  if (ib_host) cudaFreeHost(ib_host);
  ib_host = nullptr;
  ib_host_bytes = 0;
  if (ib_done) cudaEventDestroy(ib_done);
  ib_done = nullptr;
  for (cudaEvent_t ev : events) cudaEventDestroy(ev);
  events.clear();
  for (cudaStream_t st : post_streams) cudaStreamDestroy(st);
  post_streams.clear();
  if (aux_stream) cudaStreamDestroy(aux_stream);
  aux_stream = nullptr;
  release_tape(this);
  if (small_host) cudaFreeHost(small_host);
  small_host = nullptr;
  if (small_done) cudaEventDestroy(small_done);
  small_done = nullptr;
  for (cudaEvent_t& ev : result_ev) {
    if (ev) cudaEventDestroy(ev);
    ev = nullptr;
  }
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
    small_bytes = 0;       // no buffer until both allocations below succeed
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
      cudaError_t e = launch_step(view(0, B.cur, nxt), desc.storage, B.bx, B.by, stream, B.minb);
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

// Without a tape, steps are replayed from captured graphs of `chunk` reference steps (a
// multiple of the level-rotation period, at least 16 steps); the remainder launches directly.
// m reference steps of a continuous-scale domain from one-step graphs captured per level
// assignment (the schedule of one step is 16 launches with forks and joins on several
// streams; replaying it as one graph leaves the GPU no gaps between them).  Single-block
// domains launch their one kernel directly.
lbm_status lbm_domain::advance_single(int m) {
  if (blocks.size() == 1 || !graphs) return advance_direct(m);
  for (int i = 0; i < m; ++i) {
    std::vector<int> key(blocks.size());
    for (size_t b = 0; b < blocks.size(); ++b) key[b] = blocks[b].cur;
    cudaGraphExec_t exec = nullptr;
    for (auto& kv : graphs->single)
      if (kv.first == key) exec = kv.second;
    if (!exec) {
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
      const lbm_status st = multiscale_step(this);
      cudaError_t e2 = cudaStreamEndCapture(stream, &g);
      for (size_t b = 0; b < blocks.size(); ++b) blocks[b].cur = key[b];
      if (st != LBM_OK || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return st != LBM_OK ? st : cuda_fail(e2, "step graph capture");
      }
      e = cudaGraphInstantiate(&exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
      graphs->single.push_back({key, exec});
    }
    const cudaError_t e = cudaGraphLaunch(exec, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    const std::vector<int> s = next_levels(blocks, key);
    for (size_t b = 0; b < blocks.size(); ++b) blocks[b].cur = s[b];
    ++steps;
  }
  return LBM_OK;
}

lbm_status lbm_domain::advance(int n) {
  if (n > 0) {
    for (size_t b = 0; b < blocks.size(); ++b) {
      const bool was = blocks[b].tuned;
      lbm_status st = autotune_tiles((int)b);
      if (st != LBM_OK) return st;
      if (!was) invalidate_graphs();
    }
  }
  if (blocks.size() > 1) {  // stream and events of the fork/join schedule exist before capture
    cudaStream_t a = nullptr;
    lbm_status st = aux(&a);
    if (st != LBM_OK) return st;
    if (!event(10 + 3 * (int)blocks.size())) return fail(LBM_ERR_CUDA, "cudaEventCreate");
    if (!post_stream((int)blocks.size())) return fail(LBM_ERR_CUDA, "cudaStreamCreate");
  }
  if (tape != nullptr) return advance_direct(n);
  std::vector<int> start(blocks.size());
  for (size_t b = 0; b < blocks.size(); ++b) start[b] = blocks[b].cur;
  if (!graphs) {
    int period = 1;
    std::vector<int> s = next_levels(blocks, start);
    while (s != start && period < 64) { s = next_levels(blocks, s); ++period; }
    if (s != start) return advance_direct(n);
    graphs = new GraphCache();
    graphs->chunk = period * ((16 + period - 1) / period);
  }
  const int chunk = graphs->chunk;
  if (n < 2 * chunk) return advance_single(n);
  int done = 0;
  while (n - done >= chunk) {
    std::vector<int> key(blocks.size());
    for (size_t b = 0; b < blocks.size(); ++b) key[b] = blocks[b].cur;
    cudaGraphExec_t exec = nullptr;
    for (auto& kv : graphs->exec)
      if (kv.first == key) exec = kv.second;
    if (!exec) {
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
      lbm_status st = LBM_OK;
      for (int i = 0; i < chunk && st == LBM_OK; ++i) {
        if (blocks.size() == 1) {
          Block& B = blocks[0];
          const cudaError_t el = launch_step(view(0, B.cur, B.cur ^ 1), desc.storage, B.bx, B.by, stream, B.minb);
          if (el != cudaSuccess) st = cuda_fail(el, "collide-stream launch");
          B.cur ^= 1;
        } else {
          st = multiscale_step(this);
        }
      }
      cudaError_t e2 = cudaStreamEndCapture(stream, &g);
      for (size_t b = 0; b < blocks.size(); ++b) blocks[b].cur = key[b];
      if (st != LBM_OK || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return st != LBM_OK ? st : cuda_fail(e2, "step graph capture");
      }
      e = cudaGraphInstantiate(&exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
      graphs->exec.push_back({key, exec});
    }
    cudaError_t e = cudaGraphLaunch(exec, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    std::vector<int> s = key;
    for (int i = 0; i < chunk; ++i) s = next_levels(blocks, s);
    for (size_t b = 0; b < blocks.size(); ++b) blocks[b].cur = s[b];
    steps += chunk;
    done += chunk;
  }
  return advance_single(n - done);
}

// lbm_step_reduce: n reference steps whose last one (on a single-block domain with 32-bit
// indexing) also sums the diagnostics of the state it stores, so that reading mass, momentum
// and energy back after a step costs no second pass over the populations.  Other domains
// take the n steps and lbm_reduce of block 0.
// Enqueues n steps and the diagnostics of block 0's new state: the 6 sums into dom->d_red
// and, when out5 (device) is given, the 5 combined values.  On a single-block domain with
// 27 N < 2^32 the last step's own kernel sums them; otherwise a separate reduction follows.
static lbm_status enqueue_step_reduce(lbm_domain* dom, int32_t n, double* out5) {
  Block& B = dom->blocks[0];
  if (dom->blocks.size() > 1 || !fits_32bit_index(B.N)) {
    lbm_status st = dom->advance(n);
    if (st != LBM_OK) return st;
    const cudaError_t e = launch_reduce(B.lv[B.cur].f, dom->desc.storage, B.flags, B.N,
                                        dom->d_partials, dom->d_red, dom->stream, out5);
    return e == cudaSuccess ? LBM_OK : dom->cuda_fail(e, "reduce");
  }
  lbm_status st = dom->advance(n - 1);
  if (st == LBM_OK) st = dom->autotune_tiles(0);
  if (st == LBM_OK) st = tape_before_step(dom);
  if (st != LBM_OK) return st;
  const int nxt = B.cur ^ 1;
  const BlockView v = dom->view(0, B.cur, nxt);
  const size_t ctas = step_reduce_ctas(v, B.bx, B.by);
  if (ctas > dom->step_partials_n) {
    if (dom->d_step_partials) dom->dev_free(dom->d_step_partials);
    dom->step_partials_n = 0;
    dom->d_step_partials = static_cast<double*>(dom->dev_alloc((ctas * 8 + 6 * 128) * sizeof(double)));
    if (!dom->d_step_partials) return dom->fail(LBM_ERR_OOM, "step-reduce partials");
    dom->step_partials_n = ctas;
  }
  const cudaError_t e = launch_step_reduce(v, dom->desc.storage, B.bx, B.by, dom->stream, B.minb,
                                           dom->d_step_partials, dom->d_red, out5);
  if (e != cudaSuccess) return dom->cuda_fail(e, "collide-stream launch");
  B.cur = nxt;
  ++dom->steps;
  return LBM_OK;
}

lbm_status lbm_step_reduce(lbm_domain* dom, int32_t n, double out[5]) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  if (n < 1) return dom->fail(LBM_ERR_INVALID_ARG, "lbm_step_reduce needs at least one step");
  if (!out) return dom->fail(LBM_ERR_INVALID_ARG, "null output");
  if (*dom->h_err & 1) return dom->fail(LBM_ERR_DIVERGED, "divergence recorded by an earlier step");
  lbm_status st = enqueue_step_reduce(dom, n, nullptr);
  if (st != LBM_OK) return st;
  const cudaError_t e = cudaMemcpyAsync(dom->h_red, dom->d_red, 6 * sizeof(double),
                                        cudaMemcpyDeviceToHost, dom->stream);
  if (e != cudaSuccess) return dom->cuda_fail(e, "reduce read-back");
  st = dom->sync_and_check();
  const double* r = dom->h_red;
  out[0] = r[0] + r[1];
  out[1] = r[2];
  out[2] = r[3];
  out[3] = r[4];
  out[4] = r[5];
  return st;
}

lbm_status lbm_step_reduce_async(lbm_domain* dom, int32_t n, double out[5], int64_t* ticket) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  if (n < 1) return dom->fail(LBM_ERR_INVALID_ARG, "lbm_step_reduce_async needs at least one step");
  if (!out || !ticket) return dom->fail(LBM_ERR_INVALID_ARG, "null output or ticket");
  if (*dom->h_err & 1) return dom->fail(LBM_ERR_DIVERGED, "divergence recorded by an earlier step");
  const int slot = (int)(dom->results_issued % lbm_domain::kResultSlots);
  if (!dom->result_ev[slot] &&
      cudaEventCreateWithFlags(&dom->result_ev[slot], cudaEventDisableTiming) != cudaSuccess) {
    dom->result_ev[slot] = nullptr;
    return dom->fail(LBM_ERR_CUDA, "cudaEventCreate");
  }
  double* d_out5 = dom->d_red + 8;
  lbm_status st = enqueue_step_reduce(dom, n, d_out5);
  if (st != LBM_OK) return st;
  cudaError_t e = cudaMemcpyAsync(out, d_out5, 5 * sizeof(double), cudaMemcpyDeviceToHost,
                                  dom->stream);
  if (e == cudaSuccess) {
    dom->post_error_probe();
    e = cudaEventRecord(dom->result_ev[slot], dom->stream);
  }
  if (e != cudaSuccess) return dom->cuda_fail(e, "reduce read-back");
  *ticket = ++dom->results_issued;
  return LBM_OK;
}

lbm_status lbm_wait_results(lbm_domain* dom, int64_t ticket) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  if (ticket < 1 || ticket > dom->results_issued)
    return dom->fail(LBM_ERR_INVALID_ARG, "not a ticket of lbm_step_reduce_async on this domain");
  const int slot = (int)((ticket - 1) % lbm_domain::kResultSlots);
  const cudaError_t e = cudaEventSynchronize(dom->result_ev[slot]);
  if (e != cudaSuccess) return dom->cuda_fail(e, "cudaEventSynchronize");
  return dom->error_status();
}
