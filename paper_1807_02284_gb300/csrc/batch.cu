// Batched persistent stepping of many independent single-block domains of uneven sizes.
//
// All domains' nodes are cut into chunks of consecutive node indices; one cooperative,
// persistent kernel walks the joint chunk list for every step and separates the steps with a
// device-wide barrier.  The barrier's waits are bounded by a clock limit: a CTA that waits too
// long sets the TIMEOUT bit of the error word and every CTA leaves the kernel, so a lost CTA
// can never hang the GPU.  The launch (plus the reset of the barrier counters) is captured in
// a CUDA graph and replayed.  Every node runs the same cell_update as the single-block kernel,
// so results are bit-identical to stepping each domain on its own.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "lbm_cell.cuh"
#include "runtime.h"

namespace lbm {

struct BatchItem {
  int dom;        // domain index in the batch
  uint32_t start; // first node of the chunk
};

struct BarrierState {
  unsigned int count;
  unsigned int gen;
};

constexpr long long kBarrierLimitCycles = 4000000000LL;  // ~2 s at 2 GHz

// Device-wide barrier with a bounded wait.  Returns false when the wait gave up.
__device__ __forceinline__ bool grid_barrier(BarrierState* bs, unsigned int nblocks, int* err,
                                             long long limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned int* vgen = &bs->gen;
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&bs->count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&bs->count, 0u);
      __threadfence();
      atomicAdd(&bs->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if (clock64() - t0 > limit) {
          atomicOr(err, 8);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <typename T, typename IT>
__global__ void __launch_bounds__(256) k_batch(const BlockView* __restrict__ views,
                                               const BatchItem* __restrict__ items, int n_items,
                                               int chunk, int steps, BarrierState* bs,
                                               unsigned int expected_blocks, int* err,
                                               long long limit) {
  for (int s = 0; s < steps; ++s) {
    const int p = s & 1;
    for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
      const BatchItem it = items[w];
      const BlockView& v = views[2 * it.dom + p];
      const uint32_t nx = (uint32_t)v.nx, nxy = (uint32_t)v.nx * (uint32_t)v.ny;
      const uint32_t end = min((uint32_t)v.N, it.start + (uint32_t)chunk);
      for (uint32_t idx = it.start + threadIdx.x; idx < end; idx += blockDim.x) {
        const uint32_t z = idx / nxy;
        const uint32_t r = idx - z * nxy;
        const uint32_t y = r / nx;
        cell_update<T, IT>(v, (int)(r - y * nx), (int)y, (int)z);
      }
    }
    if (s + 1 < steps) {
      if (!grid_barrier(bs, expected_blocks, err, limit)) return;
      if (*((volatile int*)err) & 8) return;
    }
  }
}

// k_batch with the diagnostics fused into the last step (lbm_step_batch_reduce): in that
// step each node adds its moments (from cell_update, into a per-thread shared-memory slot)
// to its thread's accumulator, and every work item ends with a CTA sum (shuffle tree per
// warp, warps in order, FP32) stored as one record of 8 doubles, records[item * 8 + value].
// The populations, velocities and scalars are those of k_batch.
template <typename T>
__global__ void __launch_bounds__(256, 2) k_batch_red(const BlockView* __restrict__ views,
                                                   const BatchItem* __restrict__ items,
                                                   int n_items, int chunk, int steps,
                                                   BarrierState* bs, unsigned int expected_blocks,
                                                   int* err, long long limit, double* records) {
  __shared__ float tmp[6][256];
  __shared__ float acc[6][256];
  __shared__ float swarp[8][6];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const NodeMomentsOut out{&tmp[0][t], 256};
  for (int s = 0; s < steps; ++s) {
    const int p = s & 1;
    const bool last = s + 1 == steps;
    for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
      const BatchItem it = items[w];
      const BlockView& v = views[2 * it.dom + p];
      const uint32_t nx = (uint32_t)v.nx, nxy = (uint32_t)v.nx * (uint32_t)v.ny;
      const uint32_t end = min((uint32_t)v.N, it.start + (uint32_t)chunk);
      if (!last) {
        for (uint32_t idx = it.start + t; idx < end; idx += blockDim.x) {
          const uint32_t z = idx / nxy;
          const uint32_t r = idx - z * nxy;
          const uint32_t y = r / nx;
          cell_update<T, uint32_t>(v, (int)(r - y * nx), (int)y, (int)z);
        }
        continue;
      }
#pragma unroll
      for (int i = 0; i < 6; ++i) acc[i][t] = 0.0f;
      for (uint32_t idx = it.start + t; idx < end; idx += blockDim.x) {
        const uint32_t z = idx / nxy;
        const uint32_t r = idx - z * nxy;
        const uint32_t y = r / nx;
#pragma unroll
        for (int i = 0; i < 6; ++i) tmp[i][t] = 0.0f;
        cell_update<T, uint32_t, false, false, true>(v, (int)(r - y * nx), (int)y, (int)z, &out);
#pragma unroll
        for (int i = 0; i < 6; ++i) acc[i][t] += tmp[i][t];
      }
      float val[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) val[i] = acc[i][t];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < 6; ++i) val[i] += __shfl_xor_sync(0xffffffffu, val[i], o);
      if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 6; ++i) swarp[wid][i] = val[i];
      }
      __syncthreads();
      if (t < 8) {
        float sum = 0.0f;
        if (t < 6)
          for (int k = 0; k < (int)(blockDim.x >> 5); ++k) sum += swarp[k][t];
        records[(size_t)w * 8 + t] = (double)sum;
      }
      __syncthreads();
    }
    if (s + 1 < steps) {
      if (!grid_barrier(bs, expected_blocks, err, limit)) return;
      if (*((volatile int*)err) & 8) return;
    }
  }
}

template <typename T>
static cudaError_t launch_batch_red_t(const BlockView* views, const BatchItem* items, int n_items,
                                      int chunk, int steps, BarrierState* bs, int threads,
                                      int grid, unsigned int expected, int* err, long long limit,
                                      double* records, cudaStream_t s) {
  void* args[] = {(void*)&views, (void*)&items, (void*)&n_items, (void*)&chunk, (void*)&steps,
                  (void*)&bs, (void*)&expected, (void*)&err, (void*)&limit, (void*)&records};
  return cudaLaunchCooperativeKernel((const void*)k_batch_red<T>, dim3(grid), dim3(threads),
                                     args, 0, s);
}

template <typename T, typename IT>
static cudaError_t launch_batch_t(const BlockView* views, const BatchItem* items, int n_items,
                                  int chunk, int steps, BarrierState* bs, int threads, int grid,
                                  unsigned int expected, int* err, long long limit,
                                  bool cooperative, cudaStream_t s) {
  if (!cooperative) {
    k_batch<T, IT><<<grid, threads, 0, s>>>(views, items, n_items, chunk, steps, bs, expected,
                                            err, limit);
    return cudaGetLastError();
  }
  void* args[] = {(void*)&views, (void*)&items, (void*)&n_items, (void*)&chunk, (void*)&steps,
                  (void*)&bs, (void*)&expected, (void*)&err, (void*)&limit};
  return cudaLaunchCooperativeKernel((const void*)k_batch<T, IT>, dim3(grid), dim3(threads),
                                     args, 0, s);
}

static cudaError_t launch_batch(int storage, bool i32, const BlockView* views,
                                const BatchItem* items, int n_items, int chunk, int steps,
                                BarrierState* bs, int threads, int grid, unsigned int expected,
                                int* err, long long limit, bool cooperative, cudaStream_t s) {
  if (storage == ST_FP16) {
    if (i32) return launch_batch_t<__half, uint32_t>(views, items, n_items, chunk, steps, bs, threads, grid, expected, err, limit, cooperative, s);
    return launch_batch_t<__half, uint64_t>(views, items, n_items, chunk, steps, bs, threads, grid, expected, err, limit, cooperative, s);
  }
  if (i32) return launch_batch_t<float, uint32_t>(views, items, n_items, chunk, steps, bs, threads, grid, expected, err, limit, cooperative, s);
  return launch_batch_t<float, uint64_t>(views, items, n_items, chunk, steps, bs, threads, grid, expected, err, limit, cooperative, s);
}

static int resident_blocks(int storage, bool i32, int threads, bool red = false) {
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void* fn = red ? (storage == ST_FP16 ? (const void*)k_batch_red<__half> : (const void*)k_batch_red<float>)
                 : storage == ST_FP16
                       ? (i32 ? (const void*)k_batch<__half, uint32_t> : (const void*)k_batch<__half, uint64_t>)
                       : (i32 ? (const void*)k_batch<float, uint32_t> : (const void*)k_batch<float, uint64_t>);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0);
  return std::max(1, per_sm) * std::max(1, sms);
}

// One captured batched launch: the work list and views of a set of domains, starting from a
// given assignment of time levels and advancing a given number of steps.
struct BatchPlan {
  std::vector<unsigned long long> serials;   // members (domain serials, in call order)
  std::vector<int> curs;
  int steps = 0;
  int chunk = 0, threads = 0;
  BlockView* views = nullptr;
  BatchItem* items = nullptr;
  BarrierState* bar = nullptr;
  int n_items = 0;
  bool i32 = true;
  int grid = 0;
  cudaGraphExec_t exec = nullptr;
  bool captured = false;
  // fused diagnostics (lbm_step_batch_reduce): per-item records, per-member sums (sums and
  // error word, 8 doubles each) copied to pinned host memory by the same graph
  bool red = false;
  double* records = nullptr;
  RedMember* members = nullptr;
  double* out_dev = nullptr;
  double* out_host = nullptr;
  double* out5_dev = nullptr;   // lbm_step_batch_reduce_async: 5 values per member
};

// Plans cached by the first domain of a batch.  A call with an odd step count flips every
// member's current level, so alternating calls need two plans; a few more cover a caller
// that alternates between batches.  Members are matched by serial, never by address, so a
// plan never refers to a destroyed domain's memory once it is chosen.
struct BatchCache {
  std::vector<BatchPlan*> plans;   // most recently used last
  int chunk = 0, threads = 0;      // tuned once per cache
};
constexpr size_t kMaxBatchPlans = 4;

}  // namespace lbm

using namespace lbm;

static void free_plan(lbm_domain* dom, BatchPlan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  dom->dev_free(p->views);
  dom->dev_free(p->items);
  dom->dev_free(p->bar);
  if (p->records) dom->dev_free(p->records);
  if (p->members) dom->dev_free(p->members);
  if (p->out_dev) dom->dev_free(p->out_dev);
  if (p->out5_dev) dom->dev_free(p->out5_dev);
  if (p->out_host) cudaFreeHost(p->out_host);
  delete p;
}

// The diagnostics buffers of a plan: one record per work item, the members' item ranges and
// error words, the per-member sums on the device and in pinned host memory.
static lbm_status add_red_buffers(lbm_domain* const* doms, int n, BatchPlan* p) {
  lbm_domain* d0 = doms[0];
  std::vector<RedMember> hm(n);
  int at = 0;
  for (int i = 0; i < n; ++i) {
    const Block& B = doms[i]->blocks[0];
    const int cnt = (int)((B.N + (size_t)p->chunk - 1) / (size_t)p->chunk);
    hm[i] = RedMember{nullptr, nullptr, doms[i]->d_err, B.N, at, cnt};
    at += cnt;
  }
  if (at != p->n_items) return d0->fail(LBM_ERR_STATE, "batch work list and members disagree");
  p->records = static_cast<double*>(d0->dev_alloc((size_t)p->n_items * 8 * sizeof(double)));
  p->members = static_cast<RedMember*>(d0->dev_alloc((size_t)n * sizeof(RedMember)));
  p->out_dev = static_cast<double*>(d0->dev_alloc((size_t)n * 8 * sizeof(double)));
  p->out5_dev = static_cast<double*>(d0->dev_alloc((size_t)n * 5 * sizeof(double)));
  if (!p->records || !p->members || !p->out_dev || !p->out5_dev)
    return d0->fail(LBM_ERR_OOM, "batch diagnostics buffers");
  if (cudaMallocHost(&p->out_host, (size_t)n * 8 * sizeof(double)) != cudaSuccess) {
    p->out_host = nullptr;
    return d0->fail(LBM_ERR_OOM, "batch diagnostics staging");
  }
  cudaError_t e = cudaMemcpyAsync(p->members, hm.data(), (size_t)n * sizeof(RedMember),
                                  cudaMemcpyHostToDevice, d0->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d0->stream);
  if (e != cudaSuccess) return d0->cuda_fail(e, "batch diagnostics upload");
  p->red = true;
  return LBM_OK;
}

// The work of one batched call on stream s: reset the barrier, the persistent launch, and with
// fused diagnostics the per-member sums and their copy to pinned host memory.
static cudaError_t enqueue_batch(lbm_domain* d0, BatchPlan* p, int steps, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(p->bar, 0, sizeof(BarrierState), s);
  if (e != cudaSuccess) return e;
  if (!p->red)
    return launch_batch(d0->desc.storage, p->i32, p->views, p->items, p->n_items, p->chunk, steps,
                        p->bar, p->threads, p->grid, (unsigned)p->grid, d0->d_err,
                        kBarrierLimitCycles, true, s);
  e = d0->desc.storage == ST_FP16
          ? launch_batch_red_t<__half>(p->views, p->items, p->n_items, p->chunk, steps, p->bar,
                                       p->threads, p->grid, (unsigned)p->grid, d0->d_err,
                                       kBarrierLimitCycles, p->records, s)
          : launch_batch_red_t<float>(p->views, p->items, p->n_items, p->chunk, steps, p->bar,
                                      p->threads, p->grid, (unsigned)p->grid, d0->d_err,
                                      kBarrierLimitCycles, p->records, s);
  const int n = (int)p->serials.size();
  if (e == cudaSuccess) e = launch_reduce_item_records(p->records, p->members, n, p->out_dev, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->out_host, p->out_dev, (size_t)n * 8 * sizeof(double),
                        cudaMemcpyDeviceToHost, s);
  return e;
}

void release_batch_plan(lbm_domain* dom) {
  BatchCache* c = static_cast<BatchCache*>(dom->batch_plan);
  if (!c) return;
  for (BatchPlan* p : c->plans) free_plan(dom, p);
  delete c;
  dom->batch_plan = nullptr;
}

// Views for both step parities and the chunk list of the current batch.
static lbm_status build_plan(lbm_domain* const* doms, int n, int chunk, BatchPlan* p) {
  lbm_domain* d0 = doms[0];
  std::vector<BlockView> hv(2 * (size_t)n);
  std::vector<BatchItem> hi;
  p->i32 = true;
  for (int i = 0; i < n; ++i) {
    const Block& B = doms[i]->blocks[0];
    hv[2 * i + 0] = doms[i]->view(0, B.cur, B.cur ^ 1);
    hv[2 * i + 1] = doms[i]->view(0, B.cur ^ 1, B.cur);
    if (27ull * B.N >= 0xFFFFFFFFull) p->i32 = false;
    for (size_t s = 0; s < B.N; s += (size_t)chunk) hi.push_back(BatchItem{i, (uint32_t)s});
  }
  if (!p->i32) return d0->fail(LBM_ERR_UNSUPPORTED, "batched domains must have 27 N < 2^32");
  p->views = static_cast<BlockView*>(d0->dev_alloc(hv.size() * sizeof(BlockView)));
  p->items = static_cast<BatchItem*>(d0->dev_alloc(hi.size() * sizeof(BatchItem)));
  p->bar = static_cast<BarrierState*>(d0->dev_alloc(sizeof(BarrierState)));
  if (!p->views || !p->items || !p->bar) return d0->fail(LBM_ERR_OOM, "batch plan allocation failed");
  cudaError_t e = cudaMemcpyAsync(p->views, hv.data(), hv.size() * sizeof(BlockView),
                                  cudaMemcpyHostToDevice, d0->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->items, hi.data(), hi.size() * sizeof(BatchItem), cudaMemcpyHostToDevice,
                        d0->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d0->stream);
  if (e != cudaSuccess) return d0->cuda_fail(e, "batch plan upload");
  p->n_items = (int)hi.size();
  p->chunk = chunk;
  p->serials.resize(n);
  p->curs.resize(n);
  for (int i = 0; i < n; ++i) {
    p->serials[i] = doms[i]->serial;
    p->curs[i] = doms[i]->blocks[0].cur;
  }
  return LBM_OK;
}

// Picks the chunk size of the work list by timing single-step launches that write the next
// level without advancing any domain (no result changes).
static lbm_status tune_chunk(lbm_domain* const* doms, int n, int* chunk_out, int* threads_out) {
  lbm_domain* d0 = doms[0];
  const int cand[][2] = {{256, 256}, {256, 512}, {256, 1024}, {128, 128}, {128, 256}};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  *chunk_out = 256;
  *threads_out = 256;
  for (const auto& c : cand) {
    BatchPlan p;
    lbm_status st = build_plan(doms, n, c[1], &p);
    if (st != LBM_OK) { d0->dev_free(p.views); d0->dev_free(p.items); d0->dev_free(p.bar); cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
    const int grid = resident_blocks(d0->desc.storage, p.i32, c[0]);
    cudaError_t e = launch_batch(d0->desc.storage, p.i32, p.views, p.items, p.n_items, p.chunk, 1,
                                 p.bar, c[0], grid, (unsigned)grid, d0->d_err,
                                 kBarrierLimitCycles, false, d0->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e0, d0->stream);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r)
      e = launch_batch(d0->desc.storage, p.i32, p.views, p.items, p.n_items, p.chunk, 1, p.bar,
                       c[0], grid, (unsigned)grid, d0->d_err, kBarrierLimitCycles, false,
                       d0->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, d0->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    d0->dev_free(p.views);
    d0->dev_free(p.items);
    d0->dev_free(p.bar);
    if (e != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return d0->cuda_fail(e, "batch tuning"); }
    if (ms < best) { best = ms; *chunk_out = c[1]; *threads_out = c[0]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return LBM_OK;
}

// Per-member sums (8 doubles: 6 sums, the member's error word, unused) to the 5 diagnostics of
// the lbm_reduce layout, and every member's error bits into the first domain's error word.
__global__ void k_batch_combine(const double* __restrict__ sums, int n, double* __restrict__ out5,
                                int* err0) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  const double* r = sums + 8 * (size_t)m;
  double* o = out5 + 5 * (size_t)m;
  o[0] = r[0] + r[1];
  o[1] = r[2];
  o[2] = r[3];
  o[3] = r[4];
  o[4] = r[5];
  const int e = (int)r[6];
  if (e) atomicOr(err0, e);
}

// ticket != nullptr: lbm_step_batch_reduce_async (the values go to out on the stream).
static lbm_status step_batch(lbm_domain* const* doms, int32_t n, int32_t steps, double* out,
                             int64_t* ticket = nullptr) {
  if (!doms || n <= 0 || !doms[0]) return LBM_ERR_INVALID_ARG;
  lbm_domain* d0 = doms[0];
  cudaSetDevice(d0->desc.device);
  const bool red = out != nullptr;
  if (steps < 0) return d0->fail(LBM_ERR_INVALID_ARG, "negative step count");
  if (red && steps < 1) return d0->fail(LBM_ERR_INVALID_ARG, "lbm_step_batch_reduce needs at least one step");
  for (int i = 0; i < n; ++i) {
    if (!doms[i]) return d0->fail(LBM_ERR_INVALID_ARG, "null domain in batch");
    for (int j = 0; j < i; ++j)
      if (doms[j] == doms[i]) return d0->fail(LBM_ERR_INVALID_ARG, "a domain appears twice");
    if (doms[i]->blocks.size() != 1) return d0->fail(LBM_ERR_UNSUPPORTED, "batched domains must be single-block");
    if (doms[i]->desc.storage != d0->desc.storage) return d0->fail(LBM_ERR_INVALID_ARG, "mixed storage in batch");
    if (doms[i]->desc.device != d0->desc.device) return d0->fail(LBM_ERR_INVALID_ARG, "mixed devices in batch");
    if (doms[i]->tape) return d0->fail(LBM_ERR_UNSUPPORTED, "batched stepping does not record tapes");
    if (doms[i]->walls) return d0->fail(LBM_ERR_UNSUPPORTED, "batched domains cannot have wall faces");
    if (*doms[i]->h_err & 1) return d0->fail(LBM_ERR_DIVERGED, "a domain of the batch has diverged");
  }
  if (steps == 0) return LBM_OK;
  cudaStream_t s = d0->stream;
  // order the batch after pending work of every domain, and every domain after the batch
  std::vector<cudaEvent_t> evs;
  for (int i = 1; i < n; ++i) {
    if (doms[i]->stream == s) continue;
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) break;
    cudaEventRecord(ev, doms[i]->stream);
    cudaStreamWaitEvent(s, ev, 0);
    evs.push_back(ev);
  }
  for (cudaEvent_t ev : evs) cudaEventDestroy(ev);

  BatchCache* cache = static_cast<BatchCache*>(d0->batch_plan);
  if (!cache) {
    cache = new (std::nothrow) BatchCache();
    if (!cache) return d0->fail(LBM_ERR_OOM, "out of host memory");
    d0->batch_plan = cache;
  }
  BatchPlan* p = nullptr;
  for (size_t k = 0; k < cache->plans.size() && !p; ++k) {
    BatchPlan* q = cache->plans[k];
    bool same = q->steps == steps && q->red == red && (int)q->serials.size() == n;
    for (int i = 0; i < n && same; ++i)
      same = q->serials[i] == doms[i]->serial && q->curs[i] == doms[i]->blocks[0].cur;
    if (same) {
      p = q;
      cache->plans.erase(cache->plans.begin() + k);
      cache->plans.push_back(p);
    }
  }
  if (!p) {
    if (!cache->chunk) {
      int chunk = 256, threads = 256;
      lbm_status st = tune_chunk(doms, n, &chunk, &threads);
      if (st != LBM_OK) return st;
      cache->chunk = chunk;
      cache->threads = threads;
    }
    while (cache->plans.size() >= kMaxBatchPlans) {
      free_plan(d0, cache->plans.front());
      cache->plans.erase(cache->plans.begin());
    }
    p = new (std::nothrow) BatchPlan();
    if (!p) return d0->fail(LBM_ERR_OOM, "out of host memory");
    // the fused diagnostics end every work item with a block-wide sum: their plans take work
    // items 4x the tuned size (measured on the 64-plume batch: 1.23 -> 1.12 ms per step;
    // the plain step does not change with the item size in that range)
    const int chunk = red ? 4 * cache->chunk : cache->chunk;
    lbm_status st = build_plan(doms, n, chunk, p);
    if (st == LBM_OK && red) {
      p->chunk = chunk;
      st = add_red_buffers(doms, n, p);
    }
    if (st != LBM_OK) { free_plan(d0, p); return st; }
    p->threads = cache->threads;
    cache->plans.push_back(p);
    p->steps = steps;
    p->grid = std::min(resident_blocks(d0->desc.storage, p->i32, p->threads, red), std::max(1, p->n_items));
    // capture: reset the barrier, then the cooperative persistent launch (and the fused
    // diagnostics' sums and read-back)
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = enqueue_batch(d0, p, steps, s);
      cudaError_t e2 = cudaStreamEndCapture(s, &g);
      if (e1 == cudaSuccess && e2 == cudaSuccess && g) {
        e = cudaGraphInstantiate(&p->exec, g, 0);
        p->captured = e == cudaSuccess;
        if (!p->captured) p->exec = nullptr;
      }
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();  // a capture the driver refused leaves the direct launch below
  }
  cudaError_t e = p->captured ? cudaGraphLaunch(p->exec, s) : enqueue_batch(d0, p, steps, s);
  if (e != cudaSuccess) return d0->cuda_fail(e, "batched launch");
  for (int i = 0; i < n; ++i) {
    Block& B = doms[i]->blocks[0];
    if (steps & 1) B.cur ^= 1;
    doms[i]->steps += steps;
  }
  // every domain's stream waits for the batch (each node reports divergence into its own
  // domain's error word; a barrier timeout is reported by the first domain)
  cudaEvent_t done;
  if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess) {
    cudaEventRecord(done, s);
    for (int i = 1; i < n; ++i)
      if (doms[i]->stream != s) cudaStreamWaitEvent(doms[i]->stream, done, 0);
    cudaEventDestroy(done);
  }
  if (!red) {
    d0->post_error_probe();
    return LBM_OK;
  }
  if (ticket) {
    const int slot = (int)(d0->results_issued % lbm_domain::kResultSlots);
    if (!d0->result_ev[slot] &&
        cudaEventCreateWithFlags(&d0->result_ev[slot], cudaEventDisableTiming) != cudaSuccess) {
      d0->result_ev[slot] = nullptr;
      return d0->fail(LBM_ERR_CUDA, "cudaEventCreate");
    }
    k_batch_combine<<<(n + 63) / 64, 64, 0, s>>>(p->out_dev, n, p->out5_dev, d0->d_err);
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out, p->out5_dev, (size_t)n * 5 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) {
      d0->post_error_probe();
      e = cudaEventRecord(d0->result_ev[slot], s);
    }
    if (e != cudaSuccess) return d0->cuda_fail(e, "batch diagnostics read-back");
    *ticket = ++d0->results_issued;
    return LBM_OK;
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return d0->cuda_fail(e, "cudaStreamSynchronize");
  lbm_status first = LBM_OK;
  for (int i = 0; i < n; ++i) {
    const double* r = p->out_host + 8 * (size_t)i;
    double* o = out + 5 * (size_t)i;
    o[0] = r[0] + r[1];
    o[1] = r[2];
    o[2] = r[3];
    o[3] = r[4];
    o[4] = r[5];
    *doms[i]->h_err = (int)r[6];
    const lbm_status st = doms[i]->error_status();
    if (st != LBM_OK && first == LBM_OK) first = st;
  }
  return first;
}

extern "C" lbm_status lbm_step_batch(lbm_domain* const* doms, int32_t n, int32_t steps) {
  return step_batch(doms, n, steps, nullptr);
}

extern "C" lbm_status lbm_step_batch_reduce(lbm_domain* const* doms, int32_t n, int32_t steps,
                                            double* out) {
  if (!out) return LBM_ERR_INVALID_ARG;
  return step_batch(doms, n, steps, out);
}

extern "C" lbm_status lbm_step_batch_reduce_async(lbm_domain* const* doms, int32_t n,
                                                  int32_t steps, double* out, int64_t* ticket) {
  if (!out || !ticket) return LBM_ERR_INVALID_ARG;
  return step_batch(doms, n, steps, out, ticket);
}

// Self-test of the bounded device barrier: a cooperative kernel waits for `extra` more CTAs
// than it launched, so every wait runs out after about `limit_ms`; the expected result is
// LBM_ERR_TIMEOUT with the context still usable.
__global__ void k_barrier_selftest(BarrierState* bs, unsigned int expected, int* err,
                                   long long limit) {
  grid_barrier(bs, expected, err, limit);
}

extern "C" lbm_status lbm_barrier_selftest(int32_t extra, double limit_ms, void* cuda_stream) {
  if (extra < 0 || !(limit_ms > 0.0) || limit_ms > 5000.0) return LBM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  BarrierState* bs = nullptr;
  int* err = nullptr;
  if (cudaMalloc(&bs, sizeof(BarrierState)) != cudaSuccess) return LBM_ERR_OOM;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) { cudaFree(bs); return LBM_ERR_OOM; }
  int dev = 0, clock_khz = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev);
  const long long limit = (long long)(limit_ms * (clock_khz > 0 ? clock_khz : 2000000));
  cudaMemsetAsync(bs, 0, sizeof(BarrierState), s);
  cudaMemsetAsync(err, 0, sizeof(int), s);
  const int grid = 4;
  const unsigned int expected = (unsigned)(grid + extra);
  void* args[] = {(void*)&bs, (void*)&expected, (void*)&err, (void*)&limit};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_barrier_selftest, dim3(grid),
                                              dim3(32), args, 0, s);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(bs);
  cudaFree(err);
  if (e != cudaSuccess) return LBM_ERR_CUDA;
  return (h & 8) ? LBM_ERR_TIMEOUT : LBM_OK;
}
