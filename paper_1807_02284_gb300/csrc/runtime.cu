// Host runtime behind the C-ABI of include/lbm.h: domain and block registry, buffer
// management through the caller's allocator, field I/O, the Algorithm 1 scheduler and the
// error word.  All GPU work goes to the domain's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"
#include "runtime.h"

using namespace lbm;

namespace {
std::string g_create_error;  // message of the last failed lbm_create_domain

lbm_status map_cuda(cudaError_t e) {
  return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}
}  // namespace

void lbm_set_global_error(const char* msg) { g_create_error = msg ? msg : ""; }

// ------------------------------------------------------------------------------ helpers

lbm_status Domain::fail(lbm_status st, const std::string& msg) {
  last_error = msg;
  return st;
}

lbm_status Domain::cuda_fail(cudaError_t e, const char* what) {
  last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return map_cuda(e);
}

void* Domain::dev_alloc(size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (desc.alloc.alloc) {
    p = desc.alloc.alloc(bytes, desc.alloc.ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) allocs.push_back({p, bytes});
  return p;
}

void Domain::dev_free(void* p) {
  if (!p) return;
  for (size_t i = 0; i < allocs.size(); ++i) {
    if (allocs[i].first == p) {
      if (desc.alloc.alloc) {
        if (desc.alloc.free) desc.alloc.free(p, allocs[i].second, desc.alloc.ctx);
      } else {
        cudaFree(p);
      }
      allocs.erase(allocs.begin() + i);
      return;
    }
  }
}

void* Domain::staging(size_t bytes) {
  if (bytes > staging_bytes) {
    if (staging_buf) {
      cudaStreamSynchronize(stream);
      dev_free(staging_buf);
    }
    staging_buf = dev_alloc(bytes);
    staging_bytes = staging_buf ? bytes : 0;
  }
  return staging_buf;
}

BlockView Domain::view(int b, int from, int to) const {
  const Block& B = blocks[b];
  BlockView v;
  v.d_in = B.lv[from].f;
  v.d_out = B.lv[to].f;
  v.u_in = B.lv[from].u;
  v.u_out = B.lv[to].u;
  v.c_in = B.lv[from].c;
  v.c_out = B.lv[to].c;
  v.flags = B.flags;
  v.nx = B.nx; v.ny = B.ny; v.nz = B.nz;
  for (int a = 0; a < 3; ++a) v.per[a] = (b == 0) ? desc.periodic[a] : 0;
  v.N = B.N;
  v.rp = B.rp;
  v.c_src = (float)desc.c_src;
  v.err = d_err;
  // wall faces are faces of the reference block; obstacle surfaces are walls in every block
  // that is not a far-field block
  v.walls = b == 0 ? walls : (B.far ? 0 : (walls & WALLS_OBSTACLES));
  return v;
}

lbm_status Domain::alloc_block_levels(Block& B, int levels) {
  B.lv.resize(levels);
  for (int l = 0; l < levels; ++l) {
    B.lv[l].f = dev_alloc(B.N * 27 * elt);
    B.lv[l].u = static_cast<float*>(dev_alloc(B.N * 3 * sizeof(float)));
    B.lv[l].c = static_cast<float*>(dev_alloc(B.N * sizeof(float)));
    if (!B.lv[l].f || !B.lv[l].u || !B.lv[l].c) return fail(LBM_ERR_OOM, "block allocation failed");
  }
  B.flags = static_cast<uint8_t*>(dev_alloc(B.N));
  if (!B.flags) return fail(LBM_ERR_OOM, "flag allocation failed");
  cudaError_t e = cudaMemsetAsync(B.flags, 0, B.N, stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  return LBM_OK;
}

RelaxParams Domain::relax_params(double nu_block) const {
  RelaxParams rp;
  rp.s_nu = (float)(1.0 / (3.0 * nu_block + 0.5));
  for (int g = 0; g < 4; ++g) rp.nuh3[g] = (float)(3.0 * desc.nu_hi[g]);
  rp.a = (float)desc.a;
  rp.b = (float)desc.b;
  rp.inv_gmax = (float)(1.0 / desc.g_max);
  rp.adaptive = desc.adaptive ? 1 : 0;
  rp.local = desc.grad_mode == LBM_GRAD_LOCAL ? 1 : 0;
  return rp;
}

// Rest equilibrium everywhere, u = 0, c = 0 for every level of a block.
lbm_status Domain::clear_block(int b) {
  Block& B = blocks[b];
  for (size_t l = 0; l < B.lv.size(); ++l) {
    cudaError_t e = cudaMemsetAsync(B.lv[l].f, 0, B.N * 27 * elt, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(B.lv[l].u, 0, B.N * 3 * sizeof(float), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(B.lv[l].c, 0, B.N * sizeof(float), stream);
    if (e != cudaSuccess) return cuda_fail(e, "clear block");
  }
  return LBM_OK;
}

lbm_status Domain::check_block(int32_t b) {
  if (b < 0 || b >= (int32_t)blocks.size()) return fail(LBM_ERR_INVALID_ARG, "bad block id");
  return LBM_OK;
}

// Reads the device error word into pinned memory (async) so later calls can see it.
void Domain::post_error_probe() {
  cudaMemcpyAsync(h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, stream);
}

lbm_status Domain::sync_and_check() {
  post_error_probe();
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  return error_status();
}

// Interprets the error word last copied to the host by post_error_probe.
lbm_status Domain::error_status() {
  if (*h_err & 1) return fail(LBM_ERR_DIVERGED, "non-finite or non-positive density detected");
  if (*h_err & 4) return fail(LBM_ERR_DIVERGED, "an inflow record outside the block or on an obstacle/ghost node was skipped");
  if (*h_err & 8) return fail(LBM_ERR_TIMEOUT, "a bounded device wait gave up");
  return LBM_OK;
}

lbm_status Domain::reset_error_word() {
  cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  *h_err = 0;
  return LBM_OK;
}

// Copies `bytes` of caller data to a device pointer usable by kernels on the stream.
// Host data goes through the staging buffer and the call waits for the copy so that the
// caller may reuse its buffer on return.
const void* Domain::device_source(const void* src, size_t bytes, int on_device,
                                  lbm_status* st) {
  *st = LBM_OK;
  if (on_device) return src;
  void* s = staging(bytes);
  if (!s) { *st = fail(LBM_ERR_OOM, "staging allocation failed"); return nullptr; }
  cudaError_t e = cudaMemcpyAsync(s, src, bytes, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) { *st = cuda_fail(e, "host to device copy"); return nullptr; }
  return s;
}

// -------------------------------------------------------------------------------- ABI

extern "C" {

int32_t lbm_abi_version(void) { return 5; }

lbm_status lbm_default_desc(lbm_domain_desc* d) {
  if (!d) return LBM_ERR_INVALID_ARG;
  std::memset(d, 0, sizeof(*d));
  d->storage = LBM_FP32;
  d->adaptive = 1;
  d->a = -4.0;
  d->b = 5.0;
  d->g_max = 0.1;
  d->nu_hi[0] = 0.005;
  d->nu_hi[1] = 0.007;
  d->nu_hi[2] = 0.009;
  d->nu_hi[3] = 0.01;
  d->c_src = 1.0;
  return LBM_OK;
}

lbm_status lbm_create_domain(const lbm_domain_desc* desc, lbm_domain** out) {
  if (!desc || !out) { g_create_error = "null argument"; return LBM_ERR_INVALID_ARG; }
  *out = nullptr;
  for (int a = 0; a < 3; ++a)
    if (desc->dims[a] < 1) { g_create_error = "dims must be >= 1"; return LBM_ERR_INVALID_ARG; }
  if (!(desc->nu > 0.0) || !std::isfinite(desc->nu)) {
    g_create_error = "nu must be positive"; return LBM_ERR_INVALID_ARG;
  }
  if (desc->storage != LBM_FP32 && desc->storage != LBM_FP16_SHIFTED) {
    g_create_error = "unknown storage"; return LBM_ERR_INVALID_ARG;
  }
  if (!(desc->g_max > 0.0)) { g_create_error = "g_max must be positive"; return LBM_ERR_INVALID_ARG; }
  if (desc->grad_mode != LBM_GRAD_LAGGED && desc->grad_mode != LBM_GRAD_LOCAL) {
    g_create_error = "unknown grad_mode"; return LBM_ERR_INVALID_ARG;
  }
  for (int g = 0; g < 4; ++g)
    if (!(desc->nu_hi[g] > 0.0)) { g_create_error = "nu_hi must be positive"; return LBM_ERR_INVALID_ARG; }
  if ((desc->alloc.alloc == nullptr) != (desc->alloc.free == nullptr)) {
    g_create_error = "allocator needs both alloc and free"; return LBM_ERR_INVALID_ARG;
  }
  const double N = (double)desc->dims[0] * desc->dims[1] * desc->dims[2];
  if (N > 4.0e9) { g_create_error = "block too large"; return LBM_ERR_INVALID_ARG; }
  if (desc->dims[2] > 65535) { g_create_error = "nz must be <= 65535"; return LBM_ERR_INVALID_ARG; }

  cudaError_t e = cudaSetDevice(desc->device);
  if (e != cudaSuccess) { g_create_error = cudaGetErrorString(e); return LBM_ERR_CUDA; }

  Domain* dom = new (std::nothrow) Domain();
  if (!dom) { g_create_error = "out of host memory"; return LBM_ERR_OOM; }
  static std::atomic<unsigned long long> next_serial{1};
  dom->desc = *desc;
  dom->serial = next_serial++;
  dom->elt = desc->storage == LBM_FP16_SHIFTED ? 2 : 4;
  if (desc->cuda_stream) {
    dom->stream = static_cast<cudaStream_t>(desc->cuda_stream);
  } else {
    e = cudaStreamCreateWithFlags(&dom->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { g_create_error = cudaGetErrorString(e); delete dom; return LBM_ERR_CUDA; }
    dom->own_stream = true;
  }
  e = cudaMallocHost(&dom->h_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&dom->h_red, 8 * sizeof(double));
  if (e != cudaSuccess) { g_create_error = cudaGetErrorString(e); lbm_destroy_domain(dom); return LBM_ERR_CUDA; }
  *dom->h_err = 0;
  dom->d_err = static_cast<int*>(dom->dev_alloc(64));
  dom->d_partials = static_cast<double*>(dom->dev_alloc(REDUCE_CTAS * 6 * sizeof(double)));
  // 8 doubles: reduction sums and other small results; 8 more: the combined diagnostics of
  // lbm_step_reduce_async
  dom->d_red = static_cast<double*>(dom->dev_alloc(16 * sizeof(double)));
  if (!dom->d_err || !dom->d_partials || !dom->d_red) {
    g_create_error = "allocation failed"; lbm_destroy_domain(dom); return LBM_ERR_OOM;
  }

  Block B;
  B.nx = desc->dims[0]; B.ny = desc->dims[1]; B.nz = desc->dims[2];
  B.N = (size_t)B.nx * B.ny * B.nz;
  B.origin[0] = B.origin[1] = B.origin[2] = 0.0;
  B.h = 1.0;
  B.nu = desc->nu;
  B.substeps = 1;
  B.rp = dom->relax_params(B.nu);
  dom->blocks.push_back(B);
  lbm_status st = dom->alloc_block_levels(dom->blocks[0], 2);
  if (st == LBM_OK) st = dom->clear_block(0);
  if (st == LBM_OK) st = dom->reset_error_word();
  if (st != LBM_OK) { g_create_error = dom->last_error; lbm_destroy_domain(dom); return st; }
  dom->pick_tiles(0);
  *out = dom;
  return LBM_OK;
}

lbm_status lbm_destroy_domain(lbm_domain* dom) {
  if (!dom) return LBM_OK;
  cudaSetDevice(dom->desc.device);
  if (dom->stream) cudaStreamSynchronize(dom->stream);
  dom->release_extras();
  while (!dom->allocs.empty()) dom->dev_free(dom->allocs.back().first);
  if (dom->h_err) cudaFreeHost(dom->h_err);
  if (dom->h_red) cudaFreeHost(dom->h_red);
  if (dom->own_stream && dom->stream) cudaStreamDestroy(dom->stream);
  delete dom;
  return LBM_OK;
}

lbm_status lbm_set_boundary(lbm_domain* dom, int32_t block_id, int32_t kind, const void* ptr,
                            size_t nbytes, int32_t on_device) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  lbm_status st = dom->check_block(block_id);
  if (st != LBM_OK) return st;
  Block& B = dom->blocks[block_id];
  if (kind == LBM_BC_FLAGS) {
    if (!ptr || nbytes < B.N) return dom->fail(LBM_ERR_INVALID_ARG, "flags need N bytes");
    const void* src = dom->device_source(ptr, B.N, on_device, &st);
    if (st != LBM_OK) return st;
    cudaError_t e = launch_merge_user_flags(B.flags, static_cast<const uint8_t*>(src), B.N,
                                            dom->stream);
    if (e == cudaSuccess) {
      int per[3] = {0, 0, 0};
      if (block_id == 0) for (int a = 0; a < 3; ++a) per[a] = dom->desc.periodic[a];
      if ((dom->walls & WALLS_OBSTACLES) && !B.far)   // the new obstacles' surfaces
        e = launch_obstacle_walls(B.flags, B.nx, B.ny, B.nz, per, 1, dom->stream);
      if (e == cudaSuccess) e = launch_near_solid(B.flags, B.nx, B.ny, B.nz, per, dom->stream);
    }
    // a block surrounded by a far-field block keeps its outer layer as scale boundary,
    // except where the new flags put obstacles or inflow nodes
    for (size_t i = 1; i < dom->blocks.size() && e == cudaSuccess; ++i)
      if (dom->blocks[i].far && dom->blocks[i].child == block_id)
        e = launch_outer_ghost(B.flags, B.nx, B.ny, B.nz, 1, dom->stream);
    if (e != cudaSuccess) return dom->cuda_fail(e, "set flags");
    dom->invalidate_graphs();
    return LBM_OK;
  }
  if (kind == LBM_BC_WALLS) {
    if (block_id != 0) return dom->fail(LBM_ERR_INVALID_ARG, "walls are faces of block 0");
    if (!ptr || nbytes < 6) return dom->fail(LBM_ERR_INVALID_ARG, "walls need 6 bytes");
    if (on_device) return dom->fail(LBM_ERR_INVALID_ARG, "the wall mask is host memory");
    const uint8_t* m = static_cast<const uint8_t*>(ptr);
    int walls = 0;
    for (int f = 0; f < 6; ++f)
      if (m[f]) {
        if (dom->desc.periodic[f / 2]) return dom->fail(LBM_ERR_INVALID_ARG, "a wall on a periodic axis");
        walls |= 1 << f;
      }
    if (nbytes >= 7 && m[6]) walls |= WALLS_OBSTACLES;
    for (size_t i = 1; i < dom->blocks.size(); ++i)
      if (dom->blocks[i].far && (walls & ~WALLS_OBSTACLES))
        return dom->fail(LBM_ERR_UNSUPPORTED, "wall faces and far-field blocks exclude each other");
    int per[3];
    for (int a = 0; a < 3; ++a) per[a] = dom->desc.periodic[a];
    cudaError_t e = launch_mark_walls(B.flags, B.nx, B.ny, B.nz, walls, dom->stream);
    if (e == cudaSuccess && ((walls | dom->walls) & WALLS_OBSTACLES)) {
      e = launch_obstacle_walls(B.flags, B.nx, B.ny, B.nz, per, (walls & WALLS_OBSTACLES) ? 1 : 0,
                                dom->stream);
      if (e == cudaSuccess) e = launch_near_solid(B.flags, B.nx, B.ny, B.nz, per, dom->stream);
    }
    // obstacle surfaces of the refined blocks (their faces are scale boundaries, not walls)
    const int zero[3] = {0, 0, 0};
    for (size_t i = 1; i < dom->blocks.size() && e == cudaSuccess; ++i) {
      Block& R = dom->blocks[i];
      if (!((walls | dom->walls) & WALLS_OBSTACLES)) break;
      if (R.far) continue;             // far-field blocks keep halfway bounce-back
      e = launch_obstacle_walls(R.flags, R.nx, R.ny, R.nz, zero, (walls & WALLS_OBSTACLES) ? 1 : 0,
                                dom->stream);
      if (e == cudaSuccess) e = launch_near_solid(R.flags, R.nx, R.ny, R.nz, zero, dom->stream);
    }
    if (e != cudaSuccess) return dom->cuda_fail(e, "wall flags");
    dom->walls = walls;
    dom->invalidate_graphs();
    return LBM_OK;
  }
  if (kind == LBM_BC_INFLOW) {
    if (nbytes % sizeof(lbm_inflow_record) != 0)
      return dom->fail(LBM_ERR_INVALID_ARG, "nbytes must be a multiple of the record size");
    const int n = (int)(nbytes / sizeof(lbm_inflow_record));
    if (n == 0) return LBM_OK;
    if (!ptr) return dom->fail(LBM_ERR_INVALID_ARG, "null records");
    const void* src = on_device ? ptr : dom->upload_small(ptr, nbytes, &st);
    if (st != LBM_OK) return st;
    std::vector<float*> lv;
    for (auto& L : B.lv) lv.push_back(L.u);
    // records never touch obstacle voxels, so the derived near-obstacle bits stay valid
    cudaError_t e = launch_inflow_records(src, n, B.flags, lv.data(), (int)lv.size(), B.nx,
                                          B.ny, B.nz, B.N, dom->d_err, dom->stream);
    if (e != cudaSuccess) return dom->cuda_fail(e, "inflow records");
    return LBM_OK;
  }
  return dom->fail(LBM_ERR_INVALID_ARG, "unknown boundary kind");
}

lbm_status lbm_init_macro(lbm_domain* dom, int32_t block_id, const float* rho, const float* u,
                          const float* c, int32_t on_device) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  lbm_status st = dom->check_block(block_id);
  if (st != LBM_OK) return st;
  if (!u) return dom->fail(LBM_ERR_INVALID_ARG, "u is required");
  Block& B = dom->blocks[block_id];
  const size_t N = B.N;
  // gather the three inputs into one device area
  const float* d_rho = nullptr; const float* d_u = nullptr; const float* d_c = nullptr;
  if (on_device) {
    d_rho = rho; d_u = u; d_c = c;
  } else {
    float* s = static_cast<float*>(dom->staging(N * 5 * sizeof(float)));
    if (!s) return dom->fail(LBM_ERR_OOM, "staging allocation failed");
    cudaError_t e = cudaMemcpyAsync(s, u, 3 * N * sizeof(float), cudaMemcpyHostToDevice, dom->stream);
    d_u = s;
    if (e == cudaSuccess && rho) {
      e = cudaMemcpyAsync(s + 3 * N, rho, N * sizeof(float), cudaMemcpyHostToDevice, dom->stream);
      d_rho = s + 3 * N;
    }
    if (e == cudaSuccess && c) {
      e = cudaMemcpyAsync(s + 4 * N, c, N * sizeof(float), cudaMemcpyHostToDevice, dom->stream);
      d_c = s + 4 * N;
    }
    if (e != cudaSuccess) return dom->cuda_fail(e, "host to device copy");
  }
  BlockView v = dom->view(block_id, B.cur, B.cur);
  cudaError_t e = launch_init(v, dom->desc.storage, d_rho, d_u, d_c, dom->stream);
  if (e != cudaSuccess) return dom->cuda_fail(e, "init kernel");
  if (!on_device) {
    e = cudaStreamSynchronize(dom->stream);
    if (e != cudaSuccess) return dom->cuda_fail(e, "cudaStreamSynchronize");
  }
  dom->on_state_reset(block_id);
  return dom->reset_error_word();
}

lbm_status lbm_step(lbm_domain* dom, int32_t n) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  if (n < 0) return dom->fail(LBM_ERR_INVALID_ARG, "negative step count");
  if (*dom->h_err & 1) return dom->fail(LBM_ERR_DIVERGED, "divergence recorded by an earlier step");
  lbm_status st = dom->advance(n);
  if (st != LBM_OK) return st;
  dom->post_error_probe();
  return LBM_OK;
}

lbm_status lbm_sync(lbm_domain* dom) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  return dom->sync_and_check();
}

lbm_status lbm_read_field(lbm_domain* dom, int32_t block_id, int32_t field, int32_t dtype,
                          void* dst, size_t dst_bytes, int32_t on_device) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  lbm_status st = dom->check_block(block_id);
  if (st != LBM_OK) return st;
  if (!dst) return dom->fail(LBM_ERR_INVALID_ARG, "null destination");
  Block& B = dom->blocks[block_id];
  const size_t N = B.N;
  const Level& L = B.lv[B.cur];
  size_t count, esz;
  if (field == LBM_FIELD_FLAGS) {
    if (dtype != LBM_U8) return dom->fail(LBM_ERR_INVALID_ARG, "flags are LBM_U8");
    count = N; esz = 1;
  } else {
    if (dtype != LBM_F32 && dtype != LBM_F64) return dom->fail(LBM_ERR_INVALID_ARG, "bad dtype");
    esz = dtype == LBM_F64 ? 8 : 4;
    count = field == LBM_FIELD_F ? 27 * N : field == LBM_FIELD_U ? 3 * N
          : (field == LBM_FIELD_SCALAR || field == LBM_FIELD_RHO) ? N : 0;
    if (!count) return dom->fail(LBM_ERR_INVALID_ARG, "unknown field");
  }
  const size_t bytes = count * esz;
  if (dst_bytes < bytes) return dom->fail(LBM_ERR_INVALID_ARG, "destination too small");
  void* out = on_device ? dst : dom->staging(bytes + (field == LBM_FIELD_RHO ? N * 4 : 0));
  if (!out) return dom->fail(LBM_ERR_OOM, "staging allocation failed");
  cudaError_t e = cudaSuccess;
  const int f64 = dtype == LBM_F64;
  switch (field) {
    case LBM_FIELD_F: e = launch_read_f(L.f, dom->desc.storage, N, out, f64, dom->stream); break;
    case LBM_FIELD_U: e = launch_convert(L.u, 0, out, f64, 3 * N, dom->stream); break;
    case LBM_FIELD_SCALAR: e = launch_convert(L.c, 0, out, f64, N, dom->stream); break;
    case LBM_FIELD_RHO: {
      float* tmp = static_cast<float*>(on_device ? dom->staging(N * 4) : (void*)((char*)out + bytes));
      if (!tmp) return dom->fail(LBM_ERR_OOM, "staging allocation failed");
      e = launch_read_rho(L.f, dom->desc.storage, N, tmp, dom->stream);
      if (e == cudaSuccess) e = launch_convert(tmp, 0, out, f64, N, dom->stream);
      break;
    }
    case LBM_FIELD_FLAGS: e = cudaMemcpyAsync(out, B.flags, N, cudaMemcpyDeviceToDevice, dom->stream); break;
  }
  if (e != cudaSuccess) return dom->cuda_fail(e, "read field");
  if (!on_device) {
    e = cudaMemcpyAsync(dst, out, bytes, cudaMemcpyDeviceToHost, dom->stream);
    if (e != cudaSuccess) return dom->cuda_fail(e, "device to host copy");
  }
  return dom->sync_and_check();
}

lbm_status lbm_read_macro(lbm_domain* dom, int32_t block_id, int32_t what, void* dst,
                          size_t dst_bytes, int32_t on_device) {
  const int32_t field = what == LBM_MACRO_RHO ? LBM_FIELD_RHO
                      : what == LBM_MACRO_U ? LBM_FIELD_U
                      : what == LBM_MACRO_SCALAR ? LBM_FIELD_SCALAR : -1;
  if (!dom) return LBM_ERR_INVALID_ARG;
  if (field < 0) return dom->fail(LBM_ERR_INVALID_ARG, "unknown macro selector");
  return lbm_read_field(dom, block_id, field, LBM_F32, dst, dst_bytes, on_device);
}

lbm_status lbm_write_field(lbm_domain* dom, int32_t block_id, int32_t field, int32_t dtype,
                           const void* src, size_t src_bytes, int32_t on_device) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  lbm_status st = dom->check_block(block_id);
  if (st != LBM_OK) return st;
  if (!src) return dom->fail(LBM_ERR_INVALID_ARG, "null source");
  if (dtype != LBM_F32 && dtype != LBM_F64) return dom->fail(LBM_ERR_INVALID_ARG, "bad dtype");
  Block& B = dom->blocks[block_id];
  const size_t N = B.N;
  const size_t count = field == LBM_FIELD_F ? 27 * N : field == LBM_FIELD_U ? 3 * N
                     : field == LBM_FIELD_SCALAR ? N : 0;
  if (!count) return dom->fail(LBM_ERR_INVALID_ARG, "field is not writable");
  const int f64 = dtype == LBM_F64;
  const size_t bytes = count * (f64 ? 8 : 4);
  if (src_bytes < bytes) return dom->fail(LBM_ERR_INVALID_ARG, "source too small");
  const void* s = dom->device_source(src, bytes, on_device, &st);
  if (st != LBM_OK) return st;
  const Level& L = B.lv[B.cur];
  cudaError_t e;
  if (field == LBM_FIELD_F) e = launch_write_f(L.f, dom->desc.storage, N, s, f64, dom->stream);
  else if (field == LBM_FIELD_U) e = launch_convert(s, f64, L.u, 0, 3 * N, dom->stream);
  else e = launch_convert(s, f64, L.c, 0, N, dom->stream);
  if (e != cudaSuccess) return dom->cuda_fail(e, "write field");
  if (!on_device) {
    e = cudaStreamSynchronize(dom->stream);
    if (e != cudaSuccess) return dom->cuda_fail(e, "cudaStreamSynchronize");
  }
  dom->on_state_reset(block_id);
  return dom->reset_error_word();
}

lbm_status lbm_reduce(lbm_domain* dom, int32_t block_id, double out[5]) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  lbm_status st = dom->check_block(block_id);
  if (st != LBM_OK) return st;
  if (!out) return dom->fail(LBM_ERR_INVALID_ARG, "null output");
  Block& B = dom->blocks[block_id];
  cudaError_t e = launch_reduce(B.lv[B.cur].f, dom->desc.storage, B.flags, B.N, dom->d_partials,
                                dom->d_red, dom->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dom->h_red, dom->d_red, 6 * sizeof(double), cudaMemcpyDeviceToHost, dom->stream);
  if (e != cudaSuccess) return dom->cuda_fail(e, "reduce");
  st = dom->sync_and_check();
  const double* r = dom->h_red;
  out[0] = r[0] + r[1];
  out[1] = r[2];
  out[2] = r[3];
  out[3] = r[4];
  out[4] = r[5];
  return st;
}

// lbm_reduce_batch for members that share device, stream and storage: one launch over a
// list of node chunks of all members, one read-back (sums and error words), one wait.
static lbm_status reduce_batch_joint(lbm_domain* const* doms, int n, int block_id, double* out) {
  lbm_domain* d0 = doms[0];
  constexpr size_t kChunk = 8192;
  std::vector<RedMember> mem(n);
  std::vector<RedItem> items;
  for (int i = 0; i < n; ++i) {
    Block& B = doms[i]->blocks[block_id];
    mem[i] = RedMember{B.lv[B.cur].f, B.flags, doms[i]->d_err, B.N, (int)items.size(), 0};
    for (size_t s = 0; s < B.N; s += kChunk)
      items.push_back(RedItem{i, 0, s, std::min(kChunk, B.N - s)});
    mem[i].n_items = (int)items.size() - mem[i].first_item;
  }
  const size_t mb = mem.size() * sizeof(RedMember), ib = items.size() * sizeof(RedItem);
  const size_t rb = items.size() * 8 * sizeof(double), ob = (size_t)n * 8 * sizeof(double);
  if (d0->rb_host_bytes < mb + ib + ob) {
    if (d0->rb_host) cudaFreeHost(d0->rb_host);
    d0->rb_host = nullptr;
    d0->rb_host_bytes = 0;
    if (cudaMallocHost(&d0->rb_host, mb + ib + ob) != cudaSuccess) {
      d0->rb_host = nullptr;
      return d0->fail(LBM_ERR_OOM, "batch reduction staging");
    }
    d0->rb_host_bytes = mb + ib + ob;
  }
  if (d0->rb_dev_bytes < mb + ib + rb + ob) {
    if (d0->rb_dev) d0->dev_free(d0->rb_dev);
    d0->rb_dev_bytes = 0;
    d0->rb_dev = d0->dev_alloc(mb + ib + rb + ob);
    if (!d0->rb_dev) return d0->fail(LBM_ERR_OOM, "batch reduction scratch");
    d0->rb_dev_bytes = mb + ib + rb + ob;
  }
  char* h = static_cast<char*>(d0->rb_host);
  char* g = static_cast<char*>(d0->rb_dev);
  std::memcpy(h, mem.data(), mb);
  std::memcpy(h + mb, items.data(), ib);
  const RedMember* g_mem = reinterpret_cast<const RedMember*>(g);
  const RedItem* g_items = reinterpret_cast<const RedItem*>(g + mb);
  double* g_rec = reinterpret_cast<double*>(g + mb + ib);
  double* g_out = reinterpret_cast<double*>(g + mb + ib + rb);
  double* h_out = reinterpret_cast<double*>(h + mb + ib);
  cudaError_t e = cudaMemcpyAsync(g, h, mb + ib, cudaMemcpyHostToDevice, d0->stream);
  if (e == cudaSuccess)
    e = launch_reduce_items(d0->desc.storage, g_items, (int)items.size(), g_mem, n, g_rec, g_out,
                            d0->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_out, g_out, ob, cudaMemcpyDeviceToHost, d0->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d0->stream);
  if (e != cudaSuccess) return d0->cuda_fail(e, "batch reduction");
  lbm_status first = LBM_OK;
  for (int i = 0; i < n; ++i) {
    const double* r = h_out + 8 * (size_t)i;
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

lbm_status lbm_reduce_batch(lbm_domain* const* doms, int32_t n, int32_t block_id, double* out) {
  if (!doms || n <= 0 || !out) return LBM_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    if (!doms[i]) return LBM_ERR_INVALID_ARG;
    cudaSetDevice(doms[i]->desc.device);
    const lbm_status st = doms[i]->check_block(block_id);
    if (st != LBM_OK) return st;
  }
  bool joint = n >= 2;
  for (int i = 1; i < n && joint; ++i)
    joint = doms[i]->desc.device == doms[0]->desc.device && doms[i]->stream == doms[0]->stream &&
            doms[i]->desc.storage == doms[0]->desc.storage;
  if (joint) {
    cudaSetDevice(doms[0]->desc.device);
    return reduce_batch_joint(doms, n, block_id, out);
  }
  // queue every reduction and its read-back before waiting on any stream
  for (int i = 0; i < n; ++i) {
    lbm_domain* d = doms[i];
    cudaSetDevice(d->desc.device);
    Block& B = d->blocks[block_id];
    cudaError_t e = launch_reduce(B.lv[B.cur].f, d->desc.storage, B.flags, B.N, d->d_partials,
                                  d->d_red, d->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d->h_red, d->d_red, 6 * sizeof(double), cudaMemcpyDeviceToHost, d->stream);
    if (e != cudaSuccess) return d->cuda_fail(e, "reduce");
    d->post_error_probe();
  }
  lbm_status first = LBM_OK;
  for (int i = 0; i < n; ++i) {
    lbm_domain* d = doms[i];
    cudaSetDevice(d->desc.device);
    const cudaError_t e = cudaStreamSynchronize(d->stream);
    const lbm_status st = e != cudaSuccess ? d->cuda_fail(e, "cudaStreamSynchronize")
                                           : d->error_status();
    if (st != LBM_OK && first == LBM_OK) first = st;
    const double* r = d->h_red;
    double* o = out + 5 * (size_t)i;
    o[0] = r[0] + r[1];
    o[1] = r[2];
    o[2] = r[3];
    o[3] = r[4];
    o[4] = r[5];
  }
  return first;
}

lbm_status lbm_get_block_info(const lbm_domain* dom, int32_t block_id, lbm_block_info* info) {
  if (!dom || !info) return LBM_ERR_INVALID_ARG;
  if (block_id < 0 || block_id >= (int32_t)dom->blocks.size()) return LBM_ERR_INVALID_ARG;
  const Block& B = dom->blocks[block_id];
  info->dims[0] = B.nx; info->dims[1] = B.ny; info->dims[2] = B.nz;
  for (int a = 0; a < 3; ++a) info->origin[a] = B.origin[a];
  info->h = B.h;
  info->nu = B.nu;
  info->substeps = B.substeps;
  info->steps = dom->steps;
  info->tile[0] = B.bx;
  info->tile[1] = B.by;
  const bool pair = step_is_pair(B.minb) && B.nx % 2 == 0;
  info->ctas_per_sm = pair ? B.minb - STEP_PAIR : step_scalar_bound(B.minb);
  info->parent = (block_id == 0 || B.far) ? -1 : B.parent;
  info->nodes_per_thread = pair ? 2 : 1;
  return LBM_OK;
}

const char* lbm_last_error(const lbm_domain* dom) {
  if (!dom) return g_create_error.c_str();
  return dom->last_error.c_str();
}

}  // extern "C"

// LBM_BC_INFLOW records of block 0 of several domains: members sharing device and stream get
// one staged upload and one launch; otherwise each member takes lbm_set_boundary.
lbm_status lbm_set_inflow_batch(lbm_domain* const* doms, int32_t n,
                                const lbm_inflow_record* const* recs, const int32_t* counts) {
  if (!doms || n <= 0 || !recs || !counts) return LBM_ERR_INVALID_ARG;
  size_t total = 0;
  for (int i = 0; i < n; ++i) {
    if (!doms[i] || counts[i] < 0 || (counts[i] > 0 && !recs[i])) return LBM_ERR_INVALID_ARG;
    total += (size_t)counts[i];
  }
  if (total > (size_t)INT32_MAX) return doms[0]->fail(LBM_ERR_INVALID_ARG, "too many records");
  bool joint = n >= 2;
  for (int i = 1; i < n && joint; ++i)
    joint = doms[i]->desc.device == doms[0]->desc.device && doms[i]->stream == doms[0]->stream;
  if (!joint) {
    for (int i = 0; i < n; ++i) {
      const lbm_status st = lbm_set_boundary(doms[i], 0, LBM_BC_INFLOW, recs[i],
                                             (size_t)counts[i] * sizeof(lbm_inflow_record), 0);
      if (st != LBM_OK) return st;
    }
    return LBM_OK;
  }
  lbm_domain* d0 = doms[0];
  cudaSetDevice(d0->desc.device);
  if (total == 0) return LBM_OK;
  const size_t rb = total * sizeof(lbm_inflow_record), ob = total * sizeof(int);
  const size_t mb = (size_t)n * sizeof(InflowMember);
  const size_t bytes = mb + rb + ob;
  if (!d0->ib_done && cudaEventCreateWithFlags(&d0->ib_done, cudaEventDisableTiming) != cudaSuccess) {
    d0->ib_done = nullptr;
    return d0->fail(LBM_ERR_CUDA, "cudaEventCreate");
  }
  // the previous upload from the staging buffer must have left it
  cudaError_t e = cudaEventSynchronize(d0->ib_done);
  if (e != cudaSuccess) return d0->cuda_fail(e, "cudaEventSynchronize");
  if (d0->ib_host_bytes < bytes) {
    if (d0->ib_host) cudaFreeHost(d0->ib_host);
    d0->ib_host = nullptr;
    d0->ib_host_bytes = 0;
    if (cudaMallocHost(&d0->ib_host, bytes) != cudaSuccess) {
      d0->ib_host = nullptr;
      return d0->fail(LBM_ERR_OOM, "inflow batch staging");
    }
    d0->ib_host_bytes = bytes;
  }
  if (d0->ib_dev_bytes < bytes) {
    if (d0->ib_dev) d0->dev_free(d0->ib_dev);
    d0->ib_dev_bytes = 0;
    d0->ib_dev = d0->dev_alloc(bytes);
    if (!d0->ib_dev) return d0->fail(LBM_ERR_OOM, "inflow batch buffer");
    d0->ib_dev_bytes = bytes;
  }
  char* h = static_cast<char*>(d0->ib_host);
  InflowMember* hm = reinterpret_cast<InflowMember*>(h);
  char* hr = h + mb;
  int* ho = reinterpret_cast<int*>(h + mb + rb);
  size_t at = 0;
  for (int i = 0; i < n; ++i) {
    Block& B = doms[i]->blocks[0];
    InflowMember m{};
    m.flags = B.flags;
    for (int l = 0; l < 3; ++l) m.u[l] = l < (int)B.lv.size() ? B.lv[l].u : nullptr;
    m.nx = B.nx; m.ny = B.ny; m.nz = B.nz;
    m.N = B.N;
    m.err = doms[i]->d_err;
    hm[i] = m;
    std::memcpy(hr + at * sizeof(lbm_inflow_record), recs[i], (size_t)counts[i] * sizeof(lbm_inflow_record));
    for (int k = 0; k < counts[i]; ++k) ho[at + k] = i;
    at += (size_t)counts[i];
  }
  char* g = static_cast<char*>(d0->ib_dev);
  e = cudaMemcpyAsync(g, h, bytes, cudaMemcpyHostToDevice, d0->stream);
  if (e == cudaSuccess) e = cudaEventRecord(d0->ib_done, d0->stream);
  if (e == cudaSuccess)
    e = launch_inflow_records_multi(g + mb, (int)total, reinterpret_cast<const int*>(g + mb + rb),
                                    reinterpret_cast<const InflowMember*>(g), d0->stream);
  if (e != cudaSuccess) return d0->cuda_fail(e, "inflow batch");
  return LBM_OK;
}
