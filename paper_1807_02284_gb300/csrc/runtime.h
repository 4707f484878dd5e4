// Host-side domain object behind the opaque lbm_domain handle.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace lbm {

struct Level {             // one time level of a block
  void* f = nullptr;       // 27 planes of shifted populations (cube order), FP32 or FP16
  float* u = nullptr;      // 3 planes, velocity stored by the step that produced this level
  float* c = nullptr;      // passive scalar
};

struct MapTable {
  MapEntry* d = nullptr;   // device array
  int n = 0;
  int src = 0, dst = 0;    // block ids
  float khat = 1.0f;       // K_hat factor of moments 4..8 for src -> dst
};

// Planes of a ghost-layer interpolant buffer: 27 shifted populations, the scalar, the status.
constexpr int GHOST_PLANES = 29;

struct Block {
  MapTable prior;                 // ghost layer <- parent (refined blocks)
  // trilinear interpolants of the ghost layer from the parent at t_n (0) and t_n + dt_0 (1),
  // GHOST_PLANES x prior.n floats each (refined blocks)
  float* gs[2] = {nullptr, nullptr};
  std::vector<MapTable> post;     // every coarser block <- this block's interior
  int nx = 0, ny = 0, nz = 0;
  size_t N = 0;
  double origin[3] = {0, 0, 0};
  double h = 1.0;          // dx_s / dx_0
  double nu = 0.0;         // viscosity in this block's lattice units
  int substeps = 1;        // l = sub-steps per reference step
  bool integer_ratio = true;
  std::vector<Level> lv;   // 2 levels for s0, 3 for refined blocks
  uint8_t* flags = nullptr;
  int cur = 0;             // level holding the current state
  int saved = 0;           // level holding the state at t_n (refined blocks)
  int parent = 0;          // nearest coarser block containing this one (prior-mapping source)
  RelaxParams rp;
  int bx = 128, by = 2;    // tile of the collide-stream launch
  int minb = 3;            // register bound of the collide-stream launch (CTAs per SM)
  bool tuned = false;      // tile shape chosen by autotune_tiles
  // far-field block (h > 1, Sec. 4.2.4-4.2.5): it surrounds block `child` (s0 or the previous
  // far block), takes its nodes inside the child's interior from the child (far_in) and
  // gives the child its outer layer (far_out)
  bool far = false;
  int child = -1;
  MapTable far_in, far_out;
};

struct TapeState;          // adjoint tape (adjoint.cu)
struct GraphCache;         // captured step graphs (scheduler.cu)

}  // namespace lbm

struct lbm_domain {
  lbm_domain_desc desc{};
  unsigned long long serial = 0;        // unique per created domain (keys cached batch plans)
  int walls = 0;                        // no-slip wall faces of block 0 (LBM_BC_WALLS bits)
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t elt = 4;
  std::vector<lbm::Block> blocks;
  std::vector<std::pair<void*, size_t>> allocs;
  int* d_err = nullptr;
  int* h_err = nullptr;                 // pinned
  double* d_partials = nullptr;         // reduction scratch: REDUCE_CTAS * 6 doubles
  double* d_step_partials = nullptr;    // per-CTA partials of lbm_step_reduce (6 per CTA)
  size_t step_partials_n = 0;           // CTAs d_step_partials has room for
  double* d_red = nullptr;
  double* h_red = nullptr;              // pinned
  void* staging_buf = nullptr;
  size_t staging_bytes = 0;
  void* small_host = nullptr;           // pinned bounce buffer for small uploads
  void* small_dev = nullptr;
  size_t small_bytes = 0;
  cudaEvent_t small_done = nullptr;
  // lbm_step_reduce_async: one event per ticket slot (ticket t uses slot (t - 1) % 16; a
  // later ticket's event in the same slot completes after it, so waiting on it is safe)
  static constexpr int kResultSlots = 16;
  cudaEvent_t result_ev[kResultSlots] = {};
  long long results_issued = 0;
  std::string last_error;
  long long steps = 0;
  lbm::TapeState* tape = nullptr;
  lbm::GraphCache* graphs = nullptr;
  // launch shapes already timed, by block size class (x extent: < 64, < 128, < 256, more;
  // nodes: < 2^20, < 2^23, more): a block of the same class (a rebuilt dynamic scale)
  // reuses the choice
  struct TunedShape { int nx_class, n_class, bx, by, minb; };
  std::vector<TunedShape> tuned_shapes;
  void* batch_plan = nullptr;           // cached plans of lbm_step_batch (batch.cu)
  // scratch of lbm_reduce_batch when this domain heads the list (device and pinned host)
  void* rb_dev = nullptr;
  size_t rb_dev_bytes = 0;
  void* rb_host = nullptr;
  size_t rb_host_bytes = 0;
  // staging of lbm_set_inflow_batch when this domain heads the list; ib_done marks the end
  // of the previous upload from ib_host
  void* ib_dev = nullptr;
  size_t ib_dev_bytes = 0;
  void* ib_host = nullptr;
  size_t ib_host_bytes = 0;
  cudaEvent_t ib_done = nullptr;
  cudaStream_t aux_stream = nullptr;    // second stream for concurrent mapping launches
  std::vector<cudaEvent_t> events;      // fork / join events (timing disabled)

  std::vector<cudaStream_t> post_streams;  // one per post-mapping target block

  // a reference step run phase by phase (lbm_step_phase): each block's level at the step
  // start, and per block 0 (nothing yet), 1 (sub-cycle done), 2 (post-mapping done)
  bool phase_open = false;
  bool phase_ref_done = false;
  std::vector<int> phase_saved;
  std::vector<char> phase_done;

  lbm_status aux(cudaStream_t* out);    // the auxiliary stream, created on first use
  cudaEvent_t event(int i);             // fork / join event i, created on first use
  cudaStream_t post_stream(int k);      // stream of post-mappings into block k

  lbm_status fail(lbm_status st, const std::string& msg);
  lbm_status cuda_fail(cudaError_t e, const char* what);
  void* dev_alloc(size_t bytes);
  void dev_free(void* p);
  void* staging(size_t bytes);
  const void* device_source(const void* src, size_t bytes, int on_device, lbm_status* st);
  const void* upload_small(const void* src, size_t bytes, lbm_status* st);
  lbm::BlockView view(int b, int from, int to) const;
  lbm_status alloc_block_levels(lbm::Block& B, int levels);
  lbm::RelaxParams relax_params(double nu_block) const;
  lbm_status clear_block(int b);
  lbm_status check_block(int32_t b);
  void post_error_probe();
  lbm_status sync_and_check();
  lbm_status error_status();
  lbm_status reset_error_word();
  void pick_tiles(int b);
  lbm_status autotune_tiles(int b);
  void invalidate_graphs();
  void release_extras();
  void on_state_reset(int b);
  lbm_status advance(int n);            // Algorithm 1, n reference steps
  lbm_status advance_direct(int n);     // same, launched without graph capture
  lbm_status advance_single(int m);     // m steps from one-step graphs (several blocks)
};

using Domain = lbm_domain;
