/* C-ABI of the GB300 continuous-scale central-moment lattice Boltzmann library.
 *
 * Method: arXiv 1807.02284 (Li, Bai, Liu, "Continuous-Scale Kinetic Fluid Simulation").
 *   - D3Q27 lattice Boltzmann equation, stream + collide            Sec. 1 (LBE), Appendix
 *   - non-orthogonal central-moment collision Omega = -T S (m-m^eq)  Sec. 3.1, Appendix
 *   - adaptive high-order relaxation                                 Sec. 4.1
 *   - continuous-scale blocks: K-hat rescale, prior-/post-mapping,
 *     trilinear + temporal interpolation, Algorithm 1 schedule       Sec. 3.2, 4.2, Alg. 1
 *   - initial equilibrium, inflow, open (Neumann) boundaries         Sec. 6.1
 *
 * Conventions for every entry point
 *   - Returns lbm_status; never throws, aborts or traps.  On failure the domain's
 *     lbm_last_error() string says why.
 *   - Pointers flagged by `on_device` != 0 are device pointers on the domain's device;
 *     otherwise host pointers (pinned or pageable).  Caller memory is never retained: the
 *     library copies what it needs before returning and never frees caller memory.
 *   - Library buffers come from desc.alloc (e.g. PyTorch's caching allocator) or, when
 *     desc.alloc.alloc is NULL, from cudaMalloc.  They are released by lbm_destroy_domain.
 *   - All GPU work is ordered on desc.cuda_stream (NULL: the library creates its own).
 *     Calls that return data to the host synchronise that stream; lbm_step only enqueues.
 *   - Device-side failures (non-finite density, bad inflow record) are recorded in a device
 *     error word and reported by the next synchronising call as LBM_ERR_DIVERGED.
 *   - Calls on one domain are not thread-safe; different domains are independent.
 *   - Array layout: node (x, y, z) of a block with dims (nx, ny, nz) has linear index
 *     (z*ny + y)*nx + x.  Vector fields are 3 planes (x, y, z components) of N = nx*ny*nz;
 *     populations are 27 planes in the order of the paper's Appendix velocity list (with
 *     index 13 read as (1,0,-1), the printed list duplicates (1,0,1)).
 *   - Units: lattice units of the block (dx = dt = 1 on the block's own grid).  Velocity
 *     is the same number on every scale because dt = dx on each scale (Sec. 4.2.4).
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_domain lbm_domain; /* opaque; owned by the library */

typedef enum {
  LBM_OK = 0,
  LBM_ERR_INVALID_ARG = 1, /* bad pointer, size, block id, enum value or geometry */
  LBM_ERR_OOM = 2,         /* allocation failed */
  LBM_ERR_CUDA = 3,        /* a CUDA runtime call failed (message in lbm_last_error) */
  LBM_ERR_DIVERGED = 4,    /* a node reached a non-finite or non-positive density */
  LBM_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
  LBM_ERR_UNSUPPORTED = 6, /* valid request outside what this build implements */
  LBM_ERR_STATE = 7        /* call not valid in the current state (e.g. no tape) */
} lbm_status;

/* storage of the populations */
enum { LBM_FP32 = 0, LBM_FP16_SHIFTED = 1 };

/* lbm_set_boundary kinds */
enum {
  LBM_BC_FLAGS = 0,  /* uint8 per node (N bytes): bit0 obstacle voxel (halfway bounce-back),
                        bit1 Dirichlet inflow node, bit2 scalar source node.  Replaces the
                        three bits on every node; other bits are library-owned. */
  LBM_BC_INFLOW = 1, /* array of lbm_inflow_record: marks the nodes as inflow and sets
                        their inflow velocity (applied to every time level).  Records outside
                        the block or on obstacle voxels / ghost nodes are skipped and
                        reported as LBM_ERR_DIVERGED by the next synchronising call. */
  LBM_BC_WALLS = 2   /* block 0 only: 6 or 7 uint8 (host).  Bytes 0..5 non-zero for a no-slip
                        wall on face x-, x+, y-, y+, z-, z+ (the paper's second-order wall for
                        the ground and box walls, Sec. 6.1, read as the regularized on-node
                        wall: the face nodes are wall nodes at rest; populations pulled
                        through the wall are completed by bounce-back, both of a pair through
                        walls take the rest equilibrium, and every population is rebuilt from
                        the equilibrium at (rho, 0) and the non-equilibrium stress of the
                        completed set before the collision).  Byte 6 (optional) non-zero: the
                        same wall on the objects, Sec. 6.1 — an obstacle voxel with a
                        non-obstacle neighbour is a wall node at rest (flag bit 6 instead of
                        bit 0 in LBM_FIELD_FLAGS), populations pulled from the inner obstacle
                        voxels are the unknown ones, the inner voxels stay inert; without it
                        obstacles use halfway bounce-back.  Byte 6 applies to every refined
                        block too (their faces are scale boundaries, never walls); the
                        continuous-scale mappings treat every obstacle voxel, surface or
                        inner, as an obstacle (a dropped interpolation corner, a destination
                        left alone).  Replaces the previous walls.
                        INVALID_ARG for a wall on a periodic axis; UNSUPPORTED for wall
                        faces (bytes 0-5) with far-field blocks; byte 6 alone combines with
                        them (far-field blocks keep halfway bounce-back on their own obstacle
                        voxels).  With byte 6 set, blocks started from their parent
                        (lbm_init_block_from_parent, dynamic and static scale construction)
                        and the adjoint of a domain with refined blocks are UNSUPPORTED. */
};

typedef struct {
  int32_t x, y, z;
  float ux, uy, uz;
} lbm_inflow_record;

/* lbm_read_field / lbm_write_field selectors */
enum {
  LBM_FIELD_F = 0,      /* populations f_i, 27*N values (read/write) */
  LBM_FIELD_U = 1,      /* velocity stored by the last step, 3*N (read/write) */
  LBM_FIELD_SCALAR = 2, /* passive scalar, N (read/write) */
  LBM_FIELD_RHO = 3,    /* density sum_i f_i, N (read only) */
  LBM_FIELD_FLAGS = 4   /* uint8 node flags, N (read only; bit3 = scale-boundary ghost) */
};
/* element types */
enum { LBM_F32 = 0, LBM_F64 = 1, LBM_U8 = 2 };

/* lbm_read_macro selectors (float32 output) */
enum { LBM_MACRO_RHO = 0, LBM_MACRO_U = 1, LBM_MACRO_SCALAR = 2 };

typedef struct {
  void* (*alloc)(size_t bytes, void* ctx);       /* returns device memory or NULL */
  void (*free)(void* p, size_t bytes, void* ctx);
  void* ctx;
} lbm_allocator;

typedef struct {
  int32_t dims[3];     /* nx, ny, nz of the reference block s0 (>= 1 each) */
  int32_t periodic[3]; /* per axis: 1 periodic, 0 open (zero-gradient copy, Sec. 6.1) */
  double nu;           /* kinematic viscosity in reference-scale lattice units; S_4..8 =
                          1/(3 nu + 1/2) (Sec. 3.1, Eq. 3); must be > 0 */
  int32_t storage;     /* LBM_FP32 or LBM_FP16_SHIFTED (f_i - w_i stored as binary16) */
  int32_t adaptive;    /* 1: adaptive high-order relaxation of Sec. 4.1; 0: fixed nu' */
  double a, b, g_max;  /* Sec. 4.1 parameters (paper: -4, 5, g_max in [0.1, 0.13]) */
  double nu_hi[4];     /* Appendix artificial viscosities of moment groups 9..16, 17..22,
                          23..25, 26 (paper: 0.005, 0.007, 0.009, 0.01) */
  double c_src;        /* scalar value imposed on scalar-source nodes */
  void* cuda_stream;   /* cudaStream_t or NULL */
  lbm_allocator alloc; /* alloc.alloc == NULL: cudaMalloc / cudaFree */
  int32_t device;      /* CUDA device ordinal */
  int32_t grad_mode;   /* |grad u| of the adaptive relaxation (Sec. 4.1):
                          LBM_GRAD_LAGGED central differences of the velocity stored by the
                          previous step (default); LBM_GRAD_LOCAL the node's own strain rate
                          from its non-equilibrium second moments, Pi^(1) = -2 c_s^2 rho
                          S_hat / S (Sec. 4.2.1), as sqrt(2 S_hat : S_hat) */
} lbm_domain_desc;

enum { LBM_GRAD_LAGGED = 0, LBM_GRAD_LOCAL = 1 };

typedef struct {
  int32_t dims[3];
  double origin[3];  /* position of node (0,0,0) in reference-scale units */
  double h;          /* node spacing relative to the reference scale (dx_s / dx_0) */
  double nu;         /* viscosity in this block's lattice units (nu_0 / h, Sec. 3.2 Eq. 4) */
  int32_t substeps;  /* sub-steps per reference step (1 for s0) */
  int64_t steps;     /* reference steps taken by the domain */
  int32_t tile[2];   /* x, y extent in nodes of one CTA of the collide-stream kernel (chosen
                        by autotuning) */
  int32_t ctas_per_sm; /* CTAs per SM the collide-stream kernel's registers are bounded for
                          (chosen by autotuning together with the tile) */
  int32_t parent;      /* a refined block's prior-mapping source (the finest coarser block
                          containing it); -1 for the reference block and far-field blocks */
  int32_t nodes_per_thread; /* 1: one node per thread (tile[0] x tile[1] threads per CTA,
                               3 or 4 CTAs per SM); 2: two neighbouring x-nodes per thread
                               with paired FP32 arithmetic (half the threads, 4 to 6 CTAs
                               per SM; blocks with an even x-extent) */
} lbm_block_info;

/* Version of this header's ABI (5: lbm_block_info ends with nodes_per_thread; a caller built
   against version 4 passes a smaller struct and must not call lbm_get_block_info). */
int32_t lbm_abi_version(void);

/* Fills *desc with the paper's defaults (a=-4, b=5, g_max=0.1, nu' table, adaptive on,
   FP32, non-periodic, c_src=1, device 0, cudaMalloc).  dims and nu are set to 0 and must be
   filled by the caller. */
lbm_status lbm_default_desc(lbm_domain_desc* desc);

/* Creates a domain whose block 0 is the reference scale s0 with h = 1 (Sec. 4.2.4,
   "reference scale").  Populations start at the rest equilibrium, u = 0, scalar 0, no
   flags.  *out receives the handle.  INVALID_ARG for bad dims/nu/storage, OOM, CUDA. */
lbm_status lbm_create_domain(const lbm_domain_desc* desc, lbm_domain** out);

/* Releases every library buffer of the domain.  NULL is accepted. */
lbm_status lbm_destroy_domain(lbm_domain* dom);

/* Adds a scale block (Sec. 4.2: blocks at arbitrary, non-integer spacing ratios).
   origin: position of its node (0,0,0) in reference units; h = dx_s/dx_0 != 1; dims >= 4
   per axis.
   h < 1, a finer block: it must lie inside block 0; its outermost node layer is its scale
   boundary (ghost layer), written by prior-mapping from the finest coarser block that
   contains it; its interior is post-mapped into every coarser block but the far-field ones.
   Refined blocks must be added coarse to fine (h not increasing).
   h > 1, a far-field block (Sec. 4.2.4-4.2.5, the paper's FFD scales): it must contain the
   outermost block (block 0, or the last far-field block); each reference step it takes one
   step of its own dt = h dt_0 and is interpolated linearly back to t_n + dt_0, its nodes
   inside the contained block's interior are mapped from that block, and the contained
   block's outer layer becomes its scale boundary, mapped from the far-field block (obstacle
   and inflow nodes keep their own update); the outermost far-field block has open faces.
   Needs block 0 without periodic faces and without wall faces (UNSUPPORTED otherwise);
   obstacle-surface walls (LBM_BC_WALLS byte 6) are allowed.
   UNSUPPORTED for FP16 storage; STATE while an adjoint tape is recording; OOM / CUDA when a
   buffer or table cannot be created, in which case the domain is left exactly as before
   the call. */
lbm_status lbm_add_scale_block(lbm_domain* dom, const double origin[3], double h,
                               const int32_t dims[3], int32_t* block_id);

/* Removes the most recently added scale block (Sec. 5: dynamic scales are discarded and
   rebuilt; a refined block's interior has already been post-mapped into every coarser block
   at the end of each reference step).  Waits for the domain's stream, then releases the
   block's buffers and tables; removing a far-field block turns the outer layer of the block
   it contained back into open faces.  INVALID_ARG unless block_id is the last block and
   >= 1; STATE while an adjoint tape is recording. */
lbm_status lbm_remove_scale_block(lbm_domain* dom, int32_t block_id);

/* Dynamic scale construction, detection (Sec. 5): among the nodes of a block that are
   neither obstacle voxels nor ghost nodes, keeps those whose velocity-gradient magnitude
   (Frobenius norm of the central-difference Jacobian of the stored velocity, the quantity
   of the adaptive factor, Sec. 4.1) is >= g_threshold and whose |u| is >= u_threshold.
   Writes their number to *count and their bounding box, in the block's node indices, to
   box = {x0, y0, z0, x1, y1, z1} (inclusive; {0,0,0,-1,-1,-1} when count is 0).  The
   thresholds are compared in FP32.  Synchronises; deterministic. */
lbm_status lbm_detect_region(lbm_domain* dom, int32_t block_id, double g_threshold,
                             double u_threshold, int64_t* count, int32_t box[6]);

/* Starts a refined block from its prior-mapping source at the current time (Sec. 5 start of
   a dynamic scale): obstacle and scalar-source bits come from the source's nearest node
   (index floor(q + 1/2), q the node's position in the source's node units), every other
   node gets the Sec. 3.2 mapping (trilinear, obstacle corners dropped, K_hat rescale) of the
   source's current populations, with the velocity of the mapped populations and the
   interpolated scalar; obstacle nodes hold the rest state.  INVALID_ARG for block 0. */
lbm_status lbm_init_block_from_parent(lbm_domain* dom, int32_t block_id);

/* Dynamic scale construction (Sec. 5), in one call: lbm_detect_region on src_block, then
   (replace_last != 0) lbm_remove_scale_block of the last block, then, if any node was kept,
   a block of spacing h (0 < h < 1) placed on the detection box widened by `margin` source
   nodes on every side and clipped to the reference block: origin = clipped lower corner
   (reference units), floor(extent / h + 1e-9) + 1 nodes per axis, at least 4 (shifted down,
   not below 0, when they would pass the reference block's upper end); it is added with
   lbm_add_scale_block and started with lbm_init_block_from_parent.  *block_id receives the
   new block's id, or -1 when nothing was kept.  The paper repeats this every 40 steps.
   INVALID_ARG for bad arguments (replace_last needs a refined last block that is not the
   source block); the errors of the calls it makes otherwise. */
lbm_status lbm_build_dynamic_scale(lbm_domain* dom, int32_t src_block, double h,
                                   double g_threshold, double u_threshold, int32_t margin,
                                   int32_t replace_last, int32_t* block_id);

/* Static scale construction (Sec. 5): the distance to the obstacle voxels of block 0 is
   quantised into n_scales scales, scale 0 being block 0 (h = 1) and scale n_scales - 1 the
   finest (h = h_min), the spacings linearly interpolated in between; scale i covers the
   nodes within d_i = d_max (n_scales - 1 - i) / (n_scales - 1) of an obstacle, extended
   downstream along flow_axis (0, 1, 2 = x, y, z) by `wake` reference units.  Blocks are
   boxes: scale i is the obstacles' bounding box widened by d_i (plus the wake), clipped to
   block 0, with floor(extent / h + 1e-9) + 1 nodes per axis, at least 4 (shifted down, not
   below 0, at block 0's upper end).  The scales are added coarse to fine with
   lbm_add_scale_block and started with lbm_init_block_from_parent; *n_added receives their
   number (0 without obstacles).  INVALID_ARG for n_scales < 2, h_min outside (0, 1),
   negative d_max or wake, a bad axis; UNSUPPORTED when the domain has obstacle-surface walls
   (LBM_BC_WALLS byte 6); the errors of the calls it makes otherwise. */
lbm_status lbm_build_static_scales(lbm_domain* dom, int32_t n_scales, double h_min, double d_max,
                                   double wake, int32_t flow_axis, int32_t* n_added);

/* Static scale construction with the wake shaped as a soft shadow (Sec. 5: the inlet seen as
   an area light source, the darker shadow behind the obstacles taking the finer scales).
   The light is sampled at M <= n_light points: the inflow nodes of block 0 in index order
   (x fastest), every ceil(count / n_light)-th one, or, with no inflow node, the nodes of
   block 0's upstream face (index 0 along flow_axis) the same way.  Every node of block 0
   that is not an obstacle voxel and lies along flow_axis between the obstacles' upstream end
   and min(floor(downstream end + wake), last node) counts the samples it sees: the segment
   to a sample is walked in 2 m steps (m its largest coordinate difference), step k checked
   at the nearest node of p + d k / (2 m) computed in integers as
   (2 (p 2m + d k) + 2m) div (4m), end points excluded, and the sample is hidden when one of
   them is an obstacle voxel.  A node that sees c samples belongs to the wake of scale i
   (1 .. n_scales - 1) when c (n_scales - 1) <= (n_scales - 1 - i) M.  Scale i's box is the
   union of the obstacles' box widened by d_i (as above, without the straight wake) and the
   bounding box of its wake nodes, clipped, sized and started as above.  INVALID_ARG as
   above and for n_light < 1 or n_scales > 8; UNSUPPORTED with obstacle-surface walls. */
lbm_status lbm_build_static_scales_shadow(lbm_domain* dom, int32_t n_scales, double h_min,
                                          double d_max, double wake, int32_t flow_axis,
                                          int32_t n_light, int32_t* n_added);

/* Sets boundary data of one block (see LBM_BC_*).  ptr/nbytes describe the caller array;
   it is copied before return (host) or before the next enqueued work (device). */
lbm_status lbm_set_boundary(lbm_domain* dom, int32_t block_id, int32_t kind, const void* ptr,
                            size_t nbytes, int32_t on_device);

/* Initialises block populations to the equilibrium f = T m^eq(rho, u) (Algorithm 1 and
   Sec. 6.1), the stored velocity to u and the scalar to c.  rho (N floats) and c (N floats)
   may be NULL (rho = 1, c = 0); u (3*N floats) is required.  Obstacle voxels get the rest
   state.  Clears the device error word and any recorded tape. */
lbm_status lbm_init_macro(lbm_domain* dom, int32_t block_id, const float* rho, const float* u,
                          const float* c, int32_t on_device);

/* Advances the whole domain by n reference steps (Algorithm 1: s0 one step, then every
   finer block coarse to fine with prior-mapping, l sub-steps, temporal alignment and
   post-mapping to all coarser blocks).  Enqueues only; returns the status of host checks
   and of previously recorded device errors. */
lbm_status lbm_step(lbm_domain* dom, int32_t n_reference_steps);

/* Waits for the domain's stream and reports device errors (DIVERGED) recorded so far. */
lbm_status lbm_sync(lbm_domain* dom);

/* Reads rho, u (3 planes) or the scalar of a block as float32 into dst (dst_bytes must be
   at least the field size).  Synchronises. */
lbm_status lbm_read_macro(lbm_domain* dom, int32_t block_id, int32_t what, void* dst,
                          size_t dst_bytes, int32_t on_device);

/* Reads a field (LBM_FIELD_*) of a block as LBM_F32 / LBM_F64 (LBM_U8 for flags).
   Populations are returned unshifted (f_i, not f_i - w_i) in the paper's velocity order.
   Synchronises. */
lbm_status lbm_read_field(lbm_domain* dom, int32_t block_id, int32_t field, int32_t dtype,
                          void* dst, size_t dst_bytes, int32_t on_device);

/* Overwrites a field (F, U or SCALAR) of a block's current state from F32/F64 data.
   Populations are unshifted and in the paper's order.  Clears the device error word. */
lbm_status lbm_write_field(lbm_domain* dom, int32_t block_id, int32_t field, int32_t dtype,
                           const void* src, size_t src_bytes, int32_t on_device);

/* FP64 diagnostics of a block over non-obstacle, non-ghost nodes:
   out[0] mass sum rho, out[1..3] momentum sum rho u, out[4] kinetic energy
   (1/2) sum rho |u|^2.  Per-node values are formed in FP32 and summed per thread with a
   compensated FP32 sum, threads are combined in FP64 in a fixed order (deterministic).
   out is a host array of 5 doubles.  Synchronises; returns DIVERGED if the device error
   word is set. */
lbm_status lbm_reduce(lbm_domain* dom, int32_t block_id, double out[5]);

/* n >= 1 reference steps (as lbm_step) followed by the lbm_reduce diagnostics of block 0's
   new state, in one call.  On a single-block domain with 27 N < 2^32 the last step's kernel
   sums the moments of the state it stores while storing it (collision conserves rho and j,
   so a fluid node's are those of its pulled populations; per CTA in FP32 within a warp and
   FP64 across warps, then a fixed-order FP64 sum): no second pass over the populations.
   The values agree with lbm_reduce of the same state to FP32 rounding of the per-node terms
   (with FP16-shifted storage they are those of the FP32 state before it is rounded for
   storage); the stored state is the one lbm_step writes.  Other domains take the steps and
   then lbm_reduce of block 0.  out is a host array of 5 doubles (the lbm_reduce layout).
   Synchronises; INVALID_ARG for n < 1 or a null out; DIVERGED as lbm_step / lbm_reduce. */
lbm_status lbm_step_reduce(lbm_domain* dom, int32_t n, double out[5]);

/* lbm_step_reduce without the wait (not in the paper: it lets a caller queue the next step,
   and that step's inflow upload, before it reads this step's diagnostics, so that the GPU
   never idles on the host).  Enqueues the same n steps and diagnostics on the domain's
   stream, followed by a copy of the 5 values (lbm_reduce layout, combined on the device)
   into out, and returns; *ticket receives this call's number (1, 2, ... per domain).  out
   is host memory that must stay valid, and unread, until lbm_wait_results(ticket) (or
   lbm_sync) returns; pinned memory keeps the copy asynchronous, pageable memory makes this
   call wait for it.  Later calls do not reuse out.  INVALID_ARG for n < 1 or a null out or
   ticket; DIVERGED when an earlier step recorded divergence; errors of enqueueing as
   lbm_step. */
lbm_status lbm_step_reduce_async(lbm_domain* dom, int32_t n, double out[5], int64_t* ticket);

/* Waits until the lbm_step_reduce_async call that returned `ticket`, and every earlier one,
   has written its out array.  Returns DIVERGED (or TIMEOUT) when the device error word
   copied with those results says so, as lbm_sync does; INVALID_ARG for a ticket this domain
   has not issued. */
lbm_status lbm_wait_results(lbm_domain* dom, int64_t ticket);

/* lbm_reduce of block `block_id` of each of n domains (no counterpart in the paper: the
   read-back of a batch).  Members that share one device, stream and storage are reduced by
   one launch over chunks of all of them, with one read-back and one wait (the same sums in
   another order: equal to lbm_reduce's to FP32 rounding of the per-thread partials);
   otherwise every member's own reduction is queued on its stream before the call waits for
   any (lbm_reduce's values exactly).  out is a host array of 5 n doubles, domain i's five
   values at out[5 i].  INVALID_ARG for a null list, out or member, n <= 0, or a block id that some
   member lacks (nothing is launched then); otherwise every member is reduced and the first
   failing member's status is returned (DIVERGED, TIMEOUT, CUDA). */
lbm_status lbm_reduce_batch(lbm_domain* const* doms, int32_t n, int32_t block_id, double* out);

/* LBM_BC_INFLOW records of block 0 of each of n domains (no counterpart in the paper: the
   input side of a batch step).  recs[i] points to counts[i] host records for domain i (may
   be null when counts[i] is 0).  Members that share one device and stream get one staged
   host-to-device copy and one launch (the call returns once the records are staged, before
   the copy ends); otherwise each member takes lbm_set_boundary(LBM_BC_INFLOW).  Same effect
   and error reporting as the per-member calls.  INVALID_ARG for a null list, member,
   recs or counts, or a negative count. */
lbm_status lbm_set_inflow_batch(lbm_domain* const* doms, int32_t n,
                                const lbm_inflow_record* const* recs, const int32_t* counts);

lbm_status lbm_get_block_info(const lbm_domain* dom, int32_t block_id, lbm_block_info* info);

/* Halo planes of a domain split into slabs along z (no counterpart in the paper: several
   devices or processes each advance one slab with one halo plane on each side, and the
   edge planes are exchanged before every step; the pull of Sec. 1 reads a halo plane only
   through the 9 populations whose c_z points into the slab).  A packed plane of block 0's
   current state holds population rows as stored (storage element size, shifted, in the
   library's internal slot order) padded to a multiple of 16 bytes — dir +1: the 9
   populations with c_z = +1, the ones a slab above pulls; dir -1: the 9 with c_z = -1;
   dir 0: all 27 — then the 3 velocity rows and the scalar row (FP32), then the node flags
   (one byte each, derived bits included), nx * ny entries per row.  The buffer is meant for
   lbm_unpack_plane of a domain with the same nx, ny and storage, not for reading.
   lbm_plane_bytes gives its size (0 for a null domain or another dir).  lbm_pack_plane
   copies plane z into dev_buf, lbm_unpack_plane copies dev_buf into plane z (the
   population slots of another dir are left as they are); both are queued on the domain's
   stream (dev_buf is device memory of at least lbm_plane_bytes
   bytes, 16-byte aligned, owned by the caller; its size cannot be checked here).
   INVALID_ARG for a null or unaligned buffer, dir outside {-1, 0, +1} or z outside
   [0, nz); UNSUPPORTED for a domain with refined or far-field blocks; STATE while a tape
   records. */
size_t lbm_plane_bytes(const lbm_domain* dom, int32_t dir);
lbm_status lbm_pack_plane(lbm_domain* dom, int32_t z, int32_t dir, void* dev_buf);
lbm_status lbm_unpack_plane(lbm_domain* dom, int32_t z, int32_t dir, const void* dev_buf);

/* One step of a slab of a domain cut along z with its halo exchange overlapped (no
   counterpart in the paper).  lo / hi (0 or 1) say whether plane 0 / plane nz - 1 is a halo
   plane (a neighbouring slab's plane) rather than an end face of the whole domain.  The
   owned planes next to the halos, 1 (lo) and nz - 2 (hi), are stepped first; once written
   they are packed into send_lo (lbm_pack_plane layout, dir -1) and send_hi (dir +1) on
   pack_stream (a cudaStream_t, or NULL for an internal stream), while the other owned planes
   are stepped on the domain's stream; then the domain's level advances as after lbm_step.
   Halo planes are not stepped: before the next step the caller puts the neighbours' planes
   into them with lbm_unpack_plane (z = 0 with dir +1, z = nz - 1 with dir -1), after waiting
   for their transport.  Owned nodes end exactly as with lbm_step.  send buffers: device
   memory of lbm_plane_bytes bytes, 16-byte aligned, owned by the caller, not to be read
   before pack_stream reaches the packing.  INVALID_ARG for a null or unaligned send buffer
   that is needed or fewer than two owned planes; UNSUPPORTED with refined or far-field
   blocks; STATE while a tape records; DIVERGED as lbm_step. */
lbm_status lbm_step_slab(lbm_domain* dom, int32_t lo, int32_t hi, void* send_lo, void* send_hi,
                         void* pack_stream);

/* One reference step of Algorithm 1 (Sec. 4.2.4-4.2.5) as a sequence of phases, so that the
   blocks of one continuous-scale domain can be placed on several devices or processes (no
   counterpart in the paper, which runs one GPU).  Every participant holds the whole domain
   (same blocks, flags and initial state) and issues the same phases in the same order:
     LBM_PHASE_BEGIN                       records every block's level at t_n;
     LBM_PHASE_REFERENCE                   the reference block's step (block ignored);
     then for every refined block b = 1, 2, ... in order:
       LBM_PHASE_BLOCK, b                  b's sub-cycle: scale boundary at t_n from its
                                           prior-mapping source (lerped between that block's
                                           levels at t_n and now), l sub-steps, the last with
                                           the temporal alignment, scale boundary at
                                           t_n + dt_0;
       LBM_PHASE_POST, b                   post-mapping of b's interior into every coarser
                                           block;
     LBM_PHASE_END                         closes the step (one step is counted).
   compute != 0 launches the phase's work on the domain's stream; compute == 0 only advances
   the block's time levels the way the work would, so the level indices stay the same on
   every participant.  A block's owner computes its phases; before LBM_PHASE_BLOCK of b the
   owner of b's prior-mapping source sends it the boxes of
   lbm_mapping_boxes(LBM_BOX_PRIOR_SOURCE) at LBM_LEVEL_START and LBM_LEVEL_CURRENT, and
   after LBM_PHASE_POST of b the owner of b sends the LBM_BOX_POST_TARGET box of every
   coarser block it post-mapped into to that block's owner.  With every phase computed the result is bit for
   bit that of lbm_step(dom, 1).  STATE for a phase out of this order or while an adjoint
   tape records; UNSUPPORTED for domains with far-field blocks; INVALID_ARG for an unknown
   phase or a block that is not refined. */
enum {
  LBM_PHASE_BEGIN = 0, LBM_PHASE_REFERENCE = 1, LBM_PHASE_BLOCK = 2, LBM_PHASE_POST = 3,
  LBM_PHASE_END = 4
};
lbm_status lbm_step_phase(lbm_domain* dom, int32_t phase, int32_t block, int32_t compute);

/* Node boxes (inclusive index ranges lo[0..2] .. hi[0..2] in x, y, z) of one block that the
   mappings of refined block `block` exchange with block `other`:
     LBM_BOX_PRIOR_SOURCE  other = block's prior-mapping source: six boxes, one per face of
                           block (every corner of the trilinear cell of a scale-boundary node
                           lies in the box of its face);
     LBM_BOX_POST_TARGET   other = a coarser block: one box holding every node of `other`
                           that block's post-mapping writes (none if it writes none).
   boxes receives 6 int32 per box (lo then hi), room for 6 boxes; *n_boxes their number.
   INVALID_ARG for null pointers, a block that is not refined or a wrong `other`. */
enum { LBM_BOX_PRIOR_SOURCE = 0, LBM_BOX_POST_TARGET = 1 };
lbm_status lbm_mapping_boxes(const lbm_domain* dom, int32_t block, int32_t kind, int32_t other,
                             int32_t* boxes, int32_t* n_boxes);

/* A node box of a block's state as a device buffer: 27 population planes as stored (shifted,
   library slot order), 3 velocity planes and the scalar plane, FP32, one value per box node
   in x-fastest order (lbm_box_bytes gives the size: 124 bytes per node; 0 for an invalid
   box).  level: LBM_LEVEL_CURRENT, or LBM_LEVEL_START (the level at LBM_PHASE_BEGIN, inside
   a phased step).  lbm_unpack_box leaves the nodes whose flags carry any bit of skip_flags
   (LBM_FIELD_FLAGS bits) unchanged.  Queued on the domain's stream; dev_buf is caller-owned
   device memory, 16-byte aligned, of lbm_box_bytes bytes.  INVALID_ARG for a box outside
   the block, a null or unaligned buffer or another level; UNSUPPORTED without FP32 storage;
   STATE for LBM_LEVEL_START outside a phased step. */
enum { LBM_LEVEL_CURRENT = 0, LBM_LEVEL_START = 1 };
size_t lbm_box_bytes(const lbm_domain* dom, int32_t block, const int32_t lo[3],
                     const int32_t hi[3]);
lbm_status lbm_pack_box(lbm_domain* dom, int32_t block, int32_t level, const int32_t lo[3],
                        const int32_t hi[3], void* dev_buf);
lbm_status lbm_unpack_box(lbm_domain* dom, int32_t block, int32_t level, const int32_t lo[3],
                          const int32_t hi[3], const void* dev_buf, int32_t skip_flags);

/* Advances n independent single-block domains by `steps` reference steps with one
   persistent kernel per step over a joint tile work list, captured in one CUDA graph and
   launched on doms[0]'s stream (tile shape chosen by the library's autotuner on first use).
   Every domain must be single-block, without wall faces, with the same storage and device.  Results are
   bit-identical to calling lbm_step on each domain. */
lbm_status lbm_step_batch(lbm_domain* const* doms, int32_t n, int32_t steps);

/* lbm_step_batch with steps >= 1 followed by the lbm_reduce diagnostics of every member's
   new state, summed by the last step's own kernel (each work item's nodes add their
   moments as they are stored; the item sums are combined per member in FP64 in a fixed
   order and copied back by the same captured graph): no second pass over the populations.
   out is a host array of 5 n doubles (the lbm_reduce_batch layout); the values agree with
   lbm_reduce's to FP32 rounding of the per-node terms.  Synchronises; INVALID_ARG for
   steps < 1 or a null out; otherwise the lbm_step_batch errors, and each member's device
   error word as lbm_reduce_batch reports it. */
lbm_status lbm_step_batch_reduce(lbm_domain* const* doms, int32_t n, int32_t steps, double* out);

/* lbm_step_batch_reduce without the wait (not in the paper; the batched counterpart of
   lbm_step_reduce_async): the same steps and diagnostics are enqueued, the 5 n values are
   combined on the device and copied into out behind them, and the call returns.  *ticket
   receives a ticket of doms[0] (the sequence lbm_step_reduce_async uses): lbm_wait_results
   (doms[0], ticket) waits for out, and reports DIVERGED when any member's error word was set
   by then (every member's error bits are folded into doms[0]'s).  out (pinned host memory
   for an asynchronous copy) must stay valid and unread until then.  INVALID_ARG for a null
   out or ticket; otherwise as lbm_step_batch_reduce. */
lbm_status lbm_step_batch_reduce_async(lbm_domain* const* doms, int32_t n, int32_t steps,
                                       double* out, int64_t* ticket);

/* Self-test of the bounded device-wide barrier used by lbm_step_batch (no counterpart in the
   paper): launches a small cooperative kernel whose barrier waits for `extra` CTAs that do
   not exist, so every wait expires after about limit_ms (0 < limit_ms <= 5000).  Returns
   LBM_ERR_TIMEOUT when the bounded wait gave up and reported it (extra > 0), LBM_OK when
   the barrier completed (extra = 0); the CUDA context stays usable either way. */
lbm_status lbm_barrier_selftest(int32_t extra, double limit_ms, void* cuda_stream);

/* Enables recording of a reverse-mode tape by lbm_step: the state is checkpointed every
   `checkpoint_every` steps from the last lbm_init_macro (k >= 1; 0 disables). */
lbm_status lbm_set_tape(lbm_domain* dom, int32_t checkpoint_every);

/* Reverse-mode gradient of a loss L(c_T, u_T) of the final scalar and velocity of block 0
   after the n_steps steps recorded since the last lbm_init_macro (n_steps must equal the
   recorded count): dL_dscalar_final (N floats, device) and dL_du_final (3N floats, device,
   may be NULL) in; dL_du0 (3N floats, device) receives dL/du_0 for the u passed to
   lbm_init_macro.  An inflow node's velocity is its stored velocity, set with u_0 and
   carried unchanged by every step, so dL_du0 at inflow nodes is the gradient with respect to
   that inflow velocity; dL_dinflow (3N floats, device, may be NULL) receives the same values
   at inflow nodes and 0 elsewhere (inflow velocities must not be changed while the tape
   records).  Continuous-scale domains (refined blocks) are reversed through the whole
   Algorithm 1 schedule (prior- and post-mapping, sub-steps, temporal alignment); the loss
   is a function of block 0's final state, dL_du0 is block 0's gradient and
   lbm_adjoint_block_grad returns the other blocks'.  No-slip walls (wall faces and
   obstacle-surface walls, LBM_BC_WALLS) are reversed through the exact transpose of their
   completion and rebuild, far-field blocks through their aligned steps and overlap and
   boundary mappings.  Every relaxation mode (lagged gradient, local strain rate, fixed
   rates).  With FP16-shifted storage the checkpoints hold the stored deviations widened
   exactly to FP32 and each segment is replayed and reversed in FP32: the gradient is that
   of the FP32 step taken from the stored states, the storage rounding being passed
   through unchanged.  Not in the paper. */
lbm_status lbm_adjoint_step(lbm_domain* dom, int32_t n_steps, const float* dL_dscalar_final,
                            const float* dL_du_final, float* dL_du0, float* dL_dinflow);

/* After lbm_adjoint_step on a domain with refined blocks: copies dL/du_0 of block block_id
   (3 N_b floats, device) to dL_du0.  STATE if no multi-block reverse sweep has run.  Not in
   the paper. */
lbm_status lbm_adjoint_block_grad(lbm_domain* dom, int32_t block_id, float* dL_du0);

/* Largest n_nodes accepted by lbm_reduce_noalloc. */
#define LBM_REDUCE_NOALLOC_MAX_NODES 67108864

/* The same diagnostics as lbm_reduce, for callers that cannot allocate device memory (the
   paper has no counterpart; this is a library service).  Such callers include processes
   whose device memory is entirely reserved by another framework's pool and latency-critical
   loops that must never reach the driver's allocator.  This entry point allocates nothing:
   its partial sums live in a fixed 192 KiB device array inside the library, which every GPU
   that loads the library keeps until the process exits.
     f       device array of unshifted populations, 27 planes of n_nodes values in the
             paper's velocity order (the layout lbm_read_field returns), LBM_F32 or LBM_F64
             as given by dtype;
     flags   device array of n_nodes node flags (as lbm_read_field returns them) or NULL;
             obstacle voxels and ghost nodes are skipped;
     n_nodes 1 .. LBM_REDUCE_NOALLOC_MAX_NODES, larger values give LBM_ERR_INVALID_ARG;
     out     device array of 5 doubles: mass, momentum x, y, z, kinetic energy;
     cuda_stream  stream the work is enqueued on (NULL = legacy default stream); the call
             does not synchronise.
   The first call on a device (with that device current) looks up the array's device
   address and keeps it for the life of the process; make that first call before any
   stream capture, and do not call this entry point again after a context reset
   (cudaDeviceReset) of that device, which invalidates the address.  All calls share the one array,
   so calls whose work overlaps on the GPU (different streams, or different host threads on
   one device) race with each other; serialise them.  Errors are reported through
   lbm_last_error(NULL). */
lbm_status lbm_reduce_noalloc(const void* f, int32_t dtype, const uint8_t* flags,
                              int64_t n_nodes, double* out, void* cuda_stream);

/* Message of the last failure on this domain (empty if none); valid until the next call
   on the domain.  NULL dom gives the message of the last failed call that has no domain
   (lbm_create_domain, lbm_reduce_noalloc). */
const char* lbm_last_error(const lbm_domain* dom);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
