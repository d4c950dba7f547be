/*
 * jacobi.h -- C ABI of the GB300 Jacobi3D library.
 *
 * The library runs the hot path of the proxy application in Sec. 4.3 of
 * "Accelerating Communication for Parallel Programming Models on GPU Systems"
 * (Choi et al., arXiv 2102.12416): the Jacobi iterative method on a 3D grid
 * that is split into equal-size cuboid blocks (the paper's chares), each
 * block exchanging halo faces with up to six neighbours every iteration.  On
 * one GPU the exchange is a device-resident "channel" (Sec. 3.2.2, Channel
 * API): the producer writes a face straight into the neighbour's
 * preallocated receive slot and the consumer reads it there, with no
 * host-side metadata message.
 *
 * Conventions for every call
 *   - Returns JACOBI_OK (0) or a positive error code; jacobi_strerror() names
 *     it and jacobi_last_error() returns a message for the calling thread.
 *   - Handles are opaque, created and freed by the library.
 *   - Device pointers passed in (workspace, channel buffers, copy targets) stay
 *     owned by the caller and must outlive the handle that uses them.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is stream-ordered and asynchronous unless a call says it
 *     synchronises.
 *   - There is no host fallback: every numeric step runs in the library's
 *     CUDA kernels (sm_103a).  Calls that need a GPU fail with JACOBI_ECUDA
 *     when none is present.
 *
 * Environment (read by jacobi_create and jacobi_autotune):
 *   JACOBI_WAIT_MS     limit of every device-side wait in milliseconds (default
 *                      1000); an expired wait ends the kernel with
 *                      JACOBI_ETIMEDOUT instead of spinning on;
 *   JACOBI_FP64_EMU=0  keeps every FP64 add on the FP64 pipe, the FP64
 *                      stencil's and the FP32 residual's (see
 *                      jacobi_selftest_dadd);
 *   JACOBI_STAGES      ring depth (3..8) of the persistent kernel (default
 *                      4, or 5 for plane stages of 8 KB and more when the
 *                      fifth stage costs no resident CTA);
 *   JACOBI_PERSIST_WS=0  keeps the persistent path on its barrier-driven
 *                      kernel (by default launches whose items are all
 *                      plane-streamed run the warp-specialised one);
 *   JACOBI_TUNE_CACHE  file that caches jacobi_autotune's choices.
 *
 * Data layout of a grid of nx*ny*nz interior points ("interior" layout): one
 * array of nz*ny*nx values, x fastest.  The "padded" layout adds the
 * Dirichlet boundary: (nz+2)*(ny+2)*(nx+2) values, x fastest, interior at
 * indices 1..n on each axis.
 *
 * Arithmetic (the paper prints no stencil; this is the library's reading):
 *   s(i,j,k) = ((u(i-1)+u(i+1)) + (u(j-1)+u(j+1))) + (u(k-1)+u(k+1)),
 *   then u' = s * RN(1/6) in FP64 and u' = RN(s / 6) in FP32 (the float
 *   nearest 1/6 is a third of an ulp too large and would bias every FP32
 *   update by 2^-25); every operation is rounded separately (no fused
 *   multiply-add in the sum), so a run is bit-exact with a monolithic CPU
 *   evaluation in the same order, for any block split.
 * Residual (an addition; the paper's Jacobi3D runs a fixed iteration count):
 *   r = s - 6u in FP64 at every interior point, |r| = sqrt(sum r^2), b the same
 *   expression with the interior set to zero, rel = |r| / |b|.
 */
#ifndef JACOBI_H
#define JACOBI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
enum {
  JACOBI_OK = 0,
  JACOBI_EINVAL = 1,    /* bad argument (sizes, ids, null pointers, state) */
  JACOBI_ENOMEM = 2,    /* device or host allocation failed, or workspace too small */
  JACOBI_EBUSY = 3,     /* serving: no slot / HBM budget left right now */
  JACOBI_EAGAIN = 4,    /* serving: result not ready yet */
  JACOBI_ETIMEDOUT = 5, /* a device-side wait gave up (bounded spin expired) */
  JACOBI_ECUDA = 6,     /* a CUDA runtime call failed (message in jacobi_last_error) */
  JACOBI_ESEQ = 7       /* channel: sequence mismatch (message order broken) */
};

typedef enum { JACOBI_F64 = 0, JACOBI_F32 = 1 } jacobi_dtype;

/* Largest block extent per axis (work items hold block coordinates, padded
 * ones included, in 16 bits). */
#define JACOBI_MAX_BLOCK_EXTENT 32764

/* Dirichlet boundary families.  Coordinates are node-centred on the unit cube,
 * x = i/(nx+1) (IEEE FP64 division), likewise y and z. */
typedef enum {
  JACOBI_BC_LINEAR = 0,       /* g = (x + 2y) + 3z                         */
  JACOBI_BC_LINEAR_NOISE = 1, /* g + noise_amp * U(bc_seed, idx)           */
  JACOBI_BC_UNIFORM = 2       /* U(bc_seed, idx)                           */
} jacobi_bc;

typedef enum {
  JACOBI_INTERIOR_ZERO = 0,    /* interior starts at 0                    */
  JACOBI_INTERIOR_UNIFORM = 1, /* U(interior_seed, idx)                   */
  JACOBI_INTERIOR_BC = 2       /* the boundary function evaluated inside  */
} jacobi_interior;

/* Synthetic initial state.  U(seed, idx) is the idx-th output of SplitMix64
 * seeded with `seed` (Steele, Lea, Flood, OOPSLA 2014), top 53 bits scaled by
 * 2^-53; idx is the global padded linear index (k*(ny+2)+j)*(nx+2)+i, so the
 * data does not depend on the block split.  FP32 states take the FP64 value
 * rounded to nearest. */
typedef struct {
  int32_t bc;        /* jacobi_bc */
  int32_t interior;  /* jacobi_interior */
  uint64_t bc_seed;
  uint64_t interior_seed;
  double noise_amp;
} jacobi_init;

typedef struct { int64_t nx, ny, nz; } jacobi_dim3;

/* Block split (Sec. 4.3: equal-size cuboid blocks).
 *   JACOBI_SPLIT_COUNT: x,y,z = blocks per axis; extents differ by at most one
 *                       point (the first n % p blocks get the extra point).
 *   JACOBI_SPLIT_SHAPE: x,y,z = block extents; the last block on an axis is
 *                       partial when the extent does not divide the grid. */
typedef enum { JACOBI_SPLIT_COUNT = 0, JACOBI_SPLIT_SHAPE = 1 } jacobi_split_mode;
typedef struct { int32_t mode; int32_t pad_; int64_t x, y, z; } jacobi_split;

/* Step paths (all give bit-identical results).
 *   FUSED:      one launch per iteration; each block's new boundary planes are
 *               written straight into its neighbours' receive slots (pack and
 *               channel transfer fused into the stencil epilogue) and read
 *               from there by the next iteration (unpack fused into the load).
 *   EXPLICIT:   stencil launch, then an explicit pack of every face into a
 *               send buffer and a channel copy into the neighbour's slot.
 *   PERSISTENT: one cooperative launch runs all iterations; the z-chunks of
 *               the blocks (units) signal the units they share data with
 *               through release/acquire progress flags in device memory
 *               instead of kernel boundaries (bounded waits).
 *   GRAPH:      the FUSED launches captured once in a CUDA graph and replayed.
 * The next three run the halo exchange the way the paper's host-driven
 * runtimes do (Sec. 3, Sec. 4.3), for comparing the exchange forms on the
 * Jacobi3D workload; each iteration is a stencil launch followed by the
 * exchange, and the host takes part in every exchange:
 *   CHANNEL:     Channel API form (Sec. 3.2.2): the host waits for the
 *                stencil, then issues the sends; every receive slot was posted
 *                in advance, so one launch packs each face of the new iterate
 *                straight into the neighbour's slot.
 *   MESSAGING:   GPU Messaging form (Sec. 3.2.1): each face is packed into its
 *                block's send buffer; after the host has waited for that, a
 *                metadata message per face (source address, size) goes through
 *                a host-side mailbox of the receiving block, whose handler
 *                posts the receive (the source -> slot copy); the posted copies
 *                run as one launch from a table of descriptors uploaded by the
 *                host.
 *   HOST_STAGED: host staging, the non-GPU-aware form (Fig. 9): faces are
 *                packed, copied device -> pinned host memory, the host waits
 *                for them, then they are copied host -> device and unpacked into
 *                the neighbours' slots. */
typedef enum {
  JACOBI_PATH_FUSED = 0,
  JACOBI_PATH_EXPLICIT = 1,
  JACOBI_PATH_PERSISTENT = 2,
  JACOBI_PATH_GRAPH = 3,
  JACOBI_PATH_CHANNEL = 4,
  JACOBI_PATH_MESSAGING = 5,
  JACOBI_PATH_HOST_STAGED = 6
} jacobi_path;

/* Solve outcome. */
typedef enum {
  JACOBI_SOLVE_CONVERGED = 0,
  JACOBI_SOLVE_MAX_ITERS = 1,
  JACOBI_SOLVE_STAGNATED = 2
} jacobi_solve_status;

/* Copy layouts for jacobi_copy_out / jacobi_set_state. */
enum { JACOBI_LAYOUT_INTERIOR = 0, JACOBI_LAYOUT_PADDED = 1 };

typedef struct jacobi_s jacobi_t;
typedef struct channel_s channel_t;

/* Block description (host-side view of the decomposition). */
typedef struct {
  int64_t grid;          /* owning grid index within the handle         */
  int64_t origin[3];     /* first interior point (x, y, z), 0-based      */
  int64_t extent[3];     /* points per axis                              */
  int64_t neighbour[6];  /* block id across face xm,xp,ym,yp,zm,zp, -1 = Dirichlet */
} jacobi_block_info;

typedef struct {
  int64_t n_grids;
  int64_t n_blocks;
  int64_t n_points;      /* interior points over all grids             */
  int64_t iteration;     /* iterations completed so far                */
  int32_t dtype;
  int32_t path;
  int64_t halo_bytes_per_iter; /* face payload moved per iteration (bytes) */
  size_t workspace_bytes;
  int32_t stages;        /* ring depth of the persistent kernel as set (by
                            JACOBI_STAGES or the autotuner; otherwise 4, which
                            large stages may raise to 5 at launch); the
                            per-step streaming kernels use 4                  */
  int32_t item_kinds;    /* kernel variants launched per iteration (fused paths) */
  int32_t fp64_int_adds; /* neighbour pair sums per update that may run on the
                            integer pipe (0 or 3) for grids inside the integer
                            adder's domain; the kernels send most of them there */
  int32_t pad_;
  int32_t kind_items[8]; /* work items per step kernel variant: [0] tiles (rows
                            too wide to stream); [1..3] plane streaming with 8,
                            4, 2 consumer warps per CTA; [4..6] the same for
                            blocks with padded (ragged) rows; [7] unused */
  int64_t zchunk;        /* work-item shape (see jacobi_set_shape): planes per item */
  int32_t cw_cap;        /*   and the consumer-warp cap of streaming CTAs         */
  int32_t pad2_;
} jacobi_info_t;

/* Outcome of jacobi_autotune. */
typedef struct {
  int32_t path;          /* chosen jacobi_path                                  */
  int32_t stages;        /* chosen ring depth                                   */
  double ms_per_iter;    /* measured time per iteration of the chosen config    */
  int32_t n_tried;       /* candidates timed (0 when taken from the cache)      */
  int32_t from_cache;
  int64_t zchunk;        /* chosen z-chunk depth (planes per work item)         */
  int32_t cw_cap;        /* chosen consumer-warp cap per streaming CTA (2/4/8; 0 = tiles) */
  int32_t pad_;
} jacobi_tune_result;

/* ---- errors -------------------------------------------------------------- */
const char* jacobi_strerror(int code);
/* Message of the last failing call on the calling thread ("" if none). */
const char* jacobi_last_error(void);

/* ---- decomposition (host only; no GPU needed) ------------------------------ */

/* Block counts px*py*pz == nblocks, p <= n per axis, minimising the total
 * block surface of the near-equal split (Sec. 4.3 chooses the cuboid split
 * with the least surface, i.e. the least halo volume); ties go to the
 * lexicographically smallest (px, py, pz).
 * JACOBI_EINVAL if no split fits. */
int jacobi_decompose(jacobi_dim3 grid, int64_t nblocks, jacobi_dim3* counts_out);

/* Device bytes jacobi_create needs for one grid (states, receive slots,
 * flags, tables, reduction partials), for a caller-supplied workspace.
 * Grids, splits and block extents are checked as by jacobi_create:
 * JACOBI_EINVAL for a non-positive or too large size (a block may span at
 * most JACOBI_MAX_BLOCK_EXTENT points per axis). */
int jacobi_workspace_bytes(jacobi_dim3 grid, jacobi_split split, jacobi_dtype dtype,
                           size_t* bytes);
int jacobi_workspace_bytes_batch(int64_t n_grids, const jacobi_dim3* grids,
                                 const jacobi_split* splits, jacobi_dtype dtype,
                                 size_t* bytes);

/* ---- lifecycle ------------------------------------------------------------- */

/* Create a solver for one grid.  `init` may be NULL (linear boundary, zero
 * interior).  `workspace` may be NULL (the library allocates and frees it)
 * or a device buffer of at least jacobi_workspace_bytes() bytes, 256-byte
 * aligned, owned by the caller.  The initial state is written by a kernel on
 * `stream`; the call returns without waiting for it. */
int jacobi_create(jacobi_dim3 grid, jacobi_split split, jacobi_dtype dtype,
                  const jacobi_init* init, void* workspace, size_t ws_bytes, void* stream,
                  jacobi_t** out);

/* Create one handle holding n_grids independent grids (batched stepping:
 * every grid advances in the same launches).  grids/splits/inits are arrays of
 * n_grids entries (inits may be NULL). */
int jacobi_create_batch(int64_t n_grids, const jacobi_dim3* grids, const jacobi_split* splits,
                        jacobi_dtype dtype, const jacobi_init* inits, void* workspace,
                        size_t ws_bytes, void* stream, jacobi_t** out);

/* Waits for the handle's outstanding work (the handle does not own the
 * caller's streams, so this synchronises the device), then frees what the
 * library allocated (never the caller's workspace). */
int jacobi_destroy(jacobi_t* h);

int jacobi_info(const jacobi_t* h, jacobi_info_t* out);
int jacobi_block(const jacobi_t* h, int64_t block, jacobi_block_info* out);

/* Select the step path (jacobi_path).  The persistent launch uses at most as
 * many CTAs as can be co-resident on the GPU.  Its warp-specialised kernel
 * hands out the launch's (iteration, unit) pairs in order from a device
 * counter, so a CTA takes its next unit when it is free; the barrier-driven
 * kernel gives CTA c the units c, c + G, c + 2G, ... */
int jacobi_set_path(jacobi_t* h, int32_t path);

/* Work-item shape of the step kernels (the library's addition; the block
 * split itself is the caller's).  zchunk: planes per work item along z (0 =
 * the library's cost model; clamped to the tallest block).  cw_cap: at most 2,
 * 4 or 8 consumer warps per plane-streaming CTA; a CTA of CW warps covers
 * 4 * 32 * CW / (row vectors) rows of a plane, so a lower cap cuts planes into
 * more, shorter row windows (a row's vectors always fit one CTA); 0 sends
 * every block to the tile kernel (32 x 8 columns per CTA, plain loads, no
 * bulk-copy ring).  Iterates do not depend on the shape (bit for bit);
 * residual sums are reproducible for a given shape.  The item tables hold the
 * finest shapes down to a quarter of the planned z-chunk: finer ones give
 * JACOBI_EINVAL.  Synchronises the stream. */
int jacobi_set_shape(jacobi_t* h, int64_t zchunk, int32_t cw_cap, void* stream);

/* Autotuner (the library's addition): times candidate step configurations
 * (each for at least iters_per_trial iterations and ~2 ms, best of two runs)
 * on a scratch handle with the same grids,
 * splits and dtype (the handle's own state is untouched): every shape of
 * jacobi_set_shape with a z-chunk of 2, 1, 1/2 or 1/4 times the cost model's
 * and a warp cap of 8, 4, 2 or 0 (tiles; shapes that give the same items are
 * timed once), each on the GRAPH path and the PERSISTENT kernel; then FUSED and the
 * persistent ring depths 3..6 at the best shape.  Applies the fastest (path,
 * ring depth, shape) to `h`.  All candidates give bit-identical iterates.
 * When the environment variable JACOBI_TUNE_CACHE names a file, results are
 * looked up there by a signature of the geometry and appended after a search.
 * Synchronises the stream. */
int jacobi_autotune(jacobi_t* h, int64_t iters_per_trial, void* stream, jacobi_tune_result* out);

/* The same search restricted to one path (JACOBI_PATH_FUSED, _GRAPH or
 * _PERSISTENT): every candidate shape on that path and, for PERSISTENT, the
 * ring depths 3..6 at its best shape; applies the path and the fastest shape
 * and depth to `h`.  For a caller that wants a given execution form (say, the
 * whole run in one persistent launch) with the shape tuned for it.  Cached
 * under a key of its own.  JACOBI_EINVAL for another path.  Synchronises the
 * stream. */
int jacobi_autotune_path(jacobi_t* h, int32_t path, int64_t iters_per_trial, void* stream,
                         jacobi_tune_result* out);

/* ---- state transfer ---------------------------------------------------------- */

/* Replace the whole state of grid `grid` (boundary and interior) from a padded
 * array (src_on_device: 0 = host memory, 1 = device memory) of the handle's
 * dtype.  Host sources are copied synchronously; device sources are read on
 * `stream`.  Resets nothing else: the iteration counter keeps counting. */
int jacobi_set_state(jacobi_t* h, int64_t grid, const void* src, int32_t src_on_device,
                     void* stream);

/* Copy grid `grid`'s current iterate out in the interior or padded layout
 * (dtype of the handle).  dst_on_device = 0 (host; the call synchronises the
 * stream) or 1 (device; asynchronous). */
int jacobi_copy_out(jacobi_t* h, int64_t grid, void* dst, int32_t dst_on_device, int32_t layout,
                    void* stream);

/* ---- the hot path ------------------------------------------------------------ */

/* Advance every grid of the handle by n_iters Jacobi iterations (Sec. 4.3),
 * halo exchange included, on the selected path.  Asynchronous. */
int jacobi_step(jacobi_t* h, int64_t n_iters, void* stream);

/* jacobi_step with the two phases of each iteration timed by CUDA events on
 * `stream`: *compute_ms receives the summed time of the stencil launches and
 * *exchange_ms the summed time from the end of each stencil launch to the end
 * of that iteration's halo exchange (pack, transfer, host hand-offs and waits,
 * unpack).  On FUSED, GRAPH and PERSISTENT the exchange is fused into the
 * stencil: the whole iteration counts as compute and *exchange_ms is 0.
 * Synchronises the stream. */
int jacobi_step_timed(jacobi_t* h, int64_t n_iters, void* stream, double* compute_ms, double* exchange_ms);

/* FP64 residual of the current iterate of every grid: rel[g] = |b-Au|/|b|,
 * abs[g] = |b-Au| (either pointer may be NULL; arrays of n_grids doubles in
 * host memory).  Partials are reduced in a fixed order, so results are
 * reproducible bit for bit.  Synchronises the stream. */
int jacobi_residual(jacobi_t* h, double* rel, double* abs_res, void* stream);

/* Iterate until rel <= tol for every grid, checking every check_every
 * iterations on the current iterate (the residual of u_k is fused into the
 * step that computes u_{k+1}); a grid whose check passes is frozen at u_k.
 * Stops at max_iters (status MAX_ITERS) or after stall_checks (> 0) checks
 * without a new best rel (STAGNATED).  Per-grid outputs (host arrays of
 * n_grids entries, NULL allowed): iterations done, rel at stop, status.
 * Synchronises the stream once per check. */
int jacobi_solve(jacobi_t* h, double tol, int64_t max_iters, int64_t check_every,
                 int64_t stall_checks, int64_t* iters_out, double* rel_out, int32_t* status_out,
                 void* stream);

/* Synchronise `stream` and report the first device-side failure of the
 * handle's persistent steps (JACOBI_ETIMEDOUT when a bounded neighbour wait
 * expired) or JACOBI_OK; clears it. */
int jacobi_sync(jacobi_t* h, void* stream);

/* Copy the receive slot that block `block` reads across face `face`
 * (0..5 = xm, xp, ym, yp, zm, zp) at its next iteration into host memory
 * `dst` (face layout: x-faces [z][y], y-faces [z][x], z-faces [y][x]; handle
 * dtype).  After a step this is the neighbour's packed boundary plane (or the
 * Dirichlet boundary).  Synchronises the stream. */
int jacobi_read_face(jacobi_t* h, int64_t block, int32_t face, void* dst, void* stream);

/* Test support for the integer-pipe FP64 adder: out[i] = a[i] + b[i] (device
 * arrays of n doubles) computed by the integer-pipe routine the FP64 step
 * kernels use for the neighbour pair sums and the FP32 residual for the pair
 * sums of its widened values.  For a[i], b[i] >= 0 with
 * exponent field < 2040 the result is the IEEE-754 round-to-nearest-even sum
 * bit for bit; other inputs give unspecified values (the step kernels never
 * pass them: a device check keeps such grids on the FP64 pipe).  Setting the
 * environment variable JACOBI_FP64_EMU=0 before jacobi_create keeps every
 * FP64 add on the FP64 pipe.  Asynchronous. */
int jacobi_selftest_dadd(const double* a, const double* b, int64_t n, double* out, void* stream);

/* Test support for the FP32 residual's exact binary32 -> binary64 widening on
 * the integer pipe: runs every one of the 2^32 binary32 bit patterns through
 * it on the device and writes to *mismatches (host) how many results differ
 * bit for bit from the conversion instruction's (NaN inputs must give a NaN).
 * Expected 0.  Synchronises the stream. */
int jacobi_selftest_widen(uint64_t* mismatches, void* stream);

/* Test support for the FP32 update's division: u' = RN(s / 6) is computed as
 * RN(s * zh + RN(s * zl)) with zh = RN(1/6), zl = RN(1/6 - zh) (a method of
 * Brisebarre, Muller and Raina for division by a constant; the paper prints no
 * stencil, see the arithmetic note at the top of this file), with the
 * division instruction sequence for the inputs outside that form's proven
 * domain.  Runs all 2^32 binary32 bit patterns through it on the device and
 * writes to *mismatches (host) how many differ bit for bit from the division
 * instruction sequence (NaN inputs must give a NaN).  Expected 0.
 * Synchronises the stream; allocates 8 bytes of scratch. */
int jacobi_selftest_div6(uint64_t* mismatches, void* stream);

/* Measured issue rates of this GPU's two add pipes (for rooflines): FP64 adds
 * per second on the FP64 pipe, and FP64 adds per second through the
 * integer-pipe routine of jacobi_selftest_dadd; each from one timed launch of
 * 8 independent add chains per thread.  Synchronises the stream; allocates a
 * small scratch buffer. */
int jacobi_pipe_rates(double* fp64_adds_per_s, double* int_adds_per_s, void* stream);

/* Host-side fault injection for tests: the next persistent steps leave block
 * `block` out of the launch (its sends never happen), so its neighbours'
 * bounded waits expire and jacobi_sync reports JACOBI_ETIMEDOUT.  block = -1
 * clears the injection. */
int jacobi_debug_drop_block(jacobi_t* h, int64_t block);

/* Measurement switch for the halo share of a step (the share of step time
 * that exchanging halos between blocks costs): with on = 1 every block stores
 * its new boundary planes into its OWN receive slots instead of its
 * neighbours' (same kernels, same bytes, same slot shapes, but each block then
 * reads its own faces as ghosts), so timing a step with and without it shows
 * what routing the faces to other blocks costs.  The iterates computed while
 * it is on are NOT Jacobi iterates of the grid; switching it off restores the
 * exchange, not the state (reset the state with jacobi_set_state).
 * Synchronises the device. */
int jacobi_measure_local_halo(jacobi_t* h, int32_t on);

/* ---- allocation-free residual ------------------------------------------------- */

/* Largest nz accepted by jacobi_residual_noalloc (size of its fixed scratch). */
#define JACOBI_NOALLOC_MAX_PLANES 16384

/* The paper has no counterpart to this call; it serves callers that cannot
 * allocate device memory when they need a residual: applications that
 * reserve all device memory at start-up and forbid later allocations (a fixed
 * footprint, or a framework whose caching allocator must account for every
 * byte), and loops that cannot afford the device-wide synchronisation a
 * cudaMalloc or cudaFree may bring.
 *
 * Computes the FP64 residual of a caller-owned padded state array u_padded
 * (device memory, (nz+2)*(ny+2)*(nx+2) values of `dtype`, x fastest, boundary
 * included) with the same per-point expression as jacobi_residual, and writes
 * out[0] = |b - Au|, out[1] = |b|, out[2] = rel (|b| = 0: rel = |b - Au|) to
 * the caller's device buffer `out` (3 doubles), asynchronously on `stream`.
 * It allocates nothing and calls no allocating routine: the reduction scratch
 * is a fixed 256 KB device array inside the library (two FP64 partials per
 * z-plane), held by every GPU that loads the library until the process exits.
 * Grids with nz > JACOBI_NOALLOC_MAX_PLANES are rejected with JACOBI_EINVAL.
 * The first call on each device looks up the array's device address (no
 * allocation, but it may load the module), so make that first call before
 * any stream capture.  All calls on a device share the array and each call
 * overwrites every partial it reads; calls whose kernels overlap on the GPU
 * (unordered streams) race on it. */
int jacobi_residual_noalloc(const void* u_padded, jacobi_dim3 grid, jacobi_dtype dtype, double* out,
                            void* stream);

/* ---- channels (Sec. 3.1 tag scheme, Sec. 3.2.2 Channel API) ------------------ */

/* Open a two-sided channel between blocks a and b with a caller-chosen id
 * that is unique within the handle (Sec. 3.2.2).  The library allocates, for
 * each endpoint, two receive slots of max_bytes (parity double buffering),
 * plus per-endpoint message counters in device memory: a message's sequence
 * number plays the role of the 32-bit per-endpoint counter of the paper's
 * channel tag (Sec. 3.1), so messages are matched in order and exactly once. */
int channel_open(jacobi_t* h, uint32_t channel_id, int64_t block_a, int64_t block_b,
                 size_t max_bytes, channel_t** out);

/* Send `bytes` from device buffer src (16-byte aligned) on behalf of endpoint
 * `from_block`.  When the peer posted the matching receive earlier (see
 * channel_recv), one launch copies the payload straight into the posted
 * buffer and completes that receive (JACOBI_ESEQ at once, nothing sent, if the
 * posted size differs).  Otherwise the payload goes into the peer's receive
 * slot and the message's sequence number is published with a release store;
 * the send waits on the device (bounded) until the peer has consumed the
 * message that used the same slot two sends ago.  Asynchronous; a failed wait
 * is reported by channel_sync. */
int channel_send(channel_t* ch, int64_t from_block, const void* src, size_t bytes, void* stream);

/* Receive the next message for endpoint `at_block`.
 *  - Posted receive: with dst (device, 16-byte aligned) given before the
 *    matching channel_send has been issued (host program order), the call only
 *    registers dst; the send delivers the payload straight into it (the
 *    Channel API's pre-posted receive, Sec. 3.2.2).  Work that reads dst must
 *    be ordered after that send (same stream, or an event).  Until then
 *    channel_sync reports JACOBI_EAGAIN.
 *  - Otherwise: acquire-wait on the device (bounded) until the message's
 *    sequence number is published, then copy it to dst and mark it consumed,
 *    or, with dst NULL (zero-copy), leave it in its slot (see channel_slot).
 *    A zero-copy message holds its slot until the next channel_recv at this
 *    endpoint or channel_release, both of which must be ordered after every
 *    read of the slot; the peer's send of the message after next waits for
 *    that release.
 * `bytes` must equal the sent size (JACOBI_ESEQ otherwise, reported by
 * channel_sync).  Asynchronous.  A waiting receive with no matching send
 * earlier in stream order times out with JACOBI_ETIMEDOUT.  After channel_sync
 * has reported JACOBI_ETIMEDOUT or JACOBI_ESEQ the channel's message counters
 * no longer match: close and reopen it. */
int channel_recv(channel_t* ch, int64_t at_block, void* dst, size_t bytes, void* stream);

/* Release the slot held by the last zero-copy receive at endpoint at_block
 * (no-op when none is held).  Asynchronous; order it after the reads. */
int channel_release(channel_t* ch, int64_t at_block, void* stream);

/* Device address of endpoint at_block's receive slot for message parity
 * `parity` (message n uses parity n & 1). */
int channel_slot(channel_t* ch, int64_t at_block, int32_t parity, void** slot);

/* Synchronise `stream` and report the first device-side failure of the
 * channel (JACOBI_ETIMEDOUT, JACOBI_ESEQ; clears it), else JACOBI_EAGAIN while
 * a posted receive still waits for its send, else JACOBI_OK. */
int channel_sync(channel_t* ch, void* stream);

/* OSU-style ping-pong between the two endpoints (Sec. 4.2.1), run entirely on
 * the device: one cooperative launch whose first `ctas_per_side` CTAs act as
 * endpoint a and the rest as endpoint b; each round trip sends `bytes` a->b
 * and back through the channel's slots and counters.  The caller times the
 * launch with events on `stream`; one-way latency = elapsed / (2*round_trips). */
int channel_pingpong(channel_t* ch, size_t bytes, int64_t round_trips, int32_t ctas_per_side,
                     void* stream);

/* OSU-style bandwidth test (Sec. 4.2.2), run on the device: one cooperative
 * launch in which endpoint a sends `window` messages of `bytes` back to back
 * into b's slot and b acknowledges, `iterations` times (with bidirectional set
 * both endpoints send a window per iteration).  Sources are each endpoint's
 * parity-1 slot.  The caller times the launch: bandwidth = (1 or 2) * window *
 * iterations * bytes / elapsed. */
int channel_bandwidth(channel_t* ch, size_t bytes, int32_t window, int64_t iterations, int32_t ctas_per_side,
                      int32_t bidirectional, void* stream);

/* The two comparison forms of the paper, for benchmarks against the channel.
 *
 * Host staging (Fig. 9, the non-GPU-aware path): channel_send_host copies the
 * payload device->host into a pinned staging buffer of the receiving endpoint
 * and waits for it; channel_recv_host copies it host->device into dst and
 * waits.  Both synchronise the stream; one host-staged message may be in
 * flight per direction.
 *
 * GPU Messaging (Sec. 3.2.1): channel_send_msg only posts a host-side
 * metadata message (source address, size, sequence number) to the peer's
 * mailbox; channel_recv_msg takes the oldest one -- the receive can only be
 * posted once the metadata has arrived -- issues the device copy src -> dst and
 * waits for it.  JACOBI_EAGAIN when no metadata message is waiting,
 * JACOBI_ESEQ on a size mismatch.  The source must stay valid until received. */
int channel_send_host(channel_t* ch, int64_t from_block, const void* src, size_t bytes, void* stream);
int channel_recv_host(channel_t* ch, int64_t at_block, void* dst, size_t bytes, void* stream);
int channel_send_msg(channel_t* ch, int64_t from_block, const void* src, size_t bytes, void* stream);
int channel_recv_msg(channel_t* ch, int64_t at_block, void* dst, size_t bytes, void* stream);

int channel_close(channel_t* ch);

/* ---- serving: continuous batching of solve requests --------------------------- */

/* The paper runs one Jacobi3D problem at a time (Sec. 4.3); the server is the
 * library's addition for many independent solves.  A background thread admits
 * requests in arrival order while a slot and the HBM budget allow, keeps every
 * admitted grid (states, receive slots, tables) resident on the device, and
 * steps all of them in the same launches.  Each grid checks its FP64 relative
 * residual every check_every iterations on the device and freezes itself when
 * it converges (or hits its cap, or stagnates); admission and retirement happen
 * between rounds of round_checks * check_every iterations.  A request's result
 * does not depend on what else is running: its blocks, work items and residual
 * summation order come from its own decomposition. */
typedef struct serve_s serve_t;

typedef struct {
  uint64_t hbm_budget_bytes; /* admitted grids' device bytes stay below this     */
  int32_t max_slots;         /* at most this many grids run at once (<= 1024)   */
  int32_t dtype;             /* jacobi_dtype of every grid                       */
  int32_t check_every;       /* iterations between convergence checks           */
  int32_t round_checks;      /* checks per scheduling round (>= 1)              */
  int64_t stall_checks;      /* > 0: STAGNATED after this many checks w/o a new best */
} serve_config;

typedef struct {
  jacobi_dim3 grid;
  jacobi_split split;
  jacobi_init init;
  double tol;           /* relative residual target                            */
  int64_t max_iters;    /* cap; must be a multiple of check_every               */
  void* out;            /* optional host buffer for the final iterate (interior
                           layout, dtype of the server), written before the
                           result is posted; owned by the caller             */
} serve_request;

typedef struct {
  int32_t status;       /* jacobi_solve_status once done                        */
  int32_t pad_;
  int64_t iters;        /* iterations at the converged / final check            */
  double rel;           /* relative residual of the returned iterate            */
  int64_t t_arrive_ns;  /* host monotonic clock: submission                     */
  int64_t t_admit_ns;   /*                       admission                      */
  int64_t t_done_ns;    /*                       result posted                  */
} serve_result;

typedef struct {
  int64_t submitted, admitted, completed, queued, running;
  int64_t rounds;
  int64_t iterations;   /* global iterations stepped                            */
  uint64_t bytes_in_use;
  int64_t lups;         /* lattice-site updates performed on admitted grids     */
} serve_stats_t;

/* Start a server; its thread and device tables live until serve_destroy. */
int serve_create(const serve_config* cfg, serve_t** out);
/* Queue a request (thread-safe, never blocks on the GPU).  JACOBI_EINVAL for
 * bad sizes or a grid larger than the budget or the per-slot table limits. */
int serve_submit(serve_t* s, const serve_request* req, uint64_t* ticket);
/* JACOBI_OK with the result when done, JACOBI_EAGAIN (result->t_arrive_ns set)
 * while pending, JACOBI_EINVAL for an unknown ticket. */
int serve_poll(serve_t* s, uint64_t ticket, serve_result* result);
int serve_stats(serve_t* s, serve_stats_t* out);
/* Stop after the current round (pending requests are dropped) and free. */
int serve_destroy(serve_t* s);

#ifdef __cplusplus
}
#endif
#endif /* JACOBI_H */
