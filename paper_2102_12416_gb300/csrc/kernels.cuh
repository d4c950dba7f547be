// Host-visible launch wrappers for the library's kernels (defined in kernels.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"

namespace jgb {

// Initial-state description of one grid, as the init kernels see it.
struct InitDev {
  int64_t NX, NY, NZ;  // grid interior size
  int32_t bc, interior;
  uint64_t bc_seed, interior_seed;
  double noise_amp;
};

// Geometry of one block needed only by init / scatter / gather.
struct BlockGeom {
  int32_t ox, oy, oz;  // origin of the first interior point
  int32_t grid;
};

// Largest dynamic shared memory a step kernel may use (sm_103a opt-in limit of
// 227 KB per CTA, minus room for the kernels' static shared memory: the
// persistent kernels keep up to 32 units' tables there, about 13.6 KB).
constexpr int kMaxStepSmem = 227 * 1024 - 16384;
// Units per CTA whose tables the barrier-driven persistent kernel caches in
// static shared memory.
constexpr int kPersistCache = 32;
// Largest dynamic shared memory (the ring) of the warp-specialised persistent
// kernel, beside its static queue of unit tables (about 2 KB).
constexpr int kPersistWsSmem = 227 * 1024 - 4096;

// A plane-streaming item encodes its consumer warps (2, 4 or 8) in the low
// bits of y0 and, in bit 4, whether its block has padding (ragged rows or
// planes).  Item kinds of a step launch: 0 = tiles; 1, 2, 3 = streaming with
// 8, 4, 2 consumer warps; 4, 5, 6 = the same for ragged blocks.  Each kind
// runs its own kernel variant.
constexpr int kItemKinds = 7;
// Ring depth of the per-step plane-streaming kernels: a compile-time 4 (the
// stage index is a mask, and 4 measured best for every block shape; the
// planner only streams blocks whose 4-stage ring fits shared memory).  The
// persistent kernel's ring depth stays a run-time choice.
constexpr int kStreamStages = 4;
static_assert((kStreamStages & (kStreamStages - 1)) == 0, "stage indices are masks: a power of two");
constexpr int kItemRagged = 16;
__host__ __device__ inline bool item_ragged(const WorkItem& w) { return (w.y0 & kItemRagged) != 0; }
__host__ __device__ inline int item_kind(const WorkItem& w) {
  if (w.x0 >= 0) return 0;
  const int cw = w.y0 & 15;
  return (cw == 8 ? 1 : cw == 4 ? 2 : 3) + (item_ragged(w) ? 3 : 0);
}

struct StepLaunch {
  const BlockDev* blocks;
  const WorkItem* items;  // active items, grouped by kind
  int32_t n_items;
  int32_t kind_off[kItemKinds + 1];  // items of kind k: [kind_off[k], kind_off[k+1])
  const GridDev* grids;
  int64_t it;             // global iteration being computed (u_it -> u_it+1)
  double* partials;       // per item slot
  int32_t dtype;          // 0 = f64, 1 = f32
  int32_t stages;         // ring stages of the plane-streaming path
  int32_t smem;           // dynamic shared memory bytes (128 + stages * max stage)
  uint32_t* err;          // device error word (bounded waits)
  uint64_t wait_ns;
  const GridNorm* norms;  // per-grid emu_bad flags (FP64 only; may be null)
  int32_t emu;            // 1: FP64 pair sums may run on the integer pipe
  int32_t pad_;
};

// Streams and events that let the item kinds of one step run side by side:
// the kinds fork from the caller's stream and join it again before anything
// after the step (the next iteration reads their faces).  Under stream
// capture the fork becomes parallel branches of the graph.
struct KindFork {
  cudaStream_t aux[kItemKinds] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kItemKinds] = {};
};
cudaError_t kind_fork_create(KindFork* f);
void kind_fork_destroy(KindFork* f);

// Step kernels.  mode flags:
enum StepMode : int { kWrite = 1, kPack = 2, kResid = 4 };
// One step over a.items (grouped by kind at a.kind_off).  With `fork`, the
// kinds run concurrently; without it they run one after another on s.
cudaError_t launch_step(const StepLaunch& a, int mode, cudaStream_t s, const KindFork* fork = nullptr);

// Explicit exchange over the blocks ids[0..n_blocks): pack every internal
// face of the NEW iterate into its staging buffer (direct: straight into the
// neighbour's receive slot), or copy staging buffers into the neighbours'
// slots.
cudaError_t launch_pack_faces(const BlockDev* blocks, const int32_t* ids, int32_t n_blocks, void* const* staging,
                              const GridDev* grids, int64_t it, int32_t dtype, cudaStream_t s,
                              bool direct = false);
cudaError_t launch_copy_faces(const BlockDev* blocks, const int32_t* ids, int32_t n_blocks, void* const* staging,
                              const GridDev* grids, int64_t it, int32_t dtype, cudaStream_t s);

// One posted receive of the GPU Messaging form: copy `bytes` (a multiple of
// 16, both addresses 16-byte aligned) from src to dst.
struct CopyDesc {
  const void* src;
  void* dst;
  int64_t bytes;
};
cudaError_t launch_copy_desc(const CopyDesc* d, int32_t n, cudaStream_t s);

// Domain check of the integer-pipe FP64 adder (sets GridNorm::emu_bad) and
// its self-test.
cudaError_t launch_emu_check(const BlockDev* blocks, int32_t n_blocks, const GridDev* grids, GridNorm* norms,
                             const int32_t* grid_ids, int32_t n_grids, int64_t it, int dtype, cudaStream_t s);
cudaError_t launch_selftest_dadd(const double* a, const double* b, int64_t n, double* out, cudaStream_t s);
cudaError_t launch_selftest_widen(unsigned long long* bad, cudaStream_t s);
cudaError_t launch_selftest_div6(unsigned long long* bad, cudaStream_t s);
cudaError_t launch_pipe_rate(bool emu, int blocks, int threads, int iters, double* out, cudaStream_t s);

// |b|^2 partials (interior = 0, only Dirichlet ghosts).
cudaError_t launch_bnorm(const StepLaunch& a, cudaStream_t s);

// Sum partials per grid in a fixed order.  which = 0: r_norm2, 1: b_norm2.
cudaError_t launch_reduce(const GridDev* grids, GridNorm* norms, const int32_t* grid_ids, int32_t n,
                          const double* partials, int which, cudaStream_t s);

// Initial state: interiors of every block and every receive slot (parity 0
// for internal faces; the shared buffer for Dirichlet faces).
cudaError_t launch_init(const BlockDev* blocks, const BlockGeom* geom, int32_t n_blocks,
                        const InitDev* inits, int32_t dtype, cudaStream_t s);

// Scatter a padded device array of one grid into its blocks (parity p buffers
// and slots); gather the current iterate back (interior or padded layout).
cudaError_t launch_scatter(const BlockDev* blocks, const BlockGeom* geom, int32_t b0, int32_t nb,
                           const void* src, int64_t NX, int64_t NY, int64_t NZ, int parity,
                           int32_t dtype, cudaStream_t s);
cudaError_t launch_gather(const BlockDev* blocks, const BlockGeom* geom, int32_t b0, int32_t nb,
                          void* dst, int64_t NX, int64_t NY, int64_t NZ, int parity, int padded,
                          int32_t dtype, cudaStream_t s);

// Persistent path: one cooperative launch runs n_iters iterations.
struct PersistLaunch {
  const BlockDev* blocks;
  const WorkItem* items;       // active items, grouped by unit (block, z-chunk)
  const int32_t* unit_items;   // per active unit: first item index (n_units + 1 entries)
  const int32_t* unit_ids;     // per active unit: its unit id (index into progress)
  const int32_t* dep_off;      // per active unit: first dependency (n_units + 1 entries)
  const int32_t* dep_ids;      // unit ids that must have finished the previous iteration
  int32_t n_units;             // active units
  const GridDev* grids;
  int64_t it0;
  const int64_t* it0_dev;      // when set, the start iteration is read here (graph replays)
  int64_t n_iters;
  int64_t* progress;           // per unit: iterations completed (absolute)
  uint32_t* err;
  uint64_t wait_ns;
  double* partials;
  int32_t resid_first;         // fuse the residual of u_it0 into the first iteration
  int32_t dtype;
  int32_t stages;
  int32_t smem;
  const GridNorm* norms;       // per-grid emu_bad flags (FP64 only)
  int32_t emu;
  int32_t threads;             // barrier-driven kernel: CTA size 64, 128 or 256 (persistent_threads)
  int32_t ws_cw;               // > 0: the warp-specialised kernel with this many consumer warps
  int32_t stage_bytes;         // ring stage stride of the warp-specialised kernel (largest stage)
  unsigned long long* ticket;  // warp-specialised kernel: work counter, zero at launch
};
cudaError_t launch_persistent(const PersistLaunch& a, int grid_ctas, cudaStream_t s);
// Co-resident CTA limit of the persistent kernel for (threads, ws_cw) (0 on error).
int persistent_max_ctas(int dtype, int smem, int threads, int ws_cw = 0);
// Smallest persistent CTA (64, 128, 256 threads) that covers every item:
// 32 * CW threads for streamed items of CW consumer warps, 256 for tiles.
inline int persistent_threads(const WorkItem* items, size_t n) {
  int t = 64;
  for (size_t i = 0; i < n; ++i) t = std::max(t, items[i].x0 >= 0 ? 256 : 32 * (items[i].y0 & 15));
  return t;
}

}  // namespace jgb
