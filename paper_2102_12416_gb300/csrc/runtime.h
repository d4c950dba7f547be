// Host-side runtime structures of the Jacobi3D library (shared by the C-ABI
// translation units; not part of the public interface).
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/jacobi.h"
#include "common.cuh"
#include "kernels.cuh"

namespace jgb {

// Thread-local message of the last failing call.
int set_error(int code, const char* fmt, ...);
#define JGB_CUDA(call)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return ::jgb::set_error(JACOBI_ECUDA, "%s failed: %s (%s:%d)", #call,                 \
                              cudaGetErrorString(e_), __FILE__, __LINE__);                 \
  } while (0)

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct BlockHost {
  int64_t grid;
  int64_t origin[3], extent[3];
  int64_t nbr[6];
  int64_t item_begin, item_end;  // items of this block in the full list
  int64_t rx, ry;                // padded row pitch and rows per plane
  int64_t pitch;                 // elements per z-plane
  size_t u_off[2];
  size_t recv_off[6][2];
  size_t stage_off[6];           // explicit-path staging (internal faces only)
};

struct GridHost {
  jacobi_dim3 dims;
  jacobi_split split;
  jacobi_init init;
  int64_t counts[3];
  int64_t block_begin, block_end;
  int64_t item_begin, item_end;
  int64_t start_iter;    // global iteration at which the local count was 0
  int64_t frozen_local;  // local iteration held while inactive
  bool active;
};

// Decomposition + workspace layout of a set of grids.
struct Plan {
  int32_t dtype;
  size_t elem;
  std::vector<GridHost> grids;
  std::vector<BlockHost> blocks;
  std::vector<WorkItem> items;
  int64_t n_points = 0;
  int64_t halo_elems = 0;  // face elements moved per iteration (internal faces)
  uint32_t max_stage = 0;  // largest ring stage (bytes) of a plane-streamed block
  int64_t zchunk = 1;      // planes per z-chunk (the last chunk of a block may be shorter)
  int32_t cw_cap = 8;      // most consumer warps per streaming CTA (sets the row windows)
  int64_t n_units = 0;     // persistent-kernel units: (block, z-chunk) pairs
  int64_t cap_items = 0;   // item / unit table capacity in the workspace (the finest shape)
  int64_t cap_units = 0;
  // byte offsets into the workspace
  size_t off_blocks, off_geom, off_items, off_active, off_kind, off_grids, off_norms, off_inits, off_gids, off_partials,
      off_progress, off_err, off_stage_tab, off_punit_items, off_punit_ids, off_pdep_off, off_pdep_ids,
      off_active_blocks, off_it0, off_ticket;
  size_t off_stage_begin = 0, off_stage_end = 0;  // the explicit-path staging buffers, contiguous
  int64_t halo_faces = 0;                         // internal faces (one message each per iteration)
  size_t bytes = 0;
};

// With target_items <= 0 (a handle) the z-chunk comes from a cost model of
// waves, per-item pipeline fill and halo re-reads; with target_items > 0 it is
// the longest chunk that still gives that many items.  The server plans each
// request alone (so its result does not depend on the mix) with
// kServeTargetItems and z-chunks of at least kServeMinChunk planes: a request
// running alone still spreads over the GPU, while the halo planes each chunk
// re-reads stay a bounded share.
constexpr int64_t kServeTargetItems = 304;
constexpr int kMaxBlockExtent = JACOBI_MAX_BLOCK_EXTENT;
constexpr int64_t kServeMinChunk = 16;
int plan_build(int64_t n_grids, const jacobi_dim3* grids, const jacobi_split* splits, jacobi_dtype dtype,
               const jacobi_init* inits, Plan* out, int64_t target_items = 0, int64_t min_chunk = 1);
// Rebuild the work items of a built plan for another shape (z-chunk zc_req,
// 0 = the cost model's; at most cw_cap consumer warps per streaming CTA).
int plan_items(Plan* P, int64_t zc_req, int cw_cap, int64_t target_items, int64_t min_chunk);

// Device block table entries of a plan whose workspace starts at `ws`; block
// and neighbour ids are offset by `base`; grid_override >= 0 replaces every
// block's grid index.  stage_tab (nullable) receives the explicit-path staging
// buffers (6 per block).  local_halo aims every block's face stores at its own
// receive slots instead of its neighbours' (the halo-share measurement).
void fill_block_tables(const Plan& P, char* ws, int64_t base, int32_t grid_override, BlockDev* bd, BlockGeom* geo,
                       void** stage_tab, bool local_halo = false);

}  // namespace jgb

struct channel_s;

struct jacobi_s {
  jgb::Plan plan;
  int device = 0;
  char* ws = nullptr;
  bool own_ws = false;
  int32_t path = JACOBI_PATH_FUSED;
  int64_t iter = 0;  // global iterations completed

  // device tables (inside ws)
  jgb::BlockDev* d_blocks = nullptr;
  jgb::BlockGeom* d_geom = nullptr;
  jgb::WorkItem* d_items = nullptr;
  jgb::WorkItem* d_active = nullptr;
  jgb::WorkItem* d_kind = nullptr;
  jgb::GridDev* d_grids = nullptr;
  jgb::GridNorm* d_norms = nullptr;
  jgb::InitDev* d_inits = nullptr;
  int32_t* d_gids = nullptr;
  double* d_partials = nullptr;
  int64_t* d_progress = nullptr;
  uint32_t* d_err = nullptr;
  void** d_stage_tab = nullptr;
  int32_t* d_punit_items = nullptr;
  int32_t* d_punit_ids = nullptr;
  int32_t* d_pdep_off = nullptr;
  int32_t* d_pdep_ids = nullptr;
  int32_t* d_active_blocks = nullptr;  // blocks of the active grids (exchange kernels)
  int64_t* d_it0 = nullptr;            // start iteration of a replayed persistent graph
  unsigned long long* d_ticket = nullptr;  // work counter of the warp-specialised persistent kernel

  // host mirrors
  std::vector<jgb::WorkItem> active_items;
  // persistent kernel: active units (block, z-chunk) in item order, their item
  // ranges in active_items and their dependency lists (unit ids, CSR)
  std::vector<int32_t> active_units;        // unit ids
  std::vector<int32_t> active_unit_items;   // n_active_units + 1 offsets into active_items
  std::vector<int32_t> active_dep_off;      // n_active_units + 1 offsets into active_deps
  std::vector<int32_t> active_deps;
  std::vector<int32_t> active_grids;
  std::vector<int32_t> active_blocks;
  std::vector<jgb::WorkItem> kind_items;        // active items grouped by kind
  int32_t kind_off[jgb::kItemKinds + 1] = {};
  bool tables_dirty = true;
  jgb::GridDev* h_grids = nullptr;   // pinned, uploaded to d_grids
  jgb::GridNorm* h_norms = nullptr;  // pinned, read back from d_norms
  uint32_t* h_err = nullptr;        // pinned

  jgb::KindFork fork;             // side-by-side launch of the step's item kinds
  // CUDA graph of the fused path
  cudaGraphExec_t graph = nullptr;
  int64_t graph_iters = 0;
  int32_t graph_items = -1;
  // PERSISTENT path: the cooperative launch captured once per shape (without /
  // with the fused residual of the first iteration) and replayed; the start
  // iteration comes from d_it0
  struct PersistGraph {
    cudaGraphExec_t exec = nullptr;
    int64_t n_iters = 0;
    int32_t n_units = -1, stages = 0, ctas = 0, threads = 0, ws_cw = 0;
  } pgraph[2];
  bool persist_ws = true;         // warp-specialised persistent kernel where it applies
  bool pgraph_off = false;        // capture of the cooperative launch failed: launch directly

  uint64_t wait_ns = 1000000000ull;
  int32_t stages = 4;             // ring stages of the persistent kernel's plane streaming
  bool stages_fixed = false;      // set by JACOBI_STAGES or the autotuner (else large stages may take 5)
  int32_t fp64_emu = 1;           // FP64 pair sums on the integer pipe when safe
  int64_t drop_block = -1;        // fault injection (persistent path)
  bool local_halo = false;        // halo-share measurement: face stores stay in the block
  void* stage = nullptr;          // device staging for host transfers
  size_t stage_bytes = 0;
  // host-driven exchange forms (CHANNEL, MESSAGING, HOST_STAGED paths)
  void* h_halo = nullptr;                       // pinned copy of the staging region (HOST_STAGED)
  jgb::CopyDesc* d_desc = nullptr;              // posted receives of one exchange (MESSAGING)
  jgb::CopyDesc* h_desc = nullptr;              // pinned
  struct HaloMeta {                             // metadata message of one face (MESSAGING)
    const void* src;
    int64_t bytes;
    int32_t face;                               // the receiver's face the payload belongs to
  };
  std::vector<std::vector<HaloMeta>> mailbox;   // per receiving block
  std::vector<channel_s*> channels;
};
