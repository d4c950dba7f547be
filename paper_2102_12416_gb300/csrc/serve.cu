// Serving: continuous batching of independent Jacobi3D solves.
//
// The paper's Jacobi3D (Sec. 4.3) runs one problem at a time with a fixed
// iteration count; the server is this library's addition.  Requests wait in
// a FIFO queue; a background thread admits them, in arrival order, while a
// slot is free and the device bytes of the admitted grids stay below the HBM
// budget.  Every admitted grid lives in one set of device tables (blocks,
// work items, grids), so all of them advance in the same step launches.
// Scheduling happens in rounds of round_checks * check_every iterations:
// admissions and retirements happen between rounds, and every admitted grid
// starts at a round boundary, so its convergence checks fall on the first
// iteration of each check interval of every round.  At a check the step
// fuses the FP64 residual of the current iterate u_k, the per-grid reduction
// follows, and a decide kernel freezes the grid at u_k when it converged, hit
// its cap or stagnated, and records the outcome; frozen grids are skipped by
// the step kernels, so a round needs no host round trip.  A grid's blocks,
// items and residual summation order come from its own decomposition, so its
// result is bit-identical whether it runs alone or among others.
#include <time.h>

#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "runtime.h"

using namespace jgb;

namespace {

constexpr int kMaxSlotsLimit = 1024;
constexpr int64_t kBlocksPerSlot = 2048;
constexpr int64_t kItemsPerSlot = 16384;

int64_t now_ns() {
  timespec t;
  clock_gettime(CLOCK_MONOTONIC, &t);
  return (int64_t)t.tv_sec * 1000000000ll + t.tv_nsec;
}

// Request parameters and convergence state of one slot (device).
struct SlotDev {
  double tol;
  int64_t max_iters;
  int64_t stall_checks;
  double best;
  int64_t since;
};

// Outcome of one slot; status -1 while running.
struct Record {
  int32_t status;
  int32_t pad_;
  int64_t iters;
  double rel;
};

// After the residual of u_it has been reduced: decide per running grid.
__global__ void k_decide(GridDev* grids, const GridNorm* norms, SlotDev* sd, Record* rec, const int32_t* gids,
                         int n, int64_t it) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int g = gids[q];
  GridDev& G = grids[g];
  if (!G.active) return;
  SlotDev& S = sd[g];
  const int64_t k = it - G.start_iter;
  const double r = norms[g].rel;
  int st = -1;
  if (r <= S.tol) {
    st = JACOBI_SOLVE_CONVERGED;
  } else if (k >= S.max_iters) {
    st = JACOBI_SOLVE_MAX_ITERS;
  } else if (r < S.best) {
    S.best = r;
    S.since = 0;
  } else if (S.stall_checks > 0 && ++S.since >= S.stall_checks) {
    st = JACOBI_SOLVE_STAGNATED;
  }
  if (st >= 0) {
    G.active = 0;
    Record R;
    R.status = st;
    R.pad_ = 0;
    R.iters = k;
    R.rel = r;
    rec[g] = R;
  }
}

struct Req {
  uint64_t ticket;
  serve_request r;
};

struct Slot {
  bool used = false;
  uint64_t ticket = 0;
  Plan plan;
  char* ws = nullptr;
  int64_t block_base = 0;
  int64_t n_points = 0;
  void* out = nullptr;
};

}  // namespace

struct serve_s {
  serve_config cfg{};
  int device = 0;
  cudaStream_t stream = nullptr;
  KindFork fork;  // side-by-side launch of a step's item kinds
  // device tables
  char* dmem = nullptr;
  BlockDev* d_blocks = nullptr;
  BlockGeom* d_geom = nullptr;
  GridDev* d_grids = nullptr;
  GridNorm* d_norms = nullptr;
  InitDev* d_inits = nullptr;
  SlotDev* d_slotdev = nullptr;
  Record* d_rec = nullptr;
  WorkItem* d_slot_items = nullptr;  // per slot: its full item list
  WorkItem* d_kind = nullptr;        // running items grouped by kind
  double* d_partials = nullptr;
  int32_t* d_ids = nullptr;          // identity 0..max_slots-1
  int32_t* d_gids = nullptr;         // running slots
  uint32_t* d_err = nullptr;
  Record* h_rec = nullptr;
  // host state
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req> queue;
  std::unordered_map<uint64_t, serve_result> results;  // status -1: pending
  uint64_t next_ticket = 1;
  bool stop = false;
  int engine_error = JACOBI_OK;
  std::string engine_msg;
  std::vector<Slot> slots;
  std::thread th;
  uint64_t bytes_in_use = 0;
  uint32_t max_stage = 0;
  int32_t stages = 4;
  int64_t it = 0;
  serve_stats_t st{};
  std::vector<WorkItem> kind_items;
  int32_t kind_off[kItemKinds + 1] = {};
  std::vector<int32_t> running;
  bool dirty = true;
};

namespace {

int validate(const serve_s* s, const serve_request* r, Plan* plan) {
  if (!r) return set_error(JACOBI_EINVAL, "null request");
  if (!(r->tol >= 0.0)) return set_error(JACOBI_EINVAL, "tol must be >= 0");
  if (r->max_iters < 0 || r->max_iters % s->cfg.check_every)
    return set_error(JACOBI_EINVAL, "max_iters must be a non-negative multiple of check_every (%d)",
                     s->cfg.check_every);
  int rc = plan_build(1, &r->grid, &r->split, (jacobi_dtype)s->cfg.dtype, &r->init, plan, kServeTargetItems, kServeMinChunk);
  if (rc) return rc;
  if ((int64_t)plan->blocks.size() > kBlocksPerSlot || (int64_t)plan->items.size() > kItemsPerSlot)
    return set_error(JACOBI_EINVAL, "request has %zu blocks / %zu work items; a slot holds %lld / %lld",
                     plan->blocks.size(), plan->items.size(), (long long)kBlocksPerSlot, (long long)kItemsPerSlot);
  if (plan->bytes > s->cfg.hbm_budget_bytes)
    return set_error(JACOBI_EINVAL, "request needs %zu device bytes, more than the budget", plan->bytes);
  return JACOBI_OK;
}

#define ENG_CUDA(call)                                                                                   \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess) {                                                                             \
      return set_error(JACOBI_ECUDA, "serve engine: %s failed: %s", #call, cudaGetErrorString(e_));      \
    }                                                                                                    \
  } while (0)

// Admit the request at the head of the queue into slot `si` (queue lock held
// by the caller only for the pop).
int admit(serve_s* s, int si, const Req& q) {
  Slot& sl = s->slots[si];
  sl.used = true;
  sl.ticket = q.ticket;
  sl.out = q.r.out;
  int rc = plan_build(1, &q.r.grid, &q.r.split, (jacobi_dtype)s->cfg.dtype, &q.r.init, &sl.plan, kServeTargetItems, kServeMinChunk);
  if (rc) return rc;
  const Plan& P = sl.plan;
  ENG_CUDA(cudaMallocAsync((void**)&sl.ws, P.bytes, s->stream));
  s->bytes_in_use += P.bytes;
  s->max_stage = std::max(s->max_stage, P.max_stage);
  sl.block_base = (int64_t)si * kBlocksPerSlot;
  sl.n_points = P.n_points;
  const int64_t nb = (int64_t)P.blocks.size(), ni = (int64_t)P.items.size();
  std::vector<BlockDev> bd(nb);
  std::vector<BlockGeom> geo(nb);
  fill_block_tables(P, sl.ws, sl.block_base, si, bd.data(), geo.data(), nullptr);
  std::vector<WorkItem> items(P.items);
  for (int64_t k = 0; k < ni; ++k) {
    items[k].block += (int32_t)sl.block_base;
    items[k].slot = (int32_t)(si * kItemsPerSlot + k);
  }
  const GridHost& G = P.grids[0];
  GridDev gd{};
  gd.start_iter = s->it;
  gd.item_begin = (int32_t)(si * kItemsPerSlot);
  gd.item_end = (int32_t)(si * kItemsPerSlot + ni);
  gd.active = 1;
  InitDev ini{G.dims.nx, G.dims.ny, G.dims.nz, G.init.bc, G.init.interior, G.init.bc_seed, G.init.interior_seed,
              G.init.noise_amp};
  SlotDev sd{q.r.tol, q.r.max_iters, s->cfg.stall_checks, INFINITY, 0};
  Record rec{-1, 0, 0, 0.0};
  cudaStream_t st = s->stream;
  ENG_CUDA(cudaMemcpyAsync(s->d_blocks + sl.block_base, bd.data(), nb * sizeof(BlockDev), cudaMemcpyHostToDevice, st));
  ENG_CUDA(cudaMemcpyAsync(s->d_geom + sl.block_base, geo.data(), nb * sizeof(BlockGeom), cudaMemcpyHostToDevice, st));
  ENG_CUDA(cudaMemcpyAsync(s->d_slot_items + si * kItemsPerSlot, items.data(), ni * sizeof(WorkItem),
                           cudaMemcpyHostToDevice, st));
  ENG_CUDA(cudaMemcpyAsync(s->d_grids + si, &gd, sizeof gd, cudaMemcpyHostToDevice, st));
  ENG_CUDA(cudaMemcpyAsync(s->d_inits + si, &ini, sizeof ini, cudaMemcpyHostToDevice, st));
  ENG_CUDA(cudaMemcpyAsync(s->d_slotdev + si, &sd, sizeof sd, cudaMemcpyHostToDevice, st));
  ENG_CUDA(cudaMemcpyAsync(s->d_rec + si, &rec, sizeof rec, cudaMemcpyHostToDevice, st));
  ENG_CUDA(cudaMemsetAsync(sl.ws, 0, P.bytes, st));  // padding starts at zero
  ENG_CUDA(launch_init(s->d_blocks + sl.block_base, s->d_geom + sl.block_base, (int32_t)nb, s->d_inits,
                       s->cfg.dtype, st));
  StepLaunch a{};
  a.blocks = s->d_blocks;
  a.items = s->d_slot_items + si * kItemsPerSlot;
  a.n_items = (int32_t)ni;
  a.grids = s->d_grids;
  a.it = s->it;
  a.partials = s->d_partials;
  a.dtype = s->cfg.dtype;
  ENG_CUDA(launch_emu_check(s->d_blocks + sl.block_base, (int32_t)nb, s->d_grids, s->d_norms, s->d_ids + si, 1,
                            s->it, s->cfg.dtype, st));
  ENG_CUDA(launch_bnorm(a, st));
  ENG_CUDA(launch_reduce(s->d_grids, s->d_norms, s->d_ids + si, 1, s->d_partials, 1, st));
  // No synchronisation: a host-to-device cudaMemcpyAsync from pageable memory
  // returns once the source has been staged, so the vectors above may go.
  s->dirty = true;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->results[q.ticket].t_admit_ns = now_ns();
    s->st.admitted += 1;
  }
  return JACOBI_OK;
}

int rebuild_lists(serve_s* s) {
  s->running.clear();
  std::vector<WorkItem> all;
  for (int si = 0; si < (int)s->slots.size(); ++si) {
    const Slot& sl = s->slots[si];
    if (!sl.used) continue;
    s->running.push_back(si);
    for (size_t k = 0; k < sl.plan.items.size(); ++k) {
      WorkItem w = sl.plan.items[k];
      w.block += (int32_t)sl.block_base;
      w.slot = (int32_t)(si * kItemsPerSlot + (int64_t)k);
      all.push_back(w);
    }
  }
  s->kind_items.clear();
  for (int k = 0; k < kItemKinds; ++k) {
    s->kind_off[k] = (int32_t)s->kind_items.size();
    for (const WorkItem& w : all)
      if (item_kind(w) == k) s->kind_items.push_back(w);
  }
  s->kind_off[kItemKinds] = (int32_t)s->kind_items.size();
  if (!s->kind_items.empty())
    ENG_CUDA(cudaMemcpyAsync(s->d_kind, s->kind_items.data(), s->kind_items.size() * sizeof(WorkItem),
                             cudaMemcpyHostToDevice, s->stream));
  if (!s->running.empty())
    ENG_CUDA(cudaMemcpyAsync(s->d_gids, s->running.data(), s->running.size() * sizeof(int32_t),
                             cudaMemcpyHostToDevice, s->stream));
  ENG_CUDA(cudaStreamSynchronize(s->stream));
  s->dirty = false;
  return JACOBI_OK;
}

int run_round(serve_s* s) {
  StepLaunch a{};
  a.blocks = s->d_blocks;
  a.items = s->d_kind;
  a.n_items = (int32_t)s->kind_items.size();
  for (int k = 0; k <= kItemKinds; ++k) a.kind_off[k] = s->kind_off[k];
  a.grids = s->d_grids;
  a.partials = s->d_partials;
  a.dtype = s->cfg.dtype;
  a.stages = kStreamStages;
  a.smem = 128 + kStreamStages * (int32_t)s->max_stage;
  a.err = s->d_err;
  a.wait_ns = 1000000000ull;
  a.norms = s->d_norms;
  a.emu = 1;
  const int n = (int)s->running.size();
  for (int c = 0; c < s->cfg.round_checks; ++c) {
    a.it = s->it;
    ENG_CUDA(launch_step(a, kWrite | kPack | kResid, s->stream, &s->fork));
    ENG_CUDA(launch_reduce(s->d_grids, s->d_norms, s->d_gids, n, s->d_partials, 0, s->stream));
    k_decide<<<(n + 127) / 128, 128, 0, s->stream>>>(s->d_grids, s->d_norms, s->d_slotdev, s->d_rec, s->d_gids, n,
                                                       s->it);
    ENG_CUDA(cudaGetLastError());
    s->it += 1;
    for (int t = 1; t < s->cfg.check_every; ++t) {
      a.it = s->it;
      ENG_CUDA(launch_step(a, kWrite | kPack, s->stream, &s->fork));
      s->it += 1;
    }
  }
  s->st.rounds += 1;
  s->st.iterations = s->it;
  return JACOBI_OK;
}

int retire_finished(serve_s* s) {
  const size_t nslot = s->slots.size();
  uint32_t* h_err = (uint32_t*)(s->h_rec + nslot);  // the word after the records
  ENG_CUDA(cudaMemcpyAsync(s->h_rec, s->d_rec, nslot * sizeof(Record), cudaMemcpyDeviceToHost, s->stream));
  ENG_CUDA(cudaMemcpyAsync(h_err, s->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s->stream));
  ENG_CUDA(cudaStreamSynchronize(s->stream));
  // A bounded wait that gave up inside a step leaves that round's iterates
  // unreliable: stop the engine (pending requests then report the error).
  if (*h_err != DEV_OK)
    return set_error(JACOBI_ETIMEDOUT, "serve engine: a device-side wait gave up (code %u)", *h_err);
  for (int si : s->running) {
    Slot& sl = s->slots[si];
    const Record R = s->h_rec[si];
    if (R.status < 0) continue;
    if (sl.out) {
      const GridHost& G = sl.plan.grids[0];
      const size_t bytes = (size_t)G.dims.nx * G.dims.ny * G.dims.nz * sl.plan.elem;
      void* tmp = nullptr;
      ENG_CUDA(cudaMallocAsync(&tmp, bytes, s->stream));
      ENG_CUDA(launch_gather(s->d_blocks, s->d_geom, (int32_t)sl.block_base, (int32_t)sl.plan.blocks.size(), tmp,
                             G.dims.nx, G.dims.ny, G.dims.nz, (int)(R.iters & 1), 0, s->cfg.dtype, s->stream));
      ENG_CUDA(cudaMemcpyAsync(sl.out, tmp, bytes, cudaMemcpyDeviceToHost, s->stream));
      ENG_CUDA(cudaFreeAsync(tmp, s->stream));
      ENG_CUDA(cudaStreamSynchronize(s->stream));
    }
    ENG_CUDA(cudaFreeAsync(sl.ws, s->stream));
    s->bytes_in_use -= sl.plan.bytes;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      serve_result& res = s->results[sl.ticket];
      res.status = R.status;
      res.iters = R.iters;
      res.rel = R.rel;
      res.t_done_ns = now_ns();
      s->st.completed += 1;
      s->st.lups += sl.n_points * (R.iters + 1);
    }
    sl = Slot();
    s->dirty = true;
  }
  return JACOBI_OK;
}

int engine_loop(serve_s* s) {
  for (;;) {
    // admission
    for (;;) {
      Req q;
      int free_slot = -1;
      {
        std::unique_lock<std::mutex> lk(s->mu);
        if (s->stop) return JACOBI_OK;
        bool any_running = false;
        for (const Slot& sl : s->slots) any_running |= sl.used;
        if (s->queue.empty()) {
          if (!any_running) s->cv.wait_for(lk, std::chrono::milliseconds(2));
          break;
        }
        for (int si = 0; si < (int)s->slots.size(); ++si)
          if (!s->slots[si].used) {
            free_slot = si;
            break;
          }
        if (free_slot < 0) break;
        Plan probe;
        const serve_request& r = s->queue.front().r;
        if (plan_build(1, &r.grid, &r.split, (jacobi_dtype)s->cfg.dtype, &r.init, &probe, kServeTargetItems, kServeMinChunk)) break;
        if (s->bytes_in_use + probe.bytes > s->cfg.hbm_budget_bytes) break;
        q = s->queue.front();
        s->queue.pop_front();
        s->st.queued = (int64_t)s->queue.size();
      }
      int rc = admit(s, free_slot, q);
      if (rc) return rc;
    }
    bool any = false;
    for (const Slot& sl : s->slots) any |= sl.used;
    if (!any) continue;
    if (s->dirty) {
      int rc = rebuild_lists(s);
      if (rc) return rc;
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->st.running = (int64_t)s->running.size();
    }
    int rc = run_round(s);
    if (rc) return rc;
    rc = retire_finished(s);
    if (rc) return rc;
  }
}

void engine_main(serve_s* s) {
  cudaSetDevice(s->device);
  const int rc = engine_loop(s);
  if (rc) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->engine_error = rc;
    s->engine_msg = jacobi_last_error();
  }
}

}  // namespace

extern "C" {

int serve_create(const serve_config* cfg, serve_t** out) {
  if (!cfg || !out) return set_error(JACOBI_EINVAL, "null argument");
  *out = nullptr;
  if (cfg->max_slots < 1 || cfg->max_slots > kMaxSlotsLimit || cfg->check_every < 1 || cfg->round_checks < 1 ||
      (cfg->dtype != JACOBI_F64 && cfg->dtype != JACOBI_F32) || cfg->hbm_budget_bytes == 0)
    return set_error(JACOBI_EINVAL, "bad serve_config");
  serve_s* s = new (std::nothrow) serve_s();
  if (!s) return set_error(JACOBI_ENOMEM, "host allocation failed");
  s->cfg = *cfg;
  s->slots.resize(cfg->max_slots);
  s->stages = 4;
  const int64_t ns = cfg->max_slots;
  size_t off = 0;
  auto take = [&](size_t b) { size_t o = off; off = align_up(off + b, 256); return o; };
  const size_t o_blocks = take(ns * kBlocksPerSlot * sizeof(BlockDev));
  const size_t o_geom = take(ns * kBlocksPerSlot * sizeof(BlockGeom));
  const size_t o_grids = take(ns * sizeof(GridDev));
  const size_t o_norms = take(ns * sizeof(GridNorm));
  const size_t o_inits = take(ns * sizeof(InitDev));
  const size_t o_sd = take(ns * sizeof(SlotDev));
  const size_t o_rec = take(ns * sizeof(Record));
  const size_t o_sitems = take(ns * kItemsPerSlot * sizeof(WorkItem));
  const size_t o_kind = take(ns * kItemsPerSlot * sizeof(WorkItem));
  const size_t o_part = take(ns * kItemsPerSlot * sizeof(double));
  const size_t o_ids = take(ns * sizeof(int32_t));
  const size_t o_gids = take(ns * sizeof(int32_t));
  const size_t o_err = take(64);
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = kind_fork_create(&s->fork);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->dmem, off);
  if (e == cudaSuccess) e = cudaMemset(s->dmem, 0, off);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&s->h_rec, ns * sizeof(Record) + 64);  // + the error word
  if (e != cudaSuccess) {
    if (s->dmem) cudaFree(s->dmem);
    if (s->h_rec) cudaFreeHost(s->h_rec);
    kind_fork_destroy(&s->fork);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return set_error(JACOBI_ENOMEM, "serve_create: %s", cudaGetErrorString(e));
  }
  s->d_blocks = (BlockDev*)(s->dmem + o_blocks);
  s->d_geom = (BlockGeom*)(s->dmem + o_geom);
  s->d_grids = (GridDev*)(s->dmem + o_grids);
  s->d_norms = (GridNorm*)(s->dmem + o_norms);
  s->d_inits = (InitDev*)(s->dmem + o_inits);
  s->d_slotdev = (SlotDev*)(s->dmem + o_sd);
  s->d_rec = (Record*)(s->dmem + o_rec);
  s->d_slot_items = (WorkItem*)(s->dmem + o_sitems);
  s->d_kind = (WorkItem*)(s->dmem + o_kind);
  s->d_partials = (double*)(s->dmem + o_part);
  s->d_ids = (int32_t*)(s->dmem + o_ids);
  s->d_gids = (int32_t*)(s->dmem + o_gids);
  s->d_err = (uint32_t*)(s->dmem + o_err);
  std::vector<int32_t> ids(ns);
  for (int64_t q = 0; q < ns; ++q) ids[q] = (int32_t)q;
  e = cudaMemcpy(s->d_ids, ids.data(), ns * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(s->dmem);
    cudaFreeHost(s->h_rec);
    kind_fork_destroy(&s->fork);
    cudaStreamDestroy(s->stream);
    delete s;
    return set_error(JACOBI_ECUDA, "serve_create: %s", cudaGetErrorString(e));
  }
  s->th = std::thread(engine_main, s);
  *out = s;
  return JACOBI_OK;
}

int serve_submit(serve_t* s, const serve_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return set_error(JACOBI_EINVAL, "null argument");
  Plan probe;
  int rc = validate(s, req, &probe);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->engine_error) return set_error(s->engine_error, "serve engine stopped: %s", s->engine_msg.c_str());
  Req q{s->next_ticket++, *req};
  serve_result res{};
  res.status = -1;
  res.t_arrive_ns = now_ns();
  s->results[q.ticket] = res;
  s->queue.push_back(q);
  s->st.submitted += 1;
  s->st.queued = (int64_t)s->queue.size();
  *ticket = q.ticket;
  s->cv.notify_one();
  return JACOBI_OK;
}

int serve_poll(serve_t* s, uint64_t ticket, serve_result* result) {
  if (!s || !result) return set_error(JACOBI_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->results.find(ticket);
  if (it == s->results.end()) return set_error(JACOBI_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
  *result = it->second;
  if (it->second.status >= 0) return JACOBI_OK;
  if (s->engine_error) return set_error(s->engine_error, "serve engine stopped: %s", s->engine_msg.c_str());
  return JACOBI_EAGAIN;
}

int serve_stats(serve_t* s, serve_stats_t* out) {
  if (!s || !out) return set_error(JACOBI_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->bytes_in_use = s->bytes_in_use;
  return JACOBI_OK;
}

int serve_destroy(serve_t* s) {
  if (!s) return JACOBI_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();
  cudaStreamSynchronize(s->stream);
  for (Slot& sl : s->slots)
    if (sl.used && sl.ws) cudaFreeAsync(sl.ws, s->stream);
  cudaStreamSynchronize(s->stream);
  cudaFree(s->dmem);
  cudaFreeHost(s->h_rec);
  kind_fork_destroy(&s->fork);
  cudaStreamDestroy(s->stream);
  delete s;
  return JACOBI_OK;
}

}  // extern "C"
