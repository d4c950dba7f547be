// C ABI of the Jacobi3D library: decomposition (Sec. 4.3: equal-size cuboid
// blocks that minimise surface area), workspace planning, handle lifecycle,
// the step paths, residual / solve and state transfer.  Every numeric step
// runs in the kernels of kernels.cu; this file only plans, uploads tables and
// launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "runtime.h"

using namespace jgb;

namespace jgb {

static thread_local std::string g_last_error;

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

// Per-axis (origin, extent) of a split.
static int axis_split(int64_t n, int32_t mode, int64_t param, std::vector<std::pair<int64_t, int64_t>>* out) {
  out->clear();
  if (n < 1 || param < 1) return set_error(JACOBI_EINVAL, "grid and split sizes must be positive");
  if (mode == JACOBI_SPLIT_SHAPE) {
    for (int64_t o = 0; o < n; o += param) out->push_back({o, std::min(param, n - o)});
  } else if (mode == JACOBI_SPLIT_COUNT) {
    if (param > n) return set_error(JACOBI_EINVAL, "more blocks (%lld) than points (%lld) on an axis",
                                    (long long)param, (long long)n);
    const int64_t q = n / param, r = n % param;
    int64_t o = 0;
    for (int64_t b = 0; b < param; ++b) {
      const int64_t e = q + (b < r ? 1 : 0);
      out->push_back({o, e});
      o += e;
    }
  } else {
    return set_error(JACOBI_EINVAL, "unknown split mode %d", mode);
  }
  return JACOBI_OK;
}

// Consumer warps per CTA for the plane-streaming path, or 0 when a padded
// row is wider than one CTA can cover (more than 256 vectors of 16 bytes).
// Each consumer thread computes 4 rows of one vector column; a CTA of CW
// consumer warps (2, 4 or 8: the smallest that covers the padded plane, at
// most cw_cap, but never fewer than one row of vector columns needs) covers a
// window of `chunk` rows (a multiple of 4), so large planes are split into
// ceil(ry / chunk) windows and small ones run in small CTAs, several per SM.
// A ring stage of a window must fit shared memory four times over.
static int stream_shape(int64_t rx, int64_t ry, size_t elem, int cw_cap, uint32_t* stage_bytes, int64_t* chunk) {
  const int64_t txv = rx / (16 / (int64_t)elem);
  if (txv > kThreads) return 0;
  int cw = 8;
  for (int c = 2; c <= 8; c *= 2)
    if (txv * (ry / 4) <= 32 * c) {
      cw = c;
      break;
    }
  cw = std::min(cw, cw_cap);
  while (32 * cw < txv) cw *= 2;
  int64_t ch = (32 * cw / txv) * 4;
  if (ch <= 0) return 0;
  ch = std::min(ch, ry);
  const uint64_t stage = ((uint64_t)((ch + 2) * rx + 2 * ch + 2 * rx) * elem + 127) / 128 * 128;
  if (128 + kStreamStages * stage > (uint64_t)kMaxStepSmem) return 0;
  *stage_bytes = (uint32_t)stage;
  *chunk = ch;
  return cw;
}

// CTAs of one streaming kind resident per SM: registers are capped at 72 per
// thread by the launch bounds; the ring (4 stages of the largest window)
// takes shared memory.
static int64_t stream_ctas_per_sm(int cw, uint32_t stage_bytes) {
  const int64_t threads = 32 * cw + 32;
  const int64_t by_regs = 65536 / (threads * 72);
  const int64_t by_smem = (228 * 1024) / (128 + 4 * (int64_t)stage_bytes + 1024);
  return std::max<int64_t>(1, std::min<int64_t>({by_regs, by_smem, 32}));
}

static int64_t device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
      sms > 0)
    return sms;
  cudaGetLastError();
  return 152;
}

// z-chunk of a handle's work items by a cost model: a launch takes
// ceil(items / C) waves of C resident CTAs, each item costs its planes plus a
// fixed pipeline fill of ~2 planes, and in FP32 (bound by memory, not by
// arithmetic) each chunk's two re-read halo planes cost about one plane of
// traffic.  C counts the CTAs of the kind with the most units.  Candidates
// halve from the tallest block down to zmin planes; ties keep the longer chunk.
// FP32 chunks start at 32 planes at most: on 768^3 in 64^3 blocks, 64-plane
// chunks measured ~2 % slower than 32 although the model prefers them.
static int64_t choose_chunk(const Plan& P, const std::vector<int>& warps, const std::vector<int64_t>& chunks,
                            int64_t maxz, int64_t zmin) {
  int64_t kind_units[4] = {0, 0, 0, 0};  // tiles, CW 8, 4, 2
  for (size_t b = 0; b < P.blocks.size(); ++b) {
    const BlockHost& B = P.blocks[b];
    const int cw = warps[b];
    const int k = cw == 0 ? 0 : cw == 8 ? 1 : cw == 4 ? 2 : 3;
    kind_units[k] += cw ? (B.ry + chunks[b] - 1) / chunks[b] : ((B.extent[0] + TX - 1) / TX) * ((B.extent[1] + TY - 1) / TY);
  }
  const int k = (int)(std::max_element(kind_units, kind_units + 4) - kind_units);
  const int64_t per_sm = k == 0 ? 8 : stream_ctas_per_sm(k == 1 ? 8 : k == 2 ? 4 : 2, P.max_stage);
  const int64_t C = device_sms() * per_sm;
  const double halo = P.dtype == JACOBI_F32 ? 1.0 : 0.0;
  const int64_t z0 = P.dtype == JACOBI_F32 ? std::max<int64_t>(std::min<int64_t>(maxz, 32), zmin) : maxz;
  int64_t best = z0;
  double best_cost = 0.0;
  for (int64_t zc = z0;; zc = (zc + 1) / 2) {
    int64_t items = 0;
    for (size_t b = 0; b < P.blocks.size(); ++b) {
      const BlockHost& B = P.blocks[b];
      const int64_t per_plane = warps[b] ? (B.ry + chunks[b] - 1) / chunks[b]
                                         : ((B.extent[0] + TX - 1) / TX) * ((B.extent[1] + TY - 1) / TY);
      items += per_plane * ((B.extent[2] + zc - 1) / zc);
    }
    const double waves = (double)((items + C - 1) / C);
    const double cost = waves * ((double)zc + 2.0) * (1.0 + halo / (double)zc);
    if (zc == z0 || cost < best_cost) {
      best = zc;
      best_cost = cost;
    }
    if (zc <= zmin || (zc + 1) / 2 < zmin) break;
  }
  return best;
}

// Entries of the padded receive slot of face f (see BlockDev), and of the
// face itself.
static int64_t face_elems_host(const BlockHost& b, int f) {
  if (f < 2) return b.ry * b.extent[2];
  if (f < 4) return b.rx * b.extent[2];
  return b.rx * b.ry;
}
static int64_t face_points_host(const BlockHost& b, int f) {
  if (f < 2) return b.extent[1] * b.extent[2];
  if (f < 4) return b.extent[0] * b.extent[2];
  return b.extent[0] * b.extent[1];
}

// Work items of a plan's blocks for one shape.  Blocks that fit the
// plane-streaming path get one item per row window and z-chunk; the others
// one item per TX x TY tile and z-chunk.  The chunk is a power-of-two fraction
// of the tallest block: zc_req (> 0, clamped to the tallest block), else the
// cost model's choice (choose_chunk) for a handle, or the longest that still
// gives at least `target_items` items (down to min_chunk planes, at least 2).
int plan_items(Plan* P, int64_t zc_req, int cw_cap, int64_t target_items, int64_t min_chunk) {
  std::vector<int> warps(P->blocks.size());
  std::vector<int64_t> chunks(P->blocks.size());
  int64_t units = 0, maxz = 0;
  P->max_stage = 0;
  for (size_t b = 0; b < P->blocks.size(); ++b) {
    BlockHost& B = P->blocks[b];
    uint32_t sb = 0;
    int64_t ch = 0;
    const int cw = cw_cap > 0 ? stream_shape(B.rx, B.ry, P->elem, cw_cap, &sb, &ch) : 0;  // 0: tiles
    warps[b] = cw;
    chunks[b] = ch;
    if (cw) P->max_stage = std::max(P->max_stage, sb);
    units += cw ? (B.ry + ch - 1) / ch : ((B.extent[0] + TX - 1) / TX) * ((B.extent[1] + TY - 1) / TY);
    maxz = std::max(maxz, B.extent[2]);
  }
  // the cost model may go down to single planes (a small problem that fits
  // one wave); the item-target rule stops at 2
  const int64_t zmin = std::max<int64_t>(min_chunk, target_items > 0 ? 2 : 1);
  int64_t zc = maxz;
  if (zc_req > 0) {
    zc = std::min(zc_req, maxz);
  } else if (target_items > 0) {
    while (zc > zmin && (zc + 1) / 2 >= zmin && units * ((maxz + zc - 1) / zc) < target_items) zc = (zc + 1) / 2;
  } else {
    zc = choose_chunk(*P, warps, chunks, maxz, zmin);
  }
  P->zchunk = zc;
  P->cw_cap = cw_cap;
  P->n_units = 0;
  for (const BlockHost& B : P->blocks) P->n_units += (B.extent[2] + zc - 1) / zc;
  P->items.clear();
  for (GridHost& G : P->grids) {
    G.item_begin = (int64_t)P->items.size();
    for (int64_t b = G.block_begin; b < G.block_end; ++b) {
      BlockHost& B = P->blocks[b];
      const int cw = warps[b];
      B.item_begin = (int64_t)P->items.size();
      for (int64_t z0 = 0; z0 < B.extent[2]; z0 += zc) {
        WorkItem w;
        w.block = (int32_t)b;
        w.z0 = (int16_t)z0;
        w.z1 = (int16_t)std::min(B.extent[2], z0 + zc);
        w.ya = w.yb = 0;
        if (cw) {
          for (int64_t ya = 0; ya < B.ry; ya += chunks[b]) {
            w.slot = (int32_t)P->items.size();
            w.x0 = -1;
            w.y0 = (int16_t)(cw | (B.rx != B.extent[0] || B.ry != B.extent[1] ? kItemRagged : 0));
            w.ya = (int16_t)ya;
            w.yb = (int16_t)std::min(B.ry, ya + chunks[b]);
            P->items.push_back(w);
          }
          continue;
        }
        for (int64_t y0 = 0; y0 < B.extent[1]; y0 += TY)
          for (int64_t x0 = 0; x0 < B.extent[0]; x0 += TX) {
            w.slot = (int32_t)P->items.size();
            w.x0 = (int16_t)x0;
            w.y0 = (int16_t)y0;
            P->items.push_back(w);
          }
      }
      B.item_end = (int64_t)P->items.size();
    }
    G.item_end = (int64_t)P->items.size();
  }
  return JACOBI_OK;
}

int plan_build(int64_t n_grids, const jacobi_dim3* grids, const jacobi_split* splits, jacobi_dtype dtype,
               const jacobi_init* inits, Plan* P, int64_t target_items, int64_t min_chunk) {
  if (n_grids < 1 || !grids || !splits) return set_error(JACOBI_EINVAL, "need at least one grid");
  if (dtype != JACOBI_F64 && dtype != JACOBI_F32) return set_error(JACOBI_EINVAL, "bad dtype %d", (int)dtype);
  *P = Plan();
  P->dtype = dtype;
  P->elem = dtype == JACOBI_F64 ? 8 : 4;
  const size_t A = 256;
  for (int64_t g = 0; g < n_grids; ++g) {
    const jacobi_dim3 d = grids[g];
    if (d.nx < 1 || d.ny < 1 || d.nz < 1 || d.nx > (1ll << 30) || d.ny > (1ll << 30) || d.nz > (1ll << 30))
      return set_error(JACOBI_EINVAL, "grid %lld: bad size %lldx%lldx%lld", (long long)g, (long long)d.nx,
                       (long long)d.ny, (long long)d.nz);
    std::vector<std::pair<int64_t, int64_t>> ax[3];
    const int64_t n3[3] = {d.nx, d.ny, d.nz};
    const int64_t s3[3] = {splits[g].x, splits[g].y, splits[g].z};
    for (int a = 0; a < 3; ++a) {
      int rc = axis_split(n3[a], splits[g].mode, s3[a], &ax[a]);
      if (rc) return rc;
      for (auto& pe : ax[a])
        // work items hold block coordinates in 16 bits, padded extents
        // included (rows are padded to a multiple of 4)
        if (pe.second > kMaxBlockExtent)
          return set_error(JACOBI_EINVAL, "block extent %lld exceeds %d", (long long)pe.second, kMaxBlockExtent);
    }
    GridHost G;
    G.dims = d;
    G.split = splits[g];
    if (inits) {
      G.init = inits[g];
    } else {
      G.init = jacobi_init{JACOBI_BC_LINEAR, JACOBI_INTERIOR_ZERO, 0, 0, 0.0};
    }
    if (G.init.bc < 0 || G.init.bc > 2 || G.init.interior < 0 || G.init.interior > 2)
      return set_error(JACOBI_EINVAL, "grid %lld: bad init", (long long)g);
    G.counts[0] = (int64_t)ax[0].size();
    G.counts[1] = (int64_t)ax[1].size();
    G.counts[2] = (int64_t)ax[2].size();
    G.block_begin = (int64_t)P->blocks.size();
    G.start_iter = 0;
    G.frozen_local = 0;
    G.active = true;
    const int64_t px = G.counts[0], py = G.counts[1], pz = G.counts[2];
    for (int64_t bz = 0; bz < pz; ++bz)
      for (int64_t by = 0; by < py; ++by)
        for (int64_t bx = 0; bx < px; ++bx) {
          BlockHost B{};
          B.grid = g;
          B.origin[0] = ax[0][bx].first; B.extent[0] = ax[0][bx].second;
          B.origin[1] = ax[1][by].first; B.extent[1] = ax[1][by].second;
          B.origin[2] = ax[2][bz].first; B.extent[2] = ax[2][bz].second;
          auto id = [&](int64_t x, int64_t y, int64_t z) { return G.block_begin + (z * py + y) * px + x; };
          B.nbr[XM] = bx > 0 ? id(bx - 1, by, bz) : -1;
          B.nbr[XP] = bx + 1 < px ? id(bx + 1, by, bz) : -1;
          B.nbr[YM] = by > 0 ? id(bx, by - 1, bz) : -1;
          B.nbr[YP] = by + 1 < py ? id(bx, by + 1, bz) : -1;
          B.nbr[ZM] = bz > 0 ? id(bx, by, bz - 1) : -1;
          B.nbr[ZP] = bz + 1 < pz ? id(bx, by, bz + 1) : -1;
          P->blocks.push_back(B);
        }
    G.block_end = (int64_t)P->blocks.size();
    if (G.block_end > (1ll << 30)) return set_error(JACOBI_EINVAL, "too many blocks");
    P->n_points += d.nx * d.ny * d.nz;
    P->grids.push_back(G);
  }
  // padded rows (a whole number of 16-byte vectors) and planes (of 4-row groups)
  const int64_t vec = 16 / (int64_t)P->elem;
  for (BlockHost& B : P->blocks) {
    B.rx = (B.extent[0] + vec - 1) / vec * vec;
    B.ry = (B.extent[1] + 3) / 4 * 4;
  }
  int rc = plan_items(P, 0, 8, target_items, min_chunk);
  if (rc) return rc;
  // Table capacity: the item and unit tables are sized for the finest shapes
  // jacobi_set_shape accepts and the autotuner tries (z-chunks down to a
  // quarter of the planned one, CTAs down to 2 consumer warps, or tiles), so a
  // handle can be re-planned in place; states and slots never move.
  P->cap_items = (int64_t)P->items.size();
  P->cap_units = P->n_units;
  if (target_items <= 0) {
    for (int cw : {2, 0}) {
      Plan probe = *P;
      rc = plan_items(&probe, std::max<int64_t>(1, P->zchunk / 4), cw, 0, 1);
      if (rc) return rc;
      P->cap_items = std::max(P->cap_items, (int64_t)probe.items.size());
      P->cap_units = std::max(P->cap_units, probe.n_units);
    }
  }
  if (P->cap_items > (1ll << 30)) return set_error(JACOBI_EINVAL, "too many work items");
  const int64_t nb = (int64_t)P->blocks.size(), ni = P->cap_items, ng = n_grids;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, A); return o; };
  P->off_blocks = take(nb * sizeof(BlockDev));
  P->off_geom = take(nb * sizeof(BlockGeom));
  P->off_items = take(ni * sizeof(WorkItem));
  P->off_active = take(ni * sizeof(WorkItem));
  P->off_kind = take(ni * sizeof(WorkItem));
  P->off_grids = take(ng * sizeof(GridDev));
  P->off_norms = take(ng * sizeof(GridNorm));
  P->off_inits = take(ng * sizeof(InitDev));
  P->off_gids = take(ng * sizeof(int32_t));
  P->off_partials = take(ni * sizeof(double));
  const int64_t nu = P->cap_units;
  P->off_progress = take(nu * sizeof(int64_t));
  P->off_err = take(64);
  P->off_stage_tab = take(nb * 6 * sizeof(void*));
  P->off_punit_items = take((nu + 1) * sizeof(int32_t));
  P->off_punit_ids = take(nu * sizeof(int32_t));
  P->off_pdep_off = take((nu + 1) * sizeof(int32_t));
  P->off_pdep_ids = take(8 * nu * sizeof(int32_t));
  P->off_active_blocks = take(nb * sizeof(int32_t));
  P->off_it0 = take(sizeof(int64_t));
  P->off_ticket = take(sizeof(unsigned long long));
  const size_t per16 = 32;  // plane pitch rounded to 32 elements
  for (auto& B : P->blocks) {
    B.pitch = (int64_t)align_up((size_t)(B.rx * B.ry), per16);
    const size_t sb = (size_t)B.pitch * B.extent[2] * P->elem;
    B.u_off[0] = take(sb);
    B.u_off[1] = take(sb);
  }
  for (auto& B : P->blocks) {
    for (int f = 0; f < 6; ++f) {
      const size_t fb = (size_t)face_elems_host(B, f) * P->elem;
      if (B.nbr[f] >= 0) {
        B.recv_off[f][0] = take(fb);
        B.recv_off[f][1] = take(fb);
        P->halo_elems += face_points_host(B, f);
        P->halo_faces += 1;
      } else {
        B.recv_off[f][0] = B.recv_off[f][1] = take(fb);
      }
    }
  }
  P->off_stage_begin = off;
  for (auto& B : P->blocks)
    for (int f = 0; f < 6; ++f)
      B.stage_off[f] = B.nbr[f] >= 0 ? take((size_t)face_elems_host(B, f) * P->elem) : 0;
  P->off_stage_end = off;
  P->bytes = off;
  return JACOBI_OK;
}

void fill_block_tables(const Plan& P, char* ws, int64_t base, int32_t grid_override, BlockDev* bd, BlockGeom* geo,
                       void** stage_tab, bool local_halo) {
  const int64_t nb = (int64_t)P.blocks.size();
  for (int64_t b = 0; b < nb; ++b) {
    const BlockHost& B = P.blocks[b];
    BlockDev& D = bd[b];
    memset(&D, 0, sizeof D);
    D.u[0] = ws + B.u_off[0];
    D.u[1] = ws + B.u_off[1];
    for (int f = 0; f < 6; ++f) {
      D.recv[f][0] = ws + B.recv_off[f][0];
      D.recv[f][1] = ws + B.recv_off[f][1];
      D.nbr[f] = B.nbr[f] >= 0 ? (int32_t)(base + B.nbr[f]) : -1;
      if (B.nbr[f] >= 0) {
        const BlockHost& N = P.blocks[B.nbr[f]];
        // (the own slot of face f has the same shape as the neighbour's slot
        // of the opposite face: both span the face the blocks share)
        D.send[f][0] = ws + (local_halo ? B.recv_off[f][0] : N.recv_off[opposite(f)][0]);
        D.send[f][1] = ws + (local_halo ? B.recv_off[f][1] : N.recv_off[opposite(f)][1]);
        if (stage_tab) stage_tab[b * 6 + f] = ws + B.stage_off[f];
      }
    }
    D.nx = (int32_t)B.extent[0];
    D.ny = (int32_t)B.extent[1];
    D.nz = (int32_t)B.extent[2];
    D.grid = grid_override >= 0 ? grid_override : (int32_t)B.grid;
    D.plane_pitch = B.pitch;
    D.rx = (int32_t)B.rx;
    D.ry = (int32_t)B.ry;
    geo[b] = BlockGeom{(int32_t)B.origin[0], (int32_t)B.origin[1], (int32_t)B.origin[2], D.grid};
  }
}

}  // namespace jgb

// ---------------------------------------------------------------------------
// internal helpers
// ---------------------------------------------------------------------------
namespace {

cudaStream_t S(void* s) { return (cudaStream_t)s; }

int upload_tables(jacobi_t* h, cudaStream_t s) {
  const Plan& P = h->plan;
  const int64_t nb = (int64_t)P.blocks.size();
  std::vector<BlockDev> bd(nb);
  std::vector<BlockGeom> geo(nb);
  std::vector<void*> stab(nb * 6, nullptr);
  fill_block_tables(P, h->ws, 0, -1, bd.data(), geo.data(), stab.data(), h->local_halo);
  const int64_t ng = (int64_t)P.grids.size();
  std::vector<InitDev> ini(ng);
  std::vector<int32_t> gids(ng);
  for (int64_t g = 0; g < ng; ++g) {
    const GridHost& G = P.grids[g];
    ini[g] = InitDev{G.dims.nx, G.dims.ny, G.dims.nz, G.init.bc, G.init.interior, G.init.bc_seed,
                     G.init.interior_seed, G.init.noise_amp};
    gids[g] = (int32_t)g;
    GridDev& D = h->h_grids[g];
    D.start_iter = G.start_iter;
    D.active = 1;
    D.pad_ = 0;
    D.item_begin = (int32_t)G.item_begin;
    D.item_end = (int32_t)G.item_end;
  }
  JGB_CUDA(cudaMemcpyAsync(h->d_blocks, bd.data(), nb * sizeof(BlockDev), cudaMemcpyHostToDevice, s));
  JGB_CUDA(cudaMemcpyAsync(h->d_geom, geo.data(), nb * sizeof(BlockGeom), cudaMemcpyHostToDevice, s));
  JGB_CUDA(cudaMemcpyAsync(h->d_items, P.items.data(), P.items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, s));
  JGB_CUDA(cudaMemcpyAsync(h->d_inits, ini.data(), ng * sizeof(InitDev), cudaMemcpyHostToDevice, s));
  JGB_CUDA(cudaMemcpyAsync(h->d_gids, gids.data(), ng * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  JGB_CUDA(cudaMemcpyAsync(h->d_stage_tab, stab.data(), stab.size() * sizeof(void*), cudaMemcpyHostToDevice, s));
  JGB_CUDA(cudaMemcpyAsync(h->d_grids, h->h_grids, ng * sizeof(GridDev), cudaMemcpyHostToDevice, s));
  JGB_CUDA(cudaMemsetAsync(h->d_norms, 0, ng * sizeof(GridNorm), s));
  JGB_CUDA(cudaMemsetAsync(h->d_progress, 0, P.n_units * sizeof(int64_t), s));
  JGB_CUDA(cudaMemsetAsync(h->d_err, 0, 64, s));
  // The host arrays above are pageable, so each copy has been staged before
  // cudaMemcpyAsync returned; they may go out of scope now.
  return JACOBI_OK;
}

// Rebuild the active item / block lists from the grids' active flags.
int refresh_active(jacobi_t* h, cudaStream_t s) {
  if (!h->tables_dirty) return JACOBI_OK;
  if (h->graph) {  // the captured launches bake in the old lists
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  const Plan& P = h->plan;
  h->active_items.clear();
  h->active_units.clear();
  h->active_unit_items.clear();
  h->active_dep_off.clear();
  h->active_deps.clear();
  h->active_grids.clear();
  h->active_blocks.clear();
  // Persistent-kernel units: the z-chunks of each block (items are ordered by
  // z-chunk within a block).  Unit (b, c) at iteration it needs iteration
  // it - 1 finished by the units it shares data with, both ways (reads of
  // what they write, writes of what they read): chunks c - 1 and c + 1 of b
  // (halo planes), chunk c of the x and y neighbours (faces over the same
  // planes; blocks side by side share nz, hence the chunking) and the facing
  // chunk of the z neighbours.  The relation is symmetric.
  std::vector<int64_t> unit0(P.blocks.size() + 1, 0);
  for (size_t b = 0; b < P.blocks.size(); ++b)
    unit0[b + 1] = unit0[b] + (P.blocks[b].extent[2] + P.zchunk - 1) / P.zchunk;
  auto chunks = [&](int64_t b) { return unit0[b + 1] - unit0[b]; };
  for (size_t g = 0; g < P.grids.size(); ++g) {
    const GridHost& G = P.grids[g];
    if (!G.active) continue;
    h->active_grids.push_back((int32_t)g);
    for (int64_t b = G.block_begin; b < G.block_end; ++b) h->active_blocks.push_back((int32_t)b);
    for (int64_t b = G.block_begin; b < G.block_end; ++b) {
      if (b == h->drop_block && h->path == JACOBI_PATH_PERSISTENT) continue;  // injected fault
      const BlockHost& B = P.blocks[b];
      const int64_t nc = chunks(b);
      const int64_t per_chunk = (B.item_end - B.item_begin) / nc;
      for (int64_t c = 0; c < nc; ++c) {
        h->active_units.push_back((int32_t)(unit0[b] + c));
        h->active_unit_items.push_back((int32_t)h->active_items.size());
        for (int64_t q = B.item_begin + c * per_chunk; q < B.item_begin + (c + 1) * per_chunk; ++q)
          h->active_items.push_back(P.items[q]);
        h->active_dep_off.push_back((int32_t)h->active_deps.size());
        if (c > 0) h->active_deps.push_back((int32_t)(unit0[b] + c - 1));
        if (c + 1 < nc) h->active_deps.push_back((int32_t)(unit0[b] + c + 1));
        for (int f = 0; f < 4; ++f)
          if (B.nbr[f] >= 0) h->active_deps.push_back((int32_t)(unit0[B.nbr[f]] + c));
        if (c == 0 && B.nbr[ZM] >= 0) h->active_deps.push_back((int32_t)(unit0[B.nbr[ZM]] + chunks(B.nbr[ZM]) - 1));
        if (c == nc - 1 && B.nbr[ZP] >= 0) h->active_deps.push_back((int32_t)unit0[B.nbr[ZP]]);
      }
    }
  }
  h->active_unit_items.push_back((int32_t)h->active_items.size());
  h->active_dep_off.push_back((int32_t)h->active_deps.size());
  // The same items grouped by kind (stable), for one kernel variant per kind.
  h->kind_items.clear();
  for (int k = 0; k < kItemKinds; ++k) {
    h->kind_off[k] = (int32_t)h->kind_items.size();
    for (const WorkItem& w : h->active_items)
      if (item_kind(w) == k) h->kind_items.push_back(w);
  }
  h->kind_off[kItemKinds] = (int32_t)h->kind_items.size();
  if (!h->active_items.empty()) {
    JGB_CUDA(cudaMemcpyAsync(h->d_active, h->active_items.data(), h->active_items.size() * sizeof(WorkItem),
                             cudaMemcpyHostToDevice, s));
    JGB_CUDA(cudaMemcpyAsync(h->d_kind, h->kind_items.data(), h->kind_items.size() * sizeof(WorkItem),
                             cudaMemcpyHostToDevice, s));
  }
  if (!h->active_blocks.empty())
    JGB_CUDA(cudaMemcpyAsync(h->d_active_blocks, h->active_blocks.data(), h->active_blocks.size() * sizeof(int32_t),
                             cudaMemcpyHostToDevice, s));
  if (!h->active_units.empty()) {
    auto up = [&](int32_t* d, const std::vector<int32_t>& v) {
      return cudaMemcpyAsync(d, v.data(), v.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    };
    JGB_CUDA(up(h->d_punit_ids, h->active_units));
    JGB_CUDA(up(h->d_punit_items, h->active_unit_items));
    JGB_CUDA(up(h->d_pdep_off, h->active_dep_off));
    if (!h->active_deps.empty()) JGB_CUDA(up(h->d_pdep_ids, h->active_deps));
  }
  // start_iter of every grid (changes when grids are frozen / re-activated)
  for (size_t g = 0; g < P.grids.size(); ++g) {
    h->h_grids[g].start_iter = P.grids[g].start_iter;
    h->h_grids[g].active = 1;  // inactive grids have no items in the launch lists
  }
  JGB_CUDA(cudaMemcpyAsync(h->d_grids, h->h_grids, P.grids.size() * sizeof(GridDev), cudaMemcpyHostToDevice, s));
  JGB_CUDA(cudaStreamSynchronize(s));  // host mirrors are reused below
  h->tables_dirty = false;
  return JACOBI_OK;
}

StepLaunch step_args(jacobi_t* h, int64_t it, bool all_items) {
  StepLaunch a;
  a.blocks = h->d_blocks;
  // The full list (table order) serves the |b| kernel; steps use the active
  // items grouped by kind.
  a.items = all_items ? h->d_items : h->d_kind;
  a.n_items = all_items ? (int32_t)h->plan.items.size() : (int32_t)h->kind_items.size();
  for (int k = 0; k <= kItemKinds; ++k) a.kind_off[k] = all_items ? 0 : h->kind_off[k];
  a.grids = h->d_grids;
  a.it = it;
  a.partials = h->d_partials;
  a.dtype = h->plan.dtype;
  a.stages = kStreamStages;
  a.smem = 128 + kStreamStages * (int32_t)h->plan.max_stage;
  a.err = h->d_err;
  a.wait_ns = h->wait_ns;
  a.norms = h->d_norms;
  a.emu = h->fp64_emu;
  return a;
}

int check_err_word(jacobi_t* h, cudaStream_t s) {
  JGB_CUDA(cudaMemcpyAsync(h->h_err, h->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  JGB_CUDA(cudaStreamSynchronize(s));
  if (*h->h_err != DEV_OK) {
    const uint32_t e = *h->h_err;
    JGB_CUDA(cudaMemsetAsync(h->d_err, 0, sizeof(uint32_t), s));
    JGB_CUDA(cudaStreamSynchronize(s));
    return set_error(e == DEV_TIMEOUT ? JACOBI_ETIMEDOUT : JACOBI_ESEQ,
                     "device-side wait failed (code %u) in the persistent step", e);
  }
  return JACOBI_OK;
}

int step_fused_direct(jacobi_t* h, int64_t it0, int64_t n, cudaStream_t s) {
  StepLaunch a = step_args(h, 0, false);
  for (int64_t t = 0; t < n; ++t) {
    a.it = it0 + t;
    JGB_CUDA(launch_step(a, kWrite | kPack, s, &h->fork));
  }
  return JACOBI_OK;
}

int step_graph(jacobi_t* h, int64_t it0, int64_t n, cudaStream_t s) {
  const int64_t K = 32;  // iterations per graph replay (even, so parity repeats)
  int64_t done = 0;
  if ((it0 & 1) && n > 0) {
    int rc = step_fused_direct(h, it0, 1, s);
    if (rc) return rc;
    done = 1;
  }
  if (n - done >= K) {
    if (!h->graph || h->graph_items != (int32_t)h->active_items.size()) {
      if (h->graph) cudaGraphExecDestroy(h->graph);
      h->graph = nullptr;
      cudaStream_t cs;
      JGB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        StepLaunch a = step_args(h, 0, false);
        for (int64_t t = 0; t < K && e == cudaSuccess; ++t) {
          a.it = t;
          e = launch_step(a, kWrite | kPack, cs, &h->fork);
        }
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = e2;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph, g, 0);
      if (g) cudaGraphDestroy(g);
      cudaStreamDestroy(cs);
      if (e != cudaSuccess) return set_error(JACOBI_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
      h->graph_items = (int32_t)h->active_items.size();
      h->graph_iters = K;
    }
    while (n - done >= K) {
      JGB_CUDA(cudaGraphLaunch(h->graph, s));
      done += K;
    }
  }
  return step_fused_direct(h, it0 + done, n - done, s);
}

int step_persistent(jacobi_t* h, int64_t it0, int64_t n, bool resid_first, cudaStream_t s) {
  int stages = h->stages;
  int smem = 128 + stages * (int32_t)h->plan.max_stage;
  const int threads = persistent_threads(h->active_items.data(), h->active_items.size());
  // The warp-specialised kernel takes launches whose items are all streamed
  // (no tiles) and whose units have at most 8 partners; the barrier-driven
  // kernel takes the others.
  int ws_cw = 0, maxc = 0;
  if (h->persist_ws) {
    bool tiles = false;
    int cw = 2;
    for (const WorkItem& w : h->active_items) {
      tiles = tiles || w.x0 >= 0;
      cw = std::max(cw, (int)(w.y0 & 15));
    }
    int maxdep = 0;
    for (size_t u = 0; u + 1 < h->active_dep_off.size(); ++u)
      maxdep = std::max(maxdep, h->active_dep_off[u + 1] - h->active_dep_off[u]);
    if (!tiles && maxdep <= 8 && !h->active_units.empty() && smem <= kPersistWsSmem) {
      const int m = persistent_max_ctas(h->plan.dtype, smem, 0, cw);
      if (m > 0) {
        ws_cw = cw;
        maxc = m;
      }
      // Large stages (whole 64-wide planes) take one more stage of lookahead
      // when it costs no resident CTA: same-box A/B, 768^3 FP32 620 -> 659
      // GLUP/s, FP64 unchanged; small stages lose with it (256 FP32 grids of
      // 32^3 blocks 539 -> 507), so they keep the default.
      const int smem5 = smem + (int32_t)h->plan.max_stage;
      if (m > 0 && !h->stages_fixed && stages == 4 && h->plan.max_stage >= 8192 && smem5 <= kPersistWsSmem &&
          persistent_max_ctas(h->plan.dtype, smem5, 0, cw) == m) {
        stages = 5;
        smem = smem5;
      }
    }
  }
  if (!ws_cw) maxc = persistent_max_ctas(h->plan.dtype, smem, threads);
  if (maxc <= 0) return set_error(JACOBI_ECUDA, "occupancy query for the persistent kernel failed");
  if (ws_cw && resid_first && n > 1) {  // its residual launches run one iteration
    int rc = step_persistent(h, it0, 1, true, s);
    return rc ? rc : step_persistent(h, it0 + 1, n - 1, false, s);
  }
  PersistLaunch a;
  a.blocks = h->d_blocks;
  a.items = h->d_active;
  a.unit_items = h->d_punit_items;
  a.unit_ids = h->d_punit_ids;
  a.dep_off = h->d_pdep_off;
  a.dep_ids = h->d_pdep_ids;
  a.n_units = (int32_t)h->active_units.size();
  a.grids = h->d_grids;
  a.it0 = it0;
  a.it0_dev = nullptr;
  a.n_iters = n;
  a.progress = h->d_progress;
  a.err = h->d_err;
  a.wait_ns = h->wait_ns;
  a.partials = h->d_partials;
  a.resid_first = resid_first ? 1 : 0;
  a.dtype = h->plan.dtype;
  a.stages = stages;
  a.smem = smem;
  a.norms = h->d_norms;
  a.emu = h->fp64_emu;
  a.threads = threads;
  a.ws_cw = ws_cw;
  a.stage_bytes = (int32_t)h->plan.max_stage;
  a.ticket = h->d_ticket;
  const int ctas = std::min(maxc, a.n_units);
  // Replay a captured graph of the same launch shape; the start iteration
  // goes to device memory first (a pageable source is staged before the call
  // returns, so the stack variable may go).
  jacobi_s::PersistGraph& pg = h->pgraph[resid_first ? 1 : 0];
  if (!h->pgraph_off && (!pg.exec || pg.n_iters != n || pg.n_units != a.n_units || pg.stages != a.stages ||
                         pg.ctas != ctas || pg.threads != threads || pg.ws_cw != ws_cw)) {
    if (pg.exec) cudaGraphExecDestroy(pg.exec);
    pg.exec = nullptr;
    PersistLaunch c = a;
    c.it0_dev = h->d_it0;
    cudaStream_t cs = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = launch_persistent(c, ctas, cs);
      cudaError_t e2 = cudaStreamEndCapture(cs, &g);
      e = e1 != cudaSuccess ? e1 : e2;
    }
    if (e == cudaSuccess) {
      // the graph must hold exactly the one kernel node, launched
      // cooperatively (its CTAs wait on each other's flags)
      cudaGraphNode_t node = nullptr;
      size_t nn = 1;
      cudaGraphNodeType ty;
      e = cudaGraphGetNodes(g, &node, &nn);
      if (e == cudaSuccess && (nn != 1 || cudaGraphNodeGetType(node, &ty) != cudaSuccess ||
                               ty != cudaGraphNodeTypeKernel))
        e = cudaErrorNotSupported;
      if (e == cudaSuccess) {
        cudaLaunchAttributeValue v{};
        v.cooperative = 1;
        e = cudaGraphKernelNodeSetAttribute(node, cudaLaunchAttributeCooperative, &v);
      }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&pg.exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      cudaGetLastError();  // a refused capture leaves no sticky error; launch directly from now on
      pg.exec = nullptr;
      h->pgraph_off = true;
    } else {
      pg.n_iters = n;
      pg.n_units = a.n_units;
      pg.stages = a.stages;
      pg.ctas = ctas;
      pg.threads = threads;
      pg.ws_cw = ws_cw;
    }
  }
  // the warp-specialised kernel hands out its work from a counter that starts at zero
  if (ws_cw) JGB_CUDA(cudaMemsetAsync(h->d_ticket, 0, sizeof(unsigned long long), s));
  if (!h->pgraph_off && pg.exec) {
    const int64_t v = it0;
    JGB_CUDA(cudaMemcpyAsync(h->d_it0, &v, sizeof v, cudaMemcpyHostToDevice, s));
    JGB_CUDA(cudaGraphLaunch(pg.exec, s));
    return JACOBI_OK;
  }
  JGB_CUDA(launch_persistent(a, ctas, s));
  return JACOBI_OK;
}

// The halo exchange that follows the stencil launch of iteration `it` on the
// unfused paths (the new iterate has parity p ^ 1 of each grid's own count):
//   EXPLICIT:    device-side pack into the staging buffers, device-side copy
//                into the neighbours' slots (no host step);
//   CHANNEL:     the host waits for the stencil, then one launch packs every
//                face straight into the neighbour's pre-posted slot;
//   MESSAGING:   pack into the staging buffers (the send buffers); the host
//                waits, routes one metadata message per face through the
//                receiving block's mailbox, and each receiver posts its copy
//                (source from the message, destination its own slot); the
//                posted copies run as one launch from an uploaded descriptor
//                table;
//   HOST_STAGED: pack, copy the staging buffers device -> pinned host, the
//                host waits for them, copy them host -> device, unpack into the
//                neighbours' slots.
int exchange(jacobi_t* h, int64_t it, cudaStream_t s) {
  const Plan& P = h->plan;
  const int32_t na = (int32_t)h->active_blocks.size();
  const int32_t* ids = h->d_active_blocks;
  switch (h->path) {
    case JACOBI_PATH_EXPLICIT:
      JGB_CUDA(launch_pack_faces(h->d_blocks, ids, na, h->d_stage_tab, h->d_grids, it, P.dtype, s));
      JGB_CUDA(launch_copy_faces(h->d_blocks, ids, na, h->d_stage_tab, h->d_grids, it, P.dtype, s));
      return JACOBI_OK;
    case JACOBI_PATH_CHANNEL:
      JGB_CUDA(cudaStreamSynchronize(s));
      JGB_CUDA(launch_pack_faces(h->d_blocks, ids, na, h->d_stage_tab, h->d_grids, it, P.dtype, s, true));
      return JACOBI_OK;
    case JACOBI_PATH_MESSAGING: {
      JGB_CUDA(launch_pack_faces(h->d_blocks, ids, na, h->d_stage_tab, h->d_grids, it, P.dtype, s));
      if (!h->d_desc) {
        const size_t n = (size_t)std::max<int64_t>(P.halo_faces, 1);
        JGB_CUDA(cudaMalloc((void**)&h->d_desc, n * sizeof(CopyDesc)));
        JGB_CUDA(cudaMallocHost((void**)&h->h_desc, n * sizeof(CopyDesc)));
        h->mailbox.assign(P.blocks.size(), {});
      }
      JGB_CUDA(cudaStreamSynchronize(s));  // the send buffers are ready: post the metadata
      for (int32_t b : h->active_blocks) {
        const BlockHost& B = P.blocks[b];
        for (int f = 0; f < 6; ++f)
          if (B.nbr[f] >= 0)
            h->mailbox[B.nbr[f]].push_back(jacobi_s::HaloMeta{h->ws + B.stage_off[f],
                                                               face_elems_host(B, f) * (int64_t)P.elem,
                                                               opposite(f)});
      }
      int32_t nd = 0;
      for (int32_t r : h->active_blocks) {  // each receiver handles its messages
        const BlockHost& R = P.blocks[r];
        const int pn = (int)((it - P.grids[R.grid].start_iter + 1) & 1);
        for (const jacobi_s::HaloMeta& m : h->mailbox[r]) {
          if (m.bytes != face_elems_host(R, m.face) * (int64_t)P.elem)
            return set_error(JACOBI_ESEQ, "halo message of %lld bytes for a %lld-byte slot", (long long)m.bytes,
                             (long long)(face_elems_host(R, m.face) * (int64_t)P.elem));
          h->h_desc[nd++] = CopyDesc{m.src, h->ws + R.recv_off[m.face][pn], m.bytes};
        }
        h->mailbox[r].clear();
      }
      JGB_CUDA(cudaMemcpyAsync(h->d_desc, h->h_desc, (size_t)nd * sizeof(CopyDesc), cudaMemcpyHostToDevice, s));
      JGB_CUDA(launch_copy_desc(h->d_desc, nd, s));
      // the pinned descriptor table is rewritten by the next exchange only
      // after its stream synchronisation, which follows this copy
      return JACOBI_OK;
    }
    case JACOBI_PATH_HOST_STAGED: {
      const size_t bytes = P.off_stage_end - P.off_stage_begin;
      JGB_CUDA(launch_pack_faces(h->d_blocks, ids, na, h->d_stage_tab, h->d_grids, it, P.dtype, s));
      if (bytes == 0) return JACOBI_OK;
      if (!h->h_halo) JGB_CUDA(cudaMallocHost(&h->h_halo, bytes));
      JGB_CUDA(cudaMemcpyAsync(h->h_halo, h->ws + P.off_stage_begin, bytes, cudaMemcpyDeviceToHost, s));
      JGB_CUDA(cudaStreamSynchronize(s));  // the faces are in host memory: hand them on
      JGB_CUDA(cudaMemcpyAsync(h->ws + P.off_stage_begin, h->h_halo, bytes, cudaMemcpyHostToDevice, s));
      JGB_CUDA(launch_copy_faces(h->d_blocks, ids, na, h->d_stage_tab, h->d_grids, it, P.dtype, s));
      return JACOBI_OK;
    }
    default:
      return set_error(JACOBI_EINVAL, "path %d has no separate exchange", h->path);
  }
}

// Stencil launch + exchange per iteration on the unfused paths.  With `ev`
// (2n + 1 events) ev[2t] / ev[2t + 1] / ev[2t + 2] bracket iteration t's
// stencil and exchange on the stream.
int step_exchange(jacobi_t* h, int64_t it0, int64_t n, cudaStream_t s, cudaEvent_t* ev = nullptr) {
  StepLaunch a = step_args(h, 0, false);
  if (ev) JGB_CUDA(cudaEventRecord(ev[0], s));
  for (int64_t t = 0; t < n; ++t) {
    a.it = it0 + t;
    JGB_CUDA(launch_step(a, kWrite, s, &h->fork));
    if (ev) JGB_CUDA(cudaEventRecord(ev[2 * t + 1], s));
    int rc = exchange(h, a.it, s);
    if (rc) return rc;
    if (ev) JGB_CUDA(cudaEventRecord(ev[2 * t + 2], s));
  }
  return JACOBI_OK;
}

// Advance active grids by n iterations on the selected path.
int do_step(jacobi_t* h, int64_t n, cudaStream_t s) {
  int rc = refresh_active(h, s);
  if (rc) return rc;
  if (n <= 0 || h->active_items.empty()) {
    h->iter += std::max<int64_t>(n, 0);
    return JACOBI_OK;
  }
  switch (h->path) {
    case JACOBI_PATH_FUSED: rc = step_fused_direct(h, h->iter, n, s); break;
    case JACOBI_PATH_GRAPH: rc = step_graph(h, h->iter, n, s); break;
    case JACOBI_PATH_PERSISTENT: rc = step_persistent(h, h->iter, n, false, s); break;
    case JACOBI_PATH_EXPLICIT:
    case JACOBI_PATH_CHANNEL:
    case JACOBI_PATH_MESSAGING:
    case JACOBI_PATH_HOST_STAGED: rc = step_exchange(h, h->iter, n, s); break;
    default: return set_error(JACOBI_EINVAL, "bad path");
  }
  if (rc) return rc;
  h->iter += n;
  return JACOBI_OK;
}

// One step that also produces the residual of the current iterate (fused),
// followed by the per-grid reduction.  Does not synchronise.
int step_with_residual(jacobi_t* h, cudaStream_t s) {
  int rc = refresh_active(h, s);
  if (rc) return rc;
  if (h->path == JACOBI_PATH_PERSISTENT) {
    rc = step_persistent(h, h->iter, 1, true, s);
    if (rc) return rc;
  } else {
    // every other path takes the fused step here: its pack delivers the
    // faces, so the explicit path has nothing left to move either
    StepLaunch a = step_args(h, h->iter, false);
    JGB_CUDA(launch_step(a, kWrite | kPack | kResid, s, &h->fork));
  }
  JGB_CUDA(launch_reduce(h->d_grids, h->d_norms, h->d_gids, (int32_t)h->plan.grids.size(), h->d_partials, 0, s));
  h->iter += 1;
  return JACOBI_OK;
}

int residual_only(jacobi_t* h, cudaStream_t s) {
  int rc = refresh_active(h, s);
  if (rc) return rc;
  StepLaunch a = step_args(h, h->iter, false);
  JGB_CUDA(launch_step(a, kResid, s, &h->fork));
  JGB_CUDA(launch_reduce(h->d_grids, h->d_norms, h->d_gids, (int32_t)h->plan.grids.size(), h->d_partials, 0, s));
  return JACOBI_OK;
}

// |b|^2 and the FP64 adder-domain check of every grid (grid < 0) or of one
// grid (after its state was replaced).
int compute_bnorm(jacobi_t* h, cudaStream_t s, int64_t grid) {
  StepLaunch a = step_args(h, h->iter, true);
  int32_t b0 = 0, nb = (int32_t)h->plan.blocks.size(), g0 = 0, ng = (int32_t)h->plan.grids.size();
  if (grid >= 0) {
    const GridHost& G = h->plan.grids[grid];
    a.items += G.item_begin;
    a.n_items = (int32_t)(G.item_end - G.item_begin);
    b0 = (int32_t)G.block_begin;
    nb = (int32_t)(G.block_end - G.block_begin);
    g0 = (int32_t)grid;
    ng = 1;
  }
  JGB_CUDA(launch_emu_check(h->d_blocks + b0, nb, h->d_grids, h->d_norms, h->d_gids + g0, ng, h->iter, h->plan.dtype, s));
  JGB_CUDA(launch_bnorm(a, s));
  JGB_CUDA(launch_reduce(h->d_grids, h->d_norms, h->d_gids + g0, ng, h->d_partials, 1, s));
  return JACOBI_OK;
}

int read_norms(jacobi_t* h, cudaStream_t s) {
  JGB_CUDA(cudaMemcpyAsync(h->h_norms, h->d_norms, h->plan.grids.size() * sizeof(GridNorm), cudaMemcpyDeviceToHost, s));
  JGB_CUDA(cudaStreamSynchronize(s));
  return JACOBI_OK;
}

// Host-transfer staging buffer: sized once for the largest padded grid of the
// handle (growing it grid by grid would free and allocate, both synchronous,
// on many calls of a batch).
int stage_get(jacobi_t* h, size_t bytes, void** out) {
  if (h->stage_bytes < bytes) {
    size_t want = bytes;
    for (const GridHost& G : h->plan.grids)
      want = std::max(want, (size_t)(G.dims.nx + 2) * (G.dims.ny + 2) * (G.dims.nz + 2) * h->plan.elem);
    if (h->stage) cudaFree(h->stage);
    h->stage = nullptr;
    h->stage_bytes = 0;
    JGB_CUDA(cudaMalloc(&h->stage, want));
    h->stage_bytes = want;
  }
  *out = h->stage;
  return JACOBI_OK;
}

int64_t grid_local_iter(const jacobi_t* h, int64_t g) {
  const GridHost& G = h->plan.grids[g];
  return G.active ? h->iter - G.start_iter : G.frozen_local;
}

void freeze_grid(jacobi_t* h, int64_t g, int64_t local) {
  GridHost& G = h->plan.grids[g];
  G.frozen_local = local;
  G.active = false;
  h->tables_dirty = true;
}

void activate_grid(jacobi_t* h, int64_t g) {
  GridHost& G = h->plan.grids[g];
  if (G.active) return;
  G.start_iter = h->iter - G.frozen_local;
  G.active = true;
  h->tables_dirty = true;
}

// Re-plan the work items of a live handle for another shape (the states,
// slots and every table offset stay where they are; the item and unit tables
// were sized for the finest accepted shape).  Recomputes |b| (its summation
// order follows the items) and drops captured graphs.
int apply_shape(jacobi_t* h, int64_t zchunk, int32_t cw_cap, cudaStream_t s) {
  if (zchunk < 0 || (cw_cap != 0 && cw_cap != 2 && cw_cap != 4 && cw_cap != 8))
    return set_error(JACOBI_EINVAL, "bad shape: zchunk %lld, cw_cap %d", (long long)zchunk, cw_cap);
  Plan Q = h->plan;
  int rc = plan_items(&Q, zchunk, cw_cap, 0, 1);
  if (rc) return rc;
  if ((int64_t)Q.items.size() > Q.cap_items || Q.n_units > Q.cap_units)
    return set_error(JACOBI_EINVAL, "shape (zchunk %lld, cw_cap %d) needs %lld items / %lld units; the tables hold "
                     "%lld / %lld", (long long)zchunk, cw_cap, (long long)Q.items.size(), (long long)Q.n_units,
                     (long long)Q.cap_items, (long long)Q.cap_units);
  JGB_CUDA(cudaStreamSynchronize(s));  // no launch may still read the old items
  h->plan = std::move(Q);
  const Plan& P = h->plan;
  for (size_t g = 0; g < P.grids.size(); ++g) {
    h->h_grids[g].item_begin = (int32_t)P.grids[g].item_begin;
    h->h_grids[g].item_end = (int32_t)P.grids[g].item_end;
  }
  JGB_CUDA(cudaMemcpyAsync(h->d_items, P.items.data(), P.items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, s));
  JGB_CUDA(cudaMemcpyAsync(h->d_grids, h->h_grids, P.grids.size() * sizeof(GridDev), cudaMemcpyHostToDevice, s));
  JGB_CUDA(cudaMemsetAsync(h->d_progress, 0, P.cap_units * sizeof(int64_t), s));
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
  for (auto& pg : h->pgraph) {
    if (pg.exec) cudaGraphExecDestroy(pg.exec);
    pg = jacobi_s::PersistGraph();
  }
  if (128 + h->stages * (int64_t)P.max_stage > kMaxStepSmem) h->stages = 3;
  h->tables_dirty = true;
  rc = compute_bnorm(h, s, -1);
  if (rc) return rc;
  return refresh_active(h, s);
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* jacobi_strerror(int code) {
  switch (code) {
    case JACOBI_OK: return "ok";
    case JACOBI_EINVAL: return "invalid argument";
    case JACOBI_ENOMEM: return "out of memory";
    case JACOBI_EBUSY: return "busy";
    case JACOBI_EAGAIN: return "not ready";
    case JACOBI_ETIMEDOUT: return "device wait timed out";
    case JACOBI_ECUDA: return "CUDA error";
    case JACOBI_ESEQ: return "channel sequence mismatch";
    default: return "unknown error";
  }
}

const char* jacobi_last_error(void) { return jgb::g_last_error.c_str(); }

int jacobi_decompose(jacobi_dim3 grid, int64_t nblocks, jacobi_dim3* out) {
  const int64_t kMax = 1ll << 30;  // the sizes plan_build accepts
  if (!out || nblocks < 1 || grid.nx < 1 || grid.ny < 1 || grid.nz < 1 || nblocks > kMax || grid.nx > kMax ||
      grid.ny > kMax || grid.nz > kMax)
    return set_error(JACOBI_EINVAL, "bad arguments to jacobi_decompose");
  // Total block surface of a near-equal split: sum over blocks of
  // 2(ex*ey + ey*ez + ez*ex) = 2(nx*ny*pz + ny*nz*px + nz*nx*py), which can
  // exceed 64 bits at the largest accepted sizes.
  bool found = false;
  unsigned __int128 best = 0;
  jacobi_dim3 arg{0, 0, 0};
  // the divisors of nblocks in ascending order (trial division to its root)
  std::vector<int64_t> divs, upper;
  for (int64_t d = 1; d * d <= nblocks; ++d)
    if (nblocks % d == 0) {
      divs.push_back(d);
      if (d * d != nblocks) upper.push_back(nblocks / d);
    }
  divs.insert(divs.end(), upper.rbegin(), upper.rend());
  for (int64_t px : divs) {
    if (px > grid.nx) break;
    for (int64_t py : divs) {
      if (py > grid.ny || py > nblocks / px) break;
      if ((nblocks / px) % py) continue;
      const int64_t pz = nblocks / px / py;
      if (pz > grid.nz) continue;
      using U = unsigned __int128;
      const U area = 2 * ((U)grid.nx * (U)grid.ny * (U)pz + (U)grid.ny * (U)grid.nz * (U)px +
                          (U)grid.nz * (U)grid.nx * (U)py);
      if (!found || area < best) {  // loop order is lexicographic, so ties keep the first
        found = true;
        best = area;
        arg = jacobi_dim3{px, py, pz};
      }
    }
  }
  if (!found) return set_error(JACOBI_EINVAL, "no split of %lld blocks fits the grid", (long long)nblocks);
  *out = arg;
  return JACOBI_OK;
}

int jacobi_workspace_bytes_batch(int64_t n_grids, const jacobi_dim3* grids, const jacobi_split* splits,
                                 jacobi_dtype dtype, size_t* bytes) {
  if (!bytes) return set_error(JACOBI_EINVAL, "bytes is null");
  Plan P;
  int rc = plan_build(n_grids, grids, splits, dtype, nullptr, &P);
  if (rc) return rc;
  *bytes = P.bytes;
  return JACOBI_OK;
}

int jacobi_workspace_bytes(jacobi_dim3 grid, jacobi_split split, jacobi_dtype dtype, size_t* bytes) {
  return jacobi_workspace_bytes_batch(1, &grid, &split, dtype, bytes);
}

int jacobi_create_batch(int64_t n_grids, const jacobi_dim3* grids, const jacobi_split* splits, jacobi_dtype dtype,
                        const jacobi_init* inits, void* workspace, size_t ws_bytes, void* stream, jacobi_t** out) {
  if (!out) return set_error(JACOBI_EINVAL, "out is null");
  *out = nullptr;
  jacobi_t* h = new (std::nothrow) jacobi_t();
  if (!h) return set_error(JACOBI_ENOMEM, "host allocation failed");
  int rc = plan_build(n_grids, grids, splits, dtype, inits, &h->plan);
  if (rc) {
    delete h;
    return rc;
  }
  const cudaStream_t s = S(stream);
  auto fail = [&](int code) {
    kind_fork_destroy(&h->fork);
    if (h->own_ws && h->ws) cudaFree(h->ws);
    if (h->h_grids) cudaFreeHost(h->h_grids);
    if (h->h_norms) cudaFreeHost(h->h_norms);
    if (h->h_err) cudaFreeHost(h->h_err);
    delete h;
    return code;
  };
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) return fail(set_error(JACOBI_ECUDA, "no CUDA device: %s", cudaGetErrorString(e)));
  e = kind_fork_create(&h->fork);
  if (e != cudaSuccess) return fail(set_error(JACOBI_ECUDA, "stream creation failed: %s", cudaGetErrorString(e)));
  if (workspace) {
    if (ws_bytes < h->plan.bytes)
      return fail(set_error(JACOBI_ENOMEM, "workspace too small: %zu < %zu bytes", ws_bytes, h->plan.bytes));
    if ((uintptr_t)workspace % 256) return fail(set_error(JACOBI_EINVAL, "workspace must be 256-byte aligned"));
    h->ws = (char*)workspace;
  } else {
    e = cudaMalloc((void**)&h->ws, h->plan.bytes);
    if (e != cudaSuccess) {
      h->ws = nullptr;
      return fail(set_error(JACOBI_ENOMEM, "cudaMalloc(%zu) failed: %s", h->plan.bytes, cudaGetErrorString(e)));
    }
    h->own_ws = true;
  }
  if (cudaMallocHost((void**)&h->h_grids, h->plan.grids.size() * sizeof(GridDev)) != cudaSuccess ||
      cudaMallocHost((void**)&h->h_norms, h->plan.grids.size() * sizeof(GridNorm)) != cudaSuccess ||
      cudaMallocHost((void**)&h->h_err, 64) != cudaSuccess)
    return fail(set_error(JACOBI_ENOMEM, "pinned host allocation failed"));
  const Plan& P = h->plan;
  h->d_blocks = (BlockDev*)(h->ws + P.off_blocks);
  h->d_geom = (BlockGeom*)(h->ws + P.off_geom);
  h->d_items = (WorkItem*)(h->ws + P.off_items);
  h->d_active = (WorkItem*)(h->ws + P.off_active);
  h->d_kind = (WorkItem*)(h->ws + P.off_kind);
  h->d_grids = (GridDev*)(h->ws + P.off_grids);
  h->d_norms = (GridNorm*)(h->ws + P.off_norms);
  h->d_inits = (InitDev*)(h->ws + P.off_inits);
  h->d_gids = (int32_t*)(h->ws + P.off_gids);
  h->d_partials = (double*)(h->ws + P.off_partials);
  h->d_progress = (int64_t*)(h->ws + P.off_progress);
  h->d_err = (uint32_t*)(h->ws + P.off_err);
  h->d_stage_tab = (void**)(h->ws + P.off_stage_tab);
  h->d_punit_items = (int32_t*)(h->ws + P.off_punit_items);
  h->d_punit_ids = (int32_t*)(h->ws + P.off_punit_ids);
  h->d_pdep_off = (int32_t*)(h->ws + P.off_pdep_off);
  h->d_pdep_ids = (int32_t*)(h->ws + P.off_pdep_ids);
  h->d_active_blocks = (int32_t*)(h->ws + P.off_active_blocks);
  h->d_it0 = (int64_t*)(h->ws + P.off_it0);
  h->d_ticket = (unsigned long long*)(h->ws + P.off_ticket);
  if (const char* w = getenv("JACOBI_WAIT_MS")) {
    const double ms = atof(w);
    if (ms > 0) h->wait_ns = (uint64_t)(ms * 1e6);
  }
  // Ring depth of the persistent kernel's plane streaming: four stages keep
  // one plane in flight beyond the three a consumer reads (the autotuner may
  // pick another); the per-step kernels always use kStreamStages.
  h->stages = 4;
  if (const char* em = getenv("JACOBI_FP64_EMU")) h->fp64_emu = atoi(em) != 0 ? 1 : 0;
  if (const char* pw = getenv("JACOBI_PERSIST_WS")) h->persist_ws = atoi(pw) != 0;
  if (const char* st = getenv("JACOBI_STAGES")) {
    const int v = atoi(st);
    if (v >= 3 && v <= 8) {
      h->stages = v;
      h->stages_fixed = true;
    }
  }
  if (128 + h->stages * (int64_t)P.max_stage > kMaxStepSmem) h->stages = 3;
  // Zero the workspace so the padding of every row, plane and slot starts
  // finite (and inside the FP64 integer adder's domain).
  e = cudaMemsetAsync(h->ws, 0, P.bytes, s);
  if (e != cudaSuccess) return fail(set_error(JACOBI_ECUDA, "workspace clear failed: %s", cudaGetErrorString(e)));
  rc = upload_tables(h, s);
  if (rc) return fail(rc);
  e = launch_init(h->d_blocks, h->d_geom, (int32_t)P.blocks.size(), h->d_inits, P.dtype, s);
  if (e != cudaSuccess) return fail(set_error(JACOBI_ECUDA, "init launch failed: %s", cudaGetErrorString(e)));
  rc = compute_bnorm(h, s, -1);
  if (rc) return fail(rc);
  rc = refresh_active(h, s);
  if (rc) return fail(rc);
  *out = h;
  return JACOBI_OK;
}

int jacobi_create(jacobi_dim3 grid, jacobi_split split, jacobi_dtype dtype, const jacobi_init* init, void* workspace,
                  size_t ws_bytes, void* stream, jacobi_t** out) {
  return jacobi_create_batch(1, &grid, &split, dtype, init, workspace, ws_bytes, stream, out);
}

int jacobi_destroy(jacobi_t* h) {
  if (!h) return JACOBI_OK;
  cudaDeviceSynchronize();
  for (channel_s* c : std::vector<channel_s*>(h->channels)) channel_close(c);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  for (auto& pg : h->pgraph)
    if (pg.exec) cudaGraphExecDestroy(pg.exec);
  kind_fork_destroy(&h->fork);
  if (h->stage) cudaFree(h->stage);
  if (h->d_desc) cudaFree(h->d_desc);
  if (h->h_desc) cudaFreeHost(h->h_desc);
  if (h->h_halo) cudaFreeHost(h->h_halo);
  if (h->own_ws && h->ws) cudaFree(h->ws);
  if (h->h_grids) cudaFreeHost(h->h_grids);
  if (h->h_norms) cudaFreeHost(h->h_norms);
  if (h->h_err) cudaFreeHost(h->h_err);
  delete h;
  return JACOBI_OK;
}

int jacobi_info(const jacobi_t* h, jacobi_info_t* out) {
  if (!h || !out) return set_error(JACOBI_EINVAL, "null argument");
  out->n_grids = (int64_t)h->plan.grids.size();
  out->n_blocks = (int64_t)h->plan.blocks.size();
  out->n_points = h->plan.n_points;
  out->iteration = h->iter;
  out->dtype = h->plan.dtype;
  out->path = h->path;
  out->halo_bytes_per_iter = h->plan.halo_elems * (int64_t)h->plan.elem;
  out->workspace_bytes = h->plan.bytes;
  out->stages = h->stages;
  out->fp64_int_adds = (h->plan.dtype == JACOBI_F64 && h->fp64_emu) ? 3 : 0;
  int kinds = 0;
  for (int k = 0; k < kItemKinds; ++k) kinds += h->kind_off[k + 1] > h->kind_off[k] ? 1 : 0;
  out->item_kinds = kinds;
  for (int k = 0; k < 8; ++k) out->kind_items[k] = k < kItemKinds ? h->kind_off[k + 1] - h->kind_off[k] : 0;
  out->zchunk = h->plan.zchunk;
  out->cw_cap = h->plan.cw_cap;
  out->pad2_ = 0;
  return JACOBI_OK;
}

// ---- autotuner ------------------------------------------------------------------
namespace {

uint64_t geometry_signature(const Plan& P) {
  uint64_t x = 1469598103934665603ull;  // FNV-1a
  auto mix = [&](int64_t v) {
    for (int b = 0; b < 8; ++b) {
      x ^= (uint64_t)((v >> (8 * b)) & 0xff);
      x *= 1099511628211ull;
    }
  };
  mix(P.dtype);
  mix((int64_t)P.grids.size());
  for (const GridHost& G : P.grids) {
    mix(G.dims.nx); mix(G.dims.ny); mix(G.dims.nz);
    mix(G.split.mode); mix(G.split.x); mix(G.split.y); mix(G.split.z);
  }
  return x;
}

// Cache lines: "v2 <signature> <path> <stages> <zchunk> <cw_cap> <ms per iteration>".
bool cache_lookup(uint64_t key, jacobi_tune_result* r) {
  const char* f = getenv("JACOBI_TUNE_CACHE");
  if (!f || !*f) return false;
  FILE* fp = fopen(f, "r");
  if (!fp) return false;
  char line[256];
  bool found = false;
  while (fgets(line, sizeof line, fp)) {
    unsigned long long k;
    int p, st, cw;
    long long zc;
    double t;
    if (sscanf(line, "v2 %llx %d %d %lld %d %lf", &k, &p, &st, &zc, &cw, &t) == 6 && k == key) {
      r->path = p; r->stages = st; r->zchunk = zc; r->cw_cap = cw; r->ms_per_iter = t;
      found = true;  // the last entry wins
    }
  }
  fclose(fp);
  return found;
}

void cache_store(uint64_t key, const jacobi_tune_result& r) {
  const char* f = getenv("JACOBI_TUNE_CACHE");
  if (!f || !*f) return;
  FILE* fp = fopen(f, "a");
  if (!fp) return;
  fprintf(fp, "v2 %016llx %d %d %lld %d %.6f\n", (unsigned long long)key, r.path, r.stages, (long long)r.zchunk,
          r.cw_cap, r.ms_per_iter);
  fclose(fp);
}

}  // namespace

extern "C" int jacobi_set_shape(jacobi_t* h, int64_t zchunk, int32_t cw_cap, void* stream) {
  if (!h) return set_error(JACOBI_EINVAL, "null handle");
  return apply_shape(h, zchunk, cw_cap, S(stream));
}

// The search of jacobi_autotune; only_path >= 0 restricts it to that path
// (jacobi_autotune_path), cached under its own key.
static int autotune_search(jacobi_t* h, int64_t iters_per_trial, void* stream, jacobi_tune_result* out, int32_t only_path) {
  const cudaStream_t s = S(stream);
  const Plan& P = h->plan;
  const uint64_t key = geometry_signature(P) ^ (only_path < 0 ? 0ull : 0x9E3779B97F4A7C15ull * (uint64_t)(only_path + 1));
  jacobi_tune_result r{};
  if (cache_lookup(key, &r)) {
    r.from_cache = 1;
  } else {
    std::vector<jacobi_dim3> grids;
    std::vector<jacobi_split> splits;
    std::vector<jacobi_init> inits;
    for (const GridHost& G : P.grids) {
      grids.push_back(G.dims);
      splits.push_back(G.split);
      inits.push_back(G.init);
    }
    jacobi_t* t = nullptr;
    int rc = jacobi_create_batch((int64_t)grids.size(), grids.data(), splits.data(), (jacobi_dtype)P.dtype,
                                 inits.data(), nullptr, 0, stream, &t);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = INFINITY;
    // Candidate shapes: the cost model's z-chunk, twice, half and a quarter of
    // it; CTAs of up to 8, 4 or 2 consumer warps (row windows of the
    // corresponding height).  Shapes that plan the same items are tried once.
    const int64_t zc0 = t->plan.zchunk;
    std::vector<std::pair<int64_t, int32_t>> shapes;
    std::vector<std::vector<WorkItem>> seen;
    for (int64_t zc : {zc0, 2 * zc0, std::max<int64_t>(1, zc0 / 2), std::max<int64_t>(1, zc0 / 4)})
      for (int32_t cw : {8, 4, 2, 0}) {
        Plan q = t->plan;
        if (plan_items(&q, zc, cw, 0, 1) || (int64_t)q.items.size() > q.cap_items || q.n_units > q.cap_units) continue;
        bool dup = false;
        for (const auto& v : seen)
          dup = dup || (v.size() == q.items.size() &&
                        std::equal(v.begin(), v.end(), q.items.begin(), [](const WorkItem& a, const WorkItem& b) {
                          return a.block == b.block && a.x0 == b.x0 && a.y0 == b.y0 && a.z0 == b.z0 && a.z1 == b.z1 &&
                                 a.ya == b.ya && a.yb == b.yb;
                        }));
        if (dup) continue;
        seen.push_back(q.items);
        shapes.push_back({zc, cw});
      }
    // One timed run of n iterations (ms per iteration), after the warm-up.
    auto timed = [&](int64_t n, double* per) -> int {
      int rc2 = JACOBI_OK;
      if (cudaEventRecord(e0, s) != cudaSuccess) rc2 = JACOBI_ECUDA;
      if (!rc2) rc2 = do_step(t, n, s);
      if (!rc2 && cudaEventRecord(e1, s) != cudaSuccess) rc2 = JACOBI_ECUDA;
      if (!rc2 && cudaEventSynchronize(e1) != cudaSuccess) rc2 = JACOBI_ECUDA;
      if (!rc2) rc2 = check_err_word(t, s);
      float ms = 0.f;
      if (!rc2) cudaEventElapsedTime(&ms, e0, e1);
      *per = ms / (double)n;
      return rc2;
    };
    // A trial runs at least iters_per_trial iterations and at least ~2 ms (a
    // short problem's iteration takes microseconds, too short to rank
    // candidates from one run), best of two runs.
    auto trial = [&](int32_t path, int32_t st, int64_t zc, int32_t cw) -> int {
      int rc2 = apply_shape(t, zc, cw, s);
      if (rc2) return rc2;
      t->stages = st;
      t->stages_fixed = true;
      t->path = path;
      t->tables_dirty = true;
      double est = 0.0;
      rc2 = timed(std::max<int64_t>(iters_per_trial / 4, 2), &est);  // warm-up (graph capture etc.)
      if (rc2) return rc2;
      const int64_t n = std::min<int64_t>(std::max<int64_t>(iters_per_trial, (int64_t)std::ceil(2.0 / std::max(est, 1e-4))),
                                          50 * iters_per_trial);
      double per = INFINITY;
      for (int rep = 0; rep < 2 && !rc2; ++rep) {
        double p1 = 0.0;
        rc2 = timed(n, &p1);
        per = std::min(per, p1);
      }
      if (rc2) return rc2;
      r.n_tried += 1;
      if (per < best) {
        best = per;
        r.path = path;
        r.stages = st;
        r.zchunk = zc;
        r.cw_cap = cw;
        r.ms_per_iter = per;
      }
      return JACOBI_OK;
    };
    // every shape on the graph path and on the persistent kernel (4 stages),
    // then the fused path and the other ring depths at the best shape
    for (const auto& sh : shapes)
      for (int32_t path : {(int32_t)JACOBI_PATH_GRAPH, (int32_t)JACOBI_PATH_PERSISTENT, (int32_t)JACOBI_PATH_FUSED})
        if (!rc && (only_path < 0 ? path != JACOBI_PATH_FUSED : path == only_path))
          rc = trial(path, kStreamStages, sh.first, sh.second);
    const int64_t bz = r.zchunk;
    const int32_t bc = r.cw_cap;
    if (!rc && only_path < 0) rc = trial(JACOBI_PATH_FUSED, kStreamStages, bz, bc);
    for (int32_t st = 3; st <= 6 && !rc && (only_path < 0 || only_path == JACOBI_PATH_PERSISTENT); ++st) {
      if (st == kStreamStages || t->plan.max_stage == 0) continue;  // no plane-streamed blocks: depth irrelevant
      Plan q = t->plan;
      plan_items(&q, bz, bc, 0, 1);
      if (128 + st * (int64_t)q.max_stage > kMaxStepSmem) continue;
      rc = trial(JACOBI_PATH_PERSISTENT, st, bz, bc);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    jacobi_destroy(t);
    if (rc) return rc;
    cache_store(key, r);
  }
  int rc = apply_shape(h, r.zchunk, r.cw_cap, s);
  if (rc) return rc;
  h->path = r.path;
  h->stages = r.stages;
  h->stages_fixed = true;
  h->tables_dirty = true;
  if (out) *out = r;
  return JACOBI_OK;
}

extern "C" int jacobi_autotune(jacobi_t* h, int64_t iters_per_trial, void* stream, jacobi_tune_result* out) {
  if (!h || iters_per_trial < 1) return set_error(JACOBI_EINVAL, "bad arguments to jacobi_autotune");
  return autotune_search(h, iters_per_trial, stream, out, -1);
}

extern "C" int jacobi_autotune_path(jacobi_t* h, int32_t path, int64_t iters_per_trial, void* stream,
                                    jacobi_tune_result* out) {
  if (!h || iters_per_trial < 1 ||
      (path != JACOBI_PATH_FUSED && path != JACOBI_PATH_GRAPH && path != JACOBI_PATH_PERSISTENT))
    return set_error(JACOBI_EINVAL, "bad arguments to jacobi_autotune_path");
  return autotune_search(h, iters_per_trial, stream, out, path);
}

int jacobi_block(const jacobi_t* h, int64_t block, jacobi_block_info* out) {
  if (!h || !out || block < 0 || block >= (int64_t)h->plan.blocks.size())
    return set_error(JACOBI_EINVAL, "bad block index");
  const BlockHost& B = h->plan.blocks[block];
  out->grid = B.grid;
  for (int a = 0; a < 3; ++a) {
    out->origin[a] = B.origin[a];
    out->extent[a] = B.extent[a];
  }
  for (int f = 0; f < 6; ++f) out->neighbour[f] = B.nbr[f];
  return JACOBI_OK;
}

int jacobi_set_path(jacobi_t* h, int32_t path) {
  if (!h || path < JACOBI_PATH_FUSED || path > JACOBI_PATH_HOST_STAGED) return set_error(JACOBI_EINVAL, "bad path");
  if (h->path != path) h->tables_dirty = true;
  h->path = path;
  return JACOBI_OK;
}

int jacobi_step(jacobi_t* h, int64_t n_iters, void* stream) {
  if (!h || n_iters < 0) return set_error(JACOBI_EINVAL, "bad arguments to jacobi_step");
  const cudaStream_t s = S(stream);
  int rc = do_step(h, n_iters, s);
  if (rc) return rc;
  if (h->path == JACOBI_PATH_PERSISTENT) {
    // The persistent kernel reports expired waits through the error word.
    cudaError_t q = cudaStreamQuery(s);
    if (q != cudaSuccess && q != cudaErrorNotReady) return set_error(JACOBI_ECUDA, "%s", cudaGetErrorString(q));
  }
  return JACOBI_OK;
}

int jacobi_step_timed(jacobi_t* h, int64_t n_iters, void* stream, double* compute_ms, double* exchange_ms) {
  if (!h || n_iters < 0 || n_iters > (1 << 20)) return set_error(JACOBI_EINVAL, "bad arguments to jacobi_step_timed");
  const cudaStream_t s = S(stream);
  int rc = refresh_active(h, s);
  if (rc) return rc;
  const bool split = h->path == JACOBI_PATH_EXPLICIT || h->path == JACOBI_PATH_CHANNEL ||
                     h->path == JACOBI_PATH_MESSAGING || h->path == JACOBI_PATH_HOST_STAGED;
  const int64_t n = (split && !h->active_items.empty()) ? n_iters : 0;
  std::vector<cudaEvent_t> ev(split ? 2 * n + 1 : 2, nullptr);
  auto destroy = [&]() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  };
  for (cudaEvent_t& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      e = nullptr;
      destroy();
      return set_error(JACOBI_ECUDA, "event creation failed");
    }
  double comp = 0.0, exch = 0.0;
  if (split) {
    rc = step_exchange(h, h->iter, n, s, n > 0 ? ev.data() : nullptr);
    if (!rc) h->iter += n_iters;
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = set_error(JACOBI_ECUDA, "stream synchronisation failed");
    for (int64_t t = 0; t < n && !rc; ++t) {
      float a = 0.f, b = 0.f;
      cudaEventElapsedTime(&a, ev[2 * t], ev[2 * t + 1]);
      cudaEventElapsedTime(&b, ev[2 * t + 1], ev[2 * t + 2]);
      comp += a;
      exch += b;
    }
  } else {
    if (cudaEventRecord(ev[0], s) != cudaSuccess) rc = set_error(JACOBI_ECUDA, "event record failed");
    if (!rc) rc = do_step(h, n_iters, s);
    if (!rc && cudaEventRecord(ev[1], s) != cudaSuccess) rc = set_error(JACOBI_ECUDA, "event record failed");
    if (!rc && cudaEventSynchronize(ev[1]) != cudaSuccess) rc = set_error(JACOBI_ECUDA, "event wait failed");
    float a = 0.f;
    if (!rc) cudaEventElapsedTime(&a, ev[0], ev[1]);
    comp = a;
    if (!rc && h->path == JACOBI_PATH_PERSISTENT) rc = check_err_word(h, s);
  }
  destroy();
  if (rc) return rc;
  if (compute_ms) *compute_ms = comp;
  if (exchange_ms) *exchange_ms = exch;
  return JACOBI_OK;
}

int jacobi_residual(jacobi_t* h, double* rel, double* abs_res, void* stream) {
  if (!h) return set_error(JACOBI_EINVAL, "null handle");
  const cudaStream_t s = S(stream);
  int rc = residual_only(h, s);
  if (rc) return rc;
  rc = read_norms(h, s);
  if (rc) return rc;
  for (size_t g = 0; g < h->plan.grids.size(); ++g) {
    if (rel) rel[g] = h->h_norms[g].rel;
    if (abs_res) abs_res[g] = h->h_norms[g].r_norm;
  }
  return JACOBI_OK;
}

int jacobi_solve(jacobi_t* h, double tol, int64_t max_iters, int64_t check_every, int64_t stall_checks,
                 int64_t* iters_out, double* rel_out, int32_t* status_out, void* stream) {
  if (!h || check_every < 1 || max_iters < 0 || !(tol >= 0.0))
    return set_error(JACOBI_EINVAL, "bad arguments to jacobi_solve");
  const cudaStream_t s = S(stream);
  Plan& P = h->plan;
  const size_t ng = P.grids.size();
  // Every grid starts its solve at its own local iteration 0 of this call.
  std::vector<int64_t> k(ng, 0), since(ng, 0);
  std::vector<double> best(ng, INFINITY), rel(ng, 0.0);
  std::vector<int32_t> status(ng, -1);
  for (size_t g = 0; g < ng; ++g) activate_grid(h, (int64_t)g);
  int64_t done_k = 0;  // common local iteration of the active grids
  for (;;) {
    const bool check = (done_k % check_every == 0) || done_k == max_iters;
    int rc;
    if (check) {
      if (done_k >= max_iters) {
        rc = residual_only(h, s);
      } else {
        rc = step_with_residual(h, s);
      }
      if (rc) return rc;
      rc = read_norms(h, s);
      if (rc) return rc;
      if (h->path == JACOBI_PATH_PERSISTENT) {
        rc = check_err_word(h, s);
        if (rc) return rc;
      }
      const bool stepped = done_k < max_iters;
      bool any_active = false;
      for (size_t g = 0; g < ng; ++g) {
        GridHost& G = P.grids[g];
        if (!G.active) continue;
        const double r = h->h_norms[g].rel;
        rel[g] = r;
        k[g] = done_k;
        int st = -1;
        if (r <= tol) st = JACOBI_SOLVE_CONVERGED;
        else if (done_k >= max_iters) st = JACOBI_SOLVE_MAX_ITERS;
        else if (r < best[g]) { best[g] = r; since[g] = 0; }
        else if (stall_checks > 0 && ++since[g] >= stall_checks) st = JACOBI_SOLVE_STAGNATED;
        if (st >= 0) {
          status[g] = st;
          // Freeze at u_k: when a step was fused with this check, the grid
          // already holds u_{k+1} in its other buffer; u_k stays intact.
          freeze_grid(h, (int64_t)g, grid_local_iter(h, (int64_t)g) - (stepped ? 1 : 0));
        } else {
          any_active = true;
        }
      }
      if (!any_active) break;
      done_k += stepped ? 1 : 0;
      if (!stepped) break;
    } else {
      const int64_t next = std::min<int64_t>((done_k / check_every + 1) * check_every, max_iters);
      rc = do_step(h, next - done_k, s);
      if (rc) return rc;
      done_k = next;
    }
  }
  // Re-activate every grid at its own iteration count.
  for (size_t g = 0; g < ng; ++g) {
    activate_grid(h, (int64_t)g);
    if (iters_out) iters_out[g] = k[g];
    if (rel_out) rel_out[g] = rel[g];
    if (status_out) status_out[g] = status[g];
  }
  return refresh_active(h, s);
}

int jacobi_set_state(jacobi_t* h, int64_t grid, const void* src, int32_t src_on_device, void* stream) {
  if (!h || !src || grid < 0 || grid >= (int64_t)h->plan.grids.size())
    return set_error(JACOBI_EINVAL, "bad arguments to jacobi_set_state");
  const cudaStream_t s = S(stream);
  const GridHost& G = h->plan.grids[grid];
  const size_t n = (size_t)(G.dims.nx + 2) * (G.dims.ny + 2) * (G.dims.nz + 2) * h->plan.elem;
  const void* dsrc = src;
  if (!src_on_device) {
    void* tmp = nullptr;
    int rc0 = stage_get(h, n, &tmp);
    if (rc0) return rc0;
    JGB_CUDA(cudaMemcpyAsync(tmp, src, n, cudaMemcpyHostToDevice, s));
    dsrc = tmp;
  }
  const int parity = (int)(grid_local_iter(h, grid) & 1);
  cudaError_t e = launch_scatter(h->d_blocks, h->d_geom, (int32_t)G.block_begin, (int32_t)(G.block_end - G.block_begin),
                                 dsrc, G.dims.nx, G.dims.ny, G.dims.nz, parity, h->plan.dtype, s);
  int rc = JACOBI_OK;
  if (e != cudaSuccess) rc = set_error(JACOBI_ECUDA, "scatter failed: %s", cudaGetErrorString(e));
  if (!rc) rc = compute_bnorm(h, s, grid);
  if (!rc && !src_on_device) {
    // the caller may reuse its host buffer as soon as the call returns
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e2 != cudaSuccess) rc = set_error(JACOBI_ECUDA, "%s", cudaGetErrorString(e2));
  }
  return rc;
}

int jacobi_copy_out(jacobi_t* h, int64_t grid, void* dst, int32_t dst_on_device, int32_t layout, void* stream) {
  if (!h || !dst || grid < 0 || grid >= (int64_t)h->plan.grids.size() ||
      (layout != JACOBI_LAYOUT_INTERIOR && layout != JACOBI_LAYOUT_PADDED))
    return set_error(JACOBI_EINVAL, "bad arguments to jacobi_copy_out");
  const cudaStream_t s = S(stream);
  const GridHost& G = h->plan.grids[grid];
  const int64_t o = layout == JACOBI_LAYOUT_PADDED ? 2 : 0;
  const size_t n = (size_t)(G.dims.nx + o) * (G.dims.ny + o) * (G.dims.nz + o) * h->plan.elem;
  void* ddst = dst;
  void* tmp = nullptr;
  if (!dst_on_device) {
    int rc0 = stage_get(h, n, &tmp);
    if (rc0) return rc0;
    ddst = tmp;
  }
  int rc = JACOBI_OK;
  cudaError_t e = cudaSuccess;
  if (layout == JACOBI_LAYOUT_PADDED) e = cudaMemsetAsync(ddst, 0, n, s);
  const int parity = (int)(grid_local_iter(h, grid) & 1);
  if (e == cudaSuccess)
    e = launch_gather(h->d_blocks, h->d_geom, (int32_t)G.block_begin, (int32_t)(G.block_end - G.block_begin), ddst,
                      G.dims.nx, G.dims.ny, G.dims.nz, parity, layout == JACOBI_LAYOUT_PADDED, h->plan.dtype, s);
  if (e == cudaSuccess && tmp) e = cudaMemcpyAsync(dst, tmp, n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && tmp) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) rc = set_error(JACOBI_ECUDA, "copy_out failed: %s", cudaGetErrorString(e));
  return rc;
}

int jacobi_selftest_widen(uint64_t* mismatches, void* stream) {
  if (!mismatches) return set_error(JACOBI_EINVAL, "null pointer");
  const cudaStream_t s = S(stream);
  unsigned long long* d = nullptr;
  JGB_CUDA(cudaMalloc((void**)&d, sizeof *d));
  unsigned long long n = 0;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof *d, s);
  if (e == cudaSuccess) e = launch_selftest_widen(d, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&n, d, sizeof n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  if (e != cudaSuccess) return set_error(JACOBI_ECUDA, "widening self-test failed: %s", cudaGetErrorString(e));
  *mismatches = (uint64_t)n;
  return JACOBI_OK;
}

int jacobi_selftest_div6(uint64_t* mismatches, void* stream) {
  if (!mismatches) return set_error(JACOBI_EINVAL, "null pointer");
  const cudaStream_t s = S(stream);
  unsigned long long* d = nullptr;
  JGB_CUDA(cudaMalloc((void**)&d, sizeof *d));
  unsigned long long n = 0;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof *d, s);
  if (e == cudaSuccess) e = launch_selftest_div6(d, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&n, d, sizeof n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  if (e != cudaSuccess) return set_error(JACOBI_ECUDA, "division self-test failed: %s", cudaGetErrorString(e));
  *mismatches = (uint64_t)n;
  return JACOBI_OK;
}

int jacobi_selftest_dadd(const double* a, const double* b, int64_t n, double* out, void* stream) {
  if ((!a || !b || !out) && n > 0) return set_error(JACOBI_EINVAL, "null pointer");
  if (n < 0) return set_error(JACOBI_EINVAL, "negative count");
  JGB_CUDA(launch_selftest_dadd(a, b, n, out, S(stream)));
  return JACOBI_OK;
}

int jacobi_pipe_rates(double* fp64_adds_per_s, double* int_adds_per_s, void* stream) {
  const cudaStream_t s = S(stream);
  int dev = 0, sms = 0;
  JGB_CUDA(cudaGetDevice(&dev));
  JGB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 256, blocks = sms * 8, iters = 1024;
  double* out = nullptr;
  JGB_CUDA(cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double rate[2] = {0.0, 0.0};
  cudaError_t e = cudaSuccess;
  for (int emu = 0; emu < 2 && e == cudaSuccess; ++emu) {
    e = launch_pipe_rate(emu != 0, blocks, threads, iters, out, s);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch_pipe_rate(emu != 0, blocks, threads, iters, out, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) rate[emu] = (double)blocks * threads * iters * 8 / (ms * 1e-3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return set_error(JACOBI_ECUDA, "pipe-rate probe: %s", cudaGetErrorString(e));
  if (fp64_adds_per_s) *fp64_adds_per_s = rate[0];
  if (int_adds_per_s) *int_adds_per_s = rate[1];
  return JACOBI_OK;
}

int jacobi_sync(jacobi_t* h, void* stream) {
  if (!h) return set_error(JACOBI_EINVAL, "null handle");
  JGB_CUDA(cudaStreamSynchronize(S(stream)));
  return check_err_word(h, S(stream));
}

int jacobi_read_face(jacobi_t* h, int64_t block, int32_t face, void* dst, void* stream) {
  if (!h || !dst || block < 0 || block >= (int64_t)h->plan.blocks.size() || face < 0 || face > 5)
    return set_error(JACOBI_EINVAL, "bad arguments to jacobi_read_face");
  const BlockHost& B = h->plan.blocks[block];
  const int parity = (int)(grid_local_iter(h, B.grid) & 1);
  // The slot rows are padded (x-faces to ry, the others to rx): copy the
  // face's own entries, row by row, into the compact layout.
  const size_t e = h->plan.elem;
  const int64_t width = face < 2 ? B.extent[1] : B.extent[0];
  const int64_t pitch = face < 2 ? B.ry : B.rx;
  const int64_t height = face < 4 ? B.extent[2] : B.extent[1];
  JGB_CUDA(cudaMemcpy2DAsync(dst, width * e, h->ws + B.recv_off[face][parity], pitch * e, width * e, height,
                             cudaMemcpyDeviceToHost, S(stream)));
  JGB_CUDA(cudaStreamSynchronize(S(stream)));
  return JACOBI_OK;
}

int jacobi_measure_local_halo(jacobi_t* h, int32_t on) {
  if (!h) return set_error(JACOBI_EINVAL, "null handle");
  if (h->local_halo == (on != 0)) return JACOBI_OK;
  h->local_halo = on != 0;
  const Plan& P = h->plan;
  const int64_t nb = (int64_t)P.blocks.size();
  std::vector<BlockDev> bd(nb);
  std::vector<BlockGeom> geo(nb);
  fill_block_tables(P, h->ws, 0, -1, bd.data(), geo.data(), nullptr, h->local_halo);
  JGB_CUDA(cudaDeviceSynchronize());  // no launch may be reading the old table
  // (captured graphs keep working: their launches read the table in device memory)
  JGB_CUDA(cudaMemcpy(h->d_blocks, bd.data(), nb * sizeof(BlockDev), cudaMemcpyHostToDevice));
  return JACOBI_OK;
}

int jacobi_debug_drop_block(jacobi_t* h, int64_t block) {
  if (!h || block < -1 || block >= (int64_t)h->plan.blocks.size()) return set_error(JACOBI_EINVAL, "bad block");
  h->drop_block = block;
  h->tables_dirty = true;
  return JACOBI_OK;
}

}  // extern "C"
