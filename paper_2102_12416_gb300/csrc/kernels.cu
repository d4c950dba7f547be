// Jacobi3D support kernels for sm_103a: initial state, state scatter/gather,
// the |b| partials, the deterministic per-grid reduction and the explicit
// pack/copy form of the halo exchange.  The stencil step kernels (Sec. 4.3
// Jacobi iteration, fused face pack, FP64 residual, persistent driver) are in
// step.cu.

#include "kernels.cuh"

namespace jgb {

namespace {

// ---------------------------------------------------------------------------
// Initial values
// ---------------------------------------------------------------------------
__device__ double init_value(const InitDev& I, int64_t gi, int64_t gj, int64_t gk) {
  const bool bnd = gi == 0 || gj == 0 || gk == 0 || gi == I.NX + 1 || gj == I.NY + 1 ||
                   gk == I.NZ + 1;
  const uint64_t idx = ((uint64_t)gk * (uint64_t)(I.NY + 2) + (uint64_t)gj) * (uint64_t)(I.NX + 2) +
                       (uint64_t)gi;
  if (!bnd) {
    if (I.interior == 0) return 0.0;
    if (I.interior == 1) return u01(I.interior_seed, idx);
  }
  if (I.bc == 2) return u01(I.bc_seed, idx);
  const double x = (double)gi / (double)(I.NX + 1);
  const double y = (double)gj / (double)(I.NY + 1);
  const double z = (double)gk / (double)(I.NZ + 1);
  double g = radd(radd(x, rmul(2.0, y)), rmul(3.0, z));
  if (I.bc == 1) g = radd(g, rmul(I.noise_amp, u01(I.bc_seed, idx)));
  return g;
}

template <typename T> __device__ __forceinline__ T to_state(double v);
template <> __device__ __forceinline__ double to_state<double>(double v) { return v; }
template <> __device__ __forceinline__ float to_state<float>(double v) { return __double2float_rn(v); }

// Entries of the (padded) receive slot of face f.
__device__ __forceinline__ int64_t face_elems(const BlockDev& B, int f) {
  if (f == XM || f == XP) return (int64_t)B.nz * B.ry;
  if (f == YM || f == YP) return (int64_t)B.nz * B.rx;
  return (int64_t)B.ry * B.rx;
}

// Global padded grid coordinates of slot entry e of face f of block (B, G);
// false for a padding entry.
__device__ __forceinline__ bool face_coords(const BlockDev& B, const BlockGeom& G, int f, int64_t e,
                                            int64_t& gi, int64_t& gj, int64_t& gk) {
  const int nx = B.nx, ny = B.ny, nz = B.nz;
  if (f == XM || f == XP) {
    const int64_t k = e / B.ry, j = e % B.ry;
    gi = G.ox + (f == XM ? 0 : nx + 1);
    gj = G.oy + 1 + j;
    gk = G.oz + 1 + k;
    return j < ny;
  }
  if (f == YM || f == YP) {
    const int64_t k = e / B.rx, i = e % B.rx;
    gi = G.ox + 1 + i;
    gj = G.oy + (f == YM ? 0 : ny + 1);
    gk = G.oz + 1 + k;
    return i < nx;
  }
  const int64_t j = e / B.rx, i = e % B.rx;
  gi = G.ox + 1 + i;
  gj = G.oy + 1 + j;
  gk = G.oz + (f == ZM ? 0 : nz + 1);
  return i < nx && j < ny;
}

// Offset of interior point (i, j, k) in the block's padded storage.
__device__ __forceinline__ int64_t cell(const BlockDev& B, int64_t i, int64_t j, int64_t k) {
  return k * B.plane_pitch + j * B.rx + i;
}

// Calls f(i, j, k) for every interior point of B: the CTA's warps take the
// rows (j, k) in turn, the lanes walk a row (coalesced; one division per row).
template <typename F>
__device__ __forceinline__ void for_interior(const BlockDev& B, F f) {
  const int nx = B.nx, ny = B.ny, rows = B.ny * B.nz;
  const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int row = threadIdx.x >> 5; row < rows; row += nwarps) {
    const int k = row / ny, j = row - k * ny;
    for (int i = lane; i < nx; i += 32) f(i, j, k);
  }
}

template <typename T>
__global__ void k_init_interior(const BlockDev* __restrict__ blocks, const BlockGeom* __restrict__ geom,
                                const InitDev* __restrict__ inits) {
  const BlockDev& B = blocks[blockIdx.x];
  const BlockGeom G = geom[blockIdx.x];
  const InitDev I = inits[G.grid];
  T* U = (T*)B.u[0];
  // a flat walk: for a zero interior this is a pure store stream, which the
  // row-wise walk issued ~3x slower
  const int64_t nx = B.nx, ny = B.ny, n = nx * ny * B.nz, pitch = B.plane_pitch, rx = B.rx;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    const int64_t i = e % nx, j = (e / nx) % ny, k = e / (nx * ny);
    U[k * pitch + j * rx + i] = to_state<T>(init_value(I, G.ox + 1 + i, G.oy + 1 + j, G.oz + 1 + k));
  }
}

template <typename T>
__global__ void k_init_slots(const BlockDev* __restrict__ blocks, const BlockGeom* __restrict__ geom,
                             const InitDev* __restrict__ inits) {
  const BlockDev& B = blocks[blockIdx.x];
  const BlockGeom G = geom[blockIdx.x];
  const InitDev I = inits[G.grid];
  const int f = blockIdx.y;
  T* S = (T*)B.recv[f][0];
  const int64_t n = face_elems(B, f);
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    int64_t gi, gj, gk;
    if (face_coords(B, G, f, e, gi, gj, gk)) S[e] = to_state<T>(init_value(I, gi, gj, gk));
  }
}

template <typename T>
__global__ void k_scatter(const BlockDev* __restrict__ blocks, const BlockGeom* __restrict__ geom, int32_t b0,
                          const T* __restrict__ src, int64_t NX, int64_t NY, int parity) {
  const int b = b0 + blockIdx.x;
  const BlockDev& B = blocks[b];
  const BlockGeom G = geom[b];
  const int64_t px = NX + 2, py = NY + 2;
  if (blockIdx.y == 0) {
    T* U = (T*)B.u[parity];
    const int64_t pitch = B.plane_pitch, rx = B.rx;
    for_interior(B, [=](int i, int j, int k) {
      U[k * pitch + j * rx + i] = src[((G.oz + 1 + k) * py + (G.oy + 1 + j)) * px + (G.ox + 1 + i)];
    });
  } else {
    const int f = blockIdx.y - 1;
    T* S = (T*)B.recv[f][parity];
    const int64_t n = face_elems(B, f);
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
      int64_t gi, gj, gk;
      if (face_coords(B, G, f, e, gi, gj, gk)) S[e] = src[(gk * py + gj) * px + gi];
    }
  }
}

template <typename T>
__global__ void k_gather(const BlockDev* __restrict__ blocks, const BlockGeom* __restrict__ geom, int32_t b0,
                         T* __restrict__ dst, int64_t NX, int64_t NY, int parity, int padded) {
  const int b = b0 + blockIdx.x;
  const BlockDev& B = blocks[b];
  const BlockGeom G = geom[b];
  const int64_t off = padded ? 1 : 0;
  const int64_t px = NX + 2 * off, py = NY + 2 * off;
  if (blockIdx.y == 0) {
    const T* U = (const T*)B.u[parity];
    const int64_t pitch = B.plane_pitch, rx = B.rx;
    for_interior(B, [=](int i, int j, int k) {
      dst[((G.oz + off + k) * py + (G.oy + off + j)) * px + (G.ox + off + i)] = U[k * pitch + j * rx + i];
    });
  } else if (padded) {
    const int f = blockIdx.y - 1;
    if (B.nbr[f] >= 0) return;  // only Dirichlet faces lie on the padded boundary
    const T* S = (const T*)B.recv[f][parity];
    const int64_t n = face_elems(B, f);
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
      int64_t gi, gj, gk;
      if (face_coords(B, G, f, e, gi, gj, gk)) dst[(gk * py + gj) * px + gi] = S[e];
    }
  }
}

// |b|^2 partials: the residual expression with every interior value set to 0,
// so only Dirichlet ghosts contribute.  A work item is either one TX x TY tile
// (x0 >= 0) or the row window [ya, yb) of its block's planes over [z0, z1)
// (x0 < 0; a plane may be split into several windows, each its own item).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_bnorm(StepLaunch a) {
  const WorkItem w = a.items[blockIdx.x];
  const BlockDev& B = a.blocks[w.block];
  const int p = (int)((a.it - a.grids[B.grid].start_iter) & 1);
  const int nx = B.nx, ny = B.ny, nz = B.nz, rx = B.rx, ry = B.ry;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int xa = w.x0 >= 0 ? w.x0 : 0, ya = w.x0 >= 0 ? w.y0 : w.ya;
  const int xb = w.x0 >= 0 ? w.x0 + TX : nx, yb = min(w.x0 >= 0 ? w.y0 + TY : (int)w.yb, ny);
  double acc = 0.0;
  for (int y0 = ya; y0 < yb; y0 += TY)
    for (int x0 = xa; x0 < xb; x0 += TX) {
      const int i = x0 + tx, j = y0 + ty;
      if (i >= nx || j >= yb) continue;
      for (int k = w.z0; k < w.z1; ++k) {
        double v[6] = {0, 0, 0, 0, 0, 0};
        if (i == 0 && B.nbr[XM] < 0) v[0] = (double)((const T*)B.recv[XM][p])[(int64_t)k * ry + j];
        if (i == nx - 1 && B.nbr[XP] < 0) v[1] = (double)((const T*)B.recv[XP][p])[(int64_t)k * ry + j];
        if (j == 0 && B.nbr[YM] < 0) v[2] = (double)((const T*)B.recv[YM][p])[(int64_t)k * rx + i];
        if (j == ny - 1 && B.nbr[YP] < 0) v[3] = (double)((const T*)B.recv[YP][p])[(int64_t)k * rx + i];
        if (k == 0 && B.nbr[ZM] < 0) v[4] = (double)((const T*)B.recv[ZM][p])[(int64_t)j * rx + i];
        if (k == nz - 1 && B.nbr[ZP] < 0) v[5] = (double)((const T*)B.recv[ZP][p])[(int64_t)j * rx + i];
        const double sb =
            __dadd_rn(__dadd_rn(__dadd_rn(v[0], v[1]), __dadd_rn(v[2], v[3])), __dadd_rn(v[4], v[5]));
        acc = fma(sb, sb, acc);
      }
    }
  __shared__ double red[kThreads / 32];
  const double s = block_sum<kThreads>(acc, red);
  if (threadIdx.x == 0) a.partials[w.slot] = s;
}

// Flag every grid whose current state (interior at its parity and all six
// receive slots) holds a value outside the domain of the integer-pipe adder
// dadd_nn; the step kernels then keep that grid's FP64 sums (the FP64
// stencil's, and the FP32 residual's of widened values) on the FP64 pipe.  By the
// discrete maximum principle Jacobi iterates stay within the range of the
// boundary and initial data, so a state that passes keeps passing.
template <typename T>
__global__ void k_emu_check(const BlockDev* __restrict__ blocks, const GridDev* grids, GridNorm* norms, int64_t it) {
  // FP64: the high word (sign clear, exponent below 2040); FP32: the whole
  // word (sign clear, finite: widened, such a value is inside the domain)
  constexpr int W = sizeof(T) / 4;
  constexpr uint32_t kLimit = sizeof(T) == 8 ? kEmuHiLimit : 0x7F800000u;
  const BlockDev& B = blocks[blockIdx.x];
  const int p = (int)((it - grids[B.grid].start_iter) & 1);
  const uint32_t* U = (const uint32_t*)B.u[p];
  bool bad = false;
  const int64_t pitch = B.plane_pitch, rx = B.rx;
  for_interior(B, [&](int i, int j, int k) { bad |= U[W * (k * pitch + j * rx + i) + W - 1] >= kLimit; });
  for (int f = 0; f < 6; ++f) {
    const uint32_t* S = (const uint32_t*)B.recv[f][p];
    const int64_t m = face_elems(B, f);
    for (int64_t e = threadIdx.x; e < m; e += blockDim.x) bad |= S[W * e + W - 1] >= kLimit;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&norms[B.grid].emu_bad, 1u);
}

__global__ void k_emu_reset(GridNorm* norms, const int32_t* grid_ids, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) norms[grid_ids[q]].emu_bad = 0u;
}

// Self-test of the integer-pipe adder: out[i] = dadd_nn(a[i], b[i]).
__global__ void k_selftest_dadd(const double* a, const double* b, int64_t n, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = i < n ? i : n - 1;  // clamped index: every lane loads in bounds
  const double r = dadd_nn(a[j], b[j]);
  if (i < n) out[i] = r;
}

// Every binary32 bit pattern through widen_f32, against the conversion
// instruction: counts results that differ bit for bit (a NaN must stay a NaN).
__global__ void k_selftest_widen(unsigned long long* bad) {
  unsigned long long n = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < (1ull << 32); x += stride) {
    const float f = __uint_as_float((uint32_t)x);
    const double a = widen_f32(f), b = (double)f;
    const bool ok = (a != a && b != b) || __double_as_longlong(a) == __double_as_longlong(b);
    n += ok ? 0ull : 1ull;
  }
  if (n) atomicAdd(bad, n);
}

// Every binary32 bit pattern through div6 (the FP32 update's RN(s / 6) in two
// operations, with its fallback), against the division instruction sequence:
// counts results that differ bit for bit (a NaN must stay a NaN).
__global__ void k_selftest_div6(unsigned long long* bad) {
  unsigned long long n = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < (1ull << 32); x += stride) {
    const float f = __uint_as_float((uint32_t)x);
    const float a = div6(f), b = __fdiv_rn(f, 6.0f);
    const bool ok = (a != a && b != b) || __float_as_uint(a) == __float_as_uint(b);
    n += ok ? 0ull : 1ull;
  }
  if (n) atomicAdd(bad, n);
}

// Pipe-rate probe: chains of FP64 adds on the FP64 pipe (EMU = false) or
// through dadd_nn on the integer pipe (EMU = true); 8 independent chains per
// thread keep either pipe busy.  The result is stored so nothing is elided.
template <bool EMU>
__global__ void k_pipe_rate(double* out, int iters) {
  double x[8];
  for (int c = 0; c < 8; ++c) x[c] = 0.25 + 1e-3 * (double)(threadIdx.x + c);
  const double inc = 1e-9 + 1e-13 * (double)blockIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = EMU ? dadd_nn(x[c], inc) : __dadd_rn(x[c], inc);
  }
  double s = 0.0;
  for (int c = 0; c < 8; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// One warp per grid: lane l sums slots item_begin + l, + l + 32, ... in order,
// then a fixed butterfly combines the lanes.
__global__ void k_reduce(const GridDev* grids, GridNorm* norms, const int32_t* grid_ids, const double* partials,
                         int which) {
  const int g = grid_ids[blockIdx.x];
  const GridDev G = grids[g];
  GridNorm& N = norms[g];
  double s = 0.0;
  for (int q = G.item_begin + threadIdx.x; q < G.item_end; q += 32) s += partials[q];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) {
    if (which == 0) {
      N.r_norm2 = s;
      N.r_norm = sqrt(s);
      const double b = sqrt(N.b_norm2);
      N.rel = b > 0.0 ? N.r_norm / b : N.r_norm;
    } else {
      N.b_norm2 = s;
    }
  }
}

// Explicit exchange, step 1: pack each internal face of the new iterate
// (parity p ^ 1 state) into a contiguous staging buffer, or (direct) straight
// into the neighbour's receive slot for the next parity.
template <typename T>
__global__ void k_pack_faces(const BlockDev* __restrict__ blocks, const int32_t* __restrict__ ids,
                             void* const* staging, const GridDev* grids, int64_t it, int direct) {
  const int b = ids[blockIdx.x], f = blockIdx.y;
  const BlockDev& B = blocks[b];
  if (B.nbr[f] < 0) return;
  const int p = (int)((it - grids[B.grid].start_iter) & 1);
  const T* U = (const T*)B.u[p ^ 1];
  T* S = direct ? (T*)B.send[f][p ^ 1] : (T*)staging[b * 6 + f];
  const int64_t nx = B.nx, ny = B.ny, nz = B.nz, rx = B.rx, ry = B.ry;
  const int64_t n = face_elems(B, f);
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {  // padding entries copy padding
    int64_t i, j, k;
    if (f == XM || f == XP) { k = e / ry; j = e % ry; i = (f == XM) ? 0 : nx - 1; }
    else if (f == YM || f == YP) { k = e / rx; i = e % rx; j = (f == YM) ? 0 : ny - 1; }
    else { j = e / rx; i = e % rx; k = (f == ZM) ? 0 : nz - 1; }
    S[e] = U[cell(B, i, j, k)];
  }
}

// Explicit exchange, step 2: the channel transfer of each packed face into the
// neighbour's receive slot for the next parity.
template <typename T>
__global__ void k_copy_faces(const BlockDev* __restrict__ blocks, const int32_t* __restrict__ ids,
                             void* const* staging, const GridDev* grids, int64_t it) {
  const int b = ids[blockIdx.x], f = blockIdx.y;
  const BlockDev& B = blocks[b];
  if (B.nbr[f] < 0) return;
  const int p = (int)((it - grids[B.grid].start_iter) & 1);
  const T* S = (const T*)staging[b * 6 + f];
  T* D = (T*)B.send[f][p ^ 1];
  const int64_t n = face_elems(B, f);
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) D[e] = S[e];
}

// Posted receives of the GPU Messaging form: one CTA per descriptor copies
// its payload (16-byte vectors; every face buffer is a whole number of them).
__global__ void k_copy_desc(const CopyDesc* __restrict__ d, int32_t n) {
  const CopyDesc c = d[blockIdx.x];
  const uint4* src = (const uint4*)c.src;
  uint4* dst = (uint4*)c.dst;
  const int64_t nv = c.bytes / 16;
  for (int64_t q = threadIdx.x; q < nv; q += blockDim.x) dst[q] = __ldcg(src + q);
}

}  // namespace

cudaError_t launch_copy_desc(const CopyDesc* d, int32_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_copy_desc<<<n, 256, 0, s>>>(d, n);
  return cudaGetLastError();
}

cudaError_t launch_bnorm(const StepLaunch& a, cudaStream_t s) {
  if (a.n_items <= 0) return cudaSuccess;
  if (a.dtype == 0) k_bnorm<double><<<a.n_items, kThreads, 0, s>>>(a);
  else k_bnorm<float><<<a.n_items, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const GridDev* grids, GridNorm* norms, const int32_t* grid_ids, int32_t n,
                          const double* partials, int which, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_reduce<<<n, 32, 0, s>>>(grids, norms, grid_ids, partials, which);
  return cudaGetLastError();
}

cudaError_t launch_pack_faces(const BlockDev* blocks, const int32_t* ids, int32_t n_blocks, void* const* staging,
                              const GridDev* grids, int64_t it, int32_t dtype, cudaStream_t s, bool direct) {
  if (n_blocks <= 0) return cudaSuccess;
  const dim3 grid(n_blocks, 6);
  if (dtype == 0) k_pack_faces<double><<<grid, 256, 0, s>>>(blocks, ids, staging, grids, it, direct ? 1 : 0);
  else k_pack_faces<float><<<grid, 256, 0, s>>>(blocks, ids, staging, grids, it, direct ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_copy_faces(const BlockDev* blocks, const int32_t* ids, int32_t n_blocks, void* const* staging,
                              const GridDev* grids, int64_t it, int32_t dtype, cudaStream_t s) {
  if (n_blocks <= 0) return cudaSuccess;
  const dim3 grid(n_blocks, 6);
  if (dtype == 0) k_copy_faces<double><<<grid, 256, 0, s>>>(blocks, ids, staging, grids, it);
  else k_copy_faces<float><<<grid, 256, 0, s>>>(blocks, ids, staging, grids, it);
  return cudaGetLastError();
}

cudaError_t launch_emu_check(const BlockDev* blocks, int32_t n_blocks, const GridDev* grids, GridNorm* norms,
                             const int32_t* grid_ids, int32_t n_grids, int64_t it, int dtype, cudaStream_t s) {
  if (n_grids > 0) k_emu_reset<<<(n_grids + 127) / 128, 128, 0, s>>>(norms, grid_ids, n_grids);
  if (n_blocks > 0) {
    if (dtype == 0) k_emu_check<double><<<n_blocks, 256, 0, s>>>(blocks, grids, norms, it);
    else k_emu_check<float><<<n_blocks, 256, 0, s>>>(blocks, grids, norms, it);
  }
  return cudaGetLastError();
}

cudaError_t launch_pipe_rate(bool emu, int blocks, int threads, int iters, double* out, cudaStream_t s) {
  if (emu) k_pipe_rate<true><<<blocks, threads, 0, s>>>(out, iters);
  else k_pipe_rate<false><<<blocks, threads, 0, s>>>(out, iters);
  return cudaGetLastError();
}

cudaError_t launch_selftest_dadd(const double* a, const double* b, int64_t n, double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_selftest_dadd<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, b, n, out);
  return cudaGetLastError();
}

cudaError_t launch_selftest_widen(unsigned long long* bad, cudaStream_t s) {
  k_selftest_widen<<<1216, 256, 0, s>>>(bad);
  return cudaGetLastError();
}

cudaError_t launch_selftest_div6(unsigned long long* bad, cudaStream_t s) {
  k_selftest_div6<<<1216, 256, 0, s>>>(bad);
  return cudaGetLastError();
}

cudaError_t launch_init(const BlockDev* blocks, const BlockGeom* geom, int32_t n_blocks, const InitDev* inits,
                        int32_t dtype, cudaStream_t s) {
  if (n_blocks <= 0) return cudaSuccess;
  if (dtype == 0) {
    k_init_interior<double><<<n_blocks, 256, 0, s>>>(blocks, geom, inits);
    k_init_slots<double><<<dim3(n_blocks, 6), 256, 0, s>>>(blocks, geom, inits);
  } else {
    k_init_interior<float><<<n_blocks, 256, 0, s>>>(blocks, geom, inits);
    k_init_slots<float><<<dim3(n_blocks, 6), 256, 0, s>>>(blocks, geom, inits);
  }
  return cudaGetLastError();
}

cudaError_t launch_scatter(const BlockDev* blocks, const BlockGeom* geom, int32_t b0, int32_t nb, const void* src,
                           int64_t NX, int64_t NY, int64_t NZ, int parity, int32_t dtype, cudaStream_t s) {
  (void)NZ;
  if (nb <= 0) return cudaSuccess;
  const dim3 grid(nb, 7);
  if (dtype == 0) k_scatter<double><<<grid, 256, 0, s>>>(blocks, geom, b0, (const double*)src, NX, NY, parity);
  else k_scatter<float><<<grid, 256, 0, s>>>(blocks, geom, b0, (const float*)src, NX, NY, parity);
  return cudaGetLastError();
}

cudaError_t launch_gather(const BlockDev* blocks, const BlockGeom* geom, int32_t b0, int32_t nb, void* dst,
                          int64_t NX, int64_t NY, int64_t NZ, int parity, int padded, int32_t dtype,
                          cudaStream_t s) {
  (void)NZ;
  if (nb <= 0) return cudaSuccess;
  const dim3 grid(nb, 7);
  if (dtype == 0) k_gather<double><<<grid, 256, 0, s>>>(blocks, geom, b0, (double*)dst, NX, NY, parity, padded);
  else k_gather<float><<<grid, 256, 0, s>>>(blocks, geom, b0, (float*)dst, NX, NY, parity, padded);
  return cudaGetLastError();
}

}  // namespace jgb
