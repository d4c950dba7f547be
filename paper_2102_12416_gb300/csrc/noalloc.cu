// Allocation-free residual of a caller-owned padded state array.
//
// Some callers cannot allocate device memory at the point where they need a
// residual: services that reserve all device memory up front and forbid
// later allocations (a fixed footprint, or a framework whose caching
// allocator must account for every byte), and loops that cannot afford the
// device-wide synchronisation a cudaMalloc or cudaFree may bring.  For them
// this file keeps the reduction scratch in a fixed file-scope device array
// instead of a workspace: every GPU that loads the library holds it (256 KB)
// until exit.
//
// The array is shared by every call on a device and keeps the last call's
// contents; each call overwrites every partial it later reads, so nothing has
// to be cleared first.  Calls whose kernels overlap on the GPU (different
// streams without ordering) race on the array and give wrong results.
#include <mutex>

#include "runtime.h"

using namespace jgb;

namespace {

constexpr int kMaxPlanes = JACOBI_NOALLOC_MAX_PLANES;
constexpr int kNaThreads = 256;

// Two partials per z-plane: sum of r^2 and sum of b^2.
static __device__ __align__(256) double g_noalloc_scratch[2 * kMaxPlanes];

template <typename T>
__global__ void __launch_bounds__(kNaThreads) k_noalloc_planes(const T* __restrict__ u, int64_t nx, int64_t ny,
                                                             int64_t nz, double* scratch) {
  const int64_t k = 1 + blockIdx.x;  // padded plane index
  const int64_t px = nx + 2, py = ny + 2;
  const int64_t n = nx * ny;
  double ar = 0.0, ab = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += kNaThreads) {
    const int64_t i = 1 + e % nx, j = 1 + e / nx;
    const int64_t o = (k * py + j) * px + i;
    const double w[6] = {(double)u[o - 1], (double)u[o + 1], (double)u[o - px],
                         (double)u[o + px], (double)u[o - px * py], (double)u[o + px * py]};
    const bool bnd[6] = {i == 1, i == nx, j == 1, j == ny, k == 1, k == nz};
    double wb[6];
    for (int q = 0; q < 6; ++q) wb[q] = bnd[q] ? w[q] : 0.0;
    const double s = __dadd_rn(__dadd_rn(__dadd_rn(w[0], w[1]), __dadd_rn(w[2], w[3])), __dadd_rn(w[4], w[5]));
    const double sb = __dadd_rn(__dadd_rn(__dadd_rn(wb[0], wb[1]), __dadd_rn(wb[2], wb[3])), __dadd_rn(wb[4], wb[5]));
    const double r = __dsub_rn(s, __dmul_rn(6.0, (double)u[o]));
    ar = fma(r, r, ar);
    ab = fma(sb, sb, ab);
  }
  __shared__ double red[kNaThreads / 32];
  const double sr = block_sum<kNaThreads>(ar, red);
  const double sbb = block_sum<kNaThreads>(ab, red);
  if (threadIdx.x == 0) {
    scratch[2 * blockIdx.x] = sr;
    scratch[2 * blockIdx.x + 1] = sbb;
  }
}

// One warp: fixed-order sum of the plane partials, then |r|, |b|, rel.
__global__ void k_noalloc_finish(const double* scratch, int64_t nz, double* out) {
  double r = 0.0, b = 0.0;
  for (int64_t q = threadIdx.x; q < nz; q += 32) {
    r += scratch[2 * q];
    b += scratch[2 * q + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    r += __shfl_xor_sync(0xffffffffu, r, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (threadIdx.x == 0) {
    const double rn = sqrt(r), bn = sqrt(b);
    out[0] = rn;
    out[1] = bn;
    out[2] = bn > 0.0 ? rn / bn : rn;
  }
}

// Device address of the scratch array, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_ptr[kMaxDevices] = {};

int scratch_for_current_device(double** out) {
  int dev = 0;
  JGB_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(JACOBI_EINVAL, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return set_error(JACOBI_ECUDA, "cudaGetSymbolAddress(scratch) failed on device %d: %s", dev,
                       cudaGetErrorString(e));
    g_ptr[dev] = (double*)p;
  }
  *out = g_ptr[dev];
  return JACOBI_OK;
}

}  // namespace

extern "C" int jacobi_residual_noalloc(const void* u_padded, jacobi_dim3 grid, jacobi_dtype dtype, double* out,
                                       void* stream) {
  if (!u_padded || !out) return set_error(JACOBI_EINVAL, "null pointer");
  if (dtype != JACOBI_F64 && dtype != JACOBI_F32) return set_error(JACOBI_EINVAL, "bad dtype");
  if (grid.nx < 1 || grid.ny < 1 || grid.nz < 1) return set_error(JACOBI_EINVAL, "grid sizes must be positive");
  if (grid.nz > kMaxPlanes)
    return set_error(JACOBI_EINVAL, "jacobi_residual_noalloc: nz = %lld exceeds the fixed scratch limit of %d planes",
                     (long long)grid.nz, kMaxPlanes);
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  const cudaStream_t s = (cudaStream_t)stream;
  if (dtype == JACOBI_F64)
    k_noalloc_planes<double><<<(unsigned)grid.nz, kNaThreads, 0, s>>>((const double*)u_padded, grid.nx, grid.ny, grid.nz,
                                                                     scratch);
  else
    k_noalloc_planes<float><<<(unsigned)grid.nz, kNaThreads, 0, s>>>((const float*)u_padded, grid.nx, grid.ny, grid.nz,
                                                                    scratch);
  JGB_CUDA(cudaGetLastError());
  k_noalloc_finish<<<1, 32, 0, s>>>(scratch, grid.nz, out);
  JGB_CUDA(cudaGetLastError());
  return JACOBI_OK;
}
