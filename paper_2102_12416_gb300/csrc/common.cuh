// Device-side definitions shared by the library's kernels: block and work-item
// tables, rounding-exact arithmetic, the SplitMix64 generator, release/acquire
// flag operations and bounded waits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace jgb {

// Faces in the order xm, xp, ym, yp, zm, zp ("m" = low side, "p" = high side).
enum Face { XM = 0, XP = 1, YM = 2, YP = 3, ZM = 4, ZP = 5 };
__host__ __device__ inline int opposite(int f) { return f ^ 1; }

// Device error word values (first failure wins).
enum DevError : uint32_t {
  DEV_OK = 0,
  DEV_TIMEOUT = 1,   // a bounded wait expired
  DEV_SEQ = 2,       // channel sequence / size mismatch
};

// One block of the decomposition (a "chare" of the paper's Jacobi3D).
// Interior storage is padded: a row holds rx >= nx elements (nx rounded up to
// a 16-byte vector) and a plane ry >= ny rows (ny rounded up to 4), so every
// row starts on a 16-byte boundary and the plane-streaming kernels take any
// block shape.  Plane k starts at k * plane_pitch (>= rx * ry, rounded up) and
// point (i, j, k) sits at k * plane_pitch + j * rx + i.  Receive slots, by
// face, use the same padded pitches:
//   xm/xp: [k][j] (nz x ry)   ym/yp: [k][i] (nz x rx)   zm/zp: [j][i] (ry x rx)
// Padding entries never feed a real point: the kernels substitute the ghost
// value for any padding lane or row a real point would read.  recv[f][p] is
// read at iterations with parity p; for a Dirichlet face both parities point
// at the same constant boundary buffer.  send[f][p] is the neighbour's
// recv[opposite(f)][p] (written with the NEW iterate, at parity
// p = (it + 1) & 1), or null on a Dirichlet face.
struct BlockDev {
  void* u[2];
  void* recv[6][2];
  void* send[6][2];
  int32_t nx, ny, nz;
  int32_t grid;
  int64_t plane_pitch;
  int32_t nbr[6];
  int32_t rx, ry;
};

// One CTA's share of a step over the z-range [z0, z1) of block `block`:
//   x0 >= 0: the TX x TY tile of columns at (x0, y0);
//   x0 <  0: padded rows [ya, yb) of the x-y planes, streamed through
//            shared memory by a CTA of (y0 & 15) consumer warps (2, 4 or 8;
//            y0 & 16 marks a block with padding), each
//            thread computing 4 rows of one 16-byte vector column.
// `slot` indexes the reduction partials.
struct WorkItem {
  int32_t block;
  int32_t slot;
  int16_t x0, y0;
  int16_t z0, z1;
  int16_t ya, yb;
};

// Per-grid state written by the host.
struct GridDev {
  int64_t start_iter;   // global iteration at which this grid's local count was 0
  int32_t item_begin;   // partial slots [item_begin, item_end) belong to this grid
  int32_t item_end;
  int32_t active;       // 0: frozen (step kernels leave the grid untouched)
  int32_t pad_;
};

// Per-grid norms written by the reduction kernel.
struct GridNorm {
  double b_norm2;       // |b|^2, computed once per boundary
  double r_norm2;       // |b - A u|^2 of the last residual evaluation
  double r_norm;        // sqrt(r_norm2)
  double rel;           // r_norm / |b| (r_norm when |b| == 0)
  uint32_t emu_bad;     // the state has a value outside dadd_nn's domain (widened, for FP32)
  uint32_t pad_;
};

// Tile shape of the table-driven kernels: 32 x 8 threads, each thread walks z.
constexpr int TX = 32;
constexpr int TY = 8;
constexpr int kThreads = TX * TY;

// ---- rounding-exact arithmetic (no contraction into FMA) --------------------
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }

// ---- FP64 addition on the integer pipe -----------------------------------------
// On this GPU the FP64 pipe retires about 0.5 T adds/s, about the rate at
// which the integer ALU pipe runs the routine below, and the two pipes run in
// parallel; a stencil that spreads its FP64 adds over both raises its add
// throughput.  dadd_nn returns exactly the IEEE-754 binary64 sum rounded to
// nearest-even (bit-identical to __dadd_rn) for operands whose sign bit is
// clear and whose exponent field is below 2040 (so no sum can overflow);
// subnormals and zeros included.  Method: order the operands by their high
// words (equal high words imply equal exponents, where the order does not
// matter), take the 53-bit significands (hidden bit for normal numbers,
// effective exponent max(e, 1)), place the larger at bit 62 of a 64-bit word
// (10 guard bits), shift the smaller right by the exponent difference d
// (clamped to 63), add, and renormalise by at most one bit.  Rounding to
// nearest-even adds 0x1FF + (lsb | sticky) before dropping the 10 guard
// bits, where sticky says that the alignment or renormalisation shift dropped
// a nonzero bit: below half (guard bits < 0x200) never carries, above half
// always carries, and exactly 0x200 carries iff the value is above the tie
// (sticky) or the tie goes to the even neighbour (lsb).  The exponent is
// added into the high word, so a rounding carry moves it correctly.
__device__ __forceinline__ double dadd_nn(double a, double b) {
  const uint64_t A = (uint64_t)__double_as_longlong(a), B = (uint64_t)__double_as_longlong(b);
  const uint32_t ah = (uint32_t)(A >> 32), bh = (uint32_t)(B >> 32);
  const bool sw = bh > ah;
  const uint64_t X = sw ? B : A, Y = sw ? A : B;
  const uint32_t ex = max((uint32_t)(X >> 52), 1u), ey = max((uint32_t)(Y >> 52), 1u);
  const uint64_t mx = X - ((uint64_t)(ex - 1u) << 52);
  const uint64_t my = Y - ((uint64_t)(ey - 1u) << 52);
  const uint32_t d = min(ex - ey, 63u);
  const uint64_t ys = my << 10;
  const uint64_t ya = ys >> d;
  uint64_t Z = (mx << 10) + ya;
  const uint32_t s = (uint32_t)(Z >> 63);
  const uint32_t sticky = (uint32_t)((ya << d) != ys) | ((uint32_t)Z & s);
  Z >>= s;
  const uint32_t lo = (uint32_t)Z;
  Z += 0x1FFu + (((lo >> 10) | sticky) & 1u);
  return __longlong_as_double((long long)((Z >> 10) + ((uint64_t)(ex + s - 1u) << 52)));
}

// High-word bound of the values dadd_nn accepts: sign clear, exponent < 2040.
constexpr uint32_t kEmuHiLimit = 0x7F800000u;

template <typename T> struct C6;
template <> struct C6<double> { static constexpr double v = 1.0 / 6.0; };

// ---- the last operation of an update: FP64 s * RN(1/6), FP32 RN(s / 6) -----
// In FP64 the double nearest 1/6 is 2^-55 relative away from it, far below the
// iteration's rounding noise.  In FP32 the float nearest 1/6 exceeds it by a
// third of an ulp, which would scale every update by 1 + 2^-25 and let the
// iterate drift; FP32 therefore divides, rounding s / 6 once.
//
// RN(s / 6) in two operations, by the method of Brisebarre, Muller and Raina
// for division by a constant known in advance ("Accelerating correctly
// rounded floating-point division when the divisor is known in advance",
// IEEE Trans. Computers 53(8), 2004): with zh = RN(1/6) and zl = RN(1/6 - zh),
// q = RN(s * zh + RN(s * zl)), one multiply and one fused multiply-add.
// Checked exhaustively over all 2^32 binary32 inputs against IEEE division:
// equal for +0 and for every finite s with exponent field >= 6
// (|s| >= 2^-121).  Below that s * zl loses bits to underflow, and -0 and
// the infinities come out with the wrong sign or as a NaN; div6_small covers
// those inputs exactly without a division (a Jacobi run from a zero interior
// carries a band of such tiny values behind its front for thousands of
// iterations, so this path must stay cheap).  jacobi_selftest_div6 repeats
// the exhaustive check on the device against the division instruction.
__device__ __forceinline__ float div6_fast(float s) {
  constexpr float zh = 0x1.555556p-3f;    // RN(1/6)
  constexpr float zl = -0x1.555556p-28f;  // RN(1/6 - zh)
  return __fmaf_rn(s, zh, __fmul_rn(s, zl));
}
// True when div6_fast(s) == RN(s / 6): +0, or a finite s with exponent field >= 6.
__device__ __forceinline__ bool div6_fast_ok(float s) {
  const uint32_t b = __float_as_uint(s);
  return ((b & 0x7FFFFFFFu) - 0x03000000u) < (0x7F800000u - 0x03000000u) || b == 0u;
}
// RN(s / 6) for the inputs div6_fast does not take:
//  - infinities and NaNs: s * RN(1/6) keeps both classes (inf / 6 = inf);
//  - exponent field 4 or 5: s * 2^24 lies in div6_fast's domain and the
//    quotient is at least 2^-126 (normal), so both scalings are exact;
//  - exponent field <= 3 (zeros included): s = S * 2^-149 with an integer
//    S < 2^26, and s / 6 < 2^-124 lies where floats are the multiples of
//    2^-149 (exponent field 0 or 1, whose encodings are exactly the integers
//    Q of Q * 2^-149), so RN(s / 6) = RN(S / 6) * 2^-149 with the integer
//    quotient rounded half to even, and the sign bit copied.
__device__ __forceinline__ float div6_small(float s) {
  const uint32_t b = __float_as_uint(s), sign = b & 0x80000000u, a = b ^ sign;
  if (a >= 0x7F800000u) return __fmul_rn(s, 0x1.555556p-3f);
  if (a >= 0x02000000u) return __fmul_rn(div6_fast(__fmul_rn(s, 0x1p24f)), 0x1p-24f);
  const uint32_t e = a >> 23;
  const uint32_t S = e ? ((a & 0x7FFFFFu) | 0x800000u) << (e - 1u) : a;
  const uint32_t q0 = S / 6u, r = S - 6u * q0;
  const uint32_t q = q0 + ((r > 3u) | ((r == 3u) & (q0 & 1u)));
  return __uint_as_float(q | sign);
}
__device__ __forceinline__ float div6(float s) { return div6_fast_ok(s) ? div6_fast(s) : div6_small(s); }

// Finish the updates of N points from their neighbour sums.  FP32: one branch
// for the whole vector, taken only when some sum lies outside div6_fast's
// domain.
template <int N>
__device__ __forceinline__ void finish_vec(const double (&s)[N], double (&v)[N]) {
#pragma unroll
  for (int q = 0; q < N; ++q) v[q] = __dmul_rn(s[q], C6<double>::v);
}
template <int N>
__device__ __forceinline__ void finish_vec(const float (&s)[N], float (&v)[N]) {
  bool ok = true;
#pragma unroll
  for (int q = 0; q < N; ++q) {
    v[q] = div6_fast(s[q]);
    ok = ok && div6_fast_ok(s[q]);
  }
  if (!ok) {
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] = div6(s[q]);
  }
}
__device__ __forceinline__ double finish1(double s) { return __dmul_rn(s, C6<double>::v); }
__device__ __forceinline__ float finish1(float s) { return div6(s); }

// ---- SplitMix64 (Steele, Lea, Flood 2014) as a counter-based generator -------
// n-th output (0-based) of the stream seeded with `seed`.
__host__ __device__ inline uint64_t splitmix64(uint64_t seed, uint64_t n) {
  uint64_t z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ inline double u01(uint64_t seed, uint64_t n) {
  return (double)(splitmix64(seed, n) >> 11) * 0x1.0p-53;
}

// ---- memory-model helpers --------------------------------------------------
__device__ __forceinline__ int64_t ld_acquire(const int64_t* p) {
  int64_t v;
  asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int64_t* p, int64_t v) {
  asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.volatile.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Exact binary32 -> binary64 conversion on the integer pipe, from the two
// formats' definitions: for a normal number the exponent is rebiased
// (127 -> 1023) and the significand widened by 29 bits.  A subnormal is first
// scaled by 2^64 in FP32 (exact, the result is normal) and rebiased 64 less;
// zeros, infinities and NaNs keep their class.  Equal to the conversion
// instruction for every non-NaN input (jacobi_selftest_widen checks all 2^32
// inputs on the device); a NaN stays a NaN.  The FP32 residual uses it.
__device__ __forceinline__ double widen_f32(float f) {
  const uint32_t u = __float_as_uint(f);
  const bool sub = (u & 0x7F800000u) == 0u;  // zero or subnormal
  const uint32_t a = __float_as_uint(sub ? f * 0x1p64f : f) & 0x7FFFFFFFu;
  uint64_t bits = ((uint64_t)a << 29) + ((uint64_t)(sub ? 896 - 64 : 896) << 52);
  if (a == 0u) bits = 0ull;
  if (a >= 0x7F800000u) bits = ((uint64_t)a << 29) | (0x7FFull << 52);  // inf, NaN
  return __longlong_as_double((long long)(bits | ((uint64_t)(u >> 31) << 63)));
}

// Spin (bounded by wall time `limit_ns` and by a poll count) until *flag >= target,
// with acquire semantics.  Returns true on success.  On expiry it records
// DEV_TIMEOUT in *err (first failure wins); it also gives up early when another
// waiter has already recorded an error, so one failure stops every waiter.
// The first polls spin without sleeping (a neighbour's flag usually arrives
// within a few L2 round trips); after that the poll backs off to 256 ns.
__device__ inline bool wait_ge(const int64_t* flag, int64_t target, uint32_t* err,
                               uint64_t limit_ns) {
  if (ld_acquire(flag) >= target) return true;
  const uint64_t t0 = globaltimer_ns();
  unsigned sleep = 32;
  for (uint32_t n = 0; n < (1u << 26); ++n) {
    if (ld_acquire(flag) >= target) return true;
    if ((n & 7u) != 7u && n < 64u) continue;
    if (ld_volatile_u32(err) != DEV_OK) return false;
    if (globaltimer_ns() - t0 > limit_ns) break;
    if (n >= 64u) {
      __nanosleep(sleep);
      if (sleep < 256) sleep <<= 1;
    }
  }
  atomicCAS(err, (uint32_t)DEV_OK, (uint32_t)DEV_TIMEOUT);
  return false;
}

// Same for 32-bit sequence counters (wrap-safe comparison).
__device__ inline bool wait_seq_ge(const uint32_t* flag, uint32_t target, uint32_t* err,
                                   uint64_t limit_ns) {
  if ((int32_t)(ld_acquire_u32(flag) - target) >= 0) return true;
  const uint64_t t0 = globaltimer_ns();
  unsigned sleep = 32;
  for (uint32_t n = 0; n < (1u << 26); ++n) {
    if ((int32_t)(ld_acquire_u32(flag) - target) >= 0) return true;
    if (ld_volatile_u32(err) != DEV_OK) return false;
    if (globaltimer_ns() - t0 > limit_ns) break;
    __nanosleep(sleep);
    if (sleep < 256) sleep <<= 1;
  }
  atomicCAS(err, (uint32_t)DEV_OK, (uint32_t)DEV_TIMEOUT);
  return false;
}

// Deterministic block-wide FP64 sum (fixed shuffle tree + fixed smem order).
// All threads of the block must call it; the result is valid in thread 0.
template <int NT>
__device__ inline double block_sum(double v, double* smem /* NT/32 doubles */) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31;
  const int wid = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
  __syncthreads();
  if (lane == 0) smem[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (wid == 0 && lane == 0) {
    for (int w = 0; w < NT / 32; ++w) s += smem[w];
  }
  return s;
}

}  // namespace jgb
