// Jacobi3D step kernels for sm_103a: the stencil update of the paper's proxy
// application (Sec. 4.3, Jacobi iteration on a 3D grid split into blocks that
// exchange halos with up to six neighbours every iteration), with the face
// pack fused into the epilogue (new boundary planes are stored straight into
// the neighbours' receive slots, the intra-device form of the Channel API of
// Sec. 3.2.2) and the FP64 residual fused in on check iterations.
//
// Stencil reading: s = ((xm + xp) + (ym + yp)) + (zm + zp), then u' = s * c6
// in FP64 (c6 = 1/6 rounded to double) and u' = RN(s / 6) in FP32, every
// operation rounded on its own (no contraction of the sum), so results are
// bit-exact with a monolithic CPU evaluation in that order.
//
// Two ways to sweep a work item:
//  * plane streaming (x0 < 0): the CTA owns whole x-y planes of one block over
//    [z0, z1).  One elected thread fills a ring of shared-memory stages with
//    1D bulk copies (cp.async.bulk, completion counted by an mbarrier
//    transaction count): each stage holds one plane plus the four x/y ghost
//    vectors of that plane from the receive slots; the z ghosts come in as
//    whole planes from the z slots.  Each thread computes a VEC x RY patch
//    (VEC = one 16-byte vector along x) from shared memory and stores it with
//    16-byte stores.  Blocks whose shape does not fit take the next path.
//  * tiles (x0 >= 0): a TX x TY tile of columns, one column per thread, read
//    straight from global memory with the z neighbours in registers.
#include "kernels.cuh"

namespace jgb {

namespace {

// ---- mbarrier / bulk-copy helpers -------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(b))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.b32 %0, 1, 0, P;\n}"
      : "=r"(r)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return r != 0;
}
// Bounded wait for the phase of parity `parity`; on expiry records DEV_TIMEOUT.
__device__ __noinline__ bool mbar_wait(uint64_t* b, uint32_t parity, uint32_t* err, uint64_t limit_ns) {
  if (mbar_test(b, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t n = 0; n < (1u << 26); ++n) {
    if (mbar_test(b, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) break;
  }
  atomicCAS(err, (uint32_t)DEV_OK, (uint32_t)DEV_TIMEOUT);
  return false;
}

// Inline fast path: the phase is usually complete already, so test once
// before calling the bounded wait.
__device__ __forceinline__ bool mbar_ready(uint64_t* b, uint32_t parity, uint32_t* err, uint64_t limit_ns) {
  return mbar_test(b, parity) || mbar_wait(b, parity, err, limit_ns);
}

// ---- 16-byte vectors ---------------------------------------------------------
template <typename T> struct V16;
template <> struct V16<float> {
  static constexpr int N = 4;
  __device__ static __forceinline__ void load(const float* p, float (&v)[4]) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  }
  __device__ static __forceinline__ void store(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <> struct V16<double> {
  static constexpr int N = 2;
  __device__ static __forceinline__ void load(const double* p, double (&v)[2]) {
    const double2 x = *reinterpret_cast<const double2*>(p);
    v[0] = x.x; v[1] = x.y;
  }
  __device__ static __forceinline__ void store(double* p, const double (&v)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
};

// FP64 residual contribution of one point: r = s - 6u with s re-evaluated in
// FP64 from the (exactly widened) neighbours in the stencil's order.  FP32
// states are widened on the integer pipe, which leaves the slow FP64 pipe
// only the additions and multiplications (same-box A/B: the 768^3 FP32
// residual 10.5 -> 7.4 ms, the whole 200-iteration step with its residual
// 684 -> 700 GLUP/s; residuals bit-identical).
// r^2 for one point: r = s - 6u in FP64 (FP32 values widened exactly, the
// neighbour sum recomputed in FP64 in the stencil's order).  With EMU (an
// FP32 state inside the integer adder's domain: no sign bit, finite) the
// three pair sums of the widened values run on the integer pipe (dadd_nn,
// bit-identical to the FP64 pipe's addition there), which leaves the FP64
// pipe five of its eight operations per point.  FP32 kernels use it only in
// residual-only launches: same-box A/B, 768^3 residual 7.07 -> 5.87 ms,
// while in the fused step-and-residual launches the extra code path spilled
// (serving 84.0 -> 81.9 solves/s).
template <typename T, bool EMU = false>
__device__ __forceinline__ double resid2(T xm, T xp, T ym, T yp, T zm, T zp, T s, T c) {
  double s64, c64;
  if constexpr (sizeof(T) == 8) {
    s64 = (double)s;
    c64 = (double)c;
  } else if constexpr (EMU) {
    s64 = __dadd_rn(__dadd_rn(dadd_nn(widen_f32(xm), widen_f32(xp)), dadd_nn(widen_f32(ym), widen_f32(yp))),
                    dadd_nn(widen_f32(zm), widen_f32(zp)));
    c64 = widen_f32(c);
  } else {
    s64 = __dadd_rn(__dadd_rn(__dadd_rn(widen_f32(xm), widen_f32(xp)), __dadd_rn(widen_f32(ym), widen_f32(yp))),
                    __dadd_rn(widen_f32(zm), widen_f32(zp)));
    c64 = widen_f32(c);
  }
  const double r = __dsub_rn(s64, __dmul_rn(6.0, c64));
  return r * r;
}

// ---------------------------------------------------------------------------
// Tile path: thread (tx, ty) owns column (x0 + tx, y0 + ty) of block B and
// walks planes [z0, z1) with k-1, k, k+1 of its column in registers.
// Neighbours across a block face come from that face's receive slot (parity
// p); with kPack the new boundary planes go to the neighbours' slots (p ^ 1).
// ---------------------------------------------------------------------------
template <typename T, int MODE>
__device__ __forceinline__ double tile_sweep(const BlockDev& B, int p, int x0, int y0, int z0, int z1, int tx,
                                             int ty) {
  const int i = x0 + tx, j = y0 + ty;
  const int nx = B.nx, ny = B.ny, nz = B.nz, rx = B.rx, ry = B.ry;
  double acc = 0.0;
  if (i >= nx || j >= ny) return acc;
  const T* __restrict__ U = (const T*)B.u[p];
  T* __restrict__ V = (T*)B.u[p ^ 1];
  const int64_t pp = B.plane_pitch;
  const T* rxm = (const T*)B.recv[XM][p];
  const T* rxp = (const T*)B.recv[XP][p];
  const T* rym = (const T*)B.recv[YM][p];
  const T* ryp = (const T*)B.recv[YP][p];
  const T* rzp = (const T*)B.recv[ZP][p];
  const int64_t col = (int64_t)j * rx + i;
  T below = (z0 == 0) ? __ldcg((const T*)B.recv[ZM][p] + col) : U[(int64_t)(z0 - 1) * pp + col];
  T cur = U[(int64_t)z0 * pp + col];
  T* sxm = nullptr; T* sxp = nullptr; T* sym = nullptr; T* syp = nullptr; T* szm = nullptr; T* szp = nullptr;
  if (MODE & kPack) {
    if (i == 0) sxm = (T*)B.send[XM][p ^ 1];
    if (i == nx - 1) sxp = (T*)B.send[XP][p ^ 1];
    if (j == 0) sym = (T*)B.send[YM][p ^ 1];
    if (j == ny - 1) syp = (T*)B.send[YP][p ^ 1];
    szm = (T*)B.send[ZM][p ^ 1];
    szp = (T*)B.send[ZP][p ^ 1];
  }
  for (int k = z0; k < z1; ++k) {
    const int64_t o = (int64_t)k * pp + col;
    const T above = (k + 1 < nz) ? U[o + pp] : __ldcg(rzp + col);
    const T xm = (i > 0) ? U[o - 1] : __ldcg(rxm + (int64_t)k * ry + j);
    const T xp = (i < nx - 1) ? U[o + 1] : __ldcg(rxp + (int64_t)k * ry + j);
    const T ym = (j > 0) ? U[o - rx] : __ldcg(rym + (int64_t)k * rx + i);
    const T yp = (j < ny - 1) ? U[o + rx] : __ldcg(ryp + (int64_t)k * rx + i);
    const T s = radd(radd(radd(xm, xp), radd(ym, yp)), radd(below, above));
    if (MODE & kWrite) {
      const T v = finish1(s);
      V[o] = v;
      if (MODE & kPack) {
        if (sxm) sxm[(int64_t)k * ry + j] = v;
        if (sxp) sxp[(int64_t)k * ry + j] = v;
        if (sym) sym[(int64_t)k * rx + i] = v;
        if (syp) syp[(int64_t)k * rx + i] = v;
        if (k == 0 && szm) szm[col] = v;
        if (k == nz - 1 && szp) szp[col] = v;
      }
    }
    if (MODE & kResid) acc += resid2<T>(xm, xp, ym, yp, below, above, s, cur);
    below = cur;
    cur = above;
  }
  return acc;
}

// ---------------------------------------------------------------------------
// Plane-streaming path.
// ---------------------------------------------------------------------------
struct Ring {
  unsigned char* stages;
  uint64_t* bars;
  int S;
  uint32_t pbits;  // parity of each stage's next fill (bit st), barrier-driven form only
};

// Sum of the six neighbours in the stencil's order.  With EMU (FP64 states
// inside the integer adder's domain) the three pair sums run on the integer
// pipe and the two outer additions on the FP64 pipe: both pipes share the
// work and the result is bit-identical.
template <typename T, bool EMU>
__device__ __forceinline__ T nsum(T xm, T xp, T ym, T yp, T zm, T zp) {
  if (EMU) {
    const double sx = dadd_nn((double)xm, (double)xp), sy = dadd_nn((double)ym, (double)yp),
                 sz = dadd_nn((double)zm, (double)zp);
    return (T)__dadd_rn(__dadd_rn(sx, sy), sz);
  }
  return radd(radd(radd(xm, xp), radd(ym, yp)), radd(zm, zp));
}

// nsum with the z pair on the FP64 pipe (bit-identical: both adders round
// to nearest-even).
template <typename T, bool EMU>
__device__ __forceinline__ T nsum_zn(T xm, T xp, T ym, T yp, T zm, T zp) {
  if (EMU) {
    const double sx = dadd_nn((double)xm, (double)xp), sy = dadd_nn((double)ym, (double)yp),
                 sz = __dadd_rn((double)zm, (double)zp);
    return (T)__dadd_rn(__dadd_rn(sx, sy), sz);
  }
  return radd(radd(radd(xm, xp), radd(ym, yp)), radd(zm, zp));
}

// Shared-memory stage of one plane of a padded row window [ya, yb) of block
// B: rows ra..rb-1 of the plane (the window plus one neighbour row on each
// side that exists), then the x ghosts of the window's rows (xm, xp), then the
// y ghost rows (ym, yp; filled only at the block's edges, where they are
// needed).  Rows have the padded pitch rx; windows start on multiples of 4
// rows, so every copy is a whole number of 16-byte vectors.
struct StageLayout {
  int ra, rb;
  uint32_t rows_bytes, xg, yg, bytes;
  uint32_t o_xm, o_xp, o_ym, o_yp;
};
template <typename T>
__device__ __forceinline__ StageLayout stage_layout(const BlockDev& B, int ya, int yb) {
  StageLayout L;
  L.ra = ya > 0 ? ya - 1 : 0;
  L.rb = yb < B.ry ? yb + 1 : B.ry;
  L.rows_bytes = (uint32_t)((L.rb - L.ra) * B.rx * sizeof(T));
  L.xg = (uint32_t)((yb - ya) * sizeof(T));
  L.yg = (uint32_t)(B.rx * sizeof(T));
  L.o_xm = L.rows_bytes;
  L.o_xp = L.o_xm + L.xg;
  L.o_ym = L.o_xp + L.xg;
  L.o_yp = L.o_ym + L.yg;
  L.bytes = (L.o_yp + L.yg + 127u) & ~127u;
  return L;
}

// Issue the bulk copies of plane q (k = z0 - 1 + q) of window [ya, yb) into
// `dst`, completing on `bar`.
template <typename T>
__device__ __forceinline__ void issue_plane(const BlockDev& B, int p, int z0, int nplanes, int q, int ya, int yb,
                                            const StageLayout& L, unsigned char* dst, uint64_t* bar) {
  const int rx = B.rx, ry = B.ry, nz = B.nz;
  const int kk = z0 - 1 + q;
  const T* src = kk < 0 ? (const T*)B.recv[ZM][p]
                        : (kk >= nz ? (const T*)B.recv[ZP][p] : (const T*)B.u[p] + (int64_t)kk * B.plane_pitch);
  const bool ghosts = q >= 1 && q <= nplanes - 2;
  const bool gym = ghosts && ya == 0, gyp = ghosts && yb == ry;
  mbar_expect_tx(bar, L.rows_bytes + (ghosts ? 2 * L.xg : 0) + (gym ? L.yg : 0) + (gyp ? L.yg : 0));
  bulk_g2s(dst, src + (int64_t)L.ra * rx, L.rows_bytes, bar);
  if (ghosts) {
    bulk_g2s(dst + L.o_xm, (const T*)B.recv[XM][p] + (int64_t)kk * ry + ya, L.xg, bar);
    bulk_g2s(dst + L.o_xp, (const T*)B.recv[XP][p] + (int64_t)kk * ry + ya, L.xg, bar);
  }
  if (gym) bulk_g2s(dst + L.o_ym, (const T*)B.recv[YM][p] + (int64_t)kk * rx, L.yg, bar);
  if (gyp) bulk_g2s(dst + L.o_yp, (const T*)B.recv[YP][p] + (int64_t)kk * rx, L.yg, bar);
}

// What a consumer thread needs from its block, read once per work item into
// registers (the block table lives in global memory and the sweep stores
// through plain pointers, so reading it in the loop would force reloads).
template <typename T>
struct PlaneView {
  int nx, ny, nz, pn;      // extents; parity of the new iterate
  int rx, ry;              // padded row pitch and rows per plane
  int64_t pitch;
  T* V;                    // new iterate
  const BlockDev* B;       // for the send pointers, read by edge threads only
  void* const* ss;         // the six send slots copied to shared memory, or null
};
template <typename T>
__device__ __forceinline__ PlaneView<T> plane_view(const BlockDev& B, int p) {
  PlaneView<T> v;
  v.nx = B.nx;
  v.ny = B.ny;
  v.nz = B.nz;
  v.pn = p ^ 1;
  v.rx = B.rx;
  v.ry = B.ry;
  v.pitch = B.plane_pitch;
  v.V = (T*)B.u[p ^ 1];
  v.B = &B;
  v.ss = nullptr;
  return v;
}
// Neighbour receive slot of face f for the new iterate: from the CTA's
// shared-memory copy (TABLE), else through the read-only path.
template <bool TABLE, typename T>
__device__ __forceinline__ T* send_slot(const PlaneView<T>& O, int f) {
  if (TABLE) return (T*)O.ss[f];
  return (T*)__ldg((const unsigned long long*)&O.B->send[f][O.pn]);
}

// Compute plane k of padded rows [j0, j0 + RY) (inside the window [ya, yb))
// from the stages holding planes k - 1, k, k + 1.  tx = vector column.  With
// RAG (a block whose nx is not a whole number of vectors or whose ny is not a
// multiple of 4), rows at or past ny and lanes at or past nx are padding:
// their values are replaced by the y (x) ghost before use, so the last real
// row (column) sees its ghost, and they are neither summed into the residual
// nor stored.  Without RAG there is no padding and none of those checks.
// TABLE: the send slots come from the CTA's shared-memory copy.  The face
// checks are kept to the rows that can hit a face (row groups start on
// multiples of 4): same-box A/B +5 % on the FP64 64^3-block step.  XB: the
// x neighbours of the vector are loaded through a base and stride chosen once
// per plane (plane row or x ghost) instead of a per-row choice; same-box A/B
// +1 to +2 % for the small CTAs (32^3 blocks, +7 % served solves/s), neutral
// for the 8-warp ones, which keep the per-row form.
template <typename T, int RY, int MODE, bool EMU, bool RAG, bool TABLE, bool XB = false>
__device__ __forceinline__ double stream_plane(const PlaneView<T>& O, int k, int ya, const StageLayout& L,
                                               const unsigned char* sm, const unsigned char* sc,
                                               const unsigned char* sp, int tx, int j0) {
  constexpr int VEC = V16<T>::N;
  // EMU: the integer-pipe adder takes the FP64 stencil's pair sums and, in
  // either precision, the residual's (FP32 sums themselves stay FP32 adds)
  constexpr bool EMU_SUM = EMU && sizeof(T) == 8;
  const int nx = O.nx, ny = O.ny, nz = O.nz;
  const int rx = RAG ? O.rx : nx, ry = RAG ? O.ry : ny;  // equal without padding
  const int i0 = tx * VEC;
  const T* Pm = (const T*)sm - L.ra * rx;  // row j of a plane at P + j * rx
  const T* Pc = (const T*)sc - L.ra * rx;
  const T* Pp = (const T*)sp - L.ra * rx;
  const T* Gxm = (const T*)(sc + L.o_xm) - ya;  // x ghost of row j at G[j]
  const T* Gxp = (const T*)(sc + L.o_xp) - ya;
  const T* Gym = (const T*)(sc + L.o_ym);
  const T* Gyp = (const T*)(sc + L.o_yp);
  T* __restrict__ V = O.V + (int64_t)k * O.pitch;
  const int ql = nx - 1 - i0;  // last real lane of this vector column (< VEC - 1: ragged)

  T c[RY][VEC];
#pragma unroll
  for (int r = 0; r < RY; ++r) V16<T>::load(!RAG || j0 + r < ny ? Pc + (j0 + r) * rx + i0 : Gyp + i0, c[r]);
  if (RAG && ql < VEC - 1) {
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      const T g = Gxp[j0 + r];
#pragma unroll
      for (int q = 1; q < VEC; ++q)
        if (q > ql) c[r][q] = g;
    }
  }
  // x neighbours (XB form): the plane row, or the x ghost at the block edge
  const T* lbase = i0 > 0 ? Pc + i0 - 1 : Gxm;
  const int lstride = i0 > 0 ? rx : 1;
  const T* rbase = i0 + VEC < nx ? Pc + i0 + VEC : Gxp;
  const int rstride = i0 + VEC < nx ? rx : 1;
  T top[VEC], bot[VEC];
  V16<T>::load(j0 > 0 ? Pc + (j0 - 1) * rx + i0 : Gym + i0, top);
  V16<T>::load(j0 + RY < ny ? Pc + (j0 + RY) * rx + i0 : Gyp + i0, bot);
  double acc = 0.0;
  // x-face values of this thread's column over its RY rows: the first column
  // gives the xm face, else the last column the xp face; stored as whole
  // 16-byte vectors after the rows (rows are consecutive in an x slot).
  // A column that is both (one vector wide) stores its xp face row by row.
  T xe[RY];
  const bool xfirst = i0 == 0, xlast = ql < VEC;
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    const int j = j0 + r;
    T zm[VEC], zp[VEC];
    V16<T>::load(Pm + j * rx + i0, zm);
    V16<T>::load(Pp + j * rx + i0, zp);
    const T* ym = r == 0 ? top : c[r > 0 ? r - 1 : 0];
    const T* yp = r == RY - 1 ? bot : c[r < RY - 1 ? r + 1 : 0];
    T left, right;
    if (XB) {
      left = lbase[j * lstride];
      right = rbase[j * rstride];
    } else {
      left = i0 > 0 ? Pc[j * rx + i0 - 1] : Gxm[j];
      right = i0 + VEC < nx ? Pc[j * rx + i0 + VEC] : Gxp[j];
    }
    T v[VEC], sv[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
      const T xm = q == 0 ? left : c[r][q > 0 ? q - 1 : 0];
      const T xp = q == VEC - 1 ? right : c[r][q < VEC - 1 ? q + 1 : 0];
      // FP64: the z pair of 2 of a thread's 8 points goes to the FP64 pipe,
      // shifting work off the busier integer pipe (same-box A/B +0.5 % on
      // 64^3 blocks, +1.9 % on 32^3; 3 or 4 of 8 gained less).
      const T s = (q == VEC - 1 && r < 2) ? nsum_zn<T, EMU_SUM>(xm, xp, ym[q], yp[q], zm[q], zp[q])
                                          : nsum<T, EMU_SUM>(xm, xp, ym[q], yp[q], zm[q], zp[q]);
      // FP64 finishes each point at once (keeping the sum live to the end of
      // the loop made ptxas spill); FP32 finishes the vector after the loop
      // (one fallback branch per vector).
      if constexpr (sizeof(T) == 8) v[q] = finish1(s);
      else sv[q] = s;
      if (MODE & kResid) {
        const double e2 = resid2<T, EMU>(xm, xp, ym[q], yp[q], zm[q], zp[q], s, c[r][q]);
        acc += (!RAG || (q <= ql && j < ny)) ? e2 : 0.0;
      }
    }
    if constexpr (sizeof(T) == 4) finish_vec(sv, v);
    if ((MODE & kWrite) && (MODE & kPack)) {
      T last = v[VEC - 1];
      if (RAG) {
#pragma unroll
        for (int q = 0; q < VEC - 1; ++q)
          if (q == ql) last = v[q];
      }
      xe[r] = xfirst ? v[0] : last;
      if (xfirst && xlast && (!RAG || j < ny)) {
        T* d = send_slot<TABLE>(O, XP);
        if (d) d[(int64_t)k * ry + j] = last;
      }
    }
    if ((MODE & kWrite) && (!RAG || j < ny)) {
      V16<T>::store(V + j * rx + i0, v);
      if (MODE & kPack) {
        if (r == 0 && j0 == 0) {  // row groups start on multiples of 4: only row 0 can be j = 0
          T* d = send_slot<TABLE>(O, YM);
          if (d) V16<T>::store(d + (int64_t)k * rx + i0, v);
        }
        // without padding ny is a multiple of 4, so only the last row of the
        // last row group can be j = ny - 1
        if (RAG ? j == ny - 1 : (r == RY - 1 && j0 + RY == ny)) {
          T* d = send_slot<TABLE>(O, YP);
          if (d) V16<T>::store(d + (int64_t)k * rx + i0, v);
        }
        if (k == 0) {
          T* d = send_slot<TABLE>(O, ZM);
          if (d) V16<T>::store(d + j * rx + i0, v);
        }
        if (k == nz - 1) {
          T* d = send_slot<TABLE>(O, ZP);
          if (d) V16<T>::store(d + j * rx + i0, v);
        }
      }
    }
  }
  if ((MODE & kWrite) && (MODE & kPack) && (xfirst || xlast)) {
    T* d = send_slot<TABLE>(O, xfirst ? XM : XP);
    if (d) {
      T* x = d + (int64_t)k * ry + j0;  // 16-byte aligned: ry and j0 are multiples of 4
#pragma unroll
      for (int r = 0; r < RY; r += VEC) {
        T w[VEC];
#pragma unroll
        for (int q = 0; q < VEC; ++q) w[q] = xe[r + q];
        V16<T>::store(x + r, w);
      }
    }
  }
  return acc;
}

// Barrier-driven form of the streaming sweep, used inside the persistent
// kernel (all threads call it; one thread issues the copies).  Returns this
// thread's r^2 sum; sets ok = false (CTA-uniform) after a bounded wait
// expired (the error word is set and issued copies drained).
template <typename T, int RY, int MODE>
__device__ double stream_item(const BlockDev& B, int p, const WorkItem& w, Ring& ring, uint32_t* err,
                              uint64_t wait_ns, bool emu, bool& ok, void* const* tab) {
  constexpr int VEC = V16<T>::N;
  const int tid = threadIdx.x;
  const int txv = B.rx / VEC;
  const int tx = tid % txv, j0 = w.ya + (tid / txv) * RY;
  const bool active = j0 < w.yb;
  const bool rag = item_ragged(w);
  const int S = ring.S;
  const StageLayout L = stage_layout<T>(B, w.ya, w.yb);
  PlaneView<T> O = plane_view<T>(B, p);
  O.ss = tab;
  constexpr bool kEmuUse = sizeof(T) == 8 || MODE == kResid;  // FP32: residual-only launches
  const int nplanes = w.z1 - w.z0 + 2;
  auto issue = [&](int q) {
    const int st = q % S;
    issue_plane<T>(B, p, w.z0, nplanes, q, w.ya, w.yb, L, ring.stages + (size_t)st * L.bytes, ring.bars + st);
  };
  auto wait = [&](int q) {
    const int st = q % S;
    const uint32_t parity = ((ring.pbits >> st) ^ (uint32_t)(q / S)) & 1u;
    return mbar_wait(ring.bars + st, parity, err, wait_ns);
  };
  if (tid == 0) {
    fence_proxy_async();
    const int n0 = min(S - 1, nplanes);
    for (int q = 0; q < n0; ++q) issue(q);
  }
  int issued = min(S - 1, nplanes);
  double acc = 0.0;
  bool good = true;
  for (int q = 1; q <= nplanes - 2; ++q) {
    // Every thread is done with plane q - 2 (read while computing q - 1).
    if (!__syncthreads_and(good)) break;
    const int qi = q - 2 + S;
    if (qi < nplanes && qi >= issued) {
      if (tid == 0) {
        fence_proxy_async();
        issue(qi);
      }
      issued = qi + 1;
    }
    if (q == 1) good = wait(0) && wait(1);
    good = good && wait(q + 1);
    if (good && active) {
      const unsigned char* sm = ring.stages + (size_t)((q - 1) % S) * L.bytes;
      const unsigned char* sc = ring.stages + (size_t)(q % S) * L.bytes;
      const unsigned char* sp = ring.stages + (size_t)((q + 1) % S) * L.bytes;
      const int kq = w.z0 - 1 + q;
      if (rag) {
        if (kEmuUse && emu) acc += stream_plane<T, RY, MODE, true, true, true>(O, kq, w.ya, L, sm, sc, sp, tx, j0);
        else acc += stream_plane<T, RY, MODE, false, true, true>(O, kq, w.ya, L, sm, sc, sp, tx, j0);
      } else {
        if (kEmuUse && emu) acc += stream_plane<T, RY, MODE, true, false, true>(O, kq, w.ya, L, sm, sc, sp, tx, j0);
        else acc += stream_plane<T, RY, MODE, false, false, true>(O, kq, w.ya, L, sm, sc, sp, tx, j0);
      }
    }
  }
  ok = __syncthreads_and(good) != 0;
  if (!ok && tid == 0) {
    // Drain: wait (bounded) for the latest fill issued into each stage.
    for (int st = 0; st < S; ++st) {
      int qlast = -1;
      for (int q = st; q < issued; q += S) qlast = q;
      if (qlast >= 0) wait(qlast);
    }
  }
  // advance the per-stage fill parities past this item's fills
  for (int st = 0; st < S; ++st) {
    const int fills = (nplanes > st) ? (nplanes - st + S - 1) / S : 0;
    ring.pbits ^= (uint32_t)(fills & 1) << st;
  }
  return acc;
}

// `tab` holds the block's six send slots for the new iterate (shared memory).
template <typename T, int MODE>
__device__ double run_item(const BlockDev& B, int p, const WorkItem& w, Ring& ring, uint32_t* err,
                           uint64_t wait_ns, bool emu, bool& ok, void* const* tab) {
  ok = true;
  if (w.x0 >= 0) return tile_sweep<T, MODE>(B, p, w.x0, w.y0, w.z0, w.z1, threadIdx.x % TX, threadIdx.x / TX);
  return stream_item<T, 4, MODE>(B, p, w, ring, err, wait_ns, emu, ok, tab);
}

__device__ __forceinline__ Ring ring_setup(unsigned char* smem, int S) {
  Ring ring;
  ring.bars = (uint64_t*)smem;
  ring.stages = smem + 128;
  ring.S = S;
  ring.pbits = 0;
  if (threadIdx.x == 0) {
    for (int st = 0; st < S; ++st) mbar_init(ring.bars + st, 1);
    mbar_fence_init();
  }
  __syncthreads();
  return ring;
}

// Tile items (x0 >= 0), one TX x TY tile per CTA.
template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_tiles(StepLaunch a) {
  const WorkItem w = a.items[blockIdx.x];
  const BlockDev& B = a.blocks[w.block];
  const GridDev G = a.grids[B.grid];
  if (!G.active) return;  // frozen grid (CTA-uniform)
  const int p = (int)((a.it - G.start_iter) & 1);
  const double acc = tile_sweep<T, MODE>(B, p, w.x0, w.y0, w.z0, w.z1, threadIdx.x % TX, threadIdx.x / TX);
  if (MODE & kResid) {
    __shared__ double red[kThreads / 32];
    const double s = block_sum<kThreads>(acc, red);
    if (threadIdx.x == 0) a.partials[w.slot] = s;
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}

// Plane-streaming items (x0 < 0), one item per CTA, warp-specialised: warp 8
// is the producer (its lane 0 issues the bulk copies of plane q into stage
// q % S once all consumer warps have released that stage through its "empty"
// mbarrier), warps 0..7 are consumers (each waits on the "full" mbarrier of
// the planes it needs, computes, and releases the stage of plane q - 1 after
// computing plane q, its last use).  There is no CTA-wide barrier inside the
// plane loop, so consumer warps drift freely within the ring.
// CW consumer warps (2, 4 or 8) plus the producer warp; small planes use
// small CTAs so that every consumer thread still computes RY = 4 rows.  The
// register cap (72 per thread) sets the minimum CTAs per SM.
template <int CW> struct StreamShape {
  static constexpr int threads = 32 * CW + 32;
  static constexpr int min_blocks = 65536 / (threads * 72);
};

template <typename T, int RY, int CW, bool RAG, int MODE>
__global__ void __launch_bounds__(StreamShape<CW>::threads, StreamShape<CW>::min_blocks) k_stream(StepLaunch a) {
  constexpr int kConsumerWarps = CW;
  constexpr int kStreamThreads = StreamShape<CW>::threads;
  constexpr int VEC = V16<T>::N;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = (uint64_t*)smem;
  uint64_t* empty = full + 8;
  unsigned char* stages = smem + 128;
  const WorkItem w = a.items[blockIdx.x];
  const BlockDev& B = a.blocks[w.block];
  const GridDev G = a.grids[B.grid];
  if (!G.active) return;  // frozen grid (CTA-uniform, before any barrier)
  const int p = (int)((a.it - G.start_iter) & 1);
  // FP32: the depth is the compile-time kStreamStages, so stage indices are
  // masks.  FP64: the same value read at run time; ptxas then allocates the
  // ALU-bound FP64 loop without spills (same-box A/B: FP32 +2 to +8 %, FP64
  // -2 % with the constant).
  const int S = sizeof(T) == 4 ? kStreamStages : a.stages;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nplanes = w.z1 - w.z0 + 2;  // planes z0-1 .. z1
  const StageLayout L = stage_layout<T>(B, w.ya, w.yb);
  // The send slots in shared memory save the consumers a dependent global
  // load before each face store.  Same-box A/B: faster in every variant but
  // the FP64 ones with fewer than 8 consumer warps, where ptxas then spills.
  constexpr bool kSendTable = !(sizeof(T) == 8 && CW < 8);
  __shared__ void* s_send[6];
  if (kSendTable && tid < 6) s_send[tid] = B.send[tid][p ^ 1];
  if (tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(full + st, 1);
      mbar_init(empty + st, kConsumerWarps);
    }
    mbar_fence_init();
  }
  __syncthreads();
  double acc = 0.0;
  if (warp == kConsumerWarps) {
    // ---- producer ----
    if (lane == 0) {
      int q = 0;
      for (; q < nplanes; ++q) {
        const int st = q % S, fill = q / S;
        if (fill > 0 && !mbar_wait(empty + st, (uint32_t)(fill - 1) & 1u, a.err, a.wait_ns)) break;
        // No proxy fence: within one launch the bulk copies read only the
        // parity-p state and slots, which earlier launches wrote (a launch
        // boundary orders them); this launch writes parity p ^ 1 only.
        issue_plane<T>(B, p, w.z0, nplanes, q, w.ya, w.yb, L, stages + (size_t)st * L.bytes, full + st);
      }
      if (q < nplanes) {
        // A wait expired: let the copies already issued land before leaving.
        for (int st = 0; st < S; ++st) {
          int qlast = -1;
          for (int r = st; r < q; r += S) qlast = r;
          if (qlast >= 0) mbar_wait(full + st, (uint32_t)(qlast / S) & 1u, a.err, a.wait_ns);
        }
      }
    }
  } else {
    // ---- consumers ----
    const bool emu = (sizeof(T) == 8 || MODE == kResid) && a.emu && a.norms && a.norms[B.grid].emu_bad == 0u;
    PlaneView<T> O = plane_view<T>(B, p);
    if (kSendTable) O.ss = s_send;
    const int txv = O.rx / VEC;
    const int tx = tid % txv, j0 = w.ya + (tid / txv) * RY;
    const bool active = j0 < w.yb;
    bool good = true;
    // S is a power of two: stage = q & (S - 1), fill = q >> log2(S).  For FP64
    // (S read at run time) this replaces four integer divisions per plane,
    // a noticeable share of the integer pipe at 8 updates per thread and
    // plane (same-box A/B: 512^3 140.8 -> 145.9 GLUP/s).
    const int Sm = S - 1, Sl = 31 - __clz(S);
    for (int q = 1; q <= nplanes - 2 && good; ++q) {
      if (q == 1) {
        good = mbar_wait(full + 0, 0u, a.err, a.wait_ns) &&
               mbar_wait(full + (1 & Sm), (uint32_t)(1 >> Sl) & 1u, a.err, a.wait_ns);
      }
      // inline test first, the bounded wait only when the plane is not there
      // yet (same-box A/B: +1 to +1.5 %)
      good = good && mbar_ready(full + ((q + 1) & Sm), (uint32_t)((q + 1) >> Sl) & 1u, a.err, a.wait_ns);
      good = __all_sync(0xffffffffu, good);
      if (!good) break;
      if (active) {
        const unsigned char* sm = stages + (size_t)((q - 1) & Sm) * L.bytes;
        const unsigned char* sc = stages + (size_t)(q & Sm) * L.bytes;
        const unsigned char* sp = stages + (size_t)((q + 1) & Sm) * L.bytes;
        if ((sizeof(T) == 8 || MODE == kResid) && emu)
          acc += stream_plane<T, RY, MODE, true, RAG, kSendTable, (CW < 8)>(O, w.z0 - 1 + q, w.ya, L, sm, sc, sp, tx, j0);
        else
          acc += stream_plane<T, RY, MODE, false, RAG, kSendTable, (CW < 8)>(O, w.z0 - 1 + q, w.ya, L, sm, sc, sp, tx, j0);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(empty + ((q - 1) & Sm));
    }
  }
  if (MODE & kResid) {
    __shared__ double red[kStreamThreads / 32];
    const double s = block_sum<kStreamThreads>(acc, red);
    if (tid == 0) a.partials[w.slot] = s;
  }
}

// ---------------------------------------------------------------------------
// Persistent kernel: the work is split into units, the z-chunks of the blocks
// (a unit's items are its row windows or tiles); CTA c owns active units c,
// c + G, c + 2G, ... for all n_iters iterations.  Before unit u computes
// iteration it (> it0) its CTA acquire-waits until the progress flag of every
// unit it shares data with reaches it (that unit finished iteration it - 1:
// its faces and halo planes of u_it are written, and it no longer reads what
// u is about to overwrite); after u's sweep the CTA release-stores
// progress[u] = it + 1.  The host lists each unit's partners (its block's
// adjacent chunks, the same chunk of the x and y neighbours, the facing chunk
// of the z neighbours).  Waits are bounded: on expiry the error word is set and
// every CTA leaves at its next wait.
// A CTA that owns at most kPersistCache units copies their tables (block
// entry, send slots by parity, item range, partners, grid start, FP64 adder
// flag) into shared memory once, so an iteration starts with its flag polls
// instead of a chain of dependent table loads from L2 (same-box A/B in the
// notes of the library's design).
// Proxy fences order the generic stores of neighbours (and of this CTA's
// previous iteration) before the bulk copies that read them; the release
// store after the CTA barrier is cumulative, so it publishes every thread's
// stores without a separate fence.
// ---------------------------------------------------------------------------
constexpr int kPersistDeps = 8;  // a unit has at most 6 partners

struct UnitCache {
  BlockDev B;
  void* send[2][6];      // send slots for a new iterate of parity 0 / 1
  int64_t start_iter;    // the block's grid start
  int32_t unit, q0, q1, ndep;
  int32_t dep[kPersistDeps];
  int32_t emu;
  int32_t pad_;
};
static_assert(kPersistCache * sizeof(UnitCache) + 512 <= 227 * 1024 - kMaxStepSmem,
              "the persistent kernel's static shared memory must fit beside the largest ring");

// NT threads per CTA (64, 128 or 256): the host picks the smallest that
// covers every streamed row window of the launch (a window of W rows and V
// vector columns needs V * W / 4 threads), or 256 when tile items are present
// (one TX x TY tile per CTA), so CTAs of small blocks keep every thread busy.
// Registers are capped at 128 per thread.
template <typename T, int NT>
__global__ void __launch_bounds__(NT, 65536 / (NT * 128)) k_persist(PersistLaunch a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double red[NT / 32];
  __shared__ int s_ok;
  __shared__ UnitCache s_u[kPersistCache];
  __shared__ void* s_tab[6];
  const int tid = threadIdx.x, lane = tid & 31;
  const int G = (int)gridDim.x;
  const int mine = a.n_units > (int)blockIdx.x ? (a.n_units - (int)blockIdx.x + G - 1) / G : 0;
  const bool cached = mine <= kPersistCache;
  if (cached) {
    for (int k = tid >> 5; k < mine; k += NT / 32) {  // one warp per unit
      const int ui = (int)blockIdx.x + k * G;
      UnitCache& U = s_u[k];
      const int q0 = a.unit_items[ui];
      const BlockDev* Bg = a.blocks + a.items[q0].block;
      const uint32_t* src = (const uint32_t*)Bg;
      uint32_t* dst = (uint32_t*)&U.B;
      for (int i = lane; i < (int)(sizeof(BlockDev) / 4); i += 32) dst[i] = src[i];
      if (lane < 12) U.send[lane / 6][lane % 6] = Bg->send[lane % 6][lane / 6];
      const int d0 = a.dep_off[ui], d1 = a.dep_off[ui + 1];
      if (lane < kPersistDeps) U.dep[lane] = d0 + lane < d1 ? a.dep_ids[d0 + lane] : 0;
      if (lane == 0) {
        U.unit = a.unit_ids[ui];
        U.q0 = q0;
        U.q1 = a.unit_items[ui + 1];
        U.ndep = d1 - d0;
        U.start_iter = a.grids[Bg->grid].start_iter;
        U.emu = (a.emu && a.norms && a.norms[Bg->grid].emu_bad == 0u) ? 1 : 0;
      }
    }
  }
  const int64_t it0 = a.it0_dev ? *a.it0_dev : a.it0;
  Ring ring = ring_setup(smem, a.stages);  // ends with a CTA barrier
  for (int64_t t = 0; t < a.n_iters; ++t) {
    const int64_t it = it0 + t;
    for (int k = 0; k < mine; ++k) {
      const int ui = (int)blockIdx.x + k * G;
      const BlockDev* Bp;
      int u, q0, q1, ndep;
      int64_t start;
      bool emu;
      if (cached) {
        const UnitCache& U = s_u[k];
        Bp = &U.B;
        u = U.unit;
        q0 = U.q0;
        q1 = U.q1;
        ndep = U.ndep;
        start = U.start_iter;
        emu = U.emu != 0;
      } else {
        q0 = a.unit_items[ui];
        q1 = a.unit_items[ui + 1];
        u = a.unit_ids[ui];
        Bp = &a.blocks[a.items[q0].block];
        ndep = a.dep_off[ui + 1] - a.dep_off[ui];
        start = a.grids[Bp->grid].start_iter;
        emu = a.emu && a.norms && a.norms[Bp->grid].emu_bad == 0u;
      }
      if (t > 0 && tid < 32) {
        // One lane per partner: the flags are polled in parallel, so the wait
        // costs one round trip instead of one per partner (same-box A/B: 64^3
        // FP64 in 2x2x2 blocks 22.0 -> 24.3 GLUP/s, 256-grid FP32 batch
        // 109.5 -> 114.0).
        bool okw = true;
        for (int d = lane; d < ndep && okw; d += 32) {
          const int dep = (cached && ndep <= kPersistDeps) ? s_u[k].dep[d] : a.dep_ids[a.dep_off[ui] + d];
          okw = wait_ge(a.progress + dep, it, a.err, a.wait_ns);
        }
        okw = __all_sync(0xffffffffu, okw);
        if (tid == 0) {
          fence_proxy_async();
          s_ok = okw ? 1 : 0;
        }
      }
      const int p = (int)((it - start) & 1);
      if (tid < 6) s_tab[tid] = cached ? s_u[k].send[p ^ 1][tid] : Bp->send[tid][p ^ 1];
      __syncthreads();
      if (t > 0 && !s_ok) return;
      const bool resid = a.resid_first && t == 0;
      for (int q = q0; q < q1; ++q) {
        const WorkItem w = a.items[q];
        bool ok;
        if (resid) {
          const double acc = run_item<T, kWrite | kPack | kResid>(*Bp, p, w, ring, a.err, a.wait_ns, emu, ok, s_tab);
          const double s = block_sum<NT>(acc, red);
          if (tid == 0) a.partials[w.slot] = s;
        } else {
          run_item<T, kWrite | kPack>(*Bp, p, w, ring, a.err, a.wait_ns, emu, ok, s_tab);
        }
        if (!ok) return;  // CTA-uniform
      }
      fence_proxy_async();
      __syncthreads();
      if (tid == 0) st_release(a.progress + u, it + 1);
    }
  }
}

// ---------------------------------------------------------------------------
// Warp-specialised persistent kernel (all items plane-streamed): CW consumer
// warps and one producer warp per CTA, as in k_stream, but the ring of S
// stages (stride: the largest stage) runs on across items, units and
// iterations, and CTAs take their work dynamically.  The launch's work is
// n_iters x n_units tickets, handed out in order by one device counter
// (ticket t = iteration t / n_units, active unit t % n_units).  The producer
// warp takes a ticket, copies the unit's tables into a slot of a small
// shared-memory queue, acquire-waits (bounded, one lane per flag) until the
// unit's partners and the unit itself have finished the previous iteration,
// publishes the slot to the consumers and streams the unit's planes into the
// ring, reusing a stage once every consumer warp has released it; so it
// prefetches the next unit while the consumers compute.  The consumers take
// the queue's slots in order, compute each plane as k_stream does, release
// stages, and at the end of every item meet on an mbarrier (bounded wait; no
// named barrier, which a warp leaving on an error could hang): then one thread
// writes the item's residual partial and, after a unit's last item,
// release-stores progress[u] = it + 1.  Every thread fences its generic stores
// against the async proxy before that meeting, since other CTAs' bulk copies
// read them.
// Progress: a ticket waits only on tickets of the previous iteration, which
// are smaller.  The smallest unfinished ticket therefore has its partners
// finished, its producer can issue its planes (the ring stages and queue
// slots it needs are released by earlier, finished tickets of its CTA or by
// its own consumers), so it finishes; all CTAs are co-resident (cooperative
// launch).  Dynamic tickets let fast CTAs take more units, where a fixed
// assignment left per-CTA busy times 20 % apart (placement, not work).
// ---------------------------------------------------------------------------
// RESID: the launch runs one iteration and fuses the residual of its state
// (separate instantiations keep the plain sweep's register allocation).
// The host zeroes *a.ticket before every launch.  Registers are capped at 96
// per thread.
constexpr int kPersistQueue = 4;  // unit slots between the producer and the consumers

template <typename T, int CW, bool RESID>
__global__ void __launch_bounds__(StreamShape<CW>::threads, 65536 / (StreamShape<CW>::threads * 96))
    k_persist_ws(PersistLaunch a) {
  constexpr int VEC = V16<T>::N;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = (uint64_t*)smem;
  uint64_t* empty = full + 8;
  unsigned char* stages = smem + 128;
  __shared__ UnitCache s_q[kPersistQueue];
  __shared__ int64_t s_qit[kPersistQueue];  // iteration of the slot's ticket; -1: no more work
  __shared__ uint64_t s_qfull[kPersistQueue], s_qempty[kPersistQueue];
  __shared__ uint64_t s_done;
  __shared__ double s_red[2][CW];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S = a.stages;
  const size_t SB = (size_t)a.stage_bytes;
  if (tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(full + st, 1);
      mbar_init(empty + st, CW);
    }
    for (int k = 0; k < kPersistQueue; ++k) {
      mbar_init(s_qfull + k, 1);
      mbar_init(s_qempty + k, CW);
    }
    mbar_init(&s_done, CW);
    mbar_fence_init();
  }
  const int64_t it0 = a.it0_dev ? *a.it0_dev : a.it0;
  __syncthreads();
  const int64_t n_units = a.n_units;
  const uint64_t total = (uint64_t)a.n_iters * (uint64_t)n_units;
  if (warp == CW) {
    // ---- producer ----
    int64_t g = 0;       // planes issued (to drain after an error)
    int pst = 0;         // ring stage of the next plane ...
    uint32_t pfill = 0;  // ... and how often that stage was filled before
    int qs = 0;          // queue slot of the next ticket ...
    uint32_t qround = 0; // ... and how often the queue was passed through before
    bool ok = true;
    for (;;) {
      unsigned long long t = 0;
      if (lane == 0) t = atomicAdd(a.ticket, 1ull);
      t = __shfl_sync(0xffffffffu, t, 0);
      // the slot is free once every consumer warp finished its previous unit
      if (qround > 0 && !mbar_ready(s_qempty + qs, (qround - 1u) & 1u, a.err, a.wait_ns)) {
        ok = false;
        break;
      }
      if (t >= total) {  // no work left: tell the consumers
        if (lane == 0) {
          s_qit[qs] = -1;
          mbar_arrive(s_qfull + qs);
        }
        break;
      }
      const int64_t it = it0 + (int64_t)(t / (uint64_t)n_units);
      const int ui = (int)(t % (uint64_t)n_units);
      UnitCache& U = s_q[qs];
      {
        const int q0 = a.unit_items[ui];
        const BlockDev* Bg = a.blocks + a.items[q0].block;
        const uint32_t* src = (const uint32_t*)Bg;
        uint32_t* dst = (uint32_t*)&U.B;
        for (int i = lane; i < (int)(sizeof(BlockDev) / 4); i += 32) dst[i] = src[i];
        if (lane < 12) U.send[lane / 6][lane % 6] = Bg->send[lane % 6][lane / 6];
        const int d0 = a.dep_off[ui], d1 = a.dep_off[ui + 1];
        if (lane < kPersistDeps) U.dep[lane] = d0 + lane < d1 ? a.dep_ids[d0 + lane] : 0;
        if (lane == 0) {
          U.unit = a.unit_ids[ui];
          U.q0 = q0;
          U.q1 = a.unit_items[ui + 1];
          U.ndep = d1 - d0;
          U.start_iter = a.grids[Bg->grid].start_iter;
          U.emu = (sizeof(T) == 8 && a.emu && a.norms && a.norms[Bg->grid].emu_bad == 0u) ? 1 : 0;
          s_qit[qs] = it;
        }
      }
      __syncwarp();
      if (it > it0) {  // the launch's first iteration follows earlier launches in stream order
        bool okw = true;
        const int nd = U.ndep;
        if (lane < nd) okw = wait_ge(a.progress + U.dep[lane], it, a.err, a.wait_ns);
        else if (lane == nd) okw = wait_ge(a.progress + U.unit, it, a.err, a.wait_ns);
        ok = __all_sync(0xffffffffu, okw) != 0;
        if (!ok) {  // the error word is set: let the consumers leave
          if (lane == 0) {
            s_qit[qs] = -1;
            mbar_arrive(s_qfull + qs);
          }
          break;
        }
      }
      if (lane == 0) {
        fence_proxy_async();
        mbar_arrive(s_qfull + qs);  // publish the slot (tables and iteration)
        const int p = (int)((it - U.start_iter) & 1);
        for (int q = U.q0; q < U.q1 && ok; ++q) {
          const WorkItem w = a.items[q];
          const StageLayout L = stage_layout<T>(U.B, w.ya, w.yb);
          const int nplanes = w.z1 - w.z0 + 2;
          for (int j = 0; j < nplanes; ++j, ++g) {
            if (pfill > 0 && !mbar_ready(empty + pst, (pfill - 1u) & 1u, a.err, a.wait_ns)) {
              ok = false;
              break;
            }
            issue_plane<T>(U.B, p, w.z0, nplanes, j, w.ya, w.yb, L, stages + (size_t)pst * SB, full + pst);
            if (++pst == S) {
              pst = 0;
              ++pfill;
            }
          }
        }
      }
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) break;
      if (++qs == kPersistQueue) {
        qs = 0;
        ++qround;
      }
    }
    if (!ok && lane == 0) {
      // A wait expired: let the copies already issued land before leaving.
      for (int st = 0; st < S; ++st) {
        int64_t glast = -1;
        for (int64_t x = st; x < g; x += S) glast = x;
        if (glast >= 0) mbar_wait(full + st, (uint32_t)(glast / S) & 1u, a.err, a.wait_ns);
      }
    }
    return;
  }
  // ---- consumers ----
  // Ring positions (stage, fill parity) are advanced incrementally: c0 is the
  // next item's first plane.  (Stage and parity from a plane counter would
  // cost a 64-bit division by the run-time depth per use.)
  struct Pos {
    int st;
    uint32_t ph;
  };
  const auto adv = [S](Pos x) {
    if (++x.st == S) {
      x.st = 0;
      x.ph ^= 1u;
    }
    return x;
  };
  Pos c0{0, 0u};
  uint32_t nitem = 0;
  int qs = 0;
  uint32_t qround = 0;
  for (;;) {
    if (!mbar_ready(s_qfull + qs, qround & 1u, a.err, a.wait_ns)) return;
    const int64_t it = s_qit[qs];
    if (it < 0) return;  // no work left (or the producer stopped on an error)
    const UnitCache& U = s_q[qs];
    constexpr bool resid = RESID;
    const int p = (int)((it - U.start_iter) & 1);
    PlaneView<T> O = plane_view<T>(U.B, p);
    O.ss = U.send[p ^ 1];
    const bool emu = U.emu != 0;
    const int txv = O.rx / VEC;
    for (int q = U.q0; q < U.q1; ++q, ++nitem) {
      const WorkItem w = a.items[q];
      const StageLayout L = stage_layout<T>(U.B, w.ya, w.yb);
      const int nplanes = w.z1 - w.z0 + 2;
      const bool rag = item_ragged(w);
      const int tx = tid % txv, j0 = w.ya + (tid / txv) * 4;
      const bool active = j0 < w.yb;
      auto ready = [&](Pos x) { return mbar_ready(full + x.st, x.ph, a.err, a.wait_ns); };
      // planes qq - 1, qq, qq + 1 of the item
      Pos pm = c0, pc = adv(c0), pp = adv(pc);
      double acc = 0.0;
      bool good = true;
      for (int qq = 1; qq <= nplanes - 2 && good; ++qq) {
        if (qq == 1) good = ready(pm) && ready(pc);
        good = good && ready(pp);
        good = __all_sync(0xffffffffu, good) != 0;
        if (!good) break;
        if (active) {
          const unsigned char* sm = stages + (size_t)pm.st * SB;
          const unsigned char* sc = stages + (size_t)pc.st * SB;
          const unsigned char* sp = stages + (size_t)pp.st * SB;
          const int kq = w.z0 - 1 + qq;
          constexpr int MODE = RESID ? (kWrite | kPack | kResid) : (kWrite | kPack);
          if (rag) {
            if (sizeof(T) == 8 && emu) acc += stream_plane<T, 4, MODE, true, true, true>(O, kq, w.ya, L, sm, sc, sp, tx, j0);
            else acc += stream_plane<T, 4, MODE, false, true, true>(O, kq, w.ya, L, sm, sc, sp, tx, j0);
          } else {
            if (sizeof(T) == 8 && emu) acc += stream_plane<T, 4, MODE, true, false, true>(O, kq, w.ya, L, sm, sc, sp, tx, j0);
            else acc += stream_plane<T, 4, MODE, false, false, true>(O, kq, w.ya, L, sm, sc, sp, tx, j0);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + pm.st);
        pm = pc;
        pc = pp;
        pp = adv(pp);
      }
      if (!good) return;  // the error word is set; the producer drains its copies
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(empty + pm.st);
        mbar_arrive(empty + pc.st);
      }
      c0 = pp;
      // item end: every consumer warp has stored its part
      if (resid) {
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) s_red[nitem & 1][warp] = acc;
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&s_done);
      if (!mbar_ready(&s_done, (uint32_t)(nitem & 1), a.err, a.wait_ns)) return;
      if (tid == 0) {
        if (resid) {
          double r = 0.0;
          for (int c = 0; c < CW; ++c) r += s_red[nitem & 1][c];
          a.partials[w.slot] = r;
        }
        if (q == U.q1 - 1) st_release(a.progress + U.unit, it + 1);
      }
    }
    // the slot may be refilled once every consumer warp is done with it
    __syncwarp();
    if (lane == 0) mbar_arrive(s_qempty + qs);
    if (++qs == kPersistQueue) {
      qs = 0;
      ++qround;
    }
  }
}

template <typename K>
cudaError_t set_smem_attr(K kernel, bool& done) {
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxStepSmem);
  if (e == cudaSuccess) done = true;
  return e;
}

template <typename T, int RY, int CW, bool RAG, int MODE>
cudaError_t launch_stream(const StepLaunch& a, cudaStream_t s) {
  static bool done = false;
  cudaError_t e = set_smem_attr(k_stream<T, RY, CW, RAG, MODE>, done);
  if (e != cudaSuccess) return e;
  k_stream<T, RY, CW, RAG, MODE><<<a.n_items, StreamShape<CW>::threads, a.smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t launch_kind(const StepLaunch& a, int kind, cudaStream_t s) {
  StepLaunch b = a;
  b.items = a.items + a.kind_off[kind];
  b.n_items = a.kind_off[kind + 1] - a.kind_off[kind];
  switch (kind) {
    case 0: k_tiles<T, MODE><<<b.n_items, kThreads, 0, s>>>(b); return cudaGetLastError();
    case 1: return launch_stream<T, 4, 8, false, MODE>(b, s);
    case 2: return launch_stream<T, 4, 4, false, MODE>(b, s);
    case 3: return launch_stream<T, 4, 2, false, MODE>(b, s);
    case 4: return launch_stream<T, 4, 8, true, MODE>(b, s);
    case 5: return launch_stream<T, 4, 4, true, MODE>(b, s);
    default: return launch_stream<T, 4, 2, true, MODE>(b, s);
  }
}

template <typename T, int MODE>
cudaError_t launch_kinds(const StepLaunch& a, cudaStream_t s, const KindFork* fork) {
  // Non-empty kinds, largest first (it is launched first and fills the GPU;
  // the smaller ones fill in around it).
  int order[kItemKinds], nk = 0;
  for (int kind = 0; kind < kItemKinds; ++kind)
    if (a.kind_off[kind + 1] > a.kind_off[kind]) order[nk++] = kind;
  auto size = [&](int k) { return a.kind_off[k + 1] - a.kind_off[k]; };
  for (int i = 1; i < nk; ++i)
    for (int j = i; j > 0 && size(order[j]) > size(order[j - 1]); --j) std::swap(order[j], order[j - 1]);
  if (!fork || nk <= 1) {
    for (int i = 0; i < nk; ++i) {
      cudaError_t e = launch_kind<T, MODE>(a, order[i], s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  cudaError_t e = cudaEventRecord(fork->fork, s);
  for (int i = 1; i < nk && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(fork->aux[i], fork->fork, 0);
  if (e == cudaSuccess) e = launch_kind<T, MODE>(a, order[0], s);
  for (int i = 1; i < nk && e == cudaSuccess; ++i) {
    e = launch_kind<T, MODE>(a, order[i], fork->aux[i]);
    if (e == cudaSuccess) e = cudaEventRecord(fork->join[i], fork->aux[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, fork->join[i], 0);
  }
  return e;
}

template <typename T>
cudaError_t launch_step_t(const StepLaunch& a, int mode, cudaStream_t s, const KindFork* f) {
  if (a.n_items <= 0) return cudaSuccess;
  switch (mode) {
    case kWrite | kPack: return launch_kinds<T, kWrite | kPack>(a, s, f);
    case kWrite | kPack | kResid: return launch_kinds<T, kWrite | kPack | kResid>(a, s, f);
    case kWrite: return launch_kinds<T, kWrite>(a, s, f);
    case kResid: return launch_kinds<T, kResid>(a, s, f);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int NT>
const void* persist_fn_t() {
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(k_persist<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxStepSmem) !=
        cudaSuccess)
      return nullptr;
    attr_set = true;
  }
  return (const void*)k_persist<T, NT>;
}

template <typename T, int CW, bool R>
const void* persist_ws_fn_t() {
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(k_persist_ws<T, CW, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPersistWsSmem) !=
        cudaSuccess)
      return nullptr;
    attr_set = true;
  }
  return (const void*)k_persist_ws<T, CW, R>;
}

template <typename T, bool R>
const void* persist_ws_fn_r(int cw) {
  return cw == 2 ? persist_ws_fn_t<T, 2, R>() : cw == 4 ? persist_ws_fn_t<T, 4, R>() : persist_ws_fn_t<T, 8, R>();
}

const void* persist_ws_fn(int dtype, int cw, bool resid) {
  if (dtype == 0) return resid ? persist_ws_fn_r<double, true>(cw) : persist_ws_fn_r<double, false>(cw);
  return resid ? persist_ws_fn_r<float, true>(cw) : persist_ws_fn_r<float, false>(cw);
}

const void* persist_fn(int dtype, int threads) {
  if (dtype == 0) {
    return threads == 64 ? persist_fn_t<double, 64>() : threads == 128 ? persist_fn_t<double, 128>()
                                                                       : persist_fn_t<double, 256>();
  }
  return threads == 64 ? persist_fn_t<float, 64>() : threads == 128 ? persist_fn_t<float, 128>()
                                                                    : persist_fn_t<float, 256>();
}

}  // namespace

cudaError_t launch_step(const StepLaunch& a, int mode, cudaStream_t s, const KindFork* fork) {
  return a.dtype == 0 ? launch_step_t<double>(a, mode, s, fork) : launch_step_t<float>(a, mode, s, fork);
}

cudaError_t kind_fork_create(KindFork* f) {
  cudaError_t e = cudaEventCreateWithFlags(&f->fork, cudaEventDisableTiming);
  for (int k = 0; k < kItemKinds && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&f->aux[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f->join[k], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) kind_fork_destroy(f);
  return e;
}

void kind_fork_destroy(KindFork* f) {
  if (f->fork) cudaEventDestroy(f->fork);
  f->fork = nullptr;
  for (int k = 0; k < kItemKinds; ++k) {
    if (f->aux[k]) cudaStreamDestroy(f->aux[k]);
    if (f->join[k]) cudaEventDestroy(f->join[k]);
    f->aux[k] = nullptr;
    f->join[k] = nullptr;
  }
}

int persistent_max_ctas(int dtype, int smem, int threads, int ws_cw) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  const void* fn = ws_cw ? persist_ws_fn(dtype, ws_cw, false) : persist_fn(dtype, threads);
  const int nt = ws_cw ? 32 * ws_cw + 32 : threads;
  if (!fn) return 0;
  if (ws_cw) {  // the residual instantiation must fit the same launch
    int r = 0;
    const void* fr = persist_ws_fn(dtype, ws_cw, true);
    if (!fr || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, fr, nt, smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nt, smem) != cudaSuccess) return 0;
    return std::min(r, per_sm) * sms;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nt, smem) != cudaSuccess) return 0;
  return per_sm * sms;
}

cudaError_t launch_persistent(const PersistLaunch& a, int grid_ctas, cudaStream_t s) {
  if (a.n_units <= 0 || a.n_iters <= 0) return cudaSuccess;
  PersistLaunch args = a;
  void* params[] = {&args};
  // the warp-specialised kernel fuses the residual only in one-iteration launches
  if (a.ws_cw && a.resid_first && a.n_iters != 1) return cudaErrorInvalidValue;
  const void* fn = a.ws_cw ? persist_ws_fn(a.dtype, a.ws_cw, a.resid_first != 0) : persist_fn(a.dtype, a.threads);
  const int nt = a.ws_cw ? 32 * a.ws_cw + 32 : a.threads;
  if (!fn) return cudaErrorInvalidValue;
  return cudaLaunchCooperativeKernel(fn, dim3(grid_ctas), dim3(nt), params, a.smem, s);
}

}  // namespace jgb
