// One operator step in one kernel (D = 3, float4 along y): the pass pair
// k_Ly4 + k_LTy4<MODE> fused through shared memory.
//
// A CTA owns a tile of TT time planes x FS_TX x-rows x the whole y extent.
//   1. x (the operand) on the tile plus a halo of 2 rows in t and x is copied
//      into shared memory with cp.async;
//   2. y = -rho L x is computed on the tile plus a halo of 1 row, into shared
//      memory (the rows of L reach +-1, or +-2 for the one-sided forms at the
//      first and last plane / row of a non-periodic dim);
//   3. q = L^T y - theta 1_B x = -(S x) on the tile, then the mode's update
//      (Chebyshev step, residual, or apply with the <x, S x> partial sums).
// y never goes to global memory and the step is one launch.  A column gathers
// rows at distance 2 only when that row is the first or last of its
// non-periodic dim; with n_t % TT == 0, n_x % FS_TX == 0 and both tile sizes
// >= 3, such a row is always inside the halo of 1.
//
// The operand is read with a halo, so the Chebyshev modes must not update it
// in place: a.x is read, a.e written (the caller alternates two buffers).  The
// Chebyshev direction is x minus the previous iterate, which a.d points to
// (the other buffer, read at the point, then overwritten by the new iterate;
// null on the first step from zero): no direction array is kept.
#pragma once
#include "mpn_device.cuh"
#include "mpn_stepargs.cuh"

#define FS_TX 4
#define FS_TPB 256

// Bulk asynchronous copies global -> shared completing on an mbarrier.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(float* dst, const float* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// Waits for phase `parity` of the barrier; gives up after `limit` polls.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int limit) {
  const unsigned a = smem_u32(bar);
  for (int i = 0; i < limit; ++i) {
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(a), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}
#define FS_WAIT_LIMIT (1 << 22)

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
// Asks L2 for the line holding p (no register, no wait).
__device__ __forceinline__ void pf_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Shared-memory floats of the tile for a y extent n2.
__host__ __device__ constexpr int fs_rows_x(int TT) { return (TT + 4) * (FS_TX + 4); }
__host__ __device__ constexpr int fs_rows_y(int TT) { return (TT + 2) * (FS_TX + 2); }

// Difference forms along a dim at a row of class cls (0 central, 1 first,
// 2 last point of a non-periodic dim) from the values at offsets -2..2.
__device__ __forceinline__ void dforms(int cls, float4 xm2, float4 xm1, float4 x0, float4 xp1, float4 xp2, float4& a1,
                                       float4& a2) {
  if (cls == 0) { a1 = 0.5f * (xp1 - xm1); a2 = xp1 - 2.f * x0 + xm1; }
  else if (cls == 1) { a1 = -1.5f * x0 + 2.f * xp1 - 0.5f * xp2; a2 = x0 - 2.f * xp1 + xp2; }
  else { a1 = 1.5f * x0 - 2.f * xm1 + 0.5f * xm2; a2 = x0 - 2.f * xm1 + xm2; }
}
__device__ __forceinline__ void dforms1(int cls, float xm2, float xm1, float x0, float xp1, float xp2, float& a1, float& a2) {
  if (cls == 0) { a1 = 0.5f * (xp1 - xm1); a2 = xp1 - 2.f * x0 + xm1; }
  else if (cls == 1) { a1 = -1.5f * x0 + 2.f * xp1 - 0.5f * xp2; a2 = x0 - 2.f * xp1 + xp2; }
  else { a1 = 1.5f * x0 - 2.f * xm1 + 0.5f * xm2; a2 = x0 - 2.f * xm1 + xm2; }
}

// Coefficient access.  MASK = FS_ANY: fields at stride 1 and per-instance
// scalars (stored four times) at stride 0, one load either way.  Otherwise
// bit v of MASK says that c_v is a field (the problem's layout is fixed at
// compile time): scalars are loaded once into registers and fields per group;
// with FS_SHARE46, c_yy reads the field of c_xx, so their loads are issued once.
template <int MASK>
struct CoefU4 {
  const float* base[7];
  int ps[7];
  float sv[7];
  __device__ __forceinline__ CoefU4(const Coef& c, int b) {
#pragma unroll
    for (int v = 0; v < 7; ++v) {
      base[v] = c.ptr4[v] + (size_t)b * c.bstride4[v];
      ps[v] = c.pstride[v];
      sv[v] = (MASK != FS_ANY && !((MASK >> v) & 1)) ? __ldg(base[v]) : 0.f;
    }
  }
  __device__ __forceinline__ float4 at4(int v, int p) const {
    if (MASK == FS_ANY) return ld4(base[v] + p * ps[v]);
    if ((MASK & FS_SHARE46) && v == 6) v = 4;
    return ((MASK >> v) & 1) ? ld4(base[v] + p) : f4(sv[v]);
  }
  // L2 prefetch of the fields at point p (compile-time layouts only)
  __device__ __forceinline__ void prefetch(int p) const {
    if (MASK == FS_ANY) return;
#pragma unroll
    for (int v = 0; v < 7; ++v)
      if (((MASK >> v) & 1) && !((MASK & FS_SHARE46) && v == 6)) pf_l2(base[v] + p);
  }
  __device__ __forceinline__ float at(int v, int p) const {
    if (MASK == FS_ANY) return __ldg(base[v] + p * ps[v]);
    if ((MASK & FS_SHARE46) && v == 6) v = 4;
    return ((MASK >> v) & 1) ? __ldg(base[v] + p) : sv[v];
  }
};

template <int MODE, int TT, bool PER1, bool PER2, int MASK>
__global__ void __launch_bounds__(FS_TPB) k_step3(Grid g, Coef cf, const float* __restrict__ rho, StepArgs a) {
  extern __shared__ __align__(16) float fsm[];
  constexpr int RXW = FS_TX + 4, RYW = FS_TX + 2;
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const int G = n2 >> 2;
  const float invG = 1.f / (float)G;
  const int b = blockIdx.y;
  const int ntx = n1 / FS_TX;
  const int t0 = (blockIdx.x / ntx) * TT, x0 = (blockIdx.x % ntx) * FS_TX;
  const size_t off = (size_t)b * g.N;
  const int pl = n1 * n2;   // points per time plane
  float* xs = fsm;
  float* ys = fsm + fs_rows_x(TT) * n2;
  const float* X = a.x + off;
  const CoefU4<MASK> C(cf, b);
  const float h1t = 0.5f * g.is1[0], h1x = 0.5f * g.is1[1], h1y = 0.5f * g.is1[2];
  const float i2t = g.is2[0], i2x = g.is2[1], i2y = g.is2[2];

  // 1. operand rows t0-2 .. t0+TT+1 x x0-2 .. x0+FS_TX+1 (rows outside a
  //    non-periodic domain are never read): per time plane one bulk copy of
  //    the consecutive x rows, split where a periodic x wraps
  //    Lane rt of warp 0 copies time plane t0-2+rt.
  __shared__ unsigned long long bar;
  if (threadIdx.x < 32) {
    const int rt = threadIdx.x, t = t0 - 2 + rt;
    const bool plane = rt < TT + 4 && t >= 0 && t < n0;
    // visits the segments (source row x, tile row, rows) of this lane's plane
    auto segments = [&](auto&& visit) {
      int rx = 0;
      while (plane && rx < RXW) {
        int x = x0 - 2 + rx, len;
        if (x < 0) {
          len = min(-x, RXW - rx);
          if (!PER1) { rx += len; continue; }
          x += n1;
        } else if (x >= n1) {
          if (!PER1) break;
          len = RXW - rx;
          x -= n1;
        } else {
          len = min(n1 - x, RXW - rx);
        }
        visit(x, rt * RXW + rx, len);
        rx += len;
      }
    };
    int rows = 0;
    segments([&](int, int, int len) { rows += len; });
    rows = __reduce_add_sync(0xffffffffu, rows);
    if (rt == 0) {
      mbar_init(&bar, 1);
      mbar_expect_tx(&bar, (unsigned)(rows * n2 * sizeof(float)));
    }
    __syncwarp();
    segments([&](int x, int r, int len) {
      bulk_g2s(xs + r * n2, X + (size_t)t * pl + (size_t)x * n2, (unsigned)(len * n2 * sizeof(float)), &bar);
    });
  }
  // PCG's direction update (mode 5): beta from the partial sums, read while
  // the operand copies are in flight
  float beta = 0.f;
  if (MODE == SM_APPLYP && a.d) {
    const double rz = a.rz_tot ? a.rz_tot[b] : sum_partials(a.rz, b, a.nrz), ro = a.rz_old[b];
    beta = cta_scalar([&] { return (ro > 0 && rz > 0) ? (float)(rz / ro) : 0.f; });
  }
  __syncthreads();
  if (!mbar_wait(&bar, 0, FS_WAIT_LIMIT) && a.err) atomicExch(a.err, 1);
  __syncthreads();
  if (MODE == SM_APPLYP) {
    // the operand p = x + beta d on the tile and its halo (x staged above),
    // and p on the tile rows to e, a buffer other than d (neighbouring tiles
    // read d as their halo)
    for (int i = threadIdx.x; i < fs_rows_x(TT) * G; i += FS_TPB) {
      int gq;
      const int row = fdivmod(i, G, invG, gq);
      const int rt = row / RXW, rx = row % RXW;
      const int t = t0 - 2 + rt;
      int x = x0 - 2 + rx;
      if (t < 0 || t >= n0) continue;
      if (PER1) { if (x < 0) x += n1; else if (x >= n1) x -= n1; }
      else if (x < 0 || x >= n1) continue;
      const size_t q = off + (size_t)t * pl + (size_t)x * n2 + 4 * gq;
      float* sp = xs + row * n2 + 4 * gq;
      float4 v = lds4(sp);
      if (a.d) v = v + beta * ld4(a.d + q);
      *reinterpret_cast<float4*>(sp) = v;
      if (rt >= 2 && rt < TT + 2 && rx >= 2 && rx < FS_TX + 2) *reinterpret_cast<float4*>(a.e + q) = v;
    }
    __syncthreads();
  }

  // each thread keeps one float4 group gi of the rows and strides over rows
  const int rstride = FS_TPB / G;
  int gi;
  const int row0 = fdivmod((int)threadIdx.x, G, invG, gi);
  const bool active = row0 < rstride;
  const int y0 = 4 * gi;
  const bool yin2 = PER2 || (y0 >= 1 && y0 + 4 <= n2 - 1);   // L rows of the group are central in y
  const bool yin3 = PER2 || (y0 >= 3 && y0 + 3 <= n2 - 4);   // L^T gathers of the group are central in y
  const int yl = y0 == 0 ? n2 - 1 : y0 - 1, yr4 = y0 + 4 == n2 ? 0 : y0 + 4;

  // 2. y = -rho L x on rows t0-1 .. t0+TT x x0-1 .. x0+FS_TX
  for (int row = active ? row0 : fs_rows_y(TT); row < fs_rows_y(TT); row += rstride) {
    const int st = row / RYW, sx = row % RYW;
    const int t = t0 - 1 + st;
    int x = x0 - 1 + sx;
    if (t < 0 || t >= n0) continue;
    if (PER1) { if (x < 0) x += n1; else if (x >= n1) x -= n1; }
    else if (x < 0 || x >= n1) continue;
    const int p = t * pl + x * n2 + y0;
    const float4 r4 = ld4(rho + off + p);                     // issued before the arithmetic
    // a compile-time layout's coefficients at the point, loaded up front too
    // (the generic layout loads them where they are used)
    float4 cpt[7];
#pragma unroll
    for (int v = 0; v < 7; ++v) cpt[v] = MASK != FS_ANY ? C.at4(v, p) : f4(0.f);
    auto cat = [&](int v) { return MASK != FS_ANY ? cpt[v] : C.at4(v, p); };
    const float* xr = xs + ((st + 1) * RXW + sx + 1) * n2;   // operand row of this y row
    const float4 xc = lds4(xr + y0);
    float4 Lx = cat(0) * xc;
    if (t > 0 && t < n0 - 1 && (PER1 || (x > 0 && x < n1 - 1))) {
      const float4 tm = lds4(xr - RXW * n2 + y0), tp = lds4(xr + RXW * n2 + y0);
      const float4 xm = lds4(xr - n2 + y0), xp = lds4(xr + n2 + y0);
      Lx = Lx + (h1t * cat(1)) * (tp - tm) + (i2t * cat(2)) * (tp - 2.f * xc + tm) +
           (h1x * cat(3)) * (xp - xm) + (i2x * cat(4)) * (xp - 2.f * xc + xm);
    } else {
      float4 a1, a2;
      {
        const int cls = t == 0 ? 1 : (t == n0 - 1 ? 2 : 0);
        const float* up = xr + RXW * n2;
        const float* dn = xr - RXW * n2;
        float4 xm1 = cls != 1 ? lds4(dn + y0) : xc, xp1 = cls != 2 ? lds4(up + y0) : xc;
        float4 xm2 = cls == 2 ? lds4(dn - RXW * n2 + y0) : xc, xp2 = cls == 1 ? lds4(up + RXW * n2 + y0) : xc;
        dforms(cls, xm2, xm1, xc, xp1, xp2, a1, a2);
        Lx = Lx + (g.is1[0] * cat(1)) * a1 + (i2t * cat(2)) * a2;
      }
      {
        const int cls = PER1 ? 0 : (x == 0 ? 1 : (x == n1 - 1 ? 2 : 0));
        float4 xm1 = cls != 1 ? lds4(xr - n2 + y0) : xc, xp1 = cls != 2 ? lds4(xr + n2 + y0) : xc;
        float4 xm2 = cls == 2 ? lds4(xr - 2 * n2 + y0) : xc, xp2 = cls == 1 ? lds4(xr + 2 * n2 + y0) : xc;
        dforms(cls, xm2, xm1, xc, xp1, xp2, a1, a2);
        Lx = Lx + (g.is1[1] * cat(3)) * a1 + (i2x * cat(4)) * a2;
      }
    }
    // y: whole row in shared memory
    if (yin2) {
      const float4 ym = make_float4(xr[yl], xc.x, xc.y, xc.z), yp = make_float4(xc.y, xc.z, xc.w, xr[yr4]);
      Lx = Lx + (h1y * cat(5)) * (yp - ym) + (i2y * cat(6)) * (yp - 2.f * xc + ym);
    } else {
      float l4[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int yy = y0 + k;
        const int cls = yy == 0 ? 1 : (yy == n2 - 1 ? 2 : 0);
        const float v0 = xr[yy];
        const float vm1 = cls != 1 ? xr[yy - 1] : v0, vp1 = cls != 2 ? xr[yy + 1] : v0;
        const float vm2 = cls == 2 ? xr[yy - 2] : v0, vp2 = cls == 1 ? xr[yy + 2] : v0;
        float b1, b2;
        dforms1(cls, vm2, vm1, v0, vp1, vp2, b1, b2);
        l4[k] = g.is1[2] * C.at(5, p + k) * b1 + i2y * C.at(6, p + k) * b2;
      }
      Lx = Lx + make_float4(l4[0], l4[1], l4[2], l4[3]);
    }
    *reinterpret_cast<float4*>(ys + row * n2 + y0) = make_float4(-r4.x * Lx.x, -r4.y * Lx.y, -r4.z * Lx.z, -r4.w * Lx.w);
  }
  __syncthreads();

  // 3. q = L^T y - theta 1_B x on the tile, then the update
  float acc = 0.f;
  for (int row = active ? row0 : TT * FS_TX; row < TT * FS_TX; row += rstride) {
    const int ot = row / FS_TX, ox = row % FS_TX;
    const int t = t0 + ot, x = x0 + ox;
    const int p = t * pl + x * n2 + y0;
    // operands of the update, loaded before the gather so that their latency
    // overlaps it
    const size_t j = off + p;
    float4 ur = make_float4(0.f, 0.f, 0.f, 0.f), udi = ur, ud = ur;
    if (MODE != SM_APPLY && MODE != SM_APPLYP) ur = ld4(a.r + j);
    if (MODE == SM_POST0 || MODE == SM_CHEB || MODE == SM_CHEB_DOT) udi = ld4(a.dinv + j);
    // previous iterate: the buffer this step overwrites at the same point, so a
    // coherent load (not the read-only path)
    if ((MODE == SM_CHEB || MODE == SM_CHEB_DOT) && a.d) ud = __ldcg(reinterpret_cast<const float4*>(a.d + j));
    const float* yr = ys + ((ot + 1) * RYW + ox + 1) * n2;
    const float4 yc = lds4(yr + y0);
    const int pxm = (PER1 && x == 0) ? p + (n1 - 1) * n2 : p - n2;
    const int pxp = (PER1 && x == n1 - 1) ? p - (n1 - 1) * n2 : p + n2;
    // a compile-time layout's coefficients of the central gathers, loaded up
    // front (a neighbour index stays at the point where its branch is not
    // taken); the generic layout loads them where they are used
    const bool tcen = t >= 3 && t <= n0 - 4, xcen = PER1 || (x >= 3 && x <= n1 - 4);
    float4 k0, k1m, k1p, k2, k2m, k2p, k3m, k3p, k4, k4m, k4p, k5, k6;
    float c5l, c5r, c6l, c6r;
    if (MASK != FS_ANY) {
      const int ptm = tcen ? p - pl : p, ptp = tcen ? p + pl : p;
      const int qxm = xcen ? pxm : p, qxp = xcen ? pxp : p;
      const int prow = p - y0;
      k0 = C.at4(0, p); k2 = C.at4(2, p); k4 = C.at4(4, p); k5 = C.at4(5, p); k6 = C.at4(6, p);
      k1m = C.at4(1, ptm); k1p = C.at4(1, ptp); k2m = C.at4(2, ptm); k2p = C.at4(2, ptp);
      k3m = C.at4(3, qxm); k3p = C.at4(3, qxp); k4m = C.at4(4, qxm); k4p = C.at4(4, qxp);
      c5l = C.at(5, prow + yl); c5r = C.at(5, prow + yr4); c6l = C.at(6, prow + yl); c6r = C.at(6, prow + yr4);
    }
    auto pick = [&](const float4& pre, int v, int q) { return MASK != FS_ANY ? pre : C.at4(v, q); };
    auto pickf = [&](float pre, int v, int q) { return MASK != FS_ANY ? pre : C.at(v, q); };
    float4 qv = pick(k0, 0, p) * yc;
    if (t >= 3 && t <= n0 - 4 && (PER1 || (x >= 3 && x <= n1 - 4))) {
      const float4 tm = lds4(yr - RYW * n2 + y0), tp = lds4(yr + RYW * n2 + y0);
      const float4 xm = lds4(yr - n2 + y0), xp = lds4(yr + n2 + y0);
      const float4 c2t = pick(k2, 2, p), c2x = pick(k4, 4, p);
      qv = qv + h1t * (pick(k1m, 1, p - pl) * tm - pick(k1p, 1, p + pl) * tp) +
           i2t * (pick(k2m, 2, p - pl) * tm - 2.f * (c2t * yc) + pick(k2p, 2, p + pl) * tp) +
           h1x * (pick(k3m, 3, pxm) * xm - pick(k3p, 3, pxp) * xp) +
           i2x * (pick(k4m, 4, pxm) * xm - 2.f * (c2x * yc) + pick(k4p, 4, pxp) * xp);
    } else {
      // t
      if (t >= 3 && t <= n0 - 4) {
        const float4 ym = lds4(yr - RYW * n2 + y0), yp = lds4(yr + RYW * n2 + y0);
        qv = qv + h1t * (pick(k1m, 1, p - pl) * ym - pick(k1p, 1, p + pl) * yp) +
             i2t * (pick(k2m, 2, p - pl) * ym - 2.f * (pick(k2, 2, p) * yc) + pick(k2p, 2, p + pl) * yp);
      } else {
#pragma unroll
        for (int o = -2; o <= 2; ++o) {
          const int ip = t - o;
          if (ip < 0 || ip >= n0) continue;
          const float w1 = dweight(1, ip, n0, 0, o), w2 = dweight(2, ip, n0, 0, o);
          if (w1 == 0.f && w2 == 0.f) continue;
          const int pi = p - o * pl;
          const float4 yv = o == 0 ? yc : lds4(yr - o * RYW * n2 + y0);
          qv = qv + yv * ((w1 * g.is1[0]) * C.at4(1, pi) + (w2 * i2t) * C.at4(2, pi));
        }
      }
      // x
      if (PER1 || (x >= 3 && x <= n1 - 4)) {
        const float4 ym = lds4(yr - n2 + y0), yp = lds4(yr + n2 + y0);
        qv = qv + h1x * (pick(k3m, 3, pxm) * ym - pick(k3p, 3, pxp) * yp) +
             i2x * (pick(k4m, 4, pxm) * ym - 2.f * (pick(k4, 4, p) * yc) + pick(k4p, 4, pxp) * yp);
      } else {
#pragma unroll
        for (int o = -2; o <= 2; ++o) {
          const int ip = x - o;
          if (ip < 0 || ip >= n1) continue;
          const float w1 = dweight(1, ip, n1, 0, o), w2 = dweight(2, ip, n1, 0, o);
          if (w1 == 0.f && w2 == 0.f) continue;
          const int pi = p - o * n2;
          const float4 yv = o == 0 ? yc : lds4(yr - o * n2 + y0);
          qv = qv + yv * ((w1 * g.is1[1]) * C.at4(3, pi) + (w2 * i2x) * C.at4(4, pi));
        }
      }
    }
    // y
    if (yin3) {
      const int prow = p - y0;
      const float4 c1 = pick(k5, 5, p), c2 = pick(k6, 6, p);
      const float c1l = pickf(c5l, 5, prow + yl), c1r = pickf(c5r, 5, prow + yr4), c2l = pickf(c6l, 6, prow + yl), c2r = pickf(c6r, 6, prow + yr4);
      const float4 ym = make_float4(yr[yl], yc.x, yc.y, yc.z), yp = make_float4(yc.y, yc.z, yc.w, yr[yr4]);
      const float4 c1m = make_float4(c1l, c1.x, c1.y, c1.z), c1p = make_float4(c1.y, c1.z, c1.w, c1r);
      const float4 c2m = make_float4(c2l, c2.x, c2.y, c2.z), c2p = make_float4(c2.y, c2.z, c2.w, c2r);
      qv = qv + h1y * (c1m * ym - c1p * yp) + i2y * (c2m * ym - 2.f * (c2 * yc) + c2p * yp);
    } else {
      float q4[4] = {0.f, 0.f, 0.f, 0.f};
      const int prow = p - y0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int yy = y0 + k;
#pragma unroll
        for (int o = -2; o <= 2; ++o) {
          const int iy = yy - o;
          if (iy < 0 || iy >= n2) continue;
          const float w1 = dweight(1, iy, n2, 0, o), w2 = dweight(2, iy, n2, 0, o);
          if (w1 == 0.f && w2 == 0.f) continue;
          q4[k] += yr[iy] * (w1 * g.is1[2] * C.at(5, prow + iy) + w2 * i2y * C.at(6, prow + iy));
        }
      }
      qv = qv + make_float4(q4[0], q4[1], q4[2], q4[3]);
    }
    const float4 xj = lds4(xs + ((ot + 2) * RXW + ox + 2) * n2 + y0);
    // Dirichlet rows: t and x faces are shared by the group, y faces per point
    const bool bnd_tx = t == 0 || (g.final_rows && t == n0 - 1) || (!PER1 && (x == 0 || x == n1 - 1));
    if (bnd_tx) {
      qv = qv - g.theta * xj;
    } else if (!PER2) {
      if (y0 == 0) qv.x -= g.theta * xj.x;
      if (y0 + 3 == n2 - 1) qv.w -= g.theta * xj.w;
    }
    // qv = -(S x) on the group
    if (MODE == SM_APPLY || MODE == SM_APPLYP) {
      *reinterpret_cast<float4*>(a.out + j) = make_float4(-qv.x, -qv.y, -qv.z, -qv.w);
      acc -= qv.x * xj.x + qv.y * xj.y + qv.z * xj.z + qv.w * xj.w;
    } else if (MODE == SM_RES) {
      *reinterpret_cast<float4*>(a.out + j) = ur + qv;
    } else {
      const float4 res = ur + qv;
      float4 dn = a.c2 * (udi * res);
      // the direction is the difference of the last two iterates, so no
      // direction array is read or written (a.d: previous iterate, null = 0)
      if (MODE == SM_CHEB || MODE == SM_CHEB_DOT) dn = dn + a.c1 * (xj - ud);
      const float4 en = xj + dn;
      *reinterpret_cast<float4*>(a.e + j) = en;
      if (MODE == SM_CHEB_DOT) acc += en.x * ur.x + en.y * ur.y + en.z * ur.z + en.w * ur.w;   // <e', r>
    }
  }
  if ((MODE == SM_APPLY || MODE == SM_APPLYP || MODE == SM_CHEB_DOT) && a.part) {
    const double s = block_sum((double)acc);
    partial_finish(s, a.part, a.cnt, a.tot, b, blockIdx.x, gridDim.x);
  }
}
