// One operator step in one kernel on tiles that split the y rows (D = 3,
// float4 along y): the variant of k_step3 for rows too wide to keep whole in
// shared memory (n_y = 256 on the finest level of the transport workload).
//
// A CTA owns a tile of TT time planes x FS_TX x-rows x TY y points.
//   1. The operand on the tile plus a halo of 2 rows in t and x and of 4
//      points on each side in y is copied into shared memory by bulk
//      asynchronous copies, one per (t, x) row segment (16-byte aligned: the
//      y halo is one float4 group), split where a periodic y wraps and clipped
//      to the domain where it does not; they complete on an mbarrier with a
//      bounded wait.
//   2. y = -rho L x on the tile plus a ring of 1 row in t and x (float4
//      groups) and one point on each side in y (two scalar points per row:
//      the rows of L reach +-1 in y there, since a tile edge inside the domain
//      is never a non-periodic edge of the grid), into shared memory.
//   3. q = L^T y - theta 1_B x = -(S x) on the tile, then the mode's update.
// Rows of L at distance 2 (the one-sided forms at a non-periodic grid edge)
// are always inside the tile or its ring: a tile's y range starts at a
// multiple of TY >= 8, so a non-periodic y edge is interior to its tile.
// Shared-memory rows have W = TY + 8 floats; column c holds y = y0t - 4 + c.
// The Chebyshev and apply modes follow k_step3 (alternating iterate buffers,
// the previous iterate read at the point, PCG's direction update in mode 5).
#pragma once
#include "mpn_fused.cuh"

__host__ __device__ constexpr int fsy_width(int TY) { return TY + 8; }
// Shared-memory bytes of a tile.
__host__ __device__ constexpr int fsy_floats(int TT, int TY) {
  return (fs_rows_x(TT) + fs_rows_y(TT)) * fsy_width(TY);
}

template <int MODE, int TT, int TY, bool PER1, bool PER2, int MASK>
__global__ void __launch_bounds__(FS_TPB) k_step3y(Grid g, Coef cf, const float* __restrict__ rho, StepArgs a) {
  extern __shared__ __align__(16) float fsm[];
  constexpr int RXW = FS_TX + 4, RYW = FS_TX + 2, W = fsy_width(TY), G = TY / 4;
  constexpr float invG = 1.f / (float)G;
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const int b = blockIdx.y;
  const int nty = n2 / TY, ntx = n1 / FS_TX;
  const int tq = blockIdx.x / nty;
  const int y0t = (blockIdx.x - tq * nty) * TY;
  const int t0 = (tq / ntx) * TT, x0 = (tq % ntx) * FS_TX;
  const size_t off = (size_t)b * g.N;
  const int pl = n1 * n2;
  float* xs = fsm;
  float* ys = fsm + fs_rows_x(TT) * W;
  const float* X = a.x + off;
  const CoefU4<MASK> C(cf, b);
  const float h1t = 0.5f * g.is1[0], h1x = 0.5f * g.is1[1], h1y = 0.5f * g.is1[2];
  const float i2t = g.is2[0], i2x = g.is2[1], i2y = g.is2[2];

  // 1. operand rows t0-2 .. t0+TT+1 x x0-2 .. x0+FS_TX+1, y0t-4 .. y0t+TY+3;
  //    warp 0 issues the copies, lane l the rows l, l + 32, ...  The barrier
  //    is initialised first, so no thread waits for the copies to be issued:
  //    meanwhile every thread asks L2 for the global data its passes read.
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x < 32) {
    // visits the segments (global point of the row's first copied y, shared
    // column, length) of shared row `row`; none when the row lies outside a
    // non-periodic domain
    auto segments = [&](int row, auto&& visit) {
      const int rt = row / RXW, rx = row - (row / RXW) * RXW;
      const int t = t0 - 2 + rt;
      int x = x0 - 2 + rx;
      if (t < 0 || t >= n0) return;
      if (PER1) { x = x < 0 ? x + n1 : (x >= n1 ? x - n1 : x); }
      else if (x < 0 || x >= n1) return;
      const int base = t * pl + x * n2;
      int c = 0;
      while (c < W) {
        int y = y0t - 4 + c, len = W - c;
        if (y < 0) {
          len = min(-y, len);
          if (!PER2) { c += len; continue; }
          y += n2;
        } else if (y >= n2) {
          if (!PER2) break;
          y -= n2;
        } else {
          len = min(n2 - y, len);
        }
        visit(base + y, row * W + c, len);
        c += len;
      }
    };
    unsigned bytes = 0;
    for (int row = threadIdx.x; row < fs_rows_x(TT); row += 32)
      segments(row, [&](int, int, int len) { bytes += (unsigned)len * 4u; });
    bytes = __reduce_add_sync(0xffffffffu, bytes);
    if (threadIdx.x == 0) mbar_expect_tx(&bar, bytes);
    __syncwarp();
    for (int row = threadIdx.x; row < fs_rows_x(TT); row += 32)
      segments(row, [&](int src, int dst, int len) { bulk_g2s(xs + dst, X + src, (unsigned)len * 4u, &bar); });
  }
  {
    // L2 prefetch of the thread's own groups: rho and the coefficient fields
    // of its pass-1 rows, the update operands and fields of its pass-2 rows
    int gq;
    const int r0 = fdivmod((int)threadIdx.x, G, invG, gq);
    constexpr int rs = FS_TPB / G;
    if (r0 < rs) {
      const int gy = y0t + 4 * gq;
      for (int row = r0; row < fs_rows_y(TT); row += rs) {
        const int t = t0 - 1 + row / RYW;
        int x = x0 - 1 + row % RYW;
        if (t < 0 || t >= n0) continue;
        if (PER1) { if (x < 0) x += n1; else if (x >= n1) x -= n1; }
        else if (x < 0 || x >= n1) continue;
        const int q = t * pl + x * n2 + gy;
        pf_l2(rho + off + q);
        C.prefetch(q);
      }
      for (int row = r0; row < TT * FS_TX; row += rs) {
        const size_t j = off + (size_t)(t0 + row / FS_TX) * pl + (size_t)(x0 + row % FS_TX) * n2 + gy;
        if (MODE != SM_APPLY && MODE != SM_APPLYP) pf_l2(a.r + j);
        if (MODE == SM_POST0 || MODE == SM_CHEB || MODE == SM_CHEB_DOT) pf_l2(a.dinv + j);
        if ((MODE == SM_CHEB || MODE == SM_CHEB_DOT) && a.d) pf_l2(a.d + j);
      }
    }
  }
  float beta = 0.f;
  if (MODE == SM_APPLYP && a.d) {
    const double rz = a.rz_tot ? a.rz_tot[b] : sum_partials(a.rz, b, a.nrz), ro = a.rz_old[b];
    beta = cta_scalar([&] { return (ro > 0 && rz > 0) ? (float)(rz / ro) : 0.f; });
  }
  if (!mbar_wait(&bar, 0, FS_WAIT_LIMIT) && a.err) atomicExch(a.err, 1);
  if (MODE == SM_APPLYP) {
    // p = x + beta d on the staged operand (tile and halo), p on the tile to e
    constexpr int GW = W / 4;
    for (int i = threadIdx.x; i < fs_rows_x(TT) * GW; i += FS_TPB) {
      const int row = i / GW, c4 = i - (i / GW) * GW;
      const int rt = row / RXW, rx = row - (row / RXW) * RXW;
      const int t = t0 - 2 + rt;
      int x = x0 - 2 + rx, y = y0t - 4 + 4 * c4;
      if (t < 0 || t >= n0) continue;
      if (PER1) { x = x < 0 ? x + n1 : (x >= n1 ? x - n1 : x); }
      else if (x < 0 || x >= n1) continue;
      if (PER2) { y = y < 0 ? y + n2 : (y >= n2 ? y - n2 : y); }
      else if (y < 0 || y >= n2) continue;
      const size_t q = off + (size_t)t * pl + (size_t)x * n2 + y;
      float* sp = xs + row * W + 4 * c4;
      float4 v = lds4(sp);
      if (a.d) v = v + beta * ld4(a.d + q);
      *reinterpret_cast<float4*>(sp) = v;
      if (rt >= 2 && rt < TT + 2 && rx >= 2 && rx < FS_TX + 2 && c4 >= 1 && c4 <= G) *reinterpret_cast<float4*>(a.e + q) = v;
    }
    __syncthreads();
  }

  constexpr int rstride = FS_TPB / G;
  int gi;
  const int row0 = fdivmod((int)threadIdx.x, G, invG, gi);
  const bool active = row0 < rstride;
  const int y0 = 4 * gi;             // local y of the thread's group
  const int gy0 = y0t + y0;          // its global y
  const bool yin2 = PER2 || (gy0 >= 1 && gy0 + 4 <= n2 - 1);
  const bool yin3 = PER2 || (gy0 >= 3 && gy0 + 3 <= n2 - 4);
  const int yl = gy0 == 0 ? n2 - 1 : gy0 - 1, yr4 = gy0 + 4 == n2 ? 0 : gy0 + 4;   // global y-neighbours (wrapped)

  // (L x) along t and x at one shared column c of operand row xr (point at t, x)
  auto Ltx1 = [&](const float* xr, int c, int t, int x, int p) -> float {
    const float xc = xr[c];
    float acc = C.at(0, p) * xc;
    {
      const int cls = t == 0 ? 1 : (t == n0 - 1 ? 2 : 0);
      const float* up = xr + RXW * W;
      const float* dn = xr - RXW * W;
      const float xm1 = cls != 1 ? dn[c] : xc, xp1 = cls != 2 ? up[c] : xc;
      const float xm2 = cls == 2 ? dn[c - RXW * W] : xc, xp2 = cls == 1 ? up[c + RXW * W] : xc;
      float a1, a2;
      dforms1(cls, xm2, xm1, xc, xp1, xp2, a1, a2);
      acc += g.is1[0] * C.at(1, p) * a1 + i2t * C.at(2, p) * a2;
    }
    {
      const int cls = PER1 ? 0 : (x == 0 ? 1 : (x == n1 - 1 ? 2 : 0));
      const float xm1 = cls != 1 ? xr[c - W] : xc, xp1 = cls != 2 ? xr[c + W] : xc;
      const float xm2 = cls == 2 ? xr[c - 2 * W] : xc, xp2 = cls == 1 ? xr[c + 2 * W] : xc;
      float a1, a2;
      dforms1(cls, xm2, xm1, xc, xp1, xp2, a1, a2);
      acc += g.is1[1] * C.at(3, p) * a1 + i2x * C.at(4, p) * a2;
    }
    return acc;
  };

  // 2. y = -rho L x on rows t0-1 .. t0+TT x x0-1 .. x0+FS_TX, the tile's y range
  for (int row = active ? row0 : fs_rows_y(TT); row < fs_rows_y(TT); row += rstride) {
    const int st = row / RYW, sx = row % RYW;
    const int t = t0 - 1 + st;
    int x = x0 - 1 + sx;
    if (t < 0 || t >= n0) continue;
    if (PER1) { if (x < 0) x += n1; else if (x >= n1) x -= n1; }
    else if (x < 0 || x >= n1) continue;
    const int p = t * pl + x * n2 + gy0;
    const float4 r4 = ld4(rho + off + p);
    float4 cpt[7];
#pragma unroll
    for (int v = 0; v < 7; ++v) cpt[v] = MASK != FS_ANY ? C.at4(v, p) : f4(0.f);
    auto cat = [&](int v) { return MASK != FS_ANY ? cpt[v] : C.at4(v, p); };
    const float* xr = xs + ((st + 1) * RXW + sx + 1) * W + 4;   // column of y0t
    const float4 xc = lds4(xr + y0);
    float4 Lx = cat(0) * xc;
    if (t > 0 && t < n0 - 1 && (PER1 || (x > 0 && x < n1 - 1))) {
      const float4 tm = lds4(xr - RXW * W + y0), tp = lds4(xr + RXW * W + y0);
      const float4 xm = lds4(xr - W + y0), xp = lds4(xr + W + y0);
      Lx = Lx + (h1t * cat(1)) * (tp - tm) + (i2t * cat(2)) * (tp - 2.f * xc + tm) +
           (h1x * cat(3)) * (xp - xm) + (i2x * cat(4)) * (xp - 2.f * xc + xm);
    } else {
      float4 a1, a2;
      {
        const int cls = t == 0 ? 1 : (t == n0 - 1 ? 2 : 0);
        const float* up = xr + RXW * W;
        const float* dn = xr - RXW * W;
        float4 xm1 = cls != 1 ? lds4(dn + y0) : xc, xp1 = cls != 2 ? lds4(up + y0) : xc;
        float4 xm2 = cls == 2 ? lds4(dn - RXW * W + y0) : xc, xp2 = cls == 1 ? lds4(up + RXW * W + y0) : xc;
        dforms(cls, xm2, xm1, xc, xp1, xp2, a1, a2);
        Lx = Lx + (g.is1[0] * cat(1)) * a1 + (i2t * cat(2)) * a2;
      }
      {
        const int cls = PER1 ? 0 : (x == 0 ? 1 : (x == n1 - 1 ? 2 : 0));
        float4 xm1 = cls != 1 ? lds4(xr - W + y0) : xc, xp1 = cls != 2 ? lds4(xr + W + y0) : xc;
        float4 xm2 = cls == 2 ? lds4(xr - 2 * W + y0) : xc, xp2 = cls == 1 ? lds4(xr + 2 * W + y0) : xc;
        dforms(cls, xm2, xm1, xc, xp1, xp2, a1, a2);
        Lx = Lx + (g.is1[1] * cat(3)) * a1 + (i2x * cat(4)) * a2;
      }
    }
    if (yin2) {
      const float4 ym = make_float4(xr[y0 - 1], xc.x, xc.y, xc.z), yp = make_float4(xc.y, xc.z, xc.w, xr[y0 + 4]);
      Lx = Lx + (h1y * cat(5)) * (yp - ym) + (i2y * cat(6)) * (yp - 2.f * xc + ym);
    } else {
      float l4[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int yy = y0 + k, gy = gy0 + k;
        const int cls = gy == 0 ? 1 : (gy == n2 - 1 ? 2 : 0);
        const float v0 = xr[yy];
        const float vm1 = cls != 1 ? xr[yy - 1] : v0, vp1 = cls != 2 ? xr[yy + 1] : v0;
        const float vm2 = cls == 2 ? xr[yy - 2] : v0, vp2 = cls == 1 ? xr[yy + 2] : v0;
        float b1, b2;
        dforms1(cls, vm2, vm1, v0, vp1, vp2, b1, b2);
        l4[k] = g.is1[2] * C.at(5, p + k) * b1 + i2y * C.at(6, p + k) * b2;
      }
      Lx = Lx + make_float4(l4[0], l4[1], l4[2], l4[3]);
    }
    *reinterpret_cast<float4*>(ys + row * W + 4 + y0) = make_float4(-r4.x * Lx.x, -r4.y * Lx.y, -r4.z * Lx.z, -r4.w * Lx.w);
  }
  // the y-neighbours of the tile: one point on each side of every ring row
  // (central in y: a tile edge inside the domain is no grid edge)
  for (int i = threadIdx.x; i < 2 * fs_rows_y(TT); i += FS_TPB) {
    const int row = i >> 1, side = i & 1;
    const int st = row / RYW, sx = row % RYW;
    const int t = t0 - 1 + st;
    int x = x0 - 1 + sx;
    int gy = side ? y0t + TY : y0t - 1;
    if (t < 0 || t >= n0) continue;
    if (PER1) { if (x < 0) x += n1; else if (x >= n1) x -= n1; }
    else if (x < 0 || x >= n1) continue;
    if (PER2) gy = gy < 0 ? gy + n2 : (gy >= n2 ? gy - n2 : gy);
    else if (gy < 0 || gy >= n2) continue;
    const int c = side ? TY + 4 : 3;
    const int p = t * pl + x * n2 + gy;
    const float* xr = xs + ((st + 1) * RXW + sx + 1) * W;
    float Lx = Ltx1(xr, c, t, x, p);
    Lx += h1y * C.at(5, p) * (xr[c + 1] - xr[c - 1]) + i2y * C.at(6, p) * (xr[c + 1] - 2.f * xr[c] + xr[c - 1]);
    ys[row * W + c] = -__ldg(rho + off + p) * Lx;
  }
  __syncthreads();

  // 3. q = L^T y - theta 1_B x on the tile, then the update
  float acc = 0.f;
  for (int row = active ? row0 : TT * FS_TX; row < TT * FS_TX; row += rstride) {
    const int ot = row / FS_TX, ox = row % FS_TX;
    const int t = t0 + ot, x = x0 + ox;
    const int p = t * pl + x * n2 + gy0;
    const size_t j = off + p;
    float4 ur = make_float4(0.f, 0.f, 0.f, 0.f), udi = ur, ud = ur;
    if (MODE != SM_APPLY && MODE != SM_APPLYP) ur = ld4(a.r + j);
    if (MODE == SM_POST0 || MODE == SM_CHEB || MODE == SM_CHEB_DOT) udi = ld4(a.dinv + j);
    // previous iterate: the buffer this step overwrites at the same point,
    // so a coherent load (not the read-only path)
    if ((MODE == SM_CHEB || MODE == SM_CHEB_DOT) && a.d) ud = __ldcg(reinterpret_cast<const float4*>(a.d + j));
    const float* yr = ys + ((ot + 1) * RYW + ox + 1) * W + 4;
    const float4 yc = lds4(yr + y0);
    const int pxm = (PER1 && x == 0) ? p + (n1 - 1) * n2 : p - n2;
    const int pxp = (PER1 && x == n1 - 1) ? p - (n1 - 1) * n2 : p + n2;
    const bool tcen = t >= 3 && t <= n0 - 4, xcen = PER1 || (x >= 3 && x <= n1 - 4);
    float4 k0, k1m, k1p, k2, k2m, k2p, k3m, k3p, k4, k4m, k4p, k5, k6;
    float c5l, c5r, c6l, c6r;
    if (MASK != FS_ANY) {
      const int ptm = tcen ? p - pl : p, ptp = tcen ? p + pl : p;
      const int qxm = xcen ? pxm : p, qxp = xcen ? pxp : p;
      const int prow = p - gy0;
      k0 = C.at4(0, p); k2 = C.at4(2, p); k4 = C.at4(4, p); k5 = C.at4(5, p); k6 = C.at4(6, p);
      k1m = C.at4(1, ptm); k1p = C.at4(1, ptp); k2m = C.at4(2, ptm); k2p = C.at4(2, ptp);
      k3m = C.at4(3, qxm); k3p = C.at4(3, qxp); k4m = C.at4(4, qxm); k4p = C.at4(4, qxp);
      c5l = C.at(5, prow + yl); c5r = C.at(5, prow + yr4); c6l = C.at(6, prow + yl); c6r = C.at(6, prow + yr4);
    }
    auto pick = [&](const float4& pre, int v, int q) { return MASK != FS_ANY ? pre : C.at4(v, q); };
    auto pickf = [&](float pre, int v, int q) { return MASK != FS_ANY ? pre : C.at(v, q); };
    float4 qv = pick(k0, 0, p) * yc;
    if (tcen && xcen) {
      const float4 tm = lds4(yr - RYW * W + y0), tp = lds4(yr + RYW * W + y0);
      const float4 xm = lds4(yr - W + y0), xp = lds4(yr + W + y0);
      const float4 c2t = pick(k2, 2, p), c2x = pick(k4, 4, p);
      qv = qv + h1t * (pick(k1m, 1, p - pl) * tm - pick(k1p, 1, p + pl) * tp) +
           i2t * (pick(k2m, 2, p - pl) * tm - 2.f * (c2t * yc) + pick(k2p, 2, p + pl) * tp) +
           h1x * (pick(k3m, 3, pxm) * xm - pick(k3p, 3, pxp) * xp) +
           i2x * (pick(k4m, 4, pxm) * xm - 2.f * (c2x * yc) + pick(k4p, 4, pxp) * xp);
    } else {
      if (tcen) {
        const float4 ym = lds4(yr - RYW * W + y0), yp = lds4(yr + RYW * W + y0);
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
          const float4 yv = o == 0 ? yc : lds4(yr - o * RYW * W + y0);
          qv = qv + yv * ((w1 * g.is1[0]) * C.at4(1, pi) + (w2 * i2t) * C.at4(2, pi));
        }
      }
      if (xcen) {
        const float4 ym = lds4(yr - W + y0), yp = lds4(yr + W + y0);
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
          const float4 yv = o == 0 ? yc : lds4(yr - o * W + y0);
          qv = qv + yv * ((w1 * g.is1[1]) * C.at4(3, pi) + (w2 * i2x) * C.at4(4, pi));
        }
      }
    }
    if (yin3) {
      const int prow = p - gy0;
      const float4 c1 = pick(k5, 5, p), c2 = pick(k6, 6, p);
      const float c1l = pickf(c5l, 5, prow + yl), c1r = pickf(c5r, 5, prow + yr4), c2l = pickf(c6l, 6, prow + yl), c2r = pickf(c6r, 6, prow + yr4);
      const float4 ym = make_float4(yr[y0 - 1], yc.x, yc.y, yc.z), yp = make_float4(yc.y, yc.z, yc.w, yr[y0 + 4]);
      const float4 c1m = make_float4(c1l, c1.x, c1.y, c1.z), c1p = make_float4(c1.y, c1.z, c1.w, c1r);
      const float4 c2m = make_float4(c2l, c2.x, c2.y, c2.z), c2p = make_float4(c2.y, c2.z, c2.w, c2r);
      qv = qv + h1y * (c1m * ym - c1p * yp) + i2y * (c2m * ym - 2.f * (c2 * yc) + c2p * yp);
    } else {
      float q4[4] = {0.f, 0.f, 0.f, 0.f};
      const int prow = p - gy0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int gy = gy0 + k;
#pragma unroll
        for (int o = -2; o <= 2; ++o) {
          const int iy = gy - o;
          if (iy < 0 || iy >= n2) continue;
          const float w1 = dweight(1, iy, n2, 0, o), w2 = dweight(2, iy, n2, 0, o);
          if (w1 == 0.f && w2 == 0.f) continue;
          q4[k] += yr[iy - y0t] * (w1 * g.is1[2] * C.at(5, prow + iy) + w2 * i2y * C.at(6, prow + iy));
        }
      }
      qv = qv + make_float4(q4[0], q4[1], q4[2], q4[3]);
    }
    const float4 xj = lds4(xs + ((ot + 2) * RXW + ox + 2) * W + 4 + y0);
    const bool bnd_tx = t == 0 || (g.final_rows && t == n0 - 1) || (!PER1 && (x == 0 || x == n1 - 1));
    if (bnd_tx) {
      qv = qv - g.theta * xj;
    } else if (!PER2) {
      if (gy0 == 0) qv.x -= g.theta * xj.x;
      if (gy0 + 3 == n2 - 1) qv.w -= g.theta * xj.w;
    }
    if (MODE == SM_APPLY || MODE == SM_APPLYP) {
      *reinterpret_cast<float4*>(a.out + j) = make_float4(-qv.x, -qv.y, -qv.z, -qv.w);
      acc -= qv.x * xj.x + qv.y * xj.y + qv.z * xj.z + qv.w * xj.w;
    } else if (MODE == SM_RES) {
      *reinterpret_cast<float4*>(a.out + j) = ur + qv;
    } else {
      const float4 res = ur + qv;
      float4 dn = a.c2 * (udi * res);
      if (MODE == SM_CHEB || MODE == SM_CHEB_DOT) dn = dn + a.c1 * (xj - ud);
      const float4 en = xj + dn;
      *reinterpret_cast<float4*>(a.e + j) = en;
      if (MODE == SM_CHEB_DOT) acc += en.x * ur.x + en.y * ur.y + en.z * ur.z + en.w * ur.w;
    }
  }
  if ((MODE == SM_APPLY || MODE == SM_APPLYP || MODE == SM_CHEB_DOT) && a.part) {
    const double s = block_sum((double)acc);
    partial_finish(s, a.part, a.cnt, a.tot, b, blockIdx.x, gridDim.x);
  }
}
