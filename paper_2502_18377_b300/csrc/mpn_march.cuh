// One operator step (D = 3, float4 along y) in one kernel that marches along
// t through a pipeline of shared-memory plane slots: the variant of k_step3y
// for levels whose x and y are periodic, with uniform steps and a
// compile-time coefficient layout whose time coefficients c_t, c_tt are
// per-instance scalars (the transport layout, and reaction-diffusion with
// c_xx = c_yy one field).
//
// A CTA owns a column of MS_X x-rows x MS_Y y points of one instance over the
// time planes [t0, t1) (the whole time extent, or a chunk of it).  For each
// plane t in order:
//   A. y = -rho L x on plane t+1, on the column plus a ring of one x-row and
//      one y point on each side, into a ring of y planes in shared memory;
//   B. one CTA barrier;
//   C. q = L^T y - theta 1_B x = -(S x) on plane t of the column, then the
//      mode's update (as k_step3y), written to global memory.
// The rows of L that reach plane t lie on planes t-1 .. t+1, and on plane 0
// (t = 2) or n0-1 (t = n0-3) through the one-sided forms of the first and last
// plane; so y(t0-1) and y(t0) are computed before the loop, and y(n0-1)
// together with y(n0-2).
//
// The operand (x-halo 2), the coefficient fields and rho (x-halo 1), each with
// a y halo of one float4 group, stream plane by plane into ring slots by
// 16-byte asynchronous copies (cp.async, one commit group per plane step,
// issued by every thread right after the barrier that frees the slots, two
// plane steps ahead of their first use; no registers are held while they are
// in flight).  Warps 0-7 read the right-hand side, the Chebyshev diagonal and
// the previous iterate of their own point one plane ahead into registers.
// Shared memory: 111.7 KB, two CTAs per SM; two CTA barriers per plane.
#pragma once
#include "mpn_fused.cuh"

#define MS_X 16                 // x rows of a column
#define MS_Y 64                 // y points of a column
#define MS_W (MS_Y + 8)         // shared row: column c holds y = y0 - 4 + c
#define MS_TPB 288              // 9 warps: all run pass A; warps 0-7 pass C, warp 8 issues copies
#define MS_CT 256               // threads of pass C
#define MS_NX 5                 // operand plane slots
#define MS_NF 4                 // field plane slots (two fields each)
#define MS_NR 3                 // rho plane slots
#define MS_NY 5                 // y plane slots
#define MS_XR (MS_X + 4)        // operand rows of a plane
#define MS_RR (MS_X + 2)        // ring rows of a plane
#define MS_MIN_TC 8             // fewest planes of a chunk

__host__ __device__ constexpr int ms_floats() {
  return (MS_NX * MS_XR + (2 * MS_NF + MS_NR + MS_NY) * MS_RR) * MS_W;
}

// Field slot (0, 1) of c_v in the layout, or -1 for a per-instance scalar.
template <int MASK>
__host__ __device__ constexpr int ms_slot(int v) {
  return MASK == FS_MASK_TR ? (v == 3 ? 0 : (v == 5 ? 1 : -1)) : (v == 0 ? 0 : ((v == 4 || v == 6) ? 1 : -1));
}
// Variable whose field is in slot k.
template <int MASK>
__host__ __device__ constexpr int ms_var(int k) {
  return MASK == FS_MASK_TR ? (k == 0 ? 3 : 5) : (k == 0 ? 0 : 4);
}

__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int MODE, int MASK>
__global__ void __launch_bounds__(MS_TPB, 2) k_march(Grid g, Coef cf, const float* __restrict__ rho, StepArgs a, int tc) {
  static_assert(MASK == FS_MASK_TR || MASK == FS_MASK_RDI, "layouts with scalar time coefficients only");
  extern __shared__ __align__(16) float msm[];
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const int pl = n1 * n2;
  const int b = blockIdx.y;
  const int nyt = n2 / MS_Y, ncol = (n1 / MS_X) * nyt;
  const int chunk = blockIdx.x / ncol, col = blockIdx.x - chunk * ncol;
  const int x0 = (col / nyt) * MS_X, y0 = (col - (col / nyt) * nyt) * MS_Y;
  const int t0 = chunk * tc, t1 = min(t0 + tc, n0);
  const size_t off = (size_t)b * g.N;
  const int tid = threadIdx.x;

  float* xs = msm;
  float* fs = xs + MS_NX * MS_XR * MS_W;
  float* rs = fs + MS_NF * 2 * MS_RR * MS_W;
  float* ys = rs + MS_NR * MS_RR * MS_W;
  // planes streamed: operand xlo..xhi, fields and rho flo..fhi (y planes too)
  const int xlo = max(t0 - 2, 0), xhi = min(t1 + 1, n0 - 1);
  const int flo = max(t0 - 1, 0), fhi = min(t1, n0 - 1);
  auto xslot = [&](int t) { return xs + ((t - xlo) % MS_NX) * (MS_XR * MS_W); };
  auto fslot = [&](int t) { return fs + ((t - flo) % MS_NF) * (2 * MS_RR * MS_W); };
  auto rslot = [&](int t) { return rs + ((t - flo) % MS_NR) * (MS_RR * MS_W); };

  const float* X = a.x + off;
  const float* R = rho + off;
  const float* F0 = cf.ptr[ms_var<MASK>(0)] + (size_t)b * cf.bstride[ms_var<MASK>(0)];
  const float* F1 = cf.ptr[ms_var<MASK>(1)] + (size_t)b * cf.bstride[ms_var<MASK>(1)];
  float sv[7];
#pragma unroll
  for (int v = 0; v < 7; ++v) sv[v] = ms_slot<MASK>(v) < 0 ? __ldg(cf.ptr[v] + (size_t)b * cf.bstride[v]) : 0.f;
  const float is1t = g.is1[0], i2t = g.is2[0];
  const float h1x = 0.5f * g.is1[1], h1y = 0.5f * g.is1[2], i2x = g.is2[1], i2y = g.is2[2];

  // copies: each thread moves the same float4 groups of every plane, at
  // offsets within a plane (x and y wrapped) and within a slot computed once:
  // operand groups k = tid, tid + MS_TPB of MS_XR x MS_W / 4, ring groups
  // (fields, rho) k = tid, tid + MS_TPB of MS_RR x MS_W / 4
  constexpr int GW = MS_W / 4, NGX = MS_XR * GW, NGR = MS_RR * GW;
  static_assert(NGX <= 2 * MS_TPB && NGR <= 2 * MS_TPB && NGR >= MS_TPB, "two copy groups per thread");
  auto goff = [&](int k, int xh, int& so) {
    const int r = k / GW, c4 = k - (k / GW) * GW;
    int x = x0 - xh + r;
    x = x < 0 ? x + n1 : (x >= n1 ? x - n1 : x);
    int y = y0 - 4 + 4 * c4;
    y = y < 0 ? y + n2 : (y >= n2 ? y - n2 : y);
    so = r * MS_W + 4 * c4;
    return x * n2 + y;
  };
  int sx0, sx1 = 0, sr0, sr1 = 0;
  const int gx0 = goff(tid, 2, sx0), gx1 = tid + MS_TPB < NGX ? goff(tid + MS_TPB, 2, sx1) : -1;
  const int gr0 = goff(tid, 1, sr0), gr1 = tid + MS_TPB < NGR ? goff(tid + MS_TPB, 1, sr1) : -1;
  int nx = xlo, nf = flo, nr = flo;   // next planes to copy
  // copies of the planes below the given limits (into slots freed by the
  // preceding barrier), as one commit group
  auto refill = [&](int xlim, int flim, int rlim) {
    for (; nx <= xhi && nx < xlim; ++nx) {
      float* d = xslot(nx);
      const float* src = X + (size_t)nx * pl;
      cp_async16(d + sx0, src + gx0);
      if (gx1 >= 0) cp_async16(d + sx1, src + gx1);
    }
    for (; nf <= fhi && nf < flim; ++nf) {
      float* d = fslot(nf);
      const float* s0 = F0 + (size_t)nf * pl;
      const float* s1 = F1 + (size_t)nf * pl;
      cp_async16(d + sr0, s0 + gr0);
      cp_async16(d + MS_RR * MS_W + sr0, s1 + gr0);
      if (gr1 >= 0) {
        cp_async16(d + sr1, s0 + gr1);
        cp_async16(d + MS_RR * MS_W + sr1, s1 + gr1);
      }
    }
    for (; nr <= fhi && nr < rlim; ++nr) {
      float* d = rslot(nr);
      const float* src = R + (size_t)nr * pl;
      cp_async16(d + sr0, src + gr0);
      if (gr1 >= 0) cp_async16(d + sr1, src + gr1);
    }
    cp_async_commit();
  };

  // coefficient c_v of plane slot fsl at shared row rr, column c
  auto cq = [&](int v, const float* fsl, int rr, int c) -> float4 {
    return ms_slot<MASK>(v) < 0 ? f4(sv[v]) : lds4(fsl + ms_slot<MASK>(v) * (MS_RR * MS_W) + rr * MS_W + c);
  };
  auto cs = [&](int v, const float* fsl, int rr, int c) -> float {
    return ms_slot<MASK>(v) < 0 ? sv[v] : fsl[ms_slot<MASK>(v) * (MS_RR * MS_W) + rr * MS_W + c];
  };

  // slot of plane t + k from the slot i of plane t (|k| small)
  auto wr = [](int i, int S) { return i >= S ? i - S : (i < 0 ? i + S : i); };
  // A. y = -rho L x on plane tp = t + k, with ix, jf, jr, jy the slots of
  //    plane t: the thread's float4 group of ring row tid / 16, then (threads
  //    0-35) one y-neighbour point of a ring row
  auto passA = [&](int tp, int k, int ix, int jf, int jr, int jy) {
    const int cls = tp == 0 ? 1 : (tp == n0 - 1 ? 2 : 0);
    const float* xpl = xs + wr(ix + k, MS_NX) * (MS_XR * MS_W);
    const float* xm1 = cls != 1 ? xs + wr(ix + k - 1, MS_NX) * (MS_XR * MS_W) : xpl;
    const float* xp1 = cls != 2 ? xs + wr(ix + k + 1, MS_NX) * (MS_XR * MS_W) : xpl;
    const float* xm2 = cls == 2 ? xs + wr(ix + k - 2, MS_NX) * (MS_XR * MS_W) : xpl;
    const float* xp2 = cls == 1 ? xs + wr(ix + k + 2, MS_NX) * (MS_XR * MS_W) : xpl;
    const float* fsl = fs + wr(jf + k, MS_NF) * (2 * MS_RR * MS_W);
    const float* rsl = rs + wr(jr + k, MS_NR) * (MS_RR * MS_W);
    float* yo = ys + wr(jy + k, MS_NY) * (MS_RR * MS_W);
    {
      const int rr = tid >> 4, c = 4 + 4 * (tid & 15);
      const int o = (rr + 1) * MS_W + c;
      const float4 xc = lds4(xpl + o);
      float4 a1, a2;
      dforms(cls, cls == 2 ? lds4(xm2 + o) : xc, cls != 1 ? lds4(xm1 + o) : xc, xc, cls != 2 ? lds4(xp1 + o) : xc,
             cls == 1 ? lds4(xp2 + o) : xc, a1, a2);
      float4 Lx = cq(0, fsl, rr, c) * xc + (is1t * sv[1]) * a1 + (i2t * sv[2]) * a2;
      const float4 xm = lds4(xpl + o - MS_W), xp = lds4(xpl + o + MS_W);
      Lx = Lx + (h1x * cq(3, fsl, rr, c)) * (xp - xm) + (i2x * cq(4, fsl, rr, c)) * (xp - 2.f * xc + xm);
      const float4 ym = make_float4(xpl[o - 1], xc.x, xc.y, xc.z), yp = make_float4(xc.y, xc.z, xc.w, xpl[o + 4]);
      Lx = Lx + (h1y * cq(5, fsl, rr, c)) * (yp - ym) + (i2y * cq(6, fsl, rr, c)) * (yp - 2.f * xc + ym);
      const float4 r4 = lds4(rsl + rr * MS_W + c);
      *reinterpret_cast<float4*>(yo + rr * MS_W + c) = make_float4(-r4.x * Lx.x, -r4.y * Lx.y, -r4.z * Lx.z, -r4.w * Lx.w);
    }
    if (tid < 2 * MS_RR) {
      const int rr = tid >> 1, c = (tid & 1) ? MS_Y + 4 : 3;
      const int o = (rr + 1) * MS_W + c;
      const float xc = xpl[o];
      float a1, a2;
      dforms1(cls, cls == 2 ? xm2[o] : xc, cls != 1 ? xm1[o] : xc, xc, cls != 2 ? xp1[o] : xc, cls == 1 ? xp2[o] : xc,
              a1, a2);
      float Lx = cs(0, fsl, rr, c) * xc + (is1t * sv[1]) * a1 + (i2t * sv[2]) * a2;
      const float xm = xpl[o - MS_W], xp = xpl[o + MS_W];
      Lx += (h1x * cs(3, fsl, rr, c)) * (xp - xm) + (i2x * cs(4, fsl, rr, c)) * (xp - 2.f * xc + xm);
      const float ym = xpl[o - 1], yp = xpl[o + 1];
      Lx += (h1y * cs(5, fsl, rr, c)) * (yp - ym) + (i2y * cs(6, fsl, rr, c)) * (yp - 2.f * xc + ym);
      yo[rr * MS_W + c] = -rsl[rr * MS_W + c] * Lx;
    }
  };

  // pass C point of this thread (warps 0-7)
  const bool cthr = tid < MS_CT;
  const int crow = (tid >> 4) & 15, cc = 4 + 4 * (tid & 15);
  const size_t pbase = off + (size_t)(x0 + crow) * n2 + (y0 + cc - 4);
  auto load_pt = [&](int t, float4& r4, float4& di4, float4& d4) {
    const size_t j = pbase + (size_t)t * pl;
    if (MODE != SM_APPLY) r4 = ld4(a.r + j);
    if (MODE == SM_POST0 || MODE == SM_CHEB || MODE == SM_CHEB_DOT) di4 = ld4(a.dinv + j);
    // previous iterate: a buffer this kernel overwrites (at other planes of
    // the thread's own points), so a coherent load
    if ((MODE == SM_CHEB || MODE == SM_CHEB_DOT) && a.d) d4 = __ldcg(reinterpret_cast<const float4*>(a.d + j));
  };
  auto prefetch_pt = [&](int t) {
    const size_t j = pbase + (size_t)t * pl;
    if (MODE != SM_APPLY) pf_l2(a.r + j);
    if (MODE == SM_POST0 || MODE == SM_CHEB || MODE == SM_CHEB_DOT) pf_l2(a.dinv + j);
    if ((MODE == SM_CHEB || MODE == SM_CHEB_DOT) && a.d) pf_l2(a.d + j);
  };

  // prologue: the first slots' planes, then y on the plane before t0 and on t0
  refill(xlo + MS_NX, flo + MS_NF, flo + MS_NR);
  float4 cr = f4(0.f), cdi = f4(0.f), cd = f4(0.f);
  if (cthr) {
    load_pt(t0, cr, cdi, cd);
    if ((tid & 7) == 0 && t0 + 1 < t1) prefetch_pt(t0 + 1);
  }
  cp_async_wait<0>();
  __syncthreads();
  {
    const int ix = (t0 - xlo) % MS_NX, jf = (t0 - flo) % MS_NF, jr = (t0 - flo) % MS_NR, jy = (t0 - flo) % MS_NY;
    for (int tp = flo; tp <= t0; ++tp) passA(tp, tp - t0, ix, jf, jr, jy);
  }

  double accd = 0.0;
  for (int t = t0; t < t1; ++t) {
    // the copies that plane t's passes read have landed (this thread's),
    // then one barrier makes every thread's visible and frees the slots of
    // the planes no later pass reads
    if (t <= t0 + 1 || t == n0 - 3) cp_async_wait<0>();
    else cp_async_wait<1>();
    __syncthreads();
    refill(t + MS_NX, t + MS_NF, t + 1 + MS_NR);
    float4 nr4 = f4(0.f), ndi4 = f4(0.f), nd4 = f4(0.f);
    if (cthr) {
      if (t + 1 < t1) load_pt(t + 1, nr4, ndi4, nd4);
      if ((tid & 7) == 0 && t + 2 < t1) prefetch_pt(t + 2);
    }
    const int ix = (t - xlo) % MS_NX, jf = (t - flo) % MS_NF, jr = (t - flo) % MS_NR, jy = (t - flo) % MS_NY;
    // A: y(t+1) (and y(n0-1) with y(n0-2))
    if (t + 1 <= n0 - 1 && t != n0 - 2) passA(t + 1, 1, ix, jf, jr, jy);
    if (t == n0 - 3) passA(n0 - 1, 2, ix, jf, jr, jy);
    __syncthreads();
    if (!cthr) continue;
    // C. q = L^T y - theta 1_B x on plane t
    auto yrow = [&](int k) { return ys + wr(jy + k, MS_NY) * (MS_RR * MS_W) + (crow + 1) * MS_W; };
    const float* fsl = fs + jf * (2 * MS_RR * MS_W);
    const float* yr = yrow(0);
    const float4 yc = lds4(yr + cc);
    float4 qv = cq(0, fsl, crow + 1, cc) * yc;
    if (t >= 3 && t <= n0 - 4) {
      const float4 tm = lds4(yrow(-1) + cc), tp = lds4(yrow(1) + cc);
      qv = qv + (0.5f * is1t * sv[1]) * (tm - tp) + (i2t * sv[2]) * (tm - 2.f * yc + tp);
    } else {
#pragma unroll
      for (int o = -2; o <= 2; ++o) {
        const int ip = t - o;
        if (ip < 0 || ip >= n0) continue;
        const float w1 = dweight(1, ip, n0, 0, o), w2 = dweight(2, ip, n0, 0, o);
        if (w1 == 0.f && w2 == 0.f) continue;
        const float4 yv = o == 0 ? yc : lds4(yrow(-o) + cc);
        qv = qv + ((w1 * is1t) * sv[1] + (w2 * i2t) * sv[2]) * yv;
      }
    }
    {
      const float4 ym = lds4(yr - MS_W + cc), yp = lds4(yr + MS_W + cc);
      qv = qv + h1x * (cq(3, fsl, crow, cc) * ym - cq(3, fsl, crow + 2, cc) * yp) +
           i2x * (cq(4, fsl, crow, cc) * ym - 2.f * (cq(4, fsl, crow + 1, cc) * yc) + cq(4, fsl, crow + 2, cc) * yp);
    }
    {
      const int rr = crow + 1;
      const float4 c1 = cq(5, fsl, rr, cc), c2 = cq(6, fsl, rr, cc);
      const float c1l = cs(5, fsl, rr, cc - 1), c1r = cs(5, fsl, rr, cc + 4);
      const float c2l = cs(6, fsl, rr, cc - 1), c2r = cs(6, fsl, rr, cc + 4);
      const float4 ym = make_float4(yr[cc - 1], yc.x, yc.y, yc.z), yp = make_float4(yc.y, yc.z, yc.w, yr[cc + 4]);
      const float4 c1m = make_float4(c1l, c1.x, c1.y, c1.z), c1p = make_float4(c1.y, c1.z, c1.w, c1r);
      const float4 c2m = make_float4(c2l, c2.x, c2.y, c2.z), c2p = make_float4(c2.y, c2.z, c2.w, c2r);
      qv = qv + h1y * (c1m * ym - c1p * yp) + i2y * (c2m * ym - 2.f * (c2 * yc) + c2p * yp);
    }
    const float4 xj = lds4(xs + ix * (MS_XR * MS_W) + (crow + 2) * MS_W + cc);
    if (t == 0 || (g.final_rows && t == n0 - 1)) qv = qv - g.theta * xj;
    const size_t j = pbase + (size_t)t * pl;
    float acc = 0.f;
    if (MODE == SM_APPLY) {
      *reinterpret_cast<float4*>(a.out + j) = make_float4(-qv.x, -qv.y, -qv.z, -qv.w);
      acc = -(qv.x * xj.x + qv.y * xj.y + qv.z * xj.z + qv.w * xj.w);
    } else if (MODE == SM_RES) {
      *reinterpret_cast<float4*>(a.out + j) = cr + qv;
    } else {
      const float4 res = cr + qv;
      float4 dn = a.c2 * (cdi * res);
      if (MODE == SM_CHEB || MODE == SM_CHEB_DOT) dn = dn + a.c1 * (xj - cd);
      const float4 en = xj + dn;
      *reinterpret_cast<float4*>(a.e + j) = en;
      if (MODE == SM_CHEB_DOT) acc = en.x * cr.x + en.y * cr.y + en.z * cr.z + en.w * cr.w;
    }
    if (MODE == SM_APPLY || MODE == SM_CHEB_DOT) accd += (double)acc;
    cr = nr4; cdi = ndi4; cd = nd4;
  }
  cp_async_wait<0>();
  if ((MODE == SM_APPLY || MODE == SM_CHEB_DOT) && a.part) {
    const double s = block_sum(accd);
    partial_finish(s, a.part, a.cnt, a.tot, b, blockIdx.x, gridDim.x);
  }
}
