// One operator step (D = 3, float4 along y) in one kernel that marches along
// t through a pipeline of shared-memory plane slots: the variant of k_step3y
// for levels whose x and y are periodic, with uniform steps and a
// compile-time coefficient layout whose time coefficients c_t, c_tt are
// per-instance scalars (the transport layout, and reaction-diffusion with
// c_xx = c_yy one field).
//
// A CTA owns a column of MX x-rows x MS_Y y points of one instance over the
// time planes [t0, t1) (the whole time extent, or a chunk of it).  For each
// plane t in order:
//   A. y = -rho L x on plane t+1, on the column plus a ring of one x-row and
//      one y point on each side, into a ring of y planes in shared memory;
//   B. one CTA barrier (then the next planes' copies are issued);
//   C. q = L^T y - theta 1_B x = -(S x) on plane t of the column, then the
//      mode's update (as k_step3y), written to global memory.
// The rows of L that reach plane t lie on planes t-1 .. t+1, and on plane 0
// (t = 2) or n0-1 (t = n0-3) through the one-sided forms of the first and last
// plane; so y(t0-1) and y(t0) are computed before the loop, and y(n0-1)
// together with y(n0-2).
//
// The operand (x-halo 2), the coefficient fields and rho (x-halo 1), each with
// a y halo of one float4 group, stream plane by plane into ring slots by
// 16-byte asynchronous copies (cp.async; each thread copies the same groups of
// every plane, at offsets computed once), one commit group per plane step,
// issued right after the step's barrier into the slots it freed and waited
// for before the next step's barrier; no registers are held while they are
// in flight.  One CTA barrier per plane publishes both the landed copies and
// the y plane of pass A.  The threads of pass C read the right-hand side, the
// Chebyshev diagonal and the previous iterate of their own point one plane
// ahead into registers, before the step's pass A.  Shared memory: 111.7 KB (16 rows, two CTAs per SM)
// or 61.9 KB (8 rows, three).
#pragma once
#include "mpn_fused.cuh"

// Columns of MX = 16 or 8 x-rows (CTAs of (MX + 2) x 16 threads: all run
// pass A, the first MX x 16 pass C; two CTAs per SM with 16 rows, three
// with 8).
#define MS_Y 64                 // y points of a column
#define MS_W (MS_Y + 8)         // shared row: column c holds y = y0 - 4 + c
#define MS_NX 5                 // operand plane slots
#define MS_NF 4                 // field plane slots (two fields each)
#define MS_NR 3                 // rho plane slots
#define MS_NY 5                 // y plane slots
#define MS_MIN_TC 8             // fewest planes of a chunk

__host__ __device__ constexpr int ms_tpb(int MX) { return (MX + 2) * (MS_Y / 4); }
__host__ __device__ constexpr int ms_ctas_per_sm(int MX) { return MX == 16 ? 2 : 3; }
__host__ __device__ constexpr int ms_floats(int MX) {
  return (MS_NX * (MX + 4) + (2 * MS_NF + MS_NR + MS_NY) * (MX + 2)) * MS_W;
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

template <int MODE, int MASK, int MX>
__global__ void __launch_bounds__(ms_tpb(MX), ms_ctas_per_sm(MX))
    k_march(Grid g, Coef cf, const float* __restrict__ rho, StepArgs a, int tc) {
  static_assert(MASK == FS_MASK_TR || MASK == FS_MASK_RDI, "layouts with scalar time coefficients only");
  static_assert(MX == 16 || MX == 8, "columns of 16 or 8 x-rows");
  constexpr int XR = MX + 4, RR = MX + 2, TPB = ms_tpb(MX), CT = MX * (MS_Y / 4);
  // slot sizes and region offsets in shared memory (floats)
  constexpr int SX = XR * MS_W, SF = 2 * RR * MS_W, SR = RR * MS_W, SY = RR * MS_W;
  constexpr int OX = 0, OF = OX + MS_NX * SX, OR = OF + MS_NF * SF, OY = OR + MS_NR * SR;
  extern __shared__ __align__(16) float msm[];
  auto L4 = [&](int o) { return *reinterpret_cast<const float4*>(&msm[o]); };
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const int pl = n1 * n2;
  const int b = blockIdx.y;
  const int nyt = n2 / MS_Y, ncol = (n1 / MX) * nyt;
  const int chunk = blockIdx.x / ncol, col = blockIdx.x - chunk * ncol;
  const int x0 = (col / nyt) * MX, y0 = (col - (col / nyt) * nyt) * MS_Y;
  const int t0 = chunk * tc, t1 = min(t0 + tc, n0);
  const size_t off = (size_t)b * g.N;
  const int tid = threadIdx.x;

  // planes streamed: operand xlo..xhi, fields and rho flo..fhi (y planes
  // too); plane p of a stream sits in slot (p - lo) mod (slots)
  const int xlo = max(t0 - 2, 0), xhi = min(t1 + 1, n0 - 1);
  const int flo = max(t0 - 1, 0), fhi = min(t1, n0 - 1);
  auto xslot = [&](int t) { return OX + ((t - xlo) % MS_NX) * SX; };
  auto fslot = [&](int t) { return OF + ((t - flo) % MS_NF) * SF; };
  auto rslot = [&](int t) { return OR + ((t - flo) % MS_NR) * SR; };
  auto yslot = [&](int t) { return OY + ((t - flo) % MS_NY) * SY; };

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
  // operand groups k = tid, tid + TPB of XR x MS_W / 4, ring groups (fields,
  // rho) k = tid, tid + TPB of RR x MS_W / 4
  constexpr int GW = MS_W / 4, NGX = XR * GW, NGR = RR * GW;
  static_assert(NGX <= 2 * TPB && NGR <= 2 * TPB && NGR >= TPB, "two copy groups per thread");
  static_assert(TPB == RR * 16, "one pass-A group per thread");
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
  const int gx0 = goff(tid, 2, sx0), gx1 = tid + TPB < NGX ? goff(tid + TPB, 2, sx1) : -1;
  const int gr0 = goff(tid, 1, sr0), gr1 = tid + TPB < NGR ? goff(tid + TPB, 1, sr1) : -1;
  int nx = xlo, nf = flo, nr = flo;   // next planes to copy
  // copies of the planes below the given limits (into slots freed by the
  // preceding barrier), as one commit group
  auto refill = [&](int xlim, int flim, int rlim) {
    for (; nx <= xhi && nx < xlim; ++nx) {
      float* d = msm + xslot(nx);
      const float* src = X + (size_t)nx * pl;
      cp_async16(d + sx0, src + gx0);
      if (gx1 >= 0) cp_async16(d + sx1, src + gx1);
    }
    for (; nf <= fhi && nf < flim; ++nf) {
      float* d = msm + fslot(nf);
      const float* s0 = F0 + (size_t)nf * pl;
      const float* s1 = F1 + (size_t)nf * pl;
      cp_async16(d + sr0, s0 + gr0);
      cp_async16(d + RR * MS_W + sr0, s1 + gr0);
      if (gr1 >= 0) {
        cp_async16(d + sr1, s0 + gr1);
        cp_async16(d + RR * MS_W + sr1, s1 + gr1);
      }
    }
    for (; nr <= fhi && nr < rlim; ++nr) {
      float* d = msm + rslot(nr);
      const float* src = R + (size_t)nr * pl;
      cp_async16(d + sr0, src + gr0);
      if (gr1 >= 0) cp_async16(d + sr1, src + gr1);
    }
    cp_async_commit();
  };

  // coefficient c_v of the field slot at offset fo, ring row rr, column c
  auto cq = [&](int v, int fo, int rr, int c) -> float4 {
    return ms_slot<MASK>(v) < 0 ? f4(sv[v]) : L4(fo + ms_slot<MASK>(v) * (RR * MS_W) + rr * MS_W + c);
  };
  auto cs = [&](int v, int fo, int rr, int c) -> float {
    return ms_slot<MASK>(v) < 0 ? sv[v] : msm[fo + ms_slot<MASK>(v) * (RR * MS_W) + rr * MS_W + c];
  };

  // A. y = -rho L x on plane tp (class cls: 0 inside, 1 first, 2 last plane)
  //    from the operand slots of planes tp-2 .. tp+2 (xm2 .. xp2; those a
  //    class does not use may be anything), the field and rho slots of tp,
  //    into the y slot yo: the thread's float4 group of ring row tid / 16,
  //    then (threads 0 .. 2 RR - 1) one y-neighbour point of a ring row
  const int arow = tid >> 4, acol = 4 + 4 * (tid & 15);
  auto passA = [&](int cls, int xm2, int xm1, int xpl, int xp1, int xp2, int fo, int ro, int yo) {
    {
      const int o = (arow + 1) * MS_W + acol;
      const float4 xc = L4(xpl + o);
      float4 a1, a2;
      if (cls == 0) {
        const float4 tm = L4(xm1 + o), tq = L4(xp1 + o);
        a1 = 0.5f * (tq - tm);
        a2 = tq - 2.f * xc + tm;
      } else {
        dforms(cls, cls == 2 ? L4(xm2 + o) : xc, cls == 2 ? L4(xm1 + o) : xc, xc, cls == 1 ? L4(xp1 + o) : xc,
               cls == 1 ? L4(xp2 + o) : xc, a1, a2);
      }
      float4 Lx = cq(0, fo, arow, acol) * xc + (is1t * sv[1]) * a1 + (i2t * sv[2]) * a2;
      const float4 xm = L4(xpl + o - MS_W), xp = L4(xpl + o + MS_W);
      Lx = Lx + (h1x * cq(3, fo, arow, acol)) * (xp - xm) + (i2x * cq(4, fo, arow, acol)) * (xp - 2.f * xc + xm);
      const float4 ym = make_float4(msm[xpl + o - 1], xc.x, xc.y, xc.z), yp = make_float4(xc.y, xc.z, xc.w, msm[xpl + o + 4]);
      Lx = Lx + (h1y * cq(5, fo, arow, acol)) * (yp - ym) + (i2y * cq(6, fo, arow, acol)) * (yp - 2.f * xc + ym);
      const float4 r4 = L4(ro + arow * MS_W + acol);
      *reinterpret_cast<float4*>(&msm[yo + arow * MS_W + acol]) =
          make_float4(-r4.x * Lx.x, -r4.y * Lx.y, -r4.z * Lx.z, -r4.w * Lx.w);
    }
    if (tid < 2 * RR) {
      const int rr = tid >> 1, c = (tid & 1) ? MS_Y + 4 : 3;
      const int o = (rr + 1) * MS_W + c;
      const float xc = msm[xpl + o];
      float a1, a2;
      dforms1(cls, cls == 2 ? msm[xm2 + o] : xc, cls != 1 ? msm[xm1 + o] : xc, xc, cls != 2 ? msm[xp1 + o] : xc,
              cls == 1 ? msm[xp2 + o] : xc, a1, a2);
      float Lx = cs(0, fo, rr, c) * xc + (is1t * sv[1]) * a1 + (i2t * sv[2]) * a2;
      const float xm = msm[xpl + o - MS_W], xp = msm[xpl + o + MS_W];
      Lx += (h1x * cs(3, fo, rr, c)) * (xp - xm) + (i2x * cs(4, fo, rr, c)) * (xp - 2.f * xc + xm);
      const float ym = msm[xpl + o - 1], yp = msm[xpl + o + 1];
      Lx += (h1y * cs(5, fo, rr, c)) * (yp - ym) + (i2y * cs(6, fo, rr, c)) * (yp - 2.f * xc + ym);
      msm[yo + rr * MS_W + c] = -msm[ro + rr * MS_W + c] * Lx;
    }
  };
  auto cls_of = [&](int tp) { return tp == 0 ? 1 : (tp == n0 - 1 ? 2 : 0); };

  // pass C point of this thread (the first CT threads)
  const bool cthr = tid < CT;
  const int crow = (tid >> 4) % MX, cc = 4 + 4 * (tid & 15);
  const float* Rp = a.r + off + (size_t)(x0 + crow) * n2 + (y0 + cc - 4);
  const float* Dp = a.dinv + off + (size_t)(x0 + crow) * n2 + (y0 + cc - 4);
  const float* Pp = a.d ? a.d + off + (size_t)(x0 + crow) * n2 + (y0 + cc - 4) : nullptr;
  const size_t jbase = off + (size_t)(x0 + crow) * n2 + (y0 + cc - 4);
  auto load_pt = [&](int t, float4& r4, float4& di4, float4& d4) {
    const int q = t * pl;
    if (MODE != SM_APPLY) r4 = ld4(Rp + q);
    if (MODE == SM_POST0 || MODE == SM_CHEB || MODE == SM_CHEB_DOT) di4 = ld4(Dp + q);
    // previous iterate: a buffer this kernel overwrites (at other planes of
    // the thread's own points), so a coherent load
    if ((MODE == SM_CHEB || MODE == SM_CHEB_DOT) && Pp) d4 = __ldcg(reinterpret_cast<const float4*>(Pp + q));
  };
  auto prefetch_pt = [&](int t) {
    const int q = t * pl;
    if (MODE != SM_APPLY) pf_l2(Rp + q);
    if (MODE == SM_POST0 || MODE == SM_CHEB || MODE == SM_CHEB_DOT) pf_l2(Dp + q);
    if ((MODE == SM_CHEB || MODE == SM_CHEB_DOT) && Pp) pf_l2(Pp + q);
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
  for (int tp = flo; tp <= t0; ++tp) {
    const int c = cls_of(tp);
    passA(c, c == 2 ? xslot(tp - 2) : 0, c != 1 ? xslot(tp - 1) : 0, xslot(tp), c != 2 ? xslot(tp + 1) : 0,
          c == 1 ? xslot(tp + 2) : 0, fslot(tp), rslot(tp), yslot(tp));
  }
  // the warm-up's planes are free: copies of the planes pass A of t0 + 1 reads
  __syncthreads();
  refill(t0 + 4, t0 + 3, t0 + 4);

  // slot offsets of the planes around t, rotated by one plane per step:
  // operand t-1 .. t+3, fields t .. t+3, rho t+1 .. t+3, y t-2 .. t+2
  int Xs[5], Fs[4], Rs[3], Ys[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) Xs[k] = OX + ((t0 - 1 + k - xlo + MS_NX) % MS_NX) * SX;
#pragma unroll
  for (int k = 0; k < 4; ++k) Fs[k] = OF + ((t0 + k - flo) % MS_NF) * SF;
#pragma unroll
  for (int k = 0; k < 3; ++k) Rs[k] = OR + ((t0 + 1 + k - flo) % MS_NR) * SR;
#pragma unroll
  for (int k = 0; k < 5; ++k) Ys[k] = OY + ((t0 - 2 + k - flo + 2 * MS_NY) % MS_NY) * SY;

  double accd = 0.0;
  for (int t = t0; t < t1; ++t) {
    // the point operands of plane t+1 (pass C of the next step), a step ahead
    float4 nr4 = f4(0.f), ndi4 = f4(0.f), nd4 = f4(0.f);
    if (cthr) {
      if (t + 1 < t1) load_pt(t + 1, nr4, ndi4, nd4);
      if ((tid & 7) == 0 && t + 2 < t1) prefetch_pt(t + 2);
    }
    // A: y(t+1) (plane t+1 is never the first; y(n0-1) is computed with
    // y(n0-2), after its field and rho planes have landed)
    if (t + 1 <= n0 - 1 && t != n0 - 2) passA(0, Xs[0], Xs[1], Xs[2], Xs[3], Xs[4], Fs[1], Rs[0], Ys[3]);
    if (t == n0 - 3) {
      cp_async_wait<0>();
      __syncthreads();
      passA(2, Xs[1], Xs[2], Xs[3], Xs[4], Xs[4], Fs[2], Rs[1], Ys[4]);
    }
    // the copies pass A of t + 1 reads have landed (this thread's); one
    // barrier publishes them and y(t+1), and frees the slots of the operand
    // and fields of t - 1 and of rho up to t + 1
    cp_async_wait<0>();
    __syncthreads();
    refill(t + MS_NX, t + MS_NF, t + 2 + MS_NR);

    if (cthr) {
      // C. q = L^T y - theta 1_B x on plane t
      const int fo = Fs[0];
      const int yr = Ys[2] + (crow + 1) * MS_W;
      const float4 yc = L4(yr + cc);
      float4 qv = cq(0, fo, crow + 1, cc) * yc;
      if (t >= 3 && t <= n0 - 4) {
        const float4 tm = L4(Ys[1] + (crow + 1) * MS_W + cc), tq = L4(Ys[3] + (crow + 1) * MS_W + cc);
        qv = qv + (0.5f * is1t * sv[1]) * (tm - tq) + (i2t * sv[2]) * (tm - 2.f * yc + tq);
      } else {
#pragma unroll
        for (int o = -2; o <= 2; ++o) {
          const int ip = t - o;
          if (ip < 0 || ip >= n0) continue;
          const float w1 = dweight(1, ip, n0, 0, o), w2 = dweight(2, ip, n0, 0, o);
          if (w1 == 0.f && w2 == 0.f) continue;
          const float4 yv = o == 0 ? yc : L4(Ys[2 - o] + (crow + 1) * MS_W + cc);
          qv = qv + ((w1 * is1t) * sv[1] + (w2 * i2t) * sv[2]) * yv;
        }
      }
      {
        const float4 ym = L4(yr - MS_W + cc), yp = L4(yr + MS_W + cc);
        qv = qv + h1x * (cq(3, fo, crow, cc) * ym - cq(3, fo, crow + 2, cc) * yp) +
             i2x * (cq(4, fo, crow, cc) * ym - 2.f * (cq(4, fo, crow + 1, cc) * yc) + cq(4, fo, crow + 2, cc) * yp);
      }
      {
        const int rr = crow + 1;
        const float4 c1 = cq(5, fo, rr, cc), c2 = cq(6, fo, rr, cc);
        const float c1l = cs(5, fo, rr, cc - 1), c1r = cs(5, fo, rr, cc + 4);
        const float c2l = cs(6, fo, rr, cc - 1), c2r = cs(6, fo, rr, cc + 4);
        const float4 ym = make_float4(msm[yr + cc - 1], yc.x, yc.y, yc.z), yp = make_float4(yc.y, yc.z, yc.w, msm[yr + cc + 4]);
        const float4 c1m = make_float4(c1l, c1.x, c1.y, c1.z), c1p = make_float4(c1.y, c1.z, c1.w, c1r);
        const float4 c2m = make_float4(c2l, c2.x, c2.y, c2.z), c2p = make_float4(c2.y, c2.z, c2.w, c2r);
        qv = qv + h1y * (c1m * ym - c1p * yp) + i2y * (c2m * ym - 2.f * (c2 * yc) + c2p * yp);
      }
      const float4 xj = L4(Xs[1] + (crow + 2) * MS_W + cc);
      if (t == 0 || (g.final_rows && t == n0 - 1)) qv = qv - g.theta * xj;
      const size_t j = jbase + (size_t)t * pl;
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
    // rotate the slot offsets by one plane
    {
      const int x_ = Xs[0]; Xs[0] = Xs[1]; Xs[1] = Xs[2]; Xs[2] = Xs[3]; Xs[3] = Xs[4]; Xs[4] = x_;
      const int f_ = Fs[0]; Fs[0] = Fs[1]; Fs[1] = Fs[2]; Fs[2] = Fs[3]; Fs[3] = f_;
      const int r_ = Rs[0]; Rs[0] = Rs[1]; Rs[1] = Rs[2]; Rs[2] = r_;
      const int y_ = Ys[0]; Ys[0] = Ys[1]; Ys[1] = Ys[2]; Ys[2] = Ys[3]; Ys[3] = Ys[4]; Ys[4] = y_;
    }
  }
  cp_async_wait<0>();
  if ((MODE == SM_APPLY || MODE == SM_CHEB_DOT) && a.part) {
    const double s = block_sum(accd);
    partial_finish(s, a.part, a.cnt, a.tot, b, blockIdx.x, gridDim.x);
  }
}
