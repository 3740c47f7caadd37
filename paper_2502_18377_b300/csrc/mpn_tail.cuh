// Fused coarse end of the V-cycle: the levels from a chosen one down to the
// coarsest run in ONE kernel launch per V-cycle instead of one launch per
// operator pass.
//
// One thread-block cluster per instance.  Time is never coarsened, so every
// level has the same n_t time planes; CTA r of the cluster owns planes
// [r P, r P + P) at every level.  Restriction and prolongation then stay
// inside a CTA, and only the operator passes read other CTAs' planes (the
// time neighbours at offsets up to +-2), through distributed shared memory.
// Each CTA keeps its planes of r, e, d, y and of the coefficient fields, rho
// and the scaled inverse diagonal in shared memory; a cluster barrier
// separates passes whose reads cross CTAs.  The arithmetic of each pass is
// that of the per-level kernels (Chebyshev-Jacobi smoothing, residual,
// full-weighting restriction, linear prolongation, explicit coarsest inverse).
#pragma once
#include <cooperative_groups.h>

#include "mpn_device.cuh"

namespace cg = cooperative_groups;

#define TAIL_TPB 512
#define TAIL_MAXL 16
// first fused level: at most TAIL_MAX_PPT points per thread and CTA (the
// reaction-diffusion benchmark, 16 x 32 x 64 x 64: fused from 32 x 8 x 8,
// 0.8 % faster per step than from 32 x 16 x 16 at 4 points per thread; 2-CTA
// clusters 2 % and 8-CTA clusters 5 % slower than 4)
#ifndef TAIL_MAX_PPT
#define TAIL_MAX_PPT 2
#endif
// clusters larger than 4 CTAs per instance only while the batch gives fewer
// CTAs than this in all (small batches leave most SMs idle otherwise)
#ifndef TAIL_TARGET_CTAS
#define TAIL_TARGET_CTAS 64
#endif
#ifndef TAIL_MAX_CLUSTER
#define TAIL_MAX_CLUSTER 16
#endif

struct TailLevel {
  Grid g;
  int cz[3];
  int plane;                // points per time plane
  int cap;                  // points per CTA (P planes)
  const float* fields;      // [F][B][N] in global memory
  const float* rho;         // [B][N]
  const float* dinv;        // [B][N]
  int o_r, o_e, o_d, o_y, o_f, o_rho, o_dinv;   // shared-memory offsets (floats)
};

struct TailArgs {
  int nl;                   // tail levels; the last one is the coarsest
  int V, F, B, M, m, P;
  float invP;
  int field_of[7];
  const float* scalars;     // [V][B]
  float c1[32], c2[32], inv_th;
  const float* Kinv;        // [B][M][M]
  int o_g;                  // gathered coarsest right-hand side (M floats)
  int o_tw;                 // time-direction weight table (P x 20 floats)
  const float* rin;         // r at the first tail level, [B][N]
  float* eout;              // e at the first tail level, [B][N]
  TailLevel lv[TAIL_MAXL];
};

extern __shared__ __align__(16) float tail_sm[];

// Load from CTA `rank`'s copy of the shared-memory word that `local` points
// to in this CTA (distributed shared memory).
__device__ __forceinline__ float dsm_ld(const float* local, int rank) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
  uint32_t ra;
  float v;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(ra));
  return v;
}

// Per-pass copy of one level's parameters (registers, not parameter space).
struct TailLv {
  Grid g;
  int cz1, cz2, plane, cap;
  int o_r, o_e, o_d, o_y, o_f, o_rho, o_dinv;
  __device__ __forceinline__ explicit TailLv(const TailLevel& L)
      : g(L.g), cz1(L.cz[1]), cz2(L.cz[2]), plane(L.plane), cap(L.cap), o_r(L.o_r), o_e(L.o_e), o_d(L.o_d),
        o_y(L.o_y), o_f(L.o_f), o_rho(L.o_rho), o_dinv(L.o_dinv) {}
};

// Position of the CTA-local point j.
template <int D>
__device__ __forceinline__ void tl_pos(const Grid& g, int plane, float invpl, float inv2, int t0, int j, int pos[3],
                                       int& rem) {
  int lt = fdivmod(j, plane, invpl, rem);
  pos[0] = t0 + lt;
  if (D == 3) {
    int i2;
    pos[1] = fdivmod(rem, g.n[2], inv2, i2);
    pos[2] = i2;
  } else {
    pos[1] = rem; pos[2] = 0;
  }
}

// In-plane offset of the neighbour at +-o along spatial dim d (wrapping when
// periodic; the caller guarantees existence otherwise).
__device__ __forceinline__ int tl_off(const Grid& g, const int pos[3], int d, int o) {
  int c = pos[d] + o;
  if (g.per[d]) { if (c < 0) c += g.n[d]; else if (c >= g.n[d]) c -= g.n[d]; }
  return (c - pos[d]) * g.stride[d];
}

// MASK: FS_ANY (coefficient kind read at run time) or bit v set when c_v is a
// field (layout fixed at compile time).
template <int MASK>
struct TailView {
  TailLv L;
  int fo[7];
  float scal[7];
  int myr, t0, ntp, P;
  float invP;
  // value of the level array at offset `o_arr` for (time plane tp, in-plane
  // index rem), wherever in the cluster that plane lives
  __device__ __forceinline__ float ld(int o_arr, int tp, int rem) const {
    int r = __float2int_rz(((float)tp + 0.5f) * invP);
    const float* a = tail_sm + o_arr + (tp - r * P) * L.plane + rem;
    return r == myr ? *a : dsm_ld(a, r);
  }
  // coefficient v at CTA-local point j
  __device__ __forceinline__ bool is_field(int v) const { return MASK == FS_ANY ? fo[v] >= 0 : ((MASK >> v) & 1); }
  // (FS_SHARE46: c_yy reads the field of c_xx, so the two share their loads)
  __device__ __forceinline__ float c(int v, int j) const {
    if ((MASK & FS_SHARE46) && v == 6) v = 4;
    return is_field(v) ? tail_sm[L.o_f + fo[v] * L.cap + j] : scal[v];
  }
  // coefficient v at (time plane tp, in-plane index rem), any CTA
  __device__ __forceinline__ float cr(int v, int tp, int rem) const {
    if ((MASK & FS_SHARE46) && v == 6) v = 4;
    return is_field(v) ? ld(L.o_f + fo[v] * L.cap, tp, rem) : scal[v];
  }
};

// Time-direction weights, per CTA-local plane lt (time t = t0 + lt), stored
// at tail_sm[o_tw + 20 lt]: [0,5) w1 and [5,10) w2 of the row at t applied to
// x(t + o); [10,15) g1 and [15,20) g2 with which the column at t gathers row
// t - o (0 where that row does not exist or does not touch t); o = -2..2.
// Time is not coarsened, so the table serves every level.
#define TW_STRIDE 20

// Spatial part (dims 1 .. D-1) of (L x)_j.
template <int D, int MASK>
__device__ __forceinline__ float ly_space(const TailView<MASK>& v, const float* X, int j, const int pos[3], float xc) {
  const Grid& g = v.L.g;
  float acc = 0.f;
#pragma unroll
  for (int d = 1; d < D; ++d) {
    float a1, a2;
    if (g.per[d] || (pos[d] >= 1 && pos[d] <= g.n[d] - 2)) {
      float xm = X[j + tl_off(g, pos, d, -1)], xp = X[j + tl_off(g, pos, d, 1)];
      a1 = 0.5f * (xp - xm); a2 = xp - 2.f * xc + xm;
    } else {
      a1 = 0.f; a2 = 0.f;
#pragma unroll
      for (int o = -2; o <= 2; ++o) {
        float w1 = dweight(1, pos[d], g.n[d], 0, o), w2 = dweight(2, pos[d], g.n[d], 0, o);
        if (w1 == 0.f && w2 == 0.f) continue;
        float xv = o == 0 ? xc : X[j + o * g.stride[d]];
        a1 += w1 * xv; a2 += w2 * xv;
      }
    }
    acc += v.c(1 + 2 * d, j) * a1 * g.is1[d] + v.c(2 + 2 * d, j) * a2 * g.is2[d];
  }
  return acc;
}

// y = -rho L e on this CTA's points.
template <int D, int MASK>
__device__ void tail_Ly(const TailView<MASK>& v, int o_tw) {
  const Grid& g = v.L.g;
  const int n0 = g.n[0];
  const int cnt = v.ntp * v.L.plane;
  const int o_e = v.L.o_e;
  const float* X = tail_sm + o_e;
  float* Y = tail_sm + v.L.o_y;
  const float* RHO = tail_sm + v.L.o_rho;
  const float invpl = 1.f / (float)v.L.plane, inv2 = 1.f / (float)g.n[2];
  const float is1t = g.is1[0], is2t = g.is2[0];
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    int pos[3], rem;
    tl_pos<D>(g, v.L.plane, invpl, inv2, v.t0, j, pos, rem);
    const int t = pos[0];
    const float xc = X[j];
    float a1, a2;
    if (t >= 1 && t <= n0 - 2) {
      float xm = v.ld(o_e, t - 1, rem), xp = v.ld(o_e, t + 1, rem);
      a1 = 0.5f * (xp - xm); a2 = xp - 2.f * xc + xm;
    } else {
      const float* tw = tail_sm + o_tw + (t - v.t0) * TW_STRIDE;
      a1 = 0.f; a2 = 0.f;
#pragma unroll
      for (int o = -2; o <= 2; ++o) {
        float w1 = tw[o + 2], w2 = tw[5 + o + 2];
        if (w1 == 0.f && w2 == 0.f) continue;
        float xv = o == 0 ? xc : v.ld(o_e, t + o, rem);
        a1 += w1 * xv; a2 += w2 * xv;
      }
    }
    float Lx = v.c(0, j) * xc + v.c(1, j) * a1 * is1t + v.c(2, j) * a2 * is2t + ly_space<D, MASK>(v, X, j, pos, xc);
    Y[j] = -RHO[j] * Lx;
  }
}

// q = L^T y - theta 1_B e = -(S e) on this CTA's points, then the mode's
// update (SM_CHEB / SM_POST0: Chebyshev step on e, d; SM_RES: d = r - S e).
template <int D, int MODE, int MASK>
__device__ void tail_LTy(const TailView<MASK>& v, int o_tw, float c1, float c2) {
  const Grid& g = v.L.g;
  const int n0 = g.n[0];
  const int cnt = v.ntp * v.L.plane;
  const int o_y = v.L.o_y;
  const float* Y = tail_sm + o_y;
  float* E = tail_sm + v.L.o_e;
  float* Dd = tail_sm + v.L.o_d;
  const float* R = tail_sm + v.L.o_r;
  const float* DI = tail_sm + v.L.o_dinv;
  const float invpl = 1.f / (float)v.L.plane, inv2 = 1.f / (float)g.n[2];
  const float is1t = g.is1[0], is2t = g.is2[0];
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    int pos[3], rem;
    tl_pos<D>(g, v.L.plane, invpl, inv2, v.t0, j, pos, rem);
    const int t = pos[0];
    const float yc = Y[j];
    float q = v.c(0, j) * yc;
    // time direction
    if (t >= 3 && t <= n0 - 4) {
      float ym = v.ld(o_y, t - 1, rem), yp = v.ld(o_y, t + 1, rem);
      float am = v.cr(1, t - 1, rem), ap = v.cr(1, t + 1, rem);
      float bm = v.cr(2, t - 1, rem), bp = v.cr(2, t + 1, rem);
      q += 0.5f * is1t * (am * ym - ap * yp) + is2t * (bm * ym - 2.f * v.c(2, j) * yc + bp * yp);
    } else {
      const float* tw = tail_sm + o_tw + (t - v.t0) * TW_STRIDE;
#pragma unroll
      for (int o = -2; o <= 2; ++o) {
        float w1 = tw[10 + o + 2], w2 = tw[15 + o + 2];
        if (w1 == 0.f && w2 == 0.f) continue;
        float yv, a, bb;
        if (o == 0) { yv = yc; a = v.c(1, j); bb = v.c(2, j); }
        else { yv = v.ld(o_y, t - o, rem); a = v.cr(1, t - o, rem); bb = v.cr(2, t - o, rem); }
        q += yv * (a * w1 * is1t + bb * w2 * is2t);
      }
    }
    // space directions
#pragma unroll
    for (int d = 1; d < D; ++d) {
      if (g.per[d] || (pos[d] >= 3 && pos[d] <= g.n[d] - 4)) {
        int jm = j + tl_off(g, pos, d, -1), jp = j + tl_off(g, pos, d, 1);
        float ym = Y[jm], yp = Y[jp];
        q += 0.5f * g.is1[d] * (v.c(1 + 2 * d, jm) * ym - v.c(1 + 2 * d, jp) * yp) +
             g.is2[d] * (v.c(2 + 2 * d, jm) * ym - 2.f * v.c(2 + 2 * d, j) * yc + v.c(2 + 2 * d, jp) * yp);
      } else {
#pragma unroll
        for (int o = -2; o <= 2; ++o) {
          int ip = pos[d] - o;
          if (ip < 0 || ip >= g.n[d]) continue;
          float w1 = dweight(1, ip, g.n[d], 0, o), w2 = dweight(2, ip, g.n[d], 0, o);
          if (w1 == 0.f && w2 == 0.f) continue;
          int jq = j - o * g.stride[d];
          q += Y[jq] * (v.c(1 + 2 * d, jq) * w1 * g.is1[d] + v.c(2 + 2 * d, jq) * w2 * g.is2[d]);
        }
      }
    }
    const float xj = E[j];
    if (is_boundary_t<D>(g, pos)) q -= g.theta * xj;
    if (MODE == SM_RES) {
      Dd[j] = R[j] + q;
    } else {
      float res = R[j] + q;
      float dn = (MODE == SM_CHEB ? c1 * Dd[j] : 0.f) + c2 * DI[j] * res;
      Dd[j] = dn;
      E[j] = xj + dn;
    }
  }
}

// Restriction along one spatial dim of coarse index J: number of candidate
// fine indices, and candidate k's (fine index, weight); weight 0 = skip.
struct RDim {
  int mode;      // 0 not coarsened, 1 periodic halving, 2 same-domain (non-periodic)
  int J, nf, nc, i0;
  __device__ __forceinline__ RDim(int coarsened, int per, int J_, int nf_, int nc_) : J(J_), nf(nf_), nc(nc_), i0(0) {
    mode = !coarsened ? 0 : (per ? 1 : 2);
    if (mode == 2) { i0 = ((J - 1) * (nf - 1)) / (nc - 1); if (i0 < 0) i0 = 0; }
  }
  __device__ __forceinline__ int count() const {
    if (mode == 0) return 1;
    if (mode == 1) return 3;
    int i1 = ((J + 1) * (nf - 1) + nc - 2) / (nc - 1);
    if (i1 > nf - 1) i1 = nf - 1;
    return i1 - i0 + 1;
  }
  __device__ __forceinline__ void entry(int k, int& i, float& w) const {
    if (mode == 0) { i = J; w = 1.f; return; }
    if (mode == 1) {
      if (k == 0) { i = 2 * J; w = 1.f; }
      else if (k == 1) { i = 2 * J + 1; w = 0.5f; }
      else { i = J >= 1 ? 2 * J - 1 : nf - 1; w = 0.5f; }
      return;
    }
    i = i0 + k;
    int Ji; float f; np_interp(i, nf, nc, Ji, f);
    w = (Ji == J ? 1.f - f : 0.f) + (Ji + 1 == J ? f : 0.f);
  }
};

// Prolongation along one spatial dim of fine index i: up to two coarse
// indices with weights.
__device__ __forceinline__ int pdim(int coarsened, int per, int i, int nf, int nc, int& J0, int& J1, float& w0,
                                    float& w1) {
  if (!coarsened) { J0 = i; w0 = 1.f; J1 = i; w1 = 0.f; return 1; }
  if (!per) {
    float f; np_interp(i, nf, nc, J0, f);
    J1 = J0 + 1; w0 = 1.f - f; w1 = f;
    return 2;
  }
  if ((i & 1) == 0) { J0 = J1 = i >> 1; w0 = 1.f; w1 = 0.f; return 1; }
  J0 = i >> 1; J1 = (J0 + 1 < nc) ? J0 + 1 : 0; w0 = w1 = 0.5f;
  return 2;
}

// Full-weighting restriction of the fine residual (in d) to the coarse r;
// both levels share this CTA's time planes.
template <int D>
__device__ void tail_restrict(const TailLv& F, const TailLv& C, int ntp) {
  const int cnt = ntp * C.plane;
  const float* fine = tail_sm + F.o_d;
  float* out = tail_sm + C.o_r;
  const float invpl = 1.f / (float)C.plane, inv2 = 1.f / (float)C.g.n[2];
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    int pos[3], rem;
    tl_pos<D>(C.g, C.plane, invpl, inv2, 0, j, pos, rem);
    const RDim r1(F.cz1, F.g.per[1], pos[1], F.g.n[1], C.g.n[1]);
    const RDim r2(D == 3 && F.cz2, F.g.per[2], pos[2], F.g.n[2], C.g.n[2]);
    const int c1 = r1.count(), c2 = r2.count();
    const float* fb = fine + pos[0] * F.plane;
    float acc = 0.f;
    for (int a = 0; a < c1; ++a) {
      int i1; float w1; r1.entry(a, i1, w1);
      if (w1 == 0.f) continue;
      float s = 0.f;
      for (int c = 0; c < c2; ++c) {
        int i2; float w2; r2.entry(c, i2, w2);
        s += w2 * fb[i1 * F.g.stride[1] + i2];
      }
      acc += w1 * s;
    }
    out[j] = acc;
  }
}

// Linear prolongation of the coarse e, added to the fine e.
template <int D>
__device__ void tail_prolong(const TailLv& F, const TailLv& C, int ntp) {
  const int cnt = ntp * F.plane;
  const float* E = tail_sm + C.o_e;
  float* ef = tail_sm + F.o_e;
  const float invpl = 1.f / (float)F.plane, inv2 = 1.f / (float)F.g.n[2];
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    int pos[3], rem;
    tl_pos<D>(F.g, F.plane, invpl, inv2, 0, j, pos, rem);
    int a0, a1, b0, b1;
    float u0, u1, v0, v1;
    pdim(F.cz1, F.g.per[1], pos[1], F.g.n[1], C.g.n[1], a0, a1, u0, u1);
    if (D == 3) pdim(F.cz2, F.g.per[2], pos[2], F.g.n[2], C.g.n[2], b0, b1, v0, v1);
    else { b0 = b1 = 0; v0 = 1.f; v1 = 0.f; }
    const float* cb = E + pos[0] * C.plane;
    const int s1 = C.g.stride[1];
    float acc = u0 * (v0 * cb[a0 * s1 + b0] + v1 * cb[a0 * s1 + b1]) + u1 * (v0 * cb[a1 * s1 + b0] + v1 * cb[a1 * s1 + b1]);
    ef[j] += acc;
  }
}

template <int D, int MASK>
__global__ void __launch_bounds__(TAIL_TPB, 1) k_vtail(const __grid_constant__ TailArgs ta) {
  float* sm = tail_sm;
  cg::cluster_group cl = cg::this_cluster();
  const int myr = (int)cl.block_rank();
  const int b = blockIdx.y;
  const int n0 = ta.lv[0].g.n[0];
  const int t0 = myr * ta.P;
  const int ntp = max(0, min(ta.P, n0 - t0));
  const int nl = ta.nl, m = ta.m, F = ta.F, B = ta.B;

  // stage this CTA's planes of the coefficients and of the right-hand side
  for (int k = 0; k + 1 < nl; ++k) {
    const TailLevel& L = ta.lv[k];
    const int cnt = ntp * L.plane, cap = L.cap, N = L.g.N;
    const int o_f = L.o_f, o_rho = L.o_rho, o_dinv = L.o_dinv;
    const float* fields = L.fields;
    const float* rho = L.rho;
    const float* dinv = L.dinv;
    const size_t base = (size_t)b * N + (size_t)t0 * L.plane;
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      for (int f = 0; f < F; ++f) sm[o_f + f * cap + j] = __ldg(fields + (size_t)f * B * N + base + j);
      sm[o_rho + j] = __ldg(rho + base + j);
      sm[o_dinv + j] = __ldg(dinv + base + j);
    }
  }
  {
    const TailLevel& L = ta.lv[0];
    const int cnt = ntp * L.plane, o_r = L.o_r;
    const float* rin = ta.rin;
    const size_t base = (size_t)b * L.g.N + (size_t)t0 * L.plane;
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) sm[o_r + j] = rin[base + j];
  }
  TailView<MASK> v0{TailLv(ta.lv[0]), {}, {}, myr, t0, ntp, ta.P, ta.invP};
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    v0.fo[q] = ta.field_of[q];
    v0.scal[q] = (q < ta.V && ta.field_of[q] < 0) ? ta.scalars[q * B + b] : 0.f;
  }
  const float inv_th = ta.inv_th;
  const int o_tw = ta.o_tw;
  for (int lt = threadIdx.x; lt < ntp; lt += blockDim.x) {
    const int t = t0 + lt;
    float* tw = sm + o_tw + lt * TW_STRIDE;
#pragma unroll
    for (int o = -2; o <= 2; ++o) {
      tw[o + 2] = dweight(1, t, n0, 0, o);
      tw[5 + o + 2] = dweight(2, t, n0, 0, o);
      const int ip = t - o;
      const bool ok = ip >= 0 && ip < n0;
      tw[10 + o + 2] = ok ? dweight(1, ip, n0, 0, o) : 0.f;
      tw[15 + o + 2] = ok ? dweight(2, ip, n0, 0, o) : 0.f;
    }
  }
  __syncthreads();

  // down: pre-smoothing from e = 0, residual, restriction
  for (int k = 0; k + 1 < nl; ++k) {
    TailView<MASK> v = v0;
    v.L = TailLv(ta.lv[k]);
    {
      const int cnt = ntp * v.L.plane, o_e = v.L.o_e, o_d = v.L.o_d, o_r = v.L.o_r, o_di = v.L.o_dinv;
      for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
        float e = inv_th * sm[o_di + j] * sm[o_r + j];
        sm[o_e + j] = e;
        sm[o_d + j] = e;
      }
    }
    cl.sync();
    for (int s = 1; s < m; ++s) {
      tail_Ly<D, MASK>(v, o_tw);
      cl.sync();
      tail_LTy<D, SM_CHEB, MASK>(v, o_tw, ta.c1[s], ta.c2[s]);
      cl.sync();
    }
    tail_Ly<D, MASK>(v, o_tw);
    cl.sync();
    tail_LTy<D, SM_RES, MASK>(v, o_tw, 0.f, 0.f);
    __syncthreads();
    tail_restrict<D>(v.L, TailLv(ta.lv[k + 1]), ntp);
    __syncthreads();
  }

  // coarsest: e = Kinv r, from the whole right-hand side gathered locally
  cl.sync();
  {
    const TailLv C(ta.lv[nl - 1]);
    const int M = ta.M;
    float* G = sm + ta.o_g;
    const float invpl = 1.f / (float)C.plane;
    for (int col = threadIdx.x; col < M; col += blockDim.x) {
      int tp = __float2int_rz(((float)col + 0.5f) * invpl);
      int rem = col - tp * C.plane;
      int r = __float2int_rz(((float)tp + 0.5f) * ta.invP);
      const float* a = sm + C.o_r + (tp - r * ta.P) * C.plane + rem;
      G[col] = r == myr ? *a : dsm_ld(a, r);
    }
    __syncthreads();
    const int rows = ntp * C.plane;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float* Kb = ta.Kinv + ((size_t)b * M + (size_t)t0 * C.plane) * M;
    for (int jr = wid; jr < rows; jr += nw) {
      const float* row = Kb + (size_t)jr * M;
      float s = 0.f;
      for (int col = lane; col < M; col += 32) s += __ldg(row + col) * G[col];
      s = warp_sum(s);
      if (lane == 0) sm[C.o_e + jr] = s;
    }
    __syncthreads();
  }

  // up: prolongation, post-smoothing
  for (int k = nl - 2; k >= 0; --k) {
    TailView<MASK> v = v0;
    v.L = TailLv(ta.lv[k]);
    tail_prolong<D>(v.L, TailLv(ta.lv[k + 1]), ntp);
    cl.sync();
    tail_Ly<D, MASK>(v, o_tw);
    cl.sync();
    tail_LTy<D, SM_POST0, MASK>(v, o_tw, 0.f, inv_th);
    cl.sync();
    for (int s = 1; s < m; ++s) {
      tail_Ly<D, MASK>(v, o_tw);
      cl.sync();
      tail_LTy<D, SM_CHEB, MASK>(v, o_tw, ta.c1[s], ta.c2[s]);
      cl.sync();
    }
  }

  {
    const TailLevel& L = ta.lv[0];
    const int cnt = ntp * L.plane, o_e = L.o_e;
    float* eout = ta.eout;
    const size_t base = (size_t)b * L.g.N + (size_t)t0 * L.plane;
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) eout[base + j] = sm[o_e + j];
  }
}
