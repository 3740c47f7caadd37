// Application of the reduced normal operator S = L^T diag(rho) L + theta 1_B
// in two passes per operator apply, one thread per grid point:
//   k_Ly:  y = -rho L x
//   k_LTy: (L^T y)_j - theta 1_B x_j = -(S x)_j, then a mode-specific update
// Every Chebyshev smoothing step, multigrid residual and PCG operator apply
// of every level uses them.  The working set of a level (x, y, r, D^{-1},
// rho, d and the coefficient fields) is L2-resident at the sizes this solver
// targets, so the extra y array costs L2 traffic only, while each point does
// its stencil arithmetic once (no halo recomputation).
//
// Chebyshev state is kept in look-ahead form: e is always the current
// iterate, d the last direction.  A step reads e at the stencil neighbours
// (pass 1) and updates e and d at its own point only (pass 2), so both passes
// can work in place.
#pragma once
#include "mpn_device.cuh"
#include "mpn_stepargs.cuh"

// p -> (t, x, y) without integer division.
__device__ __forceinline__ void decode_f(const Grid& g, int p, float inv12, float inv2, int pos[3]) {
  int rem, i2;
  pos[0] = fdivmod(p, g.n[1] * g.n[2], inv12, rem);
  pos[1] = fdivmod(rem, g.n[2], inv2, i2);
  pos[2] = i2;
}

// Neighbour at offset +-1 along d for an interior/periodic coordinate.
__device__ __forceinline__ int nb1(const Grid& g, int p, const int pos[3], int d, int o) {
  int c = pos[d] + o;
  int s = g.stride[d];
  if (c < 0) return dbg_index(g, p + (g.n[d] - 1) * s, g.N, 2);
  if (c >= g.n[d]) return dbg_index(g, p - (g.n[d] - 1) * s, g.N, 2);
  return dbg_index(g, p + o * s, g.N, 2);
}

template <int D>
__device__ __forceinline__ bool edge_any(const Grid& g, const int pos[3]) {
  if (g.st64 || g.mixed) return true;   // the general forms everywhere
  bool e = pos[0] < 3 || pos[0] > g.n[0] - 4;
#pragma unroll
  for (int d = 1; d < D; ++d) e |= !g.per[d] && (pos[d] < 3 || pos[d] > g.n[d] - 4);
  return e;
}

template <int D>
__global__ void __launch_bounds__(256) k_Ly(Grid g, Coef cf, const float* __restrict__ rho, const float* __restrict__ x,
                                            float* __restrict__ y) {
  const int b = blockIdx.y;
  const size_t off = (size_t)b * g.N;
  const float* xb = x + off;
  const float inv12 = 1.f / (float)(g.n[1] * g.n[2]), inv2 = 1.f / (float)g.n[2];
  const CoefB C(cf, b, 1 + 2 * D);
  GRID_LOOP(p, g.N) {
    int pos[3]; decode_f(g, p, inv12, inv2, pos);
    float xc = xb[p];
    float Lx;
    if (!edge_any<D>(g, pos)) {
      Lx = C(0, p) * xc;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        float xm = xb[nb1(g, p, pos, d, -1)], xp = xb[nb1(g, p, pos, d, 1)];
        Lx += C(1 + 2 * d, p) * (0.5f * (xp - xm)) * g.is1[d] + C(2 + 2 * d, p) * (xp - 2.f * xc + xm) * g.is2[d];
      }
    } else {
      Lx = Lrow<float, D>(g, cf, b, p, pos, xb, nullptr);
      const int e = mixed_axis(g, pos);
      if (e >= 1) {   // Neumann / mixed row: y = -R (L x, B x)
        const float Bx = Brow<float>(g, b, p, pos, e, xb);
        const float r12 = g.r12[off + p], r22 = g.r22[off + p];
        y[off + p] = -(rho[off + p] * Lx + r12 * Bx);
        g.y2[off + p] = -(r12 * Lx + r22 * Bx);
        continue;
      }
    }
    y[off + p] = -rho[off + p] * Lx;
  }
}

template <int D, int MODE>
__global__ void __launch_bounds__(256) k_LTy(Grid g, Coef cf, StepArgs a) {
  const int b = blockIdx.y;
  const size_t off = (size_t)b * g.N;
  const float* yb = a.y + off;
  const float inv12 = 1.f / (float)(g.n[1] * g.n[2]), inv2 = 1.f / (float)g.n[2];
  const CoefB C(cf, b, 1 + 2 * D);
  float acc = 0.f;   // one or two points per thread; the block sum is FP64
  GRID_LOOP(p, g.N) {
    int pos[3]; decode_f(g, p, inv12, inv2, pos);
    float yc = yb[p];
    float q = C(0, p) * yc;
    if (!edge_any<D>(g, pos)) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        int pm = nb1(g, p, pos, d, -1), pp = nb1(g, p, pos, d, 1);
        float ym = yb[pm], yp = yb[pp];
        q += 0.5f * g.is1[d] * (C(1 + 2 * d, pm) * ym - C(1 + 2 * d, pp) * yp) +
             g.is2[d] * (C(2 + 2 * d, pm) * ym - 2.f * C(2 + 2 * d, p) * yc + C(2 + 2 * d, pp) * yp);
      }
    } else {
      q = LTgather<float, D>(g, cf, b, p, pos, yb);
      if (g.mixed) q += BTgather<float>(g, b, p, pos, g.y2 + off);
    }
    float xj = a.x[off + p];
    if (is_boundary_t<D>(g, pos) && mixed_axis(g, pos) < 0) q -= g.theta * xj;
    // q = -(S x)_j
    const size_t j = off + p;
    if (MODE == SM_APPLY) {
      a.out[j] = -q;
      acc -= q * xj;
    } else if (MODE == SM_RES) {
      a.out[j] = a.r[j] + q;
    } else {
      float res = a.r[j] + q;
      float dn = (MODE == SM_CHEB ? a.c1 * a.d[j] : 0.f) + a.c2 * a.dinv[j] * res;
      a.d[j] = dn;
      a.e[j] = xj + dn;
    }
  }
  if (MODE == SM_APPLY && a.part) {
    double s = block_sum((double)acc);
    if (threadIdx.x == 0) a.part[b * MPN_PMAX + blockIdx.x] = s;
  }
}

// ------------------------------------------------------------ float4 versions
// D = 3 and n_y % 4 == 0: one thread owns 4 consecutive points along y.
// Along t and x the four points share their position class, so the
// (possibly one-sided) weights are uniform and neighbours come as float4;
// along y the neighbours come from the same float4 plus one value on each
// side.  A group that touches a non-periodic y-edge falls back to the scalar
// formulas point by point.

struct CoefB4 {
  const float* base[7];
  int ps[7];
  __device__ __forceinline__ CoefB4(const Coef& c, int b) {
#pragma unroll
    for (int v = 0; v < 7; ++v) { base[v] = c.ptr[v] + (size_t)b * c.bstride[v]; ps[v] = c.pstride[v]; }
  }
  __device__ __forceinline__ float4 at4(int v, int p) const { return ps[v] ? ld4(base[v] + p) : f4(__ldg(base[v])); }
  __device__ __forceinline__ float at(int v, int p) const { return __ldg(base[v] + p * ps[v]); }
};

// group (it, ix, iy0) of p0 = first point; returns false if the group needs
// the scalar fallback (touches a non-periodic y edge region)
__device__ __forceinline__ void group_pos(const Grid& g, int q, float inv_ng, float inv_n1, int pos[3]) {
  q = dbg_index(g, q, g.N >> 2, 4);
  int ng = g.n[2] >> 2, r;
  int row = fdivmod(q, ng, inv_ng, r);
  pos[2] = r << 2;
  pos[0] = fdivmod(row, g.n[1], inv_n1, pos[1]);
}
__global__ void __launch_bounds__(256, 6) k_Ly4(Grid g, Coef cf, const float* __restrict__ rho, const float* __restrict__ x,
                                             float* __restrict__ y) {
  const int b = blockIdx.y;
  const size_t off = (size_t)b * g.N;
  const float* xb = x + off;
  const CoefB4 C(cf, b);
  const int NG = g.N >> 2;
  const float inv_ng = 1.f / (float)(g.n[2] >> 2), inv_n1 = 1.f / (float)g.n[1];
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < NG; q += gridDim.x * blockDim.x) {
    int pos[3]; group_pos(g, q, inv_ng, inv_n1, pos);
    const int p0 = q << 2;
    const int n2 = g.n[2];
    bool yedge = !g.per[2] && (pos[2] < 3 || pos[2] + 3 > n2 - 4);
    if (yedge) {
      for (int k = 0; k < 4; ++k) {
        int pk[3] = {pos[0], pos[1], pos[2] + k};
        y[off + p0 + k] = -rho[off + p0 + k] * Lrow<float, 3>(g, cf, b, p0 + k, pk, xb, nullptr);
      }
      continue;
    }
    float4 xc = ld4(xb + p0);
    float4 Lx = C.at4(0, p0) * xc;
    // t and x: uniform position class
    bool txin = pos[0] > 0 && pos[0] < g.n[0] - 1 && (g.per[1] || (pos[1] > 0 && pos[1] < g.n[1] - 1));
    if (txin) {
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        float4 xm = ld4(xb + nb1(g, p0, pos, d, -1)), xp = ld4(xb + nb1(g, p0, pos, d, 1));
        Lx = Lx + ((0.5f * g.is1[d]) * C.at4(1 + 2 * d, p0)) * (xp - xm) +
             (g.is2[d] * C.at4(2 + 2 * d, p0)) * (xp - 2.f * xc + xm);
      }
    } else {
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        float4 a1 = f4(0.f), a2 = f4(0.f);
#pragma unroll
        for (int o = -2; o <= 2; ++o) {
          float w1 = dweight(1, pos[d], g.n[d], g.per[d], o), w2 = dweight(2, pos[d], g.n[d], g.per[d], o);
          if (w1 == 0.f && w2 == 0.f) continue;
          float4 xv = o == 0 ? xc : ld4(xb + nbr(g, p0, pos, d, o));
          a1 = a1 + w1 * xv; a2 = a2 + w2 * xv;
        }
        Lx = Lx + (g.is1[d] * C.at4(1 + 2 * d, p0)) * a1 + (g.is2[d] * C.at4(2 + 2 * d, p0)) * a2;
      }
    }
    // y: central, neighbours from the group plus one value each side
    {
      int row0 = p0 - pos[2];
      float xl = xb[row0 + (pos[2] == 0 ? n2 - 1 : pos[2] - 1)];
      float xr = xb[row0 + (pos[2] + 4 == n2 ? 0 : pos[2] + 4)];
      float4 xm = make_float4(xl, xc.x, xc.y, xc.z), xp = make_float4(xc.y, xc.z, xc.w, xr);
      Lx = Lx + (0.5f * g.is1[2]) * (C.at4(5, p0) * (xp - xm)) + g.is2[2] * (C.at4(6, p0) * (xp - 2.f * xc + xm));
    }
    float4 r4 = ld4(rho + off + p0);
    *reinterpret_cast<float4*>(y + off + p0) = make_float4(-r4.x * Lx.x, -r4.y * Lx.y, -r4.z * Lx.z, -r4.w * Lx.w);
  }
}

template <int MODE>
__global__ void __launch_bounds__(256, 5) k_LTy4(Grid g, Coef cf, StepArgs a) {
  const int b = blockIdx.y;
  const size_t off = (size_t)b * g.N;
  const float* yb = a.y + off;
  const CoefB4 C(cf, b);
  const int NG = g.N >> 2;
  const float inv_ng = 1.f / (float)(g.n[2] >> 2), inv_n1 = 1.f / (float)g.n[1];
  float acc = 0.f;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < NG; q += gridDim.x * blockDim.x) {
    int pos[3]; group_pos(g, q, inv_ng, inv_n1, pos);
    const int p0 = q << 2;
    const int n2 = g.n[2];
    float4 qv;
    bool yedge = !g.per[2] && (pos[2] < 3 || pos[2] + 3 > n2 - 4);
    if (yedge) {
      float t[4];
      for (int k = 0; k < 4; ++k) {
        int pk[3] = {pos[0], pos[1], pos[2] + k};
        t[k] = LTgather<float, 3>(g, cf, b, p0 + k, pk, yb);
      }
      qv = make_float4(t[0], t[1], t[2], t[3]);
    } else {
      float4 yc = ld4(yb + p0);
      qv = C.at4(0, p0) * yc;
      // t and x: rows i = j - o e_d share their position class across the group
      bool txin = pos[0] > 2 && pos[0] < g.n[0] - 3 && (g.per[1] || (pos[1] > 2 && pos[1] < g.n[1] - 3));
      if (txin) {
#pragma unroll
        for (int d = 0; d < 2; ++d) {
          int pm = nb1(g, p0, pos, d, -1), pp = nb1(g, p0, pos, d, 1);
          float4 ym = ld4(yb + pm), yp = ld4(yb + pp);
          qv = qv + (0.5f * g.is1[d]) * (C.at4(1 + 2 * d, pm) * ym - C.at4(1 + 2 * d, pp) * yp) +
               g.is2[d] * (C.at4(2 + 2 * d, pm) * ym - 2.f * (C.at4(2 + 2 * d, p0) * yc) + C.at4(2 + 2 * d, pp) * yp);
        }
      } else
#pragma unroll
      for (int d = 0; d < 2; ++d) {
#pragma unroll
        for (int o = -2; o <= 2; ++o) {
          int ip = pos[d] - o;
          if (g.per[d]) { if (ip < 0) ip += g.n[d]; else if (ip >= g.n[d]) ip -= g.n[d]; }
          else if (ip < 0 || ip >= g.n[d]) continue;
          float w1 = dweight(1, ip, g.n[d], g.per[d], o), w2 = dweight(2, ip, g.n[d], g.per[d], o);
          if (w1 == 0.f && w2 == 0.f) continue;
          int pi = p0 + (ip - pos[d]) * g.stride[d];
          float4 yv = o == 0 ? yc : ld4(yb + pi);
          qv = qv + yv * ((w1 * g.is1[d]) * C.at4(1 + 2 * d, pi) + (w2 * g.is2[d]) * C.at4(2 + 2 * d, pi));
        }
      }
      // y: central rows j-1, j, j+1
      int row0 = p0 - pos[2];
      int pl = row0 + (pos[2] == 0 ? n2 - 1 : pos[2] - 1), pr = row0 + (pos[2] + 4 == n2 ? 0 : pos[2] + 4);
      float4 c1 = C.at4(5, p0), c2 = C.at4(6, p0);
      float yl = yb[pl], yr = yb[pr], c1l = C.at(5, pl), c1r = C.at(5, pr), c2l = C.at(6, pl), c2r = C.at(6, pr);
      float4 ym = make_float4(yl, yc.x, yc.y, yc.z), yp = make_float4(yc.y, yc.z, yc.w, yr);
      float4 c1m = make_float4(c1l, c1.x, c1.y, c1.z), c1p = make_float4(c1.y, c1.z, c1.w, c1r);
      float4 c2m = make_float4(c2l, c2.x, c2.y, c2.z), c2p = make_float4(c2.y, c2.z, c2.w, c2r);
      qv = qv + (0.5f * g.is1[2]) * (c1m * ym - c1p * yp) + g.is2[2] * (c2m * ym - 2.f * (c2 * yc) + c2p * yp);
    }
    float4 xj = ld4(a.x + off + p0);
    // Dirichlet rows: t and x faces are shared by the group, y faces per point
    bool bnd_tx = pos[0] == 0 || (g.final_rows && pos[0] == g.n[0] - 1) ||
                  (!g.per[1] && (pos[1] == 0 || pos[1] == g.n[1] - 1));
    if (bnd_tx) {
      qv = qv - g.theta * xj;
    } else if (!g.per[2]) {
      float t4[4] = {qv.x, qv.y, qv.z, qv.w};
      for (int k = 0; k < 4; ++k) {
        int iy = pos[2] + k;
        if (iy == 0 || iy == n2 - 1) t4[k] -= g.theta * get(xj, k);
      }
      qv = make_float4(t4[0], t4[1], t4[2], t4[3]);
    }
    // qv = -(S x) on the group
    const size_t j = off + p0;
    if (MODE == SM_APPLY) {
      *reinterpret_cast<float4*>(a.out + j) = make_float4(-qv.x, -qv.y, -qv.z, -qv.w);
      acc -= qv.x * xj.x + qv.y * xj.y + qv.z * xj.z + qv.w * xj.w;
    } else if (MODE == SM_RES) {
      *reinterpret_cast<float4*>(a.out + j) = ld4(a.r + j) + qv;
    } else {
      float4 res = ld4(a.r + j) + qv;
      float4 dn = a.c2 * (ld4(a.dinv + j) * res);
      // the previous direction: overwritten below by this thread, so a
      // coherent load (not the read-only path)
      if (MODE == SM_CHEB) dn = dn + a.c1 * __ldcg(reinterpret_cast<const float4*>(a.d + j));
      *reinterpret_cast<float4*>(a.d + j) = dn;
      *reinterpret_cast<float4*>(a.e + j) = xj + dn;
    }
  }
  if (MODE == SM_APPLY && a.part) {
    double s = block_sum((double)acc);
    if (threadIdx.x == 0) a.part[b * MPN_PMAX + blockIdx.x] = s;
  }
}

// D = 2 and n_x % 4 == 0: the same float4 scheme with x (the contiguous axis)
// in the role of y above.  The four points of a group share their position
// class along t, so t neighbours come as float4 rows n_x apart; along x the
// neighbours come from the group plus one value on each side.  A group that
// touches a non-periodic x edge falls back to the scalar formulas point by
// point.  Uniform steps and Dirichlet rows only (as for D = 3).
__device__ __forceinline__ void group_pos2(const Grid& g, int q, float inv_ng, int pos[3]) {
  q = dbg_index(g, q, g.N >> 2, 4);
  int r;
  pos[0] = fdivmod(q, g.n[1] >> 2, inv_ng, r);
  pos[1] = r << 2;
  pos[2] = 0;
}

__device__ __forceinline__ bool xedge2(const Grid& g, const int pos[3]) {
  return !g.per[1] && (pos[1] < 3 || pos[1] + 3 > g.n[1] - 4);
}

__global__ void __launch_bounds__(256, 4) k_Ly4_2(Grid g, Coef cf, const float* __restrict__ rho,
                                               const float* __restrict__ x, float* __restrict__ y) {
  const int b = blockIdx.y;
  const size_t off = (size_t)b * g.N;
  const float* xb = x + off;
  const CoefB4 C(cf, b);
  const int NG = g.N >> 2, n1 = g.n[1];
  const float inv_ng = 1.f / (float)(n1 >> 2);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < NG; q += gridDim.x * blockDim.x) {
    int pos[3]; group_pos2(g, q, inv_ng, pos);
    const int p0 = q << 2;
    if (xedge2(g, pos)) {
      for (int k = 0; k < 4; ++k) {
        int pk[3] = {pos[0], pos[1] + k, 0};
        y[off + p0 + k] = -rho[off + p0 + k] * Lrow<float, 2>(g, cf, b, p0 + k, pk, xb, nullptr);
      }
      continue;
    }
    const float4 xc = ld4(xb + p0);
    float4 Lx = C.at4(0, p0) * xc;
    // t: central forms inside, the one-sided forms on the first and last plane
    if (pos[0] > 0 && pos[0] < g.n[0] - 1) {
      const float4 xm = ld4(xb + dbg_index(g, p0 - n1, g.N - 3, 5)), xp = ld4(xb + dbg_index(g, p0 + n1, g.N - 3, 5));
      Lx = Lx + ((0.5f * g.is1[0]) * C.at4(1, p0)) * (xp - xm) + (g.is2[0] * C.at4(2, p0)) * (xp - 2.f * xc + xm);
    } else {
      float4 a1 = f4(0.f), a2 = f4(0.f);
#pragma unroll
      for (int o = -2; o <= 2; ++o) {
        const float w1 = dweight(1, pos[0], g.n[0], 0, o), w2 = dweight(2, pos[0], g.n[0], 0, o);
        if (w1 == 0.f && w2 == 0.f) continue;
        const float4 xv = o == 0 ? xc : ld4(xb + nbr(g, p0, pos, 0, o));
        a1 = a1 + w1 * xv; a2 = a2 + w2 * xv;
      }
      Lx = Lx + (g.is1[0] * C.at4(1, p0)) * a1 + (g.is2[0] * C.at4(2, p0)) * a2;
    }
    // x: central forms (periodic, or a group away from both faces)
    {
      const int row0 = p0 - pos[1];
      const float xl = xb[row0 + (pos[1] == 0 ? n1 - 1 : pos[1] - 1)];
      const float xr = xb[row0 + (pos[1] + 4 == n1 ? 0 : pos[1] + 4)];
      const float4 xm = make_float4(xl, xc.x, xc.y, xc.z), xp = make_float4(xc.y, xc.z, xc.w, xr);
      Lx = Lx + (0.5f * g.is1[1]) * (C.at4(3, p0) * (xp - xm)) + g.is2[1] * (C.at4(4, p0) * (xp - 2.f * xc + xm));
    }
    const float4 r4 = ld4(rho + off + p0);
    *reinterpret_cast<float4*>(y + off + p0) = make_float4(-r4.x * Lx.x, -r4.y * Lx.y, -r4.z * Lx.z, -r4.w * Lx.w);
  }
}

template <int MODE>
__global__ void __launch_bounds__(256, 5) k_LTy4_2(Grid g, Coef cf, StepArgs a) {
  const int b = blockIdx.y;
  const size_t off = (size_t)b * g.N;
  const float* yb = a.y + off;
  const CoefB4 C(cf, b);
  const int NG = g.N >> 2, n1 = g.n[1];
  const float inv_ng = 1.f / (float)(n1 >> 2);
  float acc = 0.f;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < NG; q += gridDim.x * blockDim.x) {
    int pos[3]; group_pos2(g, q, inv_ng, pos);
    const int p0 = q << 2;
    float4 qv;
    if (xedge2(g, pos)) {
      float t[4];
      for (int k = 0; k < 4; ++k) {
        int pk[3] = {pos[0], pos[1] + k, 0};
        t[k] = LTgather<float, 2>(g, cf, b, p0 + k, pk, yb);
      }
      qv = make_float4(t[0], t[1], t[2], t[3]);
    } else {
      const float4 yc = ld4(yb + p0);
      qv = C.at4(0, p0) * yc;
      // t: rows i = j - o e_t share their position class across the group
      if (pos[0] > 2 && pos[0] < g.n[0] - 3) {
        const int pm = dbg_index(g, p0 - n1, g.N - 3, 5), pp = dbg_index(g, p0 + n1, g.N - 3, 5);
        const float4 ym = ld4(yb + pm), yp = ld4(yb + pp);
        qv = qv + (0.5f * g.is1[0]) * (C.at4(1, pm) * ym - C.at4(1, pp) * yp) +
             g.is2[0] * (C.at4(2, pm) * ym - 2.f * (C.at4(2, p0) * yc) + C.at4(2, pp) * yp);
      } else {
#pragma unroll
        for (int o = -2; o <= 2; ++o) {
          const int ip = pos[0] - o;
          if (ip < 0 || ip >= g.n[0]) continue;
          const float w1 = dweight(1, ip, g.n[0], 0, o), w2 = dweight(2, ip, g.n[0], 0, o);
          if (w1 == 0.f && w2 == 0.f) continue;
          const int pi = dbg_index(g, p0 + (ip - pos[0]) * n1, g.N - 3, 5);
          const float4 yv = o == 0 ? yc : ld4(yb + pi);
          qv = qv + yv * ((w1 * g.is1[0]) * C.at4(1, pi) + (w2 * g.is2[0]) * C.at4(2, pi));
        }
      }
      // x: central rows j-1, j, j+1
      const int row0 = p0 - pos[1];
      const int pl = row0 + (pos[1] == 0 ? n1 - 1 : pos[1] - 1), pr = row0 + (pos[1] + 4 == n1 ? 0 : pos[1] + 4);
      const float4 c1 = C.at4(3, p0), c2 = C.at4(4, p0);
      const float yl = yb[pl], yr = yb[pr], c1l = C.at(3, pl), c1r = C.at(3, pr), c2l = C.at(4, pl), c2r = C.at(4, pr);
      const float4 ym = make_float4(yl, yc.x, yc.y, yc.z), yp = make_float4(yc.y, yc.z, yc.w, yr);
      const float4 c1m = make_float4(c1l, c1.x, c1.y, c1.z), c1p = make_float4(c1.y, c1.z, c1.w, c1r);
      const float4 c2m = make_float4(c2l, c2.x, c2.y, c2.z), c2p = make_float4(c2.y, c2.z, c2.w, c2r);
      qv = qv + (0.5f * g.is1[1]) * (c1m * ym - c1p * yp) + g.is2[1] * (c2m * ym - 2.f * (c2 * yc) + c2p * yp);
    }
    const float4 xj = ld4(a.x + off + p0);
    // Dirichlet rows: the t faces are shared by the group, the x faces per point
    if (pos[0] == 0 || (g.final_rows && pos[0] == g.n[0] - 1)) {
      qv = qv - g.theta * xj;
    } else if (!g.per[1]) {
      float t4[4] = {qv.x, qv.y, qv.z, qv.w};
      for (int k = 0; k < 4; ++k) {
        const int ix = pos[1] + k;
        if (ix == 0 || ix == n1 - 1) t4[k] -= g.theta * get(xj, k);
      }
      qv = make_float4(t4[0], t4[1], t4[2], t4[3]);
    }
    // qv = -(S x) on the group
    const size_t j = off + p0;
    if (MODE == SM_APPLY) {
      *reinterpret_cast<float4*>(a.out + j) = make_float4(-qv.x, -qv.y, -qv.z, -qv.w);
      acc -= qv.x * xj.x + qv.y * xj.y + qv.z * xj.z + qv.w * xj.w;
    } else if (MODE == SM_RES) {
      *reinterpret_cast<float4*>(a.out + j) = ld4(a.r + j) + qv;
    } else {
      const float4 res = ld4(a.r + j) + qv;
      float4 dn = a.c2 * (ld4(a.dinv + j) * res);
      // the previous direction: overwritten below by this thread, so a
      // coherent load (not the read-only path)
      if (MODE == SM_CHEB) dn = dn + a.c1 * __ldcg(reinterpret_cast<const float4*>(a.d + j));
      *reinterpret_cast<float4*>(a.d + j) = dn;
      *reinterpret_cast<float4*>(a.e + j) = xj + dn;
    }
  }
  if (MODE == SM_APPLY && a.part) {
    double s = block_sum((double)acc);
    if (threadIdx.x == 0) a.part[b * MPN_PMAX + blockIdx.x] = s;
  }
}
