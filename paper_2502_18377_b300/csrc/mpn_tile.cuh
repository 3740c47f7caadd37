// Fused application of the reduced normal operator S = L^T diag(rho) L + theta 1_B
// on a shared-memory tile: every Chebyshev smoothing step, multigrid residual
// and PCG operator apply (FP32), and the refinement residual (FP64).
//
// One CTA owns a T0 x T1 x T2 tile of one instance (T2 along the contiguous
// dimension).  It stages on a box with a halo of two points per active
// dimension:  x (the iterate), rho and the coefficient fields, then
// y = rho (src - L x) on the box wherever the L stencil fits in it, and finally
// gathers (L^T y)_j + theta 1_B x_j for its own points.  Rows at distance two
// from a tile point only matter for one-sided edge rows, whose stencils reach
// inward and therefore always fit.  Inputs are read from one buffer and
// results written to another (neighbouring CTAs read the same points as halo).
//
// Box cells are visited by a flat loop, four cells per thread per batch with
// all loads of the batch issued before the shared-memory stores, so each warp
// keeps several global loads in flight.  Points away from non-periodic edges
// take the central three-point weights directly; edge points use the general
// one-sided weights.
#pragma once
#include "mpn_device.cuh"

enum { TM_POST0 = 0, TM_CHEB = 1, TM_RES = 2, TM_APPLY = 3, TM_RES64 = 4 };

template <class T>
struct TileArgs {
  const T* ein;       // x = ein (+ din); null => x = 0
  const T* din;       // nullable
  const float* r;     // FP32 right-hand side at this level (modes 0-2)
  const T* rho;
  const float* dinv;
  const float* src;   // mode 4: b of the equation rows (nullable)
  const float* omega; // mode 4: Dirichlet values (nullable)
  const T* base;      // mode 4: added to the output (nullable)
  T* eout;            // mode 1, 2: x written here
  T* dout;            // mode 0, 1
  T* out;             // mode 2: r - S x;  mode 3: S x;  mode 4: base + L^T y + theta 1_B (omega - x)
  double* part;       // mode 3: partials of <x, S x>;  mode 4: of ||out||^2 (nullable)
  float c1, c2;
  int tile[3];
  int ntile[3];
};

__device__ __forceinline__ int wrap_or_invalid(int c, int n, int per, bool& valid) {
  if (per) { if (c < 0) c += n; else if (c >= n) c -= n; return c; }
  if (c < 0 || c >= n) valid = false;
  return c;
}

// A coordinate needs the general (edge-aware) weights when a one-sided row is
// within two points of it along a non-periodic dimension.
__device__ __forceinline__ bool near_edge(int c, int n, int per) { return !per && (c < 3 || c > n - 4); }

// floor(c / B) for small non-negative c (exact for c < 2^21).
__device__ __forceinline__ int fdiv(int c, float invB) { return __float2int_rz(((float)c + 0.5f) * invB); }

template <int D, class T>
__global__ void __launch_bounds__(256, 3) k_tile(Grid g, Coef cf, TileArgs<T> a, int mode) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int H2 = (D == 3) ? 2 : 0;
  constexpr int V = 1 + 2 * D;
  const int T0 = a.tile[0], T1 = a.tile[1], T2 = a.tile[2];
  const int B0 = T0 + 4, B1 = T1 + 4, B2 = T2 + 2 * H2;
  const int B12 = B1 * B2;
  const int nbox = B0 * B12;
  const float invB12 = 1.f / (float)B12, invB2 = 1.f / (float)B2;
  const int sb0 = B12, sb1 = B2;
  T* xs = (T*)smraw;
  T* ys = xs + nbox;
  T* rs = ys + nbox;
  float* fs = (float*)(rs + nbox);
  __shared__ float scal[7];
  __shared__ int fof[7];
  const int b = blockIdx.y;
  int tl = blockIdx.x;
  const int o2 = (tl % a.ntile[2]) * T2; tl /= a.ntile[2];
  const int o1 = (tl % a.ntile[1]) * T1; tl /= a.ntile[1];
  const int o0 = tl * T0;
  const size_t off = (size_t)b * g.N;
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const int per1 = g.per[1], per2 = g.per[2];
  if (threadIdx.x < V) {
    fof[threadIdx.x] = cf.field_of[threadIdx.x];
    scal[threadIdx.x] = cf.field_of[threadIdx.x] < 0 ? cf.scalars[threadIdx.x * cf.B + b] : 0.f;
  }
  const int F = cf.F;
  const bool has_src = (mode == TM_RES64) && a.src;

  // 1. stage x, rho, (src) and the coefficient fields on the box
  constexpr int U = 4;
  for (int c0b = threadIdx.x; c0b < nbox; c0b += U * blockDim.x) {
    int qv[U];
    bool vv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int c = c0b + u * blockDim.x;
      bool v = c < nbox;
      int q = 0;
      if (v) {
        int i0 = fdiv(c, invB12), rem = c - i0 * B12;
        int i1 = fdiv(rem, invB2), i2 = rem - i1 * B2;
        int g0 = wrap_or_invalid(o0 + i0 - 2, n0, 0, v);
        int g1 = wrap_or_invalid(o1 + i1 - 2, n1, per1, v);
        int g2 = D == 3 ? wrap_or_invalid(o2 + i2 - H2, n2, per2, v) : 0;
        q = (g0 * n1 + g1) * n2 + g2;
      }
      qv[u] = q; vv[u] = v;
    }
    T xv[U], rv[U], sv[U];
    float fv[U][2];   // the first two coefficient fields are batched with x and rho
#pragma unroll
    for (int u = 0; u < U; ++u) {
      xv[u] = 0; rv[u] = 0; sv[u] = 0;
      if (vv[u]) {
        size_t j = off + qv[u];
        if (a.ein) xv[u] = a.ein[j];
        if (a.din) xv[u] += a.din[j];
        rv[u] = a.rho[j];
        if (has_src) sv[u] = (T)a.src[j];
      }
#pragma unroll
      for (int f = 0; f < 2; ++f)
        fv[u][f] = (f < F && vv[u]) ? __ldg(cf.fields + ((size_t)f * cf.B + b) * g.N + qv[u]) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int c = c0b + u * blockDim.x;
      if (c < nbox) {
        xs[c] = xv[u]; rs[c] = rv[u]; ys[c] = sv[u];
#pragma unroll
        for (int f = 0; f < 2; ++f)
          if (f < F) fs[f * nbox + c] = fv[u][f];
        for (int f = 2; f < F; ++f)
          fs[f * nbox + c] = vv[u] ? __ldg(cf.fields + ((size_t)f * cf.B + b) * g.N + qv[u]) : 0.f;
      }
    }
  }
  __syncthreads();
  auto coef = [&](int v, int c) -> T {
    int f = fof[v];
    return (T)(f >= 0 ? fs[f * nbox + c] : scal[v]);
  };
  const T is1[3] = {(T)(sizeof(T) == 8 ? g.ds1[0] : g.is1[0]), (T)(sizeof(T) == 8 ? g.ds1[1] : g.is1[1]),
                    (T)(sizeof(T) == 8 ? g.ds1[2] : g.is1[2])};
  const T is2[3] = {(T)(sizeof(T) == 8 ? g.ds2[0] : g.is2[0]), (T)(sizeof(T) == 8 ? g.ds2[1] : g.is2[1]),
                    (T)(sizeof(T) == 8 ? g.ds2[2] : g.is2[2])};

  // 2. y = rho (src - L x) on the box where the stencil fits (in place over src)
  for (int c = threadIdx.x; c < nbox; c += blockDim.x) {
    int i0 = fdiv(c, invB12), rem = c - i0 * B12;
    int i1 = fdiv(rem, invB2), i2 = rem - i1 * B2;
    bool v = true;
    int g0 = wrap_or_invalid(o0 + i0 - 2, n0, 0, v);
    int g1 = wrap_or_invalid(o1 + i1 - 2, n1, per1, v);
    int g2 = D == 3 ? wrap_or_invalid(o2 + i2 - H2, n2, per2, v) : 0;
    T yv = 0;
    if (v) {
      bool edge = near_edge(g0, n0, 0) || near_edge(g1, n1, per1) || (D == 3 && near_edge(g2, n2, per2));
      T xc = xs[c];
      T acc = coef(0, c) * xc;
      bool ok = true;
      if (!edge) {
        bool inside = i0 >= 1 && i0 <= B0 - 2 && i1 >= 1 && i1 <= B1 - 2 && (D == 2 || (i2 >= 1 && i2 <= B2 - 2));
        if (!inside) ok = false;
        else {
          const int sd[3] = {sb0, sb1, 1};
#pragma unroll
          for (int d = 0; d < D; ++d) {
            T xm = xs[c - sd[d]], xp = xs[c + sd[d]];
            acc += coef(1 + 2 * d, c) * ((T)0.5 * (xp - xm)) * is1[d] + coef(2 + 2 * d, c) * (xp - (T)2 * xc + xm) * is2[d];
          }
        }
      } else {
        const int gp[3] = {g0, g1, g2};
        const int cc[3] = {i0, i1, i2};
        const int Bd[3] = {B0, B1, B2};
        const int sd[3] = {sb0, sb1, 1};
#pragma unroll
        for (int d = 0; d < D; ++d) {
          T cv1 = coef(1 + 2 * d, c), cv2 = coef(2 + 2 * d, c);
          T a1 = 0, a2 = 0;
#pragma unroll
          for (int o = -2; o <= 2; ++o) {
            float w1 = dweight(1, gp[d], g.n[d], g.per[d], o), w2 = dweight(2, gp[d], g.n[d], g.per[d], o);
            if (w1 == 0.f && w2 == 0.f) continue;
            int cb = cc[d] + o;
            if (cb < 0 || cb >= Bd[d]) { ok = false; continue; }
            T xv = xs[c + o * sd[d]];
            a1 += (T)w1 * xv; a2 += (T)w2 * xv;
          }
          acc += cv1 * a1 * is1[d] + cv2 * a2 * is2[d];
        }
      }
      if (ok) yv = rs[c] * (ys[c] - acc);
    }
    ys[c] = yv;
  }
  __syncthreads();

  // 3. out_j = (L^T y)_j - theta 1_B x_j  (= -S x_j when src = 0); per mode
  double acc_part = 0.0;
  const int ntp = T0 * T1 * T2;
  const float invT12 = 1.f / (float)(T1 * T2), invT2 = 1.f / (float)T2;
  for (int t = threadIdx.x; t < ntp; t += blockDim.x) {
    int k0 = fdiv(t, invT12), rem = t - k0 * (T1 * T2);
    int k1 = fdiv(rem, invT2), k2 = rem - k1 * T2;
    int g0 = o0 + k0, g1 = o1 + k1, g2 = o2 + k2;
    if (g0 >= n0 || g1 >= n1 || g2 >= n2) continue;
    int cb = ((k0 + 2) * B1 + (k1 + 2)) * B2 + (k2 + H2);
    T q = coef(0, cb) * ys[cb];
    bool edge = near_edge(g0, n0, 0) || near_edge(g1, n1, per1) || (D == 3 && near_edge(g2, n2, per2));
    const int sd[3] = {sb0, sb1, 1};
    if (!edge) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        int cm = cb - sd[d], cp = cb + sd[d];
        T ym = ys[cm], yp = ys[cp], yc = ys[cb];
        q += (T)0.5 * is1[d] * (coef(1 + 2 * d, cm) * ym - coef(1 + 2 * d, cp) * yp) +
             is2[d] * (coef(2 + 2 * d, cm) * ym - (T)2 * coef(2 + 2 * d, cb) * yc + coef(2 + 2 * d, cp) * yp);
      }
    } else {
      const int gp[3] = {g0, g1, g2};
#pragma unroll
      for (int d = 0; d < D; ++d) {
#pragma unroll
        for (int o = -2; o <= 2; ++o) {
          bool vi = true;
          int ip = wrap_or_invalid(gp[d] - o, g.n[d], g.per[d], vi);
          if (!vi) continue;
          float w1 = dweight(1, ip, g.n[d], g.per[d], o), w2 = dweight(2, ip, g.n[d], g.per[d], o);
          if (w1 == 0.f && w2 == 0.f) continue;
          int ci = cb - o * sd[d];
          q += ys[ci] * (coef(1 + 2 * d, ci) * (T)w1 * is1[d] + coef(2 + 2 * d, ci) * (T)w2 * is2[d]);
        }
      }
    }
    T xj = xs[cb];
    const int gp[3] = {g0, g1, g2};
    bool bnd = is_boundary_t<D>(g, gp);
    size_t j = off + (g0 * n1 + g1) * n2 + g2;
    if (mode == TM_RES64) {
      if (bnd) q += (T)g.theta * ((a.omega ? (T)a.omega[j] : (T)0) - xj);
      if (a.base) q += a.base[j];
      a.out[j] = q;
      acc_part += (double)q * (double)q;
      continue;
    }
    if (bnd) q -= (T)g.theta * xj;
    // here q = -(S x)_j
    if (mode == TM_APPLY) {
      a.out[j] = -q;
      acc_part -= (double)q * (double)xj;
      continue;
    }
    float res = a.r[j] + (float)q;
    if (mode == TM_POST0) {
      a.dout[j] = (T)(a.c2 * a.dinv[j] * res);
    } else if (mode == TM_CHEB) {
      a.eout[j] = xj;
      a.dout[j] = (T)(a.c1 * (float)a.din[j] + a.c2 * a.dinv[j] * res);
    } else {
      a.eout[j] = xj;
      a.out[j] = (T)res;
    }
  }
  if ((mode == TM_APPLY || mode == TM_RES64) && a.part) {
    double s = block_sum(acc_part);
    if (threadIdx.x == 0) a.part[b * MPN_PMAX + blockIdx.x] = s;
  }
}
