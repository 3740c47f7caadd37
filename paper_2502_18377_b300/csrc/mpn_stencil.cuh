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

enum { SM_POST0 = 0, SM_CHEB = 1, SM_RES = 2, SM_APPLY = 3 };

struct StepArgs {
  const float* x;     // operand of S (pass 1 and the theta 1_B term)
  const float* y;     // pass-1 output
  const float* r;     // right-hand side at this level
  const float* dinv;  // Chebyshev-scaled inverse diagonal
  float* e;           // iterate (modes 0, 1: updated in place; it is x)
  float* d;           // direction (modes 0, 1)
  float* out;         // mode 2: r - S x;  mode 3: S x
  double* part;       // mode 3: partials of <x, S x> (nullable)
  float c1, c2;
};

// p -> (t, x, y) without integer division (exact for p < 2^21).
__device__ __forceinline__ void decode_f(const Grid& g, int p, float inv12, float inv2, int pos[3]) {
  int n12 = g.n[1] * g.n[2];
  int i0 = __float2int_rz(((float)p + 0.5f) * inv12);
  int rem = p - i0 * n12;
  int i1 = __float2int_rz(((float)rem + 0.5f) * inv2);
  pos[0] = i0; pos[1] = i1; pos[2] = rem - i1 * g.n[2];
}

// Neighbour at offset +-1 along d for an interior/periodic coordinate.
__device__ __forceinline__ int nb1(const Grid& g, int p, const int pos[3], int d, int o) {
  int c = pos[d] + o;
  int s = g.stride[d];
  if (c < 0) return p + (g.n[d] - 1) * s;
  if (c >= g.n[d]) return p - (g.n[d] - 1) * s;
  return p + o * s;
}

template <int D>
__device__ __forceinline__ bool edge_any(const Grid& g, const int pos[3]) {
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
    }
    float xj = a.x[off + p];
    if (is_boundary_t<D>(g, pos)) q -= g.theta * xj;
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
