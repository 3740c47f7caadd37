// Per-interval steps (Section 2, "discretization": every interval of every
// axis has a step of its own, produced by the encoder and learnable) and the
// gradient of the loss with respect to them (the gradient formula after
// Eq. 11 through the entries of A that depend on the steps).
//
// Rows of position i along axis d with unequal steps (hm = x_i - x_{i-1},
// hp = x_{i+1} - x_i; periodic axes wrap, their last interval closing the
// period):
//   derivative rows (Eq. 5): sbar^k z_k = sbar^k q^(k)(x_i), q the quadratic
//     through three neighbouring points: i-1, i, i+1 inside and on periodic
//     axes (sbar = (hm + hp) / 2), i, i+1, i+2 at the first point of an open
//     axis and i-2, i-1, i at the last (sbar = the adjacent interval);
//   Taylor rows (Eqs. 6-7): u_i + hp u' + hp^2/2 u'' = u_{i+1} and
//     u_i - hm u' + hm^2/2 u'' = u_{i-1} where the neighbour exists.
// A quadratic's Taylor expansion is exact, so with w = (sbar u', sbar^2 u'')
// = q-forms + delta the Taylor rows are p delta_1 + p^2/2 delta_2 (p =
// hp / sbar) and -m delta_1 + m^2/2 delta_2 (m = hm / sbar): the exact
// point-by-point elimination keeps its form, with the position's own
// W = I + v_p v_p^T + v_m v_m^T, v_p = (p, p^2/2), v_m = (-m, m^2/2) (each
// term where its Taylor row exists).  Equal steps give W = [[3, 0], [0, 3/2]]
// inside and [[2, +-1/2], [+-1/2, 5/4]] at the ends.
//
// Multigrid levels: a coarsened periodic axis keeps every second point (a
// coarse interval is the sum of two fine ones); a coarsened open axis puts
// its nc points at the fine fractional indices J (nf - 1) / (nc - 1) (both
// ends kept), each at the coordinate interpolated linearly between the two
// fine points around it.
#pragma once
#include "mpn_device.cuh"

// Value and the partial derivatives with respect to two steps (hA, hB).
struct Dual2 {
  double v, a, b;
};
__device__ __forceinline__ Dual2 dc(double v) { return Dual2{v, 0.0, 0.0}; }
__device__ __forceinline__ Dual2 operator+(Dual2 x, Dual2 y) { return Dual2{x.v + y.v, x.a + y.a, x.b + y.b}; }
__device__ __forceinline__ Dual2 operator-(Dual2 x, Dual2 y) { return Dual2{x.v - y.v, x.a - y.a, x.b - y.b}; }
__device__ __forceinline__ Dual2 operator-(Dual2 x) { return Dual2{-x.v, -x.a, -x.b}; }
__device__ __forceinline__ Dual2 operator*(Dual2 x, Dual2 y) {
  return Dual2{x.v * y.v, x.a * y.v + x.v * y.a, x.b * y.v + x.v * y.b};
}
__device__ __forceinline__ Dual2 operator*(double s, Dual2 y) { return Dual2{s * y.v, s * y.a, s * y.b}; }
__device__ __forceinline__ Dual2 operator/(Dual2 x, Dual2 y) {
  const double iv = 1.0 / y.v;
  const double q = x.v * iv;
  return Dual2{q, (x.a - q * y.a) * iv, (x.b - q * y.b) * iv};
}
// A constant of type T.
template <class T> __device__ __forceinline__ T cst(double v);
template <> __device__ __forceinline__ double cst<double>(double v) { return v; }
template <> __device__ __forceinline__ Dual2 cst<Dual2>(double v) { return dc(v); }

// Local geometry of position i along an axis with n points: the two steps
// its rows depend on, the positions of the three points of its forms
// relative to x_i, the first offset, the row scale and which Taylor rows
// exist with their steps.  T = double, or Dual2 seeded on (hA, hB).
template <class T>
struct Local {
  T X[3];      // coordinates of u at offsets base, base+1, base+2, relative to x_i
  int base;
  T sbar;
  bool has_f, has_b;
  T hp, hm;    // steps of the forward / backward Taylor rows
};

// Interval indices (ia, ib) that position i's rows depend on.
__device__ __forceinline__ void local_idx(int i, int n, int per, int& ia, int& ib, int& cls) {
  if (per) { cls = 0; ia = i == 0 ? n - 1 : i - 1; ib = i; return; }
  if (i == 0) { cls = 1; ia = 0; ib = 1; return; }
  if (i == n - 1) { cls = 2; ia = n - 2; ib = n - 3; return; }
  cls = 0; ia = i - 1; ib = i;
}

template <class T>
__device__ __forceinline__ Local<T> make_local(int cls, T hA, T hB) {
  Local<T> L;
  if (cls == 0) {          // hA = hm, hB = hp
    L.base = -1;
    L.X[0] = -hA; L.X[1] = cst<T>(0.0); L.X[2] = hB;
    L.sbar = 0.5 * (hA + hB);
    L.has_f = L.has_b = true;
    L.hp = hB; L.hm = hA;
  } else if (cls == 1) {   // first point: hA = h_0, hB = h_1
    L.base = 0;
    L.X[0] = cst<T>(0.0); L.X[1] = hA; L.X[2] = hA + hB;
    L.sbar = hA;
    L.has_f = true; L.has_b = false;
    L.hp = hA; L.hm = hA;
  } else {                 // last point: hA = h_{n-2}, hB = h_{n-3}
    L.base = -2;
    L.X[0] = -(hA + hB); L.X[1] = -hA; L.X[2] = cst<T>(0.0);
    L.sbar = hA;
    L.has_f = false; L.has_b = true;
    L.hp = hA; L.hm = hA;
  }
  return L;
}

// Weights of the quadratic through (X_k, u_k) for its first and second
// derivative at 0 (Lagrange basis: l_k(x) = prod_{m != k} (x - X_m) / den_k,
// den_k = prod_{m != k} (X_k - X_m)), times sbar and sbar^2.
template <class T>
__device__ __forceinline__ void form_weights(const Local<T>& L, T w1[3], T w2[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int m0 = k == 0 ? 1 : 0, m1 = k == 2 ? 1 : 2;
    const T den = (L.X[k] - L.X[m0]) * (L.X[k] - L.X[m1]);
    w1[k] = L.sbar * (-(L.X[m0] + L.X[m1]) / den);
    w2[k] = (L.sbar * L.sbar) * (cst<T>(2.0) / den);
  }
}

// Intervals of level k + 1 from those of level k, one thread per (b, d):
// h[(b * 3 + d) * stn + i] (n_d - 1 intervals on open axes, n_d periodic).
__global__ void k_level_steps(Grid gf, Grid gc, int c0, int c1, int c2, const double* __restrict__ hf,
                              double* __restrict__ hc, int B) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * gf.D) return;
  const int b = t / gf.D, d = t % gf.D;
  const int cz = d == 0 ? c0 : (d == 1 ? c1 : c2);
  const int nf = gf.n[d], nc = gc.n[d], per = gf.per[d];
  const double* f = hf + (size_t)(b * 3 + d) * gf.stn;
  double* c = hc + (size_t)(b * 3 + d) * gc.stn;
  const int mf = per ? nf : nf - 1;
  if (!cz) {
    for (int i = 0; i < mf; ++i) c[i] = f[i];
    return;
  }
  if (per) {
    for (int J = 0; J < nc; ++J) c[J] = f[2 * J] + f[2 * J + 1];
    return;
  }
  // open axis: coordinates of the coarse points at fractional fine indices
  double xprev = 0.0;   // coarse point 0 sits on fine point 0
  int i = 0;            // fine interval containing the current coarse point
  double xi = 0.0;      // coordinate of fine point i
  for (int J = 1; J < nc; ++J) {
    const long long num = (long long)J * (nf - 1);
    const int q = (int)(num / (nc - 1));
    const double fr = (double)(num - (long long)q * (nc - 1)) / (double)(nc - 1);
    while (i < q) { xi += f[i]; ++i; }
    const double x = q < nf - 1 ? xi + fr * f[q] : xi;
    c[J - 1] = x - xprev;
    xprev = x;
  }
}

// Step records of one level from its intervals; err[0] is set when an
// interval is not a positive finite number.
__global__ void k_step_table(Grid g, const double* __restrict__ h, double* __restrict__ st64,
                             float* __restrict__ st32, int B, int* __restrict__ err) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * 3 * g.stn) return;
  const int i = t % g.stn, bd = t / g.stn, d = bd % 3, b = bd / 3;
  double* r64 = st64 + (size_t)t * ST_REC;
  float* r32 = st32 + (size_t)t * ST_REC;
  if (d >= g.D || i >= g.n[d]) {
    for (int k = 0; k < ST_REC; ++k) { r64[k] = 0.0; r32[k] = 0.f; }
    return;
  }
  const double* hd = h + (size_t)(b * 3 + d) * g.stn;
  int ia, ib, cls;
  local_idx(i, g.n[d], g.per[d], ia, ib, cls);
  const double hA = hd[ia], hB = hd[ib];
  if (!(hA > 0.0) || !(hB > 0.0) || !isfinite(hA) || !isfinite(hB)) atomicOr(err, 1);
  const Local<double> L = make_local<double>(cls, hA, hB);
  double w1[3], w2[3];
  form_weights<double>(L, w1, w2);
  double W11 = 1.0, W12 = 0.0, W22 = 1.0;
  if (L.has_f) {
    const double p = L.hp / L.sbar, v1 = p, v2 = 0.5 * p * p;
    W11 += v1 * v1; W12 += v1 * v2; W22 += v2 * v2;
  }
  if (L.has_b) {
    const double m = L.hm / L.sbar, v1 = -m, v2 = 0.5 * m * m;
    W11 += v1 * v1; W12 += v1 * v2; W22 += v2 * v2;
  }
  const double idet = 1.0 / (W11 * W22 - W12 * W12);
  double rec[ST_REC];
  for (int k = 0; k < 3; ++k) { rec[ST_W1 + k] = w1[k]; rec[ST_W2 + k] = w2[k]; }
  rec[ST_IS1] = 1.0 / L.sbar;
  rec[ST_IS2] = rec[ST_IS1] * rec[ST_IS1];
  rec[ST_W] = W11; rec[ST_W + 1] = W12; rec[ST_W + 2] = W22;
  rec[ST_WI] = W22 * idet; rec[ST_WI + 1] = -W12 * idet; rec[ST_WI + 2] = W11 * idet;
  rec[ST_BASE] = (double)L.base;
  rec[ST_BASE + 1] = 0.0;
  for (int k = 0; k < ST_REC; ++k) { r64[k] = rec[k]; r32[k] = (float)rec[k]; }
}

// Level-0 intervals (FP64, [B][3][stn]) from the caller's FP32 steps, laid
// out axis by axis: [B][m_0], then [B][m_1] (, [B][m_2]).
// err[0] is set when a step is not a positive finite number.
__global__ void k_steps_in(Grid g, const float* __restrict__ in, double* __restrict__ h, int B,
                           int* __restrict__ err) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * 3 * g.stn) return;
  const int i = t % g.stn, bd = t / g.stn, d = bd % 3, b = bd / 3;
  double v = 0.0;
  if (d < g.D) {
    size_t off = 0;
    for (int e = 0; e < d; ++e) off += (size_t)B * (g.per[e] ? g.n[e] : g.n[e] - 1);
    const int m = g.per[d] ? g.n[d] : g.n[d] - 1;
    if (i < m) {
      v = (double)in[off + (size_t)b * m + i];
      if (!(v > 0.0) || !isfinite(v)) atomicOr(err, 1);
    }
  }
  h[t] = v;
}

// The rows of position i along d owned by point p, applied to x (z or d_z,
// [V][N] of one instance) as functions of the local steps:
// out[0..3] = D1, D2, TF, TB (zero where the row does not exist).
__device__ __forceinline__ void rows_at(const Grid& g, int d, int p, int i, const Local<Dual2>& L,
                                        const Dual2 w1[3], const Dual2 w2[3], const double* __restrict__ x,
                                        Dual2 out[4]) {
  const int N = g.N, s = g.stride[d], n = g.n[d];
  auto at = [&](int o) {   // u at offset o along d
    int c = i + o;
    if (g.per[d]) c = wrap1(c, n);
    return x[p + (c - i) * s];
  };
  const double z1 = x[(size_t)(1 + 2 * d) * N + p], z2 = x[(size_t)(2 + 2 * d) * N + p];
  Dual2 a1 = dc(0.0), a2 = dc(0.0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double uk = at(L.base + k);
    a1 = a1 + uk * w1[k];
    a2 = a2 + uk * w2[k];
  }
  out[0] = z1 * L.sbar - a1;
  out[1] = z2 * (L.sbar * L.sbar) - a2;
  const double u0 = x[p];
  out[2] = L.has_f ? dc(u0 - at(1)) + z1 * L.hp + z2 * (0.5 * (L.hp * L.hp)) : dc(0.0);
  out[3] = L.has_b ? dc(u0 - at(-1)) - z1 * L.hm + z2 * (0.5 * (L.hm * L.hm)) : dc(0.0);
}

// dl/dh for every interval (the gradient formula after Eq. 11): with
// lambda = d - A z* and d_lambda = -A d_z, and d independent of the steps,
//   dl/dh_k = sum over entries (d_lambda_r z_c + lambda_r dz_c) dA_rc/dh_k
//           = -sum over rows r of d(f_r g_r)/dh_k,  f = A z*, g = A d_z,
// the derivatives taken with z*, d_z fixed.  Only the derivative and Taylor
// rows depend on the steps.  One CTA per (instance, axis, interval): it sums
// over the points whose rows use that interval, in a fixed order.
// z, dz: [B][V][N] FP64.  out: the caller's layout of the steps (FP32).
__global__ void k_step_grads(Grid g, const double* __restrict__ h, const double* __restrict__ z,
                             const double* __restrict__ dz, float* __restrict__ out, int B) {
  const int b = blockIdx.z, d = blockIdx.y, k = blockIdx.x;
  const int n = g.n[d], per = g.per[d];
  const int m = per ? n : n - 1;
  if (d >= g.D || k >= m) return;
  const int V = 1 + 2 * g.D;
  const double* hd = h + (size_t)(b * 3 + d) * g.stn;
  const double* zb = z + (size_t)b * V * g.N;
  const double* db = dz + (size_t)b * V * g.N;
  // positions whose rows use interval k (distinct)
  int cand[4], nc = 0;
  auto add = [&](int j) {
    if (j < 0 || j >= n) return;
    for (int q = 0; q < nc; ++q) if (cand[q] == j) return;
    cand[nc++] = j;
  };
  add(k);
  add(per ? (k + 1) % n : k + 1);
  if (!per) { add(0); add(n - 1); }
  // the other axes: points of the hyperplane orthogonal to d
  const int o1 = d == 0 ? 1 : 0, o2 = d == 2 ? 1 : 2;
  const int n1 = g.n[o1], n2 = g.D == 3 ? g.n[o2] : 1;
  const int nplane = n1 * n2;
  double acc = 0.0;
  for (int c = 0; c < nc; ++c) {
    const int j = cand[c];
    int ia, ib, cls;
    local_idx(j, n, per, ia, ib, cls);
    const bool use_a = ia == k, use_b = ib == k;
    if (!use_a && !use_b) continue;
    const Dual2 hA = Dual2{hd[ia], 1.0, 0.0}, hB = Dual2{hd[ib], 0.0, 1.0};
    const Local<Dual2> L = make_local<Dual2>(cls, hA, hB);
    Dual2 w1[3], w2[3];
    form_weights<Dual2>(L, w1, w2);
    for (int t = threadIdx.x; t < nplane; t += blockDim.x) {
      const int a1 = t / n2, a2 = t - a1 * n2;
      int pos[3];
      pos[d] = j; pos[o1] = a1;
      if (g.D == 3) pos[o2] = a2;
      else pos[2] = 0;
      const int p = pos[0] * g.stride[0] + pos[1] * g.stride[1] + (g.D == 3 ? pos[2] * g.stride[2] : 0);
      Dual2 f[4], r[4];
      rows_at(g, d, p, j, L, w1, w2, zb, f);
      rows_at(g, d, p, j, L, w1, w2, db, r);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (use_a) acc -= f[q].a * r[q].v + f[q].v * r[q].a;
        if (use_b) acc -= f[q].b * r[q].v + f[q].v * r[q].b;
      }
    }
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) {
    size_t off = 0;
    for (int e = 0; e < d; ++e) off += (size_t)B * (g.per[e] ? g.n[e] : g.n[e] - 1);
    out[off + (size_t)b * m + k] = (float)s;
  }
}
