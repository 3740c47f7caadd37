// Device-side building blocks of the NeuRLP-PDE solver: grid geometry,
// coefficient access, the difference weights of the derivative rows (Eq. 5,
// three-point central, second-order one-sided at non-periodic edges) and the
// per-point algebra of the eliminated derivative unknowns.
//
// Reduced normal equations.  The derivative unknowns of point i appear only
// in the rows owned by i (its equation row, Eq. 3, and its derivative and
// Taylor rows, Eqs. 5-7), so they are eliminated exactly from A^T A z = A^T d
// (Eq. 9), point by point.  In the scaled unknowns w = (s u', s^2 u'') of one
// dimension, the Taylor rows equal D1 + D2/2 and -D1 + D2/2 as functionals,
// so the rows of dimension d contribute delta^T W delta with
// delta = w - a(u) (a = the difference forms of Eq. 5) and
//   W = [[3, 0], [0, 3/2]]         interior / periodic (D1, D2, TF, TB)
//   W = [[2, 1/2], [1/2, 5/4]]     first point of a non-periodic dim (no TB)
//   W = [[2, -1/2], [-1/2, 5/4]]   last point (no TF).
// With beta = (c_{1+2d}/s_d, c_{2+2d}/s_d^2) and e = L_i u - b_i (L the
// finite-difference operator with the same difference forms), minimising over
// delta gives the point weight rho_i = 1 / (1 + sum_d beta_d^T W_d^{-1} beta_d)
// and the u-only system
//   S u = L^T rho (b - ...) ,  S = L^T diag(rho) L + diag(1_B)
// (Schur complement of A^T A onto u), solved here by multigrid PCG.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define MPN_TPB 256
#define GRID_LOOP(p, N) for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < (N); p += gridDim.x * blockDim.x)
#define MPN_PMAX 4096  // partial sums per instance (max CTAs per instance)

// Coefficient layouts fixed at compile time (bit v: c_v is a field, else a
// per-instance scalar).  FS_ANY: the layout is read at run time.
#define FS_ANY 0x80
// c_yy reads the field of c_xx (isotropic diffusion)
#define FS_SHARE46 0x100
// reaction-diffusion: c_0, c_xx, c_yy fields
#define FS_MASK_RD ((1 << 0) | (1 << 4) | (1 << 6))
#define FS_MASK_RDI (FS_MASK_RD | FS_SHARE46)
// transport: the velocity fields c_x, c_y
#define FS_MASK_TR ((1 << 3) | (1 << 5))

struct Grid {
  int D;          // 2 or 3
  int n[3];       // n[2] = 1 when D = 2
  int per[3];     // periodic flags (per[0] = 0)
  int stride[3];  // point-index strides
  int N;          // points per instance
  int final_rows; // Dirichlet rows on t = t_f
  float theta;    // weight of the Dirichlet rows at this level
  float is1[3], is2[3];    // 1/s, 1/s^2
  double ds1[3], ds2[3];   // 1/s, 1/s^2 in FP64
  float inv_pl, inv_n2;    // 1 / (n[1] n[2]), 1 / n[2] (index decoding)
  // Per-interval steps (null: the uniform steps above).  One record of
  // ST_REC values per (instance, dimension, position), FP64 and FP32 copies:
  // record (b, d, i) at ((b * 3 + d) * stn + i) * ST_REC.
  const double* st64;
  const float* st32;
  int stn;
  // Neumann / mixed boundary rows alpha u + beta du/dx_d = omega on both
  // faces of spatial axis d where bcm[d] (the time faces and the other axes
  // keep Dirichlet rows).  Their point weights (the 2x2 matrix R of the
  // equation and boundary rows of a face point) live in per-level arrays:
  // rho holds R11, r12 / r22 the rest (zero off those points), y2 receives
  // the boundary-row part of the first operator pass; r12d / r22d / y2d are
  // the FP64 copies of the finest level.
  int mixed;
  int bcm[3];
  float bca[3], bcb[3];
  const float* r12;
  const float* r22;
  float* y2;
  const double* r12d;
  const double* r22d;
  double* y2d;
  // Bounds-checked build (MPN_DEBUG): device word receiving the code of the
  // first out-of-range index a kernel computed (null: nothing recorded).
  int* dbg;
};

// Index check of the bounds-checked build: an index outside [0, n) records
// `code` in g.dbg (first one wins) and is replaced by 0, so the access stays
// in bounds and the kernel runs on; release builds return i unchanged.
__device__ __forceinline__ int dbg_index(const Grid& g, int i, int n, int code) {
#ifdef MPN_DEBUG
  if ((unsigned)i >= (unsigned)n) {
    if (g.dbg) atomicCAS(g.dbg, 0, code);
    return 0;
  }
#endif
  (void)g; (void)n; (void)code;
  return i;
}

// Step record of one grid position along one dimension (per-interval steps).
// In the scaled unknowns w = (sbar u', sbar^2 u'') of the position, with
// sbar the scale of its derivative rows:
//   [ST_W1 + k], [ST_W2 + k]  weights of u at offset ST_BASE + k (k < 3) in
//                            sbar u' and sbar^2 u'' (the difference forms)
//   [ST_IS1], [ST_IS2]       1 / sbar, 1 / sbar^2
//   [ST_W .. ST_W + 2]       W = (w11, w12, w22), the quadratic form of the
//                            position's derivative and Taylor rows in delta
//   [ST_WI .. ST_WI + 2]     W^{-1}
//   [ST_BASE]                first offset of the forms: -1 inside or periodic,
//                            0 at the first point, -2 at the last
#define ST_REC 16
#define ST_W1 0
#define ST_W2 3
#define ST_IS1 6
#define ST_IS2 7
#define ST_W 8
#define ST_WI 11
#define ST_BASE 14

// Host: the reciprocals decode_fast() reads.
inline void grid_set_inverses(Grid& g) {
  g.inv_pl = 1.f / (float)(g.n[1] * g.n[2]);
  g.inv_n2 = 1.f / (float)g.n[2];
}

struct Coef {
  int V, F, B;
  int field_of[7];
  const float* fields;   // [F][B][N] at this level
  const float* scalars;  // [V][B]
  // c_v at (b, p) = ptr[v][b * bstride[v] + p * pstride[v]]: a field has
  // strides (N, 1), a per-instance scalar (1, 0).
  const float* ptr[7];
  int bstride[7], pstride[7];
  // the same with per-instance scalars stored 4 times ([V][B][4]), so that a
  // float4 load at stride 0 reads a scalar: c_v as float4 at (b, p) =
  // ptr4[v][b * bstride4[v] + p * pstride[v]]
  const float* ptr4[7];
  int bstride4[7];
};

__device__ __forceinline__ float coefv(const Coef& c, int v, int b, int p, int N) {
  (void)N;
  return __ldg(c.ptr[v] + (size_t)b * c.bstride[v] + (size_t)p * c.pstride[v]);
}

// Coefficient access with the instance offset hoisted out of point loops.
struct CoefB {
  const float* base[7];
  int ps[7];
  __device__ __forceinline__ CoefB(const Coef& c, int b, int V) {
#pragma unroll
    for (int v = 0; v < 7; ++v) {
      base[v] = v < V ? c.ptr[v] + (size_t)b * c.bstride[v] : nullptr;
      ps[v] = v < V ? c.pstride[v] : 0;
    }
  }
  __device__ __forceinline__ float operator()(int v, int p) const { return __ldg(base[v] + p * ps[v]); }
};

// a = q / n, r = q mod n (0 <= q, 1 <= n) without an integer division: a
// float estimate that is off by at most one while the quotient is below 2^21,
// corrected by one step.
__device__ __forceinline__ int fdivmod(int q, int n, float inv_n, int& r) {
  int a = __float2int_rz(((float)q + 0.5f) * inv_n);
  r = q - a * n;
  if (r < 0) { --a; r += n; }
  else if (r >= n) { ++a; r -= n; }
  return a;
}

// Point index -> (t, x, y) without an integer division; any_edge: the point is within 2 of a
// time edge or of a non-periodic spatial edge (one-sided forms nearby).
__device__ __forceinline__ void decode_fast(const Grid& g, int p, int pos[3]) {
  p = dbg_index(g, p, g.N, 3);
  int rem, i2;
  pos[0] = fdivmod(p, g.n[1] * g.n[2], g.inv_pl, rem);
  pos[1] = fdivmod(rem, g.n[2], g.inv_n2, i2);
  pos[2] = i2;
}
// Per-interval steps and Neumann / mixed rows count as edges everywhere:
// only the general forms read the step records and the boundary rows.
__device__ __forceinline__ bool any_edge(const Grid& g, const int pos[3]) {
  if (g.st64 || g.mixed) return true;
  bool e = pos[0] < 3 || pos[0] > g.n[0] - 4;
  for (int d = 1; d < 3; ++d)
    if (d < g.D && !g.per[d]) e |= pos[d] < 3 || pos[d] > g.n[d] - 4;
  return e;
}

// c wrapped into [0, n) for -n <= c < 2n: every periodic neighbour offset
// is at most 2 and every extent at least 3, so one add or subtract suffices.
__device__ __forceinline__ int wrap1(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

// Point index of the neighbour at offset o along d (wrapping when periodic).
// The caller guarantees the target exists for non-periodic dims.
__device__ __forceinline__ int nbr(const Grid& g, int p, const int pos[3], int d, int o) {
  int c = pos[d] + o;
  if (g.per[d]) c = wrap1(c, g.n[d]);
  return dbg_index(g, p + (c - pos[d]) * g.stride[d], g.N, 1);
}

// Weight of u_{pos+o} in the difference form of order `order` at coordinate
// `pos` (Eq. 5): s^order * u^(order) = sum_o w(o) u_{pos+o}.
__device__ __forceinline__ float dweight(int order, int pos, int n, int per, int o) {
  if (per || (pos > 0 && pos < n - 1)) {
    if (order == 1) return o == -1 ? -0.5f : (o == 1 ? 0.5f : 0.f);
    return o == 0 ? -2.f : ((o == 1 || o == -1) ? 1.f : 0.f);
  }
  if (pos == 0) {
    if (order == 1) return o == 0 ? -1.5f : (o == 1 ? 2.f : (o == 2 ? -0.5f : 0.f));
    return o == 0 ? 1.f : (o == 1 ? -2.f : (o == 2 ? 1.f : 0.f));
  }
  if (order == 1) return o == 0 ? 1.5f : (o == -1 ? -2.f : (o == -2 ? 0.5f : 0.f));
  return o == 0 ? 1.f : (o == -1 ? -2.f : (o == -2 ? 1.f : 0.f));
}

// 0 interior/periodic, 1 first point, 2 last point of a non-periodic dim.
__device__ __forceinline__ int edge_class(const Grid& g, int d, int pos) {
  if (g.per[d]) return 0;
  return pos == 0 ? 1 : (pos == g.n[d] - 1 ? 2 : 0);
}

__device__ __forceinline__ bool is_boundary(const Grid& g, const int pos[3]) {
  if (pos[0] == 0) return true;
  if (g.final_rows && pos[0] == g.n[0] - 1) return true;
  for (int d = 1; d < g.D; ++d)
    if (!g.per[d] && (pos[d] == 0 || pos[d] == g.n[d] - 1)) return true;
  return false;
}

// Axis of the boundary row of a point: -1 none, 0 a time face (Dirichlet),
// d >= 1 a face of spatial axis d.  A point on several faces has the row of
// the first in the order t = 0, t = t_f, then the spatial axes in order.
__device__ __forceinline__ int bc_axis(const Grid& g, const int pos[3]) {
  if (pos[0] == 0 || (g.final_rows && pos[0] == g.n[0] - 1)) return 0;
  for (int d = 1; d < g.D; ++d)
    if (!g.per[d] && (pos[d] == 0 || pos[d] == g.n[d] - 1)) return d;
  return -1;
}
// The spatial axis of the point's Neumann / mixed row, or -1.
__device__ __forceinline__ int mixed_axis(const Grid& g, const int pos[3]) {
  if (!g.mixed) return -1;
  const int e = bc_axis(g, pos);
  return (e >= 1 && g.bcm[e]) ? e : -1;
}
// The point has a Dirichlet row (weight theta in the reduced operator).
__device__ __forceinline__ bool dirichlet_point(const Grid& g, const int pos[3]) {
  return is_boundary(g, pos) && mixed_axis(g, pos) < 0;
}

template <int D>
__device__ __forceinline__ bool is_boundary_t(const Grid& g, const int pos[3]) {
  bool bnd = pos[0] == 0 || (g.final_rows && pos[0] == g.n[0] - 1);
#pragma unroll
  for (int d = 1; d < D; ++d)
    bnd |= !g.per[d] && (pos[d] == 0 || pos[d] == g.n[d] - 1);
  return bnd;
}

// W_d for the edge class (symmetric 2x2: w11, w12, w22).
__device__ __forceinline__ void wmat(int cls, double& w11, double& w12, double& w22) {
  if (cls == 0) { w11 = 3.0; w12 = 0.0; w22 = 1.5; }
  else { w11 = 2.0; w12 = cls == 1 ? 0.5 : -0.5; w22 = 1.25; }
}

// W_d^{-1} x (no divisions: FP64 division is slow on this part).
template <class R>
__device__ __forceinline__ void winv(int cls, R x1, R x2, R& y1, R& y2) {
  if (cls == 0) { y1 = x1 * (R)(1.0 / 3.0); y2 = x2 * (R)(2.0 / 3.0); return; }
  const R k = (R)(1.0 / 2.25);
  R sg = cls == 1 ? (R)1 : (R)-1;
  y1 = ((R)1.25 * x1 - (R)0.5 * sg * x2) * k;
  y2 = ((R)-0.5 * sg * x1 + (R)2 * x2) * k;
}

template <class T> __device__ __forceinline__ T is1_of(const Grid& g, int d);
template <> __device__ __forceinline__ float is1_of<float>(const Grid& g, int d) { return g.is1[d]; }
template <> __device__ __forceinline__ double is1_of<double>(const Grid& g, int d) { return g.ds1[d]; }
template <class T> __device__ __forceinline__ T is2_of(const Grid& g, int d);
template <> __device__ __forceinline__ float is2_of<float>(const Grid& g, int d) { return g.is2[d]; }
template <> __device__ __forceinline__ double is2_of<double>(const Grid& g, int d) { return g.ds2[d]; }

// ------------------------------------------ uniform or per-interval steps
// The record of position i along d of instance b (per-interval steps only).
template <class T> __device__ __forceinline__ const T* st_rec(const Grid& g, int b, int d, int i);
template <> __device__ __forceinline__ const double* st_rec<double>(const Grid& g, int b, int d, int i) {
  return g.st64 + ((size_t)(b * 3 + d) * g.stn + i) * ST_REC;
}
template <> __device__ __forceinline__ const float* st_rec<float>(const Grid& g, int b, int d, int i) {
  return g.st32 + ((size_t)(b * 3 + d) * g.stn + i) * ST_REC;
}

// Weight of u_{i+o} in the scaled difference form of order `order` at
// position i along d (Eq. 5): sbar^order u^(order) = sum_o w(o) u_{i+o}.
template <class T>
__device__ __forceinline__ T swt(const Grid& g, int b, int d, int i, int order, int o) {
  if (!g.st64) return (T)dweight(order, i, g.n[d], g.per[d], o);
  const T* r = st_rec<T>(g, b, d, i);
  const int k = o - (int)r[ST_BASE];
  return (k >= 0 && k < 3) ? r[(order == 1 ? ST_W1 : ST_W2) + k] : (T)0;
}
// 1 / sbar and 1 / sbar^2 at position i along d.
template <class T>
__device__ __forceinline__ T sis1(const Grid& g, int b, int d, int i) {
  return g.st64 ? st_rec<T>(g, b, d, i)[ST_IS1] : is1_of<T>(g, d);
}
template <class T>
__device__ __forceinline__ T sis2(const Grid& g, int b, int d, int i) {
  return g.st64 ? st_rec<T>(g, b, d, i)[ST_IS2] : is2_of<T>(g, d);
}
// y = W^{-1} x at position i along d.
template <class T>
__device__ __forceinline__ void swinv(const Grid& g, int b, int d, int i, T x1, T x2, T& y1, T& y2) {
  if (!g.st64) { winv<T>(edge_class(g, d, i), x1, x2, y1, y2); return; }
  const T* r = st_rec<T>(g, b, d, i);
  y1 = r[ST_WI] * x1 + r[ST_WI + 1] * x2;
  y2 = r[ST_WI + 1] * x1 + r[ST_WI + 2] * x2;
}
// W at position i along d.
__device__ __forceinline__ void swmat(const Grid& g, int b, int d, int i, double& w11, double& w12, double& w22) {
  if (!g.st64) { wmat(edge_class(g, d, i), w11, w12, w22); return; }
  const double* r = st_rec<double>(g, b, d, i);
  w11 = r[ST_W]; w12 = r[ST_W + 1]; w22 = r[ST_W + 2];
}

// Point weight rho_i = 1 / (1 + sum_d beta_d^T W_d^{-1} beta_d).
template <class T, int DD = 0>
__device__ __forceinline__ T rho_point(const Grid& g, const Coef& cf, int b, int p, const int pos[3]) {
  T gam = 0;
#pragma unroll
  for (int d = 0; d < (DD ? DD : g.D); ++d) {
    T b1 = (T)coefv(cf, 1 + 2 * d, b, p, g.N) * sis1<T>(g, b, d, pos[d]);
    T b2 = (T)coefv(cf, 2 + 2 * d, b, p, g.N) * sis2<T>(g, b, d, pos[d]);
    if (g.st64) {
      T q1, q2;
      swinv<T>(g, b, d, pos[d], b1, b2, q1, q2);
      gam += b1 * q1 + b2 * q2;
      continue;
    }
    int cls = edge_class(g, d, pos[d]);
    if (cls == 0) gam += b1 * b1 * (T)(1.0 / 3.0) + b2 * b2 * (T)(2.0 / 3.0);
    else {
      T sg = cls == 1 ? (T)1 : (T)-1;
      gam += ((T)1.25 * b1 * b1 - sg * b1 * b2 + (T)2 * b2 * b2) * (T)(1.0 / 2.25);
    }
  }
  return (T)1 / ((T)1 + gam);
}

// (L x)_i: the equation row evaluated with every derivative replaced by its
// difference form.  x2 (nullable) is added to x on the fly.  DD: number of
// grid dimensions when known at compile time (0: read g.D).
template <class T, int DD = 0>
__device__ __forceinline__ T Lrow(const Grid& g, const Coef& cf, int b, int p, const int pos[3],
                                  const T* __restrict__ x, const T* __restrict__ x2) {
  T xc = x[p]; if (x2) xc += x2[p];
  T acc = (T)coefv(cf, 0, b, p, g.N) * xc;
#pragma unroll
  for (int d = 0; d < (DD ? DD : g.D); ++d) {
    T c1 = (T)coefv(cf, 1 + 2 * d, b, p, g.N);
    T c2 = (T)coefv(cf, 2 + 2 * d, b, p, g.N);
    if (c1 == (T)0 && c2 == (T)0) continue;
    T a1 = 0, a2 = 0;
#pragma unroll
    for (int o = -2; o <= 2; ++o) {
      T w1 = swt<T>(g, b, d, pos[d], 1, o);
      T w2 = swt<T>(g, b, d, pos[d], 2, o);
      if (w1 == (T)0 && w2 == (T)0) continue;
      T xv;
      if (o == 0) xv = xc;
      else { int q = nbr(g, p, pos, d, o); xv = x[q]; if (x2) xv += x2[q]; }
      a1 += w1 * xv; a2 += w2 * xv;
    }
    acc += c1 * a1 * sis1<T>(g, b, d, pos[d]) + c2 * a2 * sis2<T>(g, b, d, pos[d]);
  }
  return acc;
}

// (L^T y)_j: gather over the rows i whose difference forms touch point j.
template <class T, int DD = 0>
__device__ __forceinline__ T LTgather(const Grid& g, const Coef& cf, int b, int p, const int pos[3],
                                      const T* __restrict__ y) {
  T acc = (T)coefv(cf, 0, b, p, g.N) * y[p];
#pragma unroll
  for (int d = 0; d < (DD ? DD : g.D); ++d) {
#pragma unroll
    for (int o = -2; o <= 2; ++o) {
      int ip = pos[d] - o;
      if (g.per[d]) ip = wrap1(ip, g.n[d]);
      else if (ip < 0 || ip >= g.n[d]) continue;
      T w1 = swt<T>(g, b, d, ip, 1, o);
      T w2 = swt<T>(g, b, d, ip, 2, o);
      if (w1 == (T)0 && w2 == (T)0) continue;
      int q = p + (ip - pos[d]) * g.stride[d];
      T c1 = (T)coefv(cf, 1 + 2 * d, b, q, g.N);
      T c2 = (T)coefv(cf, 2 + 2 * d, b, q, g.N);
      acc += y[q] * (c1 * w1 * sis1<T>(g, b, d, ip) + c2 * w2 * sis2<T>(g, b, d, ip));
    }
  }
  return acc;
}

// (B x)_i = alpha x_i + beta (du/dx_e)_i: the Neumann / mixed row of face
// point p (axis e) with the first-derivative form of its position.
template <class T>
__device__ __forceinline__ T Brow(const Grid& g, int b, int p, const int pos[3], int e, const T* __restrict__ x) {
  T a1 = 0;
#pragma unroll
  for (int o = -2; o <= 2; ++o) {
    const T w = swt<T>(g, b, e, pos[e], 1, o);
    if (w == (T)0) continue;
    a1 += w * x[o == 0 ? p : nbr(g, p, pos, e, o)];
  }
  return (T)g.bca[e] * x[p] + (T)g.bcb[e] * sis1<T>(g, b, e, pos[e]) * a1;
}

// (B^T y2)_j: gather over the Neumann / mixed rows that touch point j.
template <class T>
__device__ __forceinline__ T BTgather(const Grid& g, int b, int p, const int pos[3], const T* __restrict__ y2) {
  T acc = 0;
  for (int e = 1; e < g.D; ++e) {
    if (!g.bcm[e] || g.per[e]) continue;
#pragma unroll
    for (int o = -2; o <= 2; ++o) {
      const int ip = pos[e] - o;
      if (ip != 0 && ip != g.n[e] - 1) continue;   // rows sit on the faces of e
      int pi[3] = {pos[0], pos[1], pos[2]};
      pi[e] = ip;
      if (bc_axis(g, pi) != e) continue;
      const T w = swt<T>(g, b, e, ip, 1, o);
      T c = (T)g.bcb[e] * sis1<T>(g, b, e, ip) * w;
      if (o == 0) c += (T)g.bca[e];
      if (c == (T)0) continue;
      acc += c * y2[p + (ip - pos[e]) * g.stride[e]];
    }
  }
  return acc;
}

// Non-periodic coarsened dimension: the nc coarse points span the same
// interval as the nf fine points (both end faces kept), so fine point i sits
// at coarse coordinate x = i (nc-1)/(nf-1); linear interpolation from J, J+1.
__device__ __forceinline__ void np_interp(int i, int nf, int nc, int& J, float& f) {
  int num = i * (nc - 1);
  J = num / (nf - 1);
  int rem = num - J * (nf - 1);
  if (J >= nc - 1) { J = nc - 2; f = 1.f; }
  else f = (float)rem / (float)(nf - 1);
}

// Weights of P^T for coarse point J of a non-periodic dim: fills up to 8
// (fine index, weight) pairs; returns the count.
__device__ __forceinline__ int np_restrict_w(int J, int nf, int nc, int* idx, float* w) {
  int i0 = ((J - 1) * (nf - 1)) / (nc - 1);
  if (i0 < 0) i0 = 0;
  int i1 = ((J + 1) * (nf - 1) + nc - 2) / (nc - 1);
  if (i1 > nf - 1) i1 = nf - 1;
  int k = 0;
  for (int i = i0; i <= i1 && k < 8; ++i) {
    int Ji; float f; np_interp(i, nf, nc, Ji, f);
    float wt = 0.f;
    if (Ji == J) wt += 1.f - f;
    if (Ji + 1 == J) wt += f;
    if (wt != 0.f) { idx[k] = i; w[k] = wt; ++k; }
  }
  return k;
}

// ------------------------------------------------------------ float4 helpers
__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float4 f4(float a) { return make_float4(a, a, a, a); }
__device__ __forceinline__ float4 operator+(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ __forceinline__ float4 operator-(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }
__device__ __forceinline__ float4 operator*(float4 a, float4 b) { return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w); }
__device__ __forceinline__ float4 operator*(float a, float4 b) { return make_float4(a * b.x, a * b.y, a * b.z, a * b.w); }
__device__ __forceinline__ float get(const float4& v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w)); }

// ---------------------------------------------------------------- reductions
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; result valid in thread 0.  Fixed order: deterministic.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[32];
  v = warp_sum(v);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0;
  if (wid == 0) {
    int nw = (blockDim.x + 31) >> 5;
    r = lane < nw ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

// A float that thread 0 of the CTA computes from per-instance FP64 sums and
// gives to every thread: an FP64 division or square root in every thread
// costs more than a streaming kernel's memory traffic on this GPU, where FP64
// runs at a small fraction of the FP32 rate.  All threads must call it; f must
// not synchronise.
template <class F>
__device__ __forceinline__ float cta_scalar(F f) {
  __shared__ float v;
  __syncthreads();
  if (threadIdx.x == 0) v = f();
  __syncthreads();
  return v;
}

// Writes this CTA's partial sum s (valid in thread 0) for instance b; with a
// counter, the last of the instance's nblk CTAs to finish (a fence, then one
// atomic increment per CTA) sums all partials in a fixed order into tot[b]
// and resets the counter, so consumers read one number instead of every CTA
// of theirs summing the partials again.  Deterministic: the order of the
// final sum does not depend on which CTA is last.  All threads must call it.
__device__ __forceinline__ void partial_finish(double s, double* __restrict__ part, int* cnt, double* tot, int b,
                                               int blk, int nblk) {
  __shared__ int last;
  if (threadIdx.x == 0) {
    part[b * MPN_PMAX + blk] = s;
    int l = 0;
    if (cnt) {
      __threadfence();
      l = atomicAdd(cnt + b, 1) == nblk - 1;
    }
    last = l;
  }
  __syncthreads();
  if (last && threadIdx.x < 32) {
    __threadfence();
    double v = 0;
    for (int k = threadIdx.x; k < nblk; k += 32) v += __ldcg(part + b * MPN_PMAX + k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) {
      tot[b] = v;
      cnt[b] = 0;
    }
  }
}

// Sum of the P partials of instance b (consumer-side second stage); every
// thread of the block receives the same value.
__device__ __forceinline__ double sum_partials(const double* __restrict__ part, int b, int P) {
  __shared__ double res;
  if (threadIdx.x < 32) {
    double v = 0;
    for (int k = threadIdx.x; k < P; k += 32) v += part[b * MPN_PMAX + k];
    v = warp_sum(v);
    if (threadIdx.x == 0) res = v;
  }
  __syncthreads();
  double out = res;
  __syncthreads();
  return out;
}
