// Kernels of the NeuRLP-PDE solver.  Every kernel is batch-strided: the
// instance is blockIdx.y and the points of that instance are covered by a
// grid-stride loop over blockIdx.x (gridDim.x <= MPN_PMAX, so kernels that
// reduce write one partial per block: part[b * MPN_PMAX + blockIdx.x]).
#pragma once
#include "mpn_device.cuh"


// FP64 coefficient access.  MASK = RES_ANY: every c_v read and converted per
// use.  Otherwise bit v of MASK says c_v is a field; the per-instance scalars
// are converted once per thread and the difference forms they multiply are
// formed before the product (fewer FP64 operations: this pass is bound by the
// FP64 pipe).
// With FS_SHARE46, c_yy reads the field of c_xx, so the shared loads and
// conversions are issued once.
#define RES_ANY FS_ANY
template <int MASK>
struct Coef64 {
  const Coef& cf;
  int b;
  double sv[7];
  __device__ __forceinline__ Coef64(const Coef& c, int b_) : cf(c), b(b_) {
#pragma unroll
    for (int v = 0; v < 7; ++v) sv[v] = scal(v) ? (double)__ldg(c.ptr[v] + (size_t)b_ * c.bstride[v]) : 0.0;
  }
  __device__ __forceinline__ static constexpr bool scal(int v) { return MASK != RES_ANY && !((MASK >> v) & 1); }
  __device__ __forceinline__ double at(int v, int p) const {
    if ((MASK & FS_SHARE46) && v == 6) v = 4;
    return scal(v) ? sv[v] : (double)coefv(cf, v, b, p, 0);
  }
};


// ------------------------------------------------------------------- setup
// rho at the finest level from the coefficients.
template <int D>
__global__ void k_rho_fine(Grid g, Coef cf, float* __restrict__ rho, double* __restrict__ rho64) {
  int b = blockIdx.y;
  GRID_LOOP(p, g.N) {
    int pos[3]; decode_fast(g, p, pos);
    double r = rho_point<double, D>(g, cf, b, p, pos);
    rho[(size_t)b * g.N + p] = (float)r;
    rho64[(size_t)b * g.N + p] = r;
  }
}

// Weights of the points with a Neumann / mixed row (axis e): with
// beta = (c_{1+2d} / sbar_d, c_{2+2d} / sbar_d^2) per axis and
// gamma = b_e / sbar_e on the first derivative along e, the 2x2 weight of the
// point's (equation, boundary) rows is R = (I + K^T W^{-1} K)^{-1},
// K = [beta, gamma]: rho <- R11, r12 <- R12, r22 <- R22, each times theta
// (1 on the finest level, the level's boundary-row weight on coarser ones).
// Other points: r12 = r22 = 0, rho untouched.
__global__ void k_mixed_weights(Grid g, Coef cf, float* __restrict__ rho, float* __restrict__ r12,
                                float* __restrict__ r22, double* __restrict__ rho64, double* __restrict__ r12d,
                                double* __restrict__ r22d) {
  int b = blockIdx.y;
  const size_t off = (size_t)b * g.N;
  GRID_LOOP(p, g.N) {
    int pos[3]; decode_fast(g, p, pos);
    const int e = mixed_axis(g, pos);
    if (e < 1) {
      r12[off + p] = 0.f; r22[off + p] = 0.f;
      if (r12d) { r12d[off + p] = 0.0; r22d[off + p] = 0.0; }
      continue;
    }
    double g11 = 0.0, be1 = 0.0, be2 = 0.0;
    for (int d = 0; d < g.D; ++d) {
      const double b1 = (double)coefv(cf, 1 + 2 * d, b, p, g.N) * sis1<double>(g, b, d, pos[d]);
      const double b2 = (double)coefv(cf, 2 + 2 * d, b, p, g.N) * sis2<double>(g, b, d, pos[d]);
      double q1, q2;
      swinv<double>(g, b, d, pos[d], b1, b2, q1, q2);
      g11 += b1 * q1 + b2 * q2;
      if (d == e) { be1 = b1; be2 = b2; }
    }
    const double gm = g.bcb[e] * sis1<double>(g, b, e, pos[e]);
    double qg1, qg2;
    swinv<double>(g, b, e, pos[e], gm, 0.0, qg1, qg2);
    const double g12 = be1 * qg1 + be2 * qg2, g22 = gm * qg1;
    const double idet = (double)g.theta / ((1.0 + g11) * (1.0 + g22) - g12 * g12);
    const double R11 = (1.0 + g22) * idet, R12 = -g12 * idet, R22 = (1.0 + g11) * idet;
    rho[off + p] = (float)R11; r12[off + p] = (float)R12; r22[off + p] = (float)R22;
    if (rho64) { rho64[off + p] = R11; r12d[off + p] = R12; r22d[off + p] = R22; }
  }
}

// Full-weighting restriction of a point field (1/4, 1/2, 1/4 per coarsened
// dimension; clamped at non-periodic edges), times `scale`.  fine/coarse are
// [nb][Nf] / [nb][Nc] with the batch-like index in blockIdx.y.
__global__ void k_restrict_field(Grid gf, Grid gc, int c0, int c1, int c2, const float* __restrict__ fine,
                                 float* __restrict__ coarse, float scale) {
  int b = blockIdx.y;
  int cz[3] = {c0, c1, c2};
  const float* f = fine + (size_t)b * gf.N;
  GRID_LOOP(p, gc.N) {
    int pos[3]; decode_fast(gc, p, pos);
    int cnt[3], idx[3][8]; float w[3][8];
    for (int d = 0; d < 3; ++d) {
      if (!cz[d]) { cnt[d] = 1; idx[d][0] = pos[d]; w[d][0] = 1.f; continue; }
      int n = gf.n[d];
      if (gf.per[d]) {
        int c = 2 * pos[d];
        cnt[d] = 3;
        idx[d][0] = wrap1(c - 1, n); idx[d][1] = c; idx[d][2] = wrap1(c + 1, n);
        w[d][0] = 0.25f; w[d][1] = 0.5f; w[d][2] = 0.25f;
      } else {
        cnt[d] = np_restrict_w(pos[d], n, gc.n[d], idx[d], w[d]);
        float sw = 0.f;
        for (int k = 0; k < cnt[d]; ++k) sw += w[d][k];
        for (int k = 0; k < cnt[d]; ++k) w[d][k] /= sw;
      }
    }
    float acc = 0.f;
    for (int a = 0; a < cnt[0]; ++a)
      for (int bb = 0; bb < cnt[1]; ++bb)
        for (int c = 0; c < cnt[2]; ++c) {
          int q = (idx[0][a] * gf.n[1] + idx[1][bb]) * gf.n[2] + idx[2][c];
          acc += w[0][a] * w[1][bb] * w[2][c] * f[q];
        }
    coarse[(size_t)b * gc.N + p] = scale * acc;
  }
}

// 1 / diag(S) with S = L^T diag(rho) L + theta diag(1_B).
__global__ void k_diag_inv(Grid g, Coef cf, const float* __restrict__ rho, float* __restrict__ dinv) {
  int b = blockIdx.y;
  const float* rh = rho + (size_t)b * g.N;
  GRID_LOOP(p, g.N) {
    int pos[3]; decode_fast(g, p, pos);
    // own row: L_jj
    const size_t off = (size_t)b * g.N;
    float Ljj = coefv(cf, 0, b, p, g.N);
    for (int d = 0; d < g.D; ++d)
      Ljj += coefv(cf, 1 + 2 * d, b, p, g.N) * swt<float>(g, b, d, pos[d], 1, 0) * sis1<float>(g, b, d, pos[d]) +
             coefv(cf, 2 + 2 * d, b, p, g.N) * swt<float>(g, b, d, pos[d], 2, 0) * sis2<float>(g, b, d, pos[d]);
    float acc = rh[p] * Ljj * Ljj;
    const int ej = mixed_axis(g, pos);
    if (ej >= 1) {   // own Neumann / mixed row
      const float Bjj = g.bca[ej] + g.bcb[ej] * sis1<float>(g, b, ej, pos[ej]) * swt<float>(g, b, ej, pos[ej], 1, 0);
      acc += 2.f * g.r12[off + p] * Ljj * Bjj + g.r22[off + p] * Bjj * Bjj;
    }
    for (int d = 0; d < g.D; ++d)
      for (int o = -2; o <= 2; ++o) {
        if (o == 0) continue;
        int ip = pos[d] - o;
        if (g.per[d]) ip = wrap1(ip, g.n[d]);
        else if (ip < 0 || ip >= g.n[d]) continue;
        float w1 = swt<float>(g, b, d, ip, 1, o), w2 = swt<float>(g, b, d, ip, 2, o);
        if (w1 == 0.f && w2 == 0.f) continue;
        int q = p + (ip - pos[d]) * g.stride[d];
        float Lij = coefv(cf, 1 + 2 * d, b, q, g.N) * w1 * sis1<float>(g, b, d, ip) +
                    coefv(cf, 2 + 2 * d, b, q, g.N) * w2 * sis2<float>(g, b, d, ip);
        acc += rh[q] * Lij * Lij;
        if (g.mixed) {   // the Neumann / mixed row of point q along d
          int pq[3] = {pos[0], pos[1], pos[2]};
          pq[d] = ip;
          if (mixed_axis(g, pq) == d) {
            const float Bij = g.bcb[d] * sis1<float>(g, b, d, ip) * w1;
            acc += 2.f * g.r12[off + q] * Lij * Bij + g.r22[off + q] * Bij * Bij;
          }
        }
      }
    if (dirichlet_point(g, pos)) acc += g.theta;
    dinv[(size_t)b * g.N + p] = acc > 0 ? 1.f / acc : 0.f;
  }
}

// --------------------------------------------------- Chebyshev-Jacobi smoother
// PCG vector kernels.  V4: the instance length is a multiple of 4 and every
// thread handles float4 groups (grid from vgrid()).
// out[4 i + k] = in[i], k < 4 (per-instance scalars for stride-0 float4 loads).
__global__ void k_rep4(int n, const float* __restrict__ in, float* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) reinterpret_cast<float4*>(out)[i] = f4(in[i]);
}

template <bool V4>
__device__ __forceinline__ float4 vld(const float* a, int i) {
  if (V4) return __ldg(reinterpret_cast<const float4*>(a) + i);
  return make_float4(__ldg(a + i), 0.f, 0.f, 0.f);
}
template <bool V4>
__device__ __forceinline__ void vst(float* a, int i, float4 v) {
  if (V4) reinterpret_cast<float4*>(a)[i] = v;
  else a[i] = v.x;
}

// The smoother iterates e <- e + d with
//   d_0 = Dinv r_0 / th,  d_k = c1_k d_{k-1} + c2_k Dinv r_k,
// r_k = r - S e_k, Dinv already scaled by 1 / lambda_max(Dinv S).
// First smoothing step from e = 0 (look-ahead form): d = Dinv r / th, e = d
// (d null on levels that keep no direction array).
template <bool V4>
__global__ void k_cheb_init(int N, const float* __restrict__ r, const float* __restrict__ dinv, float inv_th,
                            float* __restrict__ e, float* __restrict__ d) {
  const size_t off = (size_t)blockIdx.y * N;
  const int n = V4 ? N >> 2 : N;
  GRID_LOOP(i, n) {
    float4 v = inv_th * (vld<V4>(dinv + off, i) * vld<V4>(r + off, i));
    vst<V4>(e + off, i, v);
    if (d) vst<V4>(d + off, i, v);
  }
}

// ------------------------------------------------------ grid transfers (P^T, P)

// Interpolation P along a coarsened dimension (nf = 2 nc fine points):
// fine 2j <- coarse j; fine 2j+1 <- (j + j+1) / 2, wrapping when periodic;
// the last fine point of a non-periodic dimension copies the last coarse one.
// Restriction is P^T.
__global__ void k_restrict_vec(Grid gf, Grid gc, int c0, int c1, int c2, const float* __restrict__ fine,
                               float* __restrict__ coarse) {
  int b = blockIdx.y;
  int cz[3] = {c0, c1, c2};
  const float* f = fine + (size_t)b * gf.N;
  GRID_LOOP(p, gc.N) {
    int pos[3]; decode_fast(gc, p, pos);
    int cnt[3], idx[3][8]; float w[3][8];
    for (int d = 0; d < 3; ++d) {
      if (!cz[d]) { cnt[d] = 1; idx[d][0] = pos[d]; w[d][0] = 1.f; continue; }
      int J = pos[d], nc = gc.n[d], nf = gf.n[d];
      if (!gf.per[d]) { cnt[d] = np_restrict_w(J, nf, nc, idx[d], w[d]); continue; }
      int k = 0;
      idx[d][k] = 2 * J; w[d][k++] = 1.f;
      idx[d][k] = 2 * J + 1; w[d][k++] = 0.5f;
      idx[d][k] = J >= 1 ? 2 * J - 1 : nf - 1; w[d][k++] = 0.5f;
      cnt[d] = k;
    }
    float acc = 0.f;
    for (int a = 0; a < cnt[0]; ++a)
      for (int bb = 0; bb < cnt[1]; ++bb)
        for (int c = 0; c < cnt[2]; ++c) {
          int q = (idx[0][a] * gf.n[1] + idx[1][bb]) * gf.n[2] + idx[2][c];
          acc += w[0][a] * w[1][bb] * w[2][c] * f[q];
        }
    coarse[(size_t)b * gc.N + p] = acc;
  }
}

// ef += P (ec + dc)   (dc nullable: pending Chebyshev step of the coarse level)
__global__ void k_prolong_add(Grid gf, Grid gc, int c0, int c1, int c2, const float* __restrict__ ec,
                              const float* __restrict__ dc, float* __restrict__ ef) {
  int b = blockIdx.y;
  int cz[3] = {c0, c1, c2};
  const float* E = ec + (size_t)b * gc.N;
  const float* Dd = dc ? dc + (size_t)b * gc.N : nullptr;
  GRID_LOOP(p, gf.N) {
    int pos[3]; decode_fast(gf, p, pos);
    int cnt[3], idx[3][2]; float w[3][2];
    for (int d = 0; d < 3; ++d) {
      if (!cz[d]) { cnt[d] = 1; idx[d][0] = pos[d]; w[d][0] = 1.f; continue; }
      int i = pos[d], nc = gc.n[d];
      if (!gf.per[d]) {
        int J; float f; np_interp(i, gf.n[d], nc, J, f);
        cnt[d] = 2; idx[d][0] = J; idx[d][1] = J + 1; w[d][0] = 1.f - f; w[d][1] = f;
      } else if ((i & 1) == 0) { cnt[d] = 1; idx[d][0] = i >> 1; w[d][0] = 1.f; }
      else {
        int j = i >> 1;
        cnt[d] = 2; idx[d][0] = j; idx[d][1] = (j + 1 < nc) ? j + 1 : 0; w[d][0] = w[d][1] = 0.5f;
      }
    }
    float acc = 0.f;
    for (int a = 0; a < cnt[0]; ++a)
      for (int bb = 0; bb < cnt[1]; ++bb)
        for (int c = 0; c < cnt[2]; ++c) {
          int q = (idx[0][a] * gc.n[1] + idx[1][bb]) * gc.n[2] + idx[2][c];
          float v = E[q];
          if (Dd) v += Dd[q];
          acc += w[0][a] * w[1][bb] * w[2][c] * v;
        }
    ef[(size_t)b * gf.N + p] += acc;
  }
}

// e_f += P e_c for the common case: t kept, x and y periodic and halved,
// n_y % 4 == 0.  One thread owns 4 fine points along y (= coarse y 2q, 2q+1
// and the next one, wrapping).
__global__ void k_prolong_add4(Grid gf, Grid gc, const float* __restrict__ ec, float* __restrict__ ef) {
  const int b = blockIdx.y;
  const float* E = ec + (size_t)b * gc.N;
  float* Fo = ef + (size_t)b * gf.N;
  const int ng = gf.n[2] >> 2;
  const int NG = gf.N >> 2;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < NG; q += gridDim.x * blockDim.x) {
    int row = q / ng;
    int j = (q - row * ng) * 2;                  // coarse y of the group's first point
    int ix = row % gf.n[1], it = row / gf.n[1];
    int jn = j + 2 == gc.n[2] ? 0 : j + 2;
    int cx0 = ix >> 1, cx1 = (ix & 1) ? ((cx0 + 1 == gc.n[1]) ? 0 : cx0 + 1) : cx0;
    float wx = (ix & 1) ? 0.5f : 1.f;
    const float* r0 = E + ((size_t)it * gc.n[1] + cx0) * gc.n[2];
    const float* r1 = E + ((size_t)it * gc.n[1] + cx1) * gc.n[2];
    float a0 = r0[j], a1 = r0[j + 1], a2 = r0[jn];
    if (ix & 1) { a0 += r1[j]; a1 += r1[j + 1]; a2 += r1[jn]; }
    a0 *= wx; a1 *= wx; a2 *= wx;
    float4* dst = reinterpret_cast<float4*>(Fo + (size_t)q * 4);
    float4 v = *dst;
    v.x += a0; v.y += 0.5f * (a0 + a1); v.z += a1; v.w += 0.5f * (a1 + a2);
    *dst = v;
  }
}

// r_c = P^T r_f for the same case with n_y % 8 == 0: one thread owns 4
// coarse points along y, i.e. fine y 2j-1 .. 2j+7 of three fine x rows.
// With dinv_c set it also starts the coarse level's smoother (k_cheb_init's
// work): d_c = e_c = inv_th D_c^-1 r_c.
__global__ void k_restrict_vec4(Grid gf, Grid gc, const float* __restrict__ fine, float* __restrict__ coarse,
                                const float* __restrict__ dinv_c, float inv_th, float* __restrict__ e_c,
                                float* __restrict__ d_c) {
  const int b = blockIdx.y;
  const float* Fi = fine + (size_t)b * gf.N;
  float* Co = coarse + (size_t)b * gc.N;
  const int n1c = gc.n[1], n2c = gc.n[2], n1f = gf.n[1], n2f = gf.n[2];
  const int G = n2c >> 2;
  const float invG = 1.f / (float)G, inv1 = 1.f / (float)n1c;
  const int NG = gc.N >> 2;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < NG; q += gridDim.x * blockDim.x) {
    int gq, X;
    const int row = fdivmod(q, G, invG, gq);
    const int t = fdivmod(row, n1c, inv1, X);
    const int fy = 8 * gq;                        // fine y of the group's first coarse point
    const size_t jc = (size_t)b * gc.N + (size_t)q * 4;
    const float4 di = dinv_c ? ld4(dinv_c + jc) : f4(0.f);
    float4 acc = f4(0.f);
#pragma unroll
    for (int r = -1; r <= 1; ++r) {
      int xf = 2 * X + r;
      if (xf < 0) xf += n1f;
      const float w = r == 0 ? 1.f : 0.5f;
      const float* base = Fi + ((size_t)t * n1f + xf) * n2f;
      const float4 a = ld4(base + fy), c = ld4(base + fy + 4);
      const float l = __ldg(base + (fy == 0 ? n2f - 1 : fy - 1));
      const float4 o = make_float4(a.x + 0.5f * (a.y + l), a.z + 0.5f * (a.w + a.y), c.x + 0.5f * (c.y + a.w),
                                   c.z + 0.5f * (c.w + c.y));
      acc = acc + w * o;
    }
    *reinterpret_cast<float4*>(Co + (size_t)q * 4) = acc;
    if (dinv_c) {
      const float4 v = inv_th * (di * acc);
      *reinterpret_cast<float4*>(e_c + jc) = v;
      if (d_c) *reinterpret_cast<float4*>(d_c + jc) = v;
    }
  }
}

// ------------------------------------------------------ coarsest-level solve
// Banded lower storage: Kb[b][j][j - k] = S[j][k] for 0 <= j - k <= bw.
__global__ void k_coarse_assemble(Grid g, Coef cf, const float* __restrict__ rho, int bw, float* __restrict__ Kb) {
  int b = blockIdx.y;
  const float* rh = rho + (size_t)b * g.N;
  float* K = Kb + (size_t)b * g.N * (bw + 1);
  GRID_LOOP(j, g.N) {
    int pj[3]; decode_fast(g, j, pj);
    float* row = K + (size_t)j * (bw + 1);
    for (int k = 0; k <= bw; ++k) row[k] = 0.f;
    if (dirichlet_point(g, pj)) row[0] += g.theta;
    // rows i of L that touch j: i = j (center) and i = j - o e_d; a point with
    // a Neumann / mixed row adds [L_ij, B_ij] R [L_ik, B_ik]^T
    for (int d0 = -1; d0 < g.D; ++d0) {
      for (int o = -2; o <= 2; ++o) {
        int i, pi[3] = {pj[0], pj[1], pj[2]};
        double Lij;
        if (d0 < 0) {
          if (o != 0) continue;
          i = j;
          Lij = coefv(cf, 0, b, i, g.N);
          for (int d = 0; d < g.D; ++d)
            Lij += (double)coefv(cf, 1 + 2 * d, b, i, g.N) * swt<double>(g, b, d, pi[d], 1, 0) * sis1<double>(g, b, d, pi[d]) +
                   (double)coefv(cf, 2 + 2 * d, b, i, g.N) * swt<double>(g, b, d, pi[d], 2, 0) * sis2<double>(g, b, d, pi[d]);
        } else {
          if (o == 0) continue;
          int ip = pj[d0] - o;
          if (g.per[d0]) ip = wrap1(ip, g.n[d0]);
          else if (ip < 0 || ip >= g.n[d0]) continue;
          double w1 = swt<double>(g, b, d0, ip, 1, o), w2 = swt<double>(g, b, d0, ip, 2, o);
          if (w1 == 0.0 && w2 == 0.0) continue;
          i = j + (ip - pj[d0]) * g.stride[d0];
          pi[d0] = ip;
          Lij = (double)coefv(cf, 1 + 2 * d0, b, i, g.N) * w1 * sis1<double>(g, b, d0, ip) +
                (double)coefv(cf, 2 + 2 * d0, b, i, g.N) * w2 * sis2<double>(g, b, d0, ip);
        }
        double f = Lij * (double)rh[i];
        const int ei = mixed_axis(g, pi);
        if (ei >= 1) {
          double Bij = 0.0;
          if (d0 < 0) Bij = g.bca[ei] + g.bcb[ei] * sis1<double>(g, b, ei, pi[ei]) * swt<double>(g, b, ei, pi[ei], 1, 0);
          else if (d0 == ei) Bij = g.bcb[ei] * sis1<double>(g, b, ei, pi[ei]) * swt<double>(g, b, ei, pi[ei], 1, o);
          const size_t oi = (size_t)b * g.N + i;
          const double r12 = g.r12[oi], r22 = g.r22[oi];
          f += Bij * r12;
          const double fB = Lij * r12 + Bij * r22;
          // row i of B: alpha at i and the first-derivative form along ei
          for (int o2 = -2; o2 <= 2; ++o2) {
            const double w = swt<double>(g, b, ei, pi[ei], 1, o2);
            double Bik = g.bcb[ei] * sis1<double>(g, b, ei, pi[ei]) * w;
            if (o2 == 0) Bik += g.bca[ei];
            if (Bik == 0.0) continue;
            const int k = o2 == 0 ? i : nbr(g, i, pi, ei, o2);
            if (k <= j && j - k <= bw) row[j - k] += (float)(fB * Bik);
          }
        }
        // row i of L: center and off-center entries
        double Lii = coefv(cf, 0, b, i, g.N);
        for (int d = 0; d < g.D; ++d)
          Lii += (double)coefv(cf, 1 + 2 * d, b, i, g.N) * swt<double>(g, b, d, pi[d], 1, 0) * sis1<double>(g, b, d, pi[d]) +
                 (double)coefv(cf, 2 + 2 * d, b, i, g.N) * swt<double>(g, b, d, pi[d], 2, 0) * sis2<double>(g, b, d, pi[d]);
        if (i <= j && j - i <= bw) row[j - i] += (float)(f * Lii);
        for (int d = 0; d < g.D; ++d)
          for (int o2 = -2; o2 <= 2; ++o2) {
            if (o2 == 0) continue;
            double w1 = swt<double>(g, b, d, pi[d], 1, o2), w2 = swt<double>(g, b, d, pi[d], 2, o2);
            if (w1 == 0.0 && w2 == 0.0) continue;
            int k = nbr(g, i, pi, d, o2);
            double Lik = (double)coefv(cf, 1 + 2 * d, b, i, g.N) * w1 * sis1<double>(g, b, d, pi[d]) +
                         (double)coefv(cf, 2 + 2 * d, b, i, g.N) * w2 * sis2<double>(g, b, d, pi[d]);
            if (k <= j && j - k <= bw) row[j - k] += (float)(f * Lik);
          }
      }
    }
  }
}

// Banded Cholesky, one block per instance, band held in shared memory.
// A non-positive pivot is replaced by 1 and flagged in err[b].
// Right-looking band Cholesky of one instance's coarsest system in shared
// memory (the band, then a column buffer of bw floats).  Step k: threads
// ii < bw scale l_ik (i = k + 1 + ii) into the column buffer; after a barrier
// the block, as 32 columns x (blockDim / 32) rows, updates the lower triangle
// S_ij -= l_ik l_jk, k < j <= i <= k + bw.  blockDim.x >= bw, a multiple of 32.
template <bool SMEM>
__global__ void k_coarse_factor(int M, int bw, float* __restrict__ Kb, int* __restrict__ err) {
  extern __shared__ float shm[];
  const int b = blockIdx.x;
  float* K = Kb + (size_t)b * M * (bw + 1);
  const int W = bw + 1;
  // SMEM: the band is staged in shared memory; else it is factorised in place
  // in global memory (L2-resident), for bands larger than shared memory
  float* sb = SMEM ? shm : K;
  float* colk = SMEM ? shm + (size_t)M * W : shm;
  if (SMEM) {
    for (int t = threadIdx.x; t < M * W; t += blockDim.x) sb[t] = K[t];
  }
  __syncthreads();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, nty = blockDim.x >> 5;
  for (int k = 0; k < M; ++k) {
    float a = sb[k * W];
    if (!(a > 0.f)) { a = 1.f; if (threadIdx.x == 0) err[b] = 1; }
    const float piv = sqrtf(a), ipiv = 1.f / piv;
    const int nr = min(bw, M - k - 1);
    const int ii = threadIdx.x;
    if (ii < nr) colk[ii] = sb[(k + 1 + ii) * W + ii + 1] * ipiv;
    __syncthreads();
    if (threadIdx.x == 0) sb[k * W] = piv;
    if (ii < nr) sb[(k + 1 + ii) * W + ii + 1] = colk[ii];
    for (int i2 = ty; i2 < nr; i2 += nty) {
      const float li = colk[i2];
      float* row = sb + (k + 1 + i2) * W + i2;   // row[-jj] is entry (k+1+i2, k+1+jj)
      for (int jj = tx; jj <= i2; jj += 32) row[-jj] -= li * colk[jj];
    }
    __syncthreads();
  }
  if (SMEM) {
    for (int t = threadIdx.x; t < M * W; t += blockDim.x) K[t] = sb[t];
  }
}

// The same factorisation for bands of at most FACT1_MAXBW, one barrier per
// column step.  Step k: every thread reads the pivot and the column-k entries
// it needs (unscaled) and scales them itself; the triangular update of the
// trailing block, bw (bw + 1) / 2 elements, is spread evenly over the block
// (at most FACT1_EPT elements per thread, decoded once); the new pivot and
// the scaled column entry a thread owns are written back at step k + 1, after
// the barrier, when nobody reads them any more.
#define FACT1_EPT 4
#define FACT1_MAXBW 63
template <bool SMEM>
__global__ void __launch_bounds__(512) k_coarse_factor1(int M, int bw, float* __restrict__ Kb, int* __restrict__ err) {
  extern __shared__ float shm[];
  const int b = blockIdx.x;
  float* K = Kb + (size_t)b * M * (bw + 1);
  const int W = bw + 1;
  float* sb = SMEM ? shm : K;
  if (SMEM)
    for (int t = threadIdx.x; t < M * W; t += blockDim.x) sb[t] = K[t];
  // this thread's elements (i2, jj), jj <= i2 < bw, of the triangular update
  int ei[FACT1_EPT], ej[FACT1_EPT];
  const int ntri = bw * (bw + 1) / 2;
#pragma unroll
  for (int q = 0; q < FACT1_EPT; ++q) {
    const int e = threadIdx.x + q * blockDim.x;
    ei[q] = -1; ej[q] = 0;
    if (e < ntri) {
      int i2 = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
      while ((i2 + 1) * (i2 + 2) / 2 <= e) ++i2;
      while (i2 * (i2 + 1) / 2 > e) --i2;
      ei[q] = i2; ej[q] = e - i2 * (i2 + 1) / 2;
    }
  }
  __syncthreads();
  float own = 0.f, piv_prev = 0.f;
  int own_at = -1;                       // sb index of the owned column entry (previous step)
  bool bad = false;
  for (int k = 0; k < M; ++k) {
    // write-backs of step k - 1 (its readers have passed the barrier)
    if (k > 0 && threadIdx.x == 0) sb[(size_t)(k - 1) * W] = piv_prev;
    if (own_at >= 0) sb[own_at] = own;
    float a = sb[(size_t)k * W];
    if (!(a > 0.f)) { a = 1.f; bad = true; }
    const float ipiv = rsqrtf(a);
    piv_prev = a * ipiv;
    const int nr = min(bw, M - k - 1);
    const float* colk = sb + (size_t)(k + 1) * W + 1;   // colk[ii * (W + 1)] = K(k+1+ii, k), unscaled
    own_at = -1;
    if ((int)threadIdx.x < nr) {
      own_at = (k + 1 + threadIdx.x) * W + threadIdx.x + 1;
      own = sb[own_at] * ipiv;
    }
#pragma unroll
    for (int q = 0; q < FACT1_EPT; ++q) {
      const int i2 = ei[q], jj = ej[q];
      if (i2 >= 0 && i2 < nr) {
        const float li = colk[(size_t)i2 * (W + 1)] * ipiv, lj = colk[(size_t)jj * (W + 1)] * ipiv;
        sb[(size_t)(k + 1 + i2) * W + (i2 - jj)] -= li * lj;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) sb[(size_t)(M - 1) * W] = piv_prev;
  if (own_at >= 0) sb[own_at] = own;
  if (bad && threadIdx.x == 0) err[b] = 1;
  __syncthreads();
  if (SMEM)
    for (int t = threadIdx.x; t < M * W; t += blockDim.x) K[t] = sb[t];
}

// Explicit inverse from the banded factor (bw < 32 NW): one warp per column c
// solves L L^T x = e_c for the rows i >= c and writes them to column and row c
// of the symmetric Kinv.  The CTA stages the band and the reciprocal diagonal
// in shared memory, plus one forward-solution vector per warp.  At step i the
// band row (or column) is split across the lanes and the dot product reduced
// by shuffles; the last 32 NW values of the substitution live in NW registers
// per lane and shift by one lane per step.
// Grid: (column blocks x instances) in one dimension, column block major, so
// the CTAs with the longest columns (small c: 2 (M - c) substitution steps)
// start first and the short ones fill in behind them.
template <int NW, bool SMEM>
__global__ void k_coarse_inverse(int M, int bw, const float* __restrict__ Lb, float* __restrict__ Kinv) {
  extern __shared__ float sL[];
  const int ncb = (M + (int)(blockDim.x >> 5) - 1) / (int)(blockDim.x >> 5);
  const int B = gridDim.x / ncb;
  const int b = blockIdx.x % B, cb = blockIdx.x / B;
  const int W = bw + 1;
  const float* src = Lb + (size_t)b * M * W;
  float* rd = SMEM ? sL + (size_t)M * W : sL;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* Y = rd + M + (size_t)wid * M;       // this warp's forward solution
  if (SMEM) {
    for (int t = threadIdx.x; t < M * W; t += blockDim.x) sL[t] = src[t];
    __syncthreads();
  }
  const float* L = SMEM ? sL : src;        // band rows: shared memory, or global (L2)
  for (int t = threadIdx.x; t < M; t += blockDim.x) rd[t] = 1.f / L[(size_t)t * W];
  __syncthreads();
  const int c = cb * (blockDim.x >> 5) + wid;   // column of this warp
  if (c >= M) return;
  float* X = Kinv + (size_t)b * M * M;
  float w[NW];
  // forward: y_i = (delta_ic - sum_{j<i} L_ij y_j) / L_ii; w[k] on lane l holds
  // y_{i-1-32k-l}
#pragma unroll
  for (int k = 0; k < NW; ++k) w[k] = 0.f;
  for (int i = c; i < M; ++i) {
    const float* Li = L + (size_t)i * W;
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
      int o = 1 + 32 * k + lane;                // offset i - j
      if (o <= bw && i - o >= c) s += Li[o] * w[k];
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    float y = ((i == c ? 1.f : 0.f) - s) * rd[i];
#pragma unroll
    for (int k = NW - 1; k >= 0; --k) {
      float carry = k > 0 ? __shfl_sync(0xffffffffu, w[k - 1], 31) : y;
      w[k] = __shfl_up_sync(0xffffffffu, w[k], 1);
      if (lane == 0) w[k] = carry;
    }
    if (lane == 0) Y[i] = y;
  }
  __syncwarp();
  // backward: x_i = (y_i - sum_{j>i} L_ji x_j) / L_ii down to i = c (the
  // rest of the column is the mirror of rows already computed by other
  // warps); w[k] on lane l holds x_{i+1+32k+l}
#pragma unroll
  for (int k = 0; k < NW; ++k) w[k] = 0.f;
  for (int i = M - 1; i >= c; --i) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
      int o = 1 + 32 * k + lane, j = i + o;
      if (o <= bw && j < M) s += L[(size_t)j * W + o] * w[k];
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    float x = (Y[i] - s) * rd[i];
#pragma unroll
    for (int k = NW - 1; k >= 0; --k) {
      float carry = k > 0 ? __shfl_sync(0xffffffffu, w[k - 1], 31) : x;
      w[k] = __shfl_up_sync(0xffffffffu, w[k], 1);
      if (lane == 0) w[k] = carry;
    }
    if (lane == 0) { X[(size_t)i * M + c] = x; X[(size_t)c * M + i] = x; }
  }
}

// e = Kinv r at the coarsest level: one warp per row.
__global__ void k_coarse_solve(int M, const float* __restrict__ Kinv, const float* __restrict__ r,
                               float* __restrict__ e) {
  int b = blockIdx.y;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= M) return;
  const float* row = Kinv + ((size_t)b * M + warp) * M;
  const float* rr = r + (size_t)b * M;
  float s = 0.f;
  for (int j = lane; j < M; j += 32) s += row[j] * rr[j];
  s = warp_sum(s);
  if (lane == 0) e[(size_t)b * M + warp] = s;
}

// ------------------------------------------------------------ power method
// x_0 of the power method (deterministic positive pseudo-random values), with
// partials of ||x_0||^2.
__global__ void k_fill_hash(int N, float* __restrict__ x, double* __restrict__ part) {
  size_t off = (size_t)blockIdx.y * N;
  double acc = 0;
  GRID_LOOP(p, N) {
    uint32_t h = (uint32_t)(p * 2654435761u) ^ (uint32_t)(blockIdx.y * 40503u + 12345u);
    h ^= h >> 15; h *= 2246822519u; h ^= h >> 13;
    const float v = (float)(h & 0xffff) / 65536.f + 0.25f;
    x[off + p] = v;
    acc += (double)v * v;
  }
  double s = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.y * MPN_PMAX + blockIdx.x] = s;
}

// One power step after q = S x_k: x_{k+1} = Dinv q / ||x_k|| (= Dinv S applied
// to the unit vector x_k / ||x_k||, so ||x_{k+1}|| estimates lambda_max), with
// partials of ||x_{k+1}||^2 into part_out (a slot other than part_in).
__global__ void k_power_w(int N, const float* __restrict__ dinv, const float* __restrict__ q,
                          const double* __restrict__ part_in, int P, float* __restrict__ x,
                          double* __restrict__ part_out) {
  int b = blockIdx.y;
  size_t off = (size_t)b * N;
  const double ss = sum_partials(part_in, b, P);
  const float inv = cta_scalar([&] { const double nn = sqrt(ss); return nn > 0 ? (float)(1.0 / nn) : 0.f; });
  double acc = 0;
  GRID_LOOP(p, N) {
    float v = dinv[off + p] * q[off + p] * inv;
    x[off + p] = v;
    acc += (double)v * v;
  }
  double s = block_sum(acc);
  if (threadIdx.x == 0) part_out[b * MPN_PMAX + blockIdx.x] = s;
}

// dinv *= 1 / (safety * lambda),  lambda = ||w|| of the last power step.
__global__ void k_scale_dinv(int N, float* __restrict__ dinv, const double* __restrict__ part, int P,
                             float safety, float* __restrict__ lam_out) {
  int b = blockIdx.y;
  const double ss = sum_partials(part, b, P);
  const float s = cta_scalar([&] {
    const double lam = sqrt(ss);
    if (blockIdx.x == 0 && lam_out) lam_out[b] = (float)lam;
    return lam > 0 ? (float)(1.0 / (safety * lam)) : 1.f;
  });
  size_t off = (size_t)b * N;
  GRID_LOOP(p, N) dinv[off + p] *= s;
}

// --------------------------------------------------------------------- PCG
// z = e + d (d nullable); partial <r, z>.
// z = e, partial <z, r> per block.
template <bool V4>
__global__ void k_final_z(int N, const float* __restrict__ e, const float* __restrict__ r, float* __restrict__ z,
                          double* __restrict__ part) {
  const int b = blockIdx.y;
  const size_t off = (size_t)b * N;
  const int n = V4 ? N >> 2 : N;
  float acc = 0.f;
  GRID_LOOP(i, n) {
    float4 v = vld<V4>(e + off, i), rr = vld<V4>(r + off, i);
    vst<V4>(z + off, i, v);
    acc += v.x * rr.x + v.y * rr.y + v.z * rr.z + v.w * rr.w;
  }
  double s = block_sum((double)acc);
  if (threadIdx.x == 0) part[b * MPN_PMAX + blockIdx.x] = s;
}
template <bool V4>
__global__ void k_pcg_init(int N, const float* __restrict__ z, float* __restrict__ x, float* __restrict__ pv) {
  const size_t off = (size_t)blockIdx.y * N;
  const int n = V4 ? N >> 2 : N;
  GRID_LOOP(i, n) { vst<V4>(x + off, i, make_float4(0.f, 0.f, 0.f, 0.f)); vst<V4>(pv + off, i, vld<V4>(z + off, i)); }
}
// The vector loads of a thread's first group are issued before the block
// sums the partial dot products, so their latency overlaps the reduction.
// With dinv set it also starts the smoother of the V-cycle that follows on
// the new r: d = e = inv_th D^-1 r.
template <bool V4>
__global__ void k_pcg_xr(int N, const double* __restrict__ part_rz, const double* __restrict__ part_pq, int P,
                         int Prz, const float* __restrict__ pv, const float* __restrict__ q, float* __restrict__ x,
                         float* __restrict__ r, double* __restrict__ rz_old, const float* __restrict__ dinv,
                         float inv_th, float* __restrict__ e, float* __restrict__ d,
                         const double* __restrict__ tot_rz, const double* __restrict__ tot_pq) {
  const int b = blockIdx.y;
  const size_t off = (size_t)b * N;
  const int n = V4 ? N >> 2 : N;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  float4 xv, pp, rv, qq, dv = f4(0.f);
  if (i0 < n) {
    xv = vld<V4>(x + off, i0); pp = vld<V4>(pv + off, i0); rv = vld<V4>(r + off, i0); qq = vld<V4>(q + off, i0);
    if (dinv) dv = vld<V4>(dinv + off, i0);
  }
  // the finished sums where the producing kernels wrote them, else the partials
  const double rz = tot_rz ? tot_rz[b] : sum_partials(part_rz, b, Prz);
  const double pq = tot_pq ? tot_pq[b] : sum_partials(part_pq, b, P);
  const float alpha = cta_scalar([&] { return (pq > 0 && rz > 0) ? (float)(rz / pq) : 0.f; });
  if (blockIdx.x == 0 && threadIdx.x == 0) rz_old[b] = rz;
  for (int i = i0; i < n; i += stride) {
    if (i != i0) {
      xv = vld<V4>(x + off, i); pp = vld<V4>(pv + off, i); rv = vld<V4>(r + off, i); qq = vld<V4>(q + off, i);
      if (dinv) dv = vld<V4>(dinv + off, i);
    }
    const float4 rn = rv - alpha * qq;
    vst<V4>(x + off, i, xv + alpha * pp);
    vst<V4>(r + off, i, rn);
    if (dinv) {
      const float4 v = inv_th * (dv * rn);
      vst<V4>(e + off, i, v);
      if (d) vst<V4>(d + off, i, v);
    }
  }
}
template <bool V4>
__global__ void k_pcg_p(int N, const double* __restrict__ part_rz, int P, const double* __restrict__ rz_old,
                        const float* __restrict__ z, float* __restrict__ pv) {
  const int b = blockIdx.y;
  const size_t off = (size_t)b * N;
  const int n = V4 ? N >> 2 : N;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  float4 zz, pp;
  if (i0 < n) { zz = vld<V4>(z + off, i0); pp = vld<V4>(pv + off, i0); }
  const double rz = sum_partials(part_rz, b, P);
  const double ro = rz_old[b];
  const float beta = cta_scalar([&] { return (ro > 0 && rz > 0) ? (float)(rz / ro) : 0.f; });
  for (int i = i0; i < n; i += stride) {
    if (i != i0) { zz = vld<V4>(z + off, i); pp = vld<V4>(pv + off, i); }
    vst<V4>(pv + off, i, zz + beta * pp);
  }
}
// p = z + beta p_old into another buffer (p_old null: p = z), beta =
// <r, z> / rz_old with <r, z> the finished sum tot_rz[b] when given, else
// the sum of P partials (the direction update ahead of an apply on the
// t-marching step).
template <bool V4>
__global__ void k_pcg_pd(int N, const double* __restrict__ tot_rz, const double* __restrict__ part_rz, int P,
                         const double* __restrict__ rz_old, const float* __restrict__ z,
                         const float* __restrict__ pold, float* __restrict__ pnew) {
  const int b = blockIdx.y;
  const size_t off = (size_t)b * N;
  const int n = V4 ? N >> 2 : N;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  float4 zz, pp = f4(0.f);
  if (i0 < n) {
    zz = vld<V4>(z + off, i0);
    if (pold) pp = vld<V4>(pold + off, i0);
  }
  float beta = 0.f;
  if (pold) {
    const double rz = tot_rz ? tot_rz[b] : sum_partials(part_rz, b, P);
    const double ro = rz_old[b];
    beta = cta_scalar([&] { return (ro > 0 && rz > 0) ? (float)(rz / ro) : 0.f; });
  }
  for (int i = i0; i < n; i += stride) {
    if (i != i0) {
      zz = vld<V4>(z + off, i);
      if (pold) pp = vld<V4>(pold + off, i);
    }
    vst<V4>(pnew + off, i, zz + beta * pp);
  }
}
// ------------------------------------------------ FGMRES (Section 3.1)
// Batched right-preconditioned flexible GMRES(m) on S x = r from x = 0, one
// restart cycle per refinement sweep: Arnoldi basis v_0..v_m (FP32 vectors),
// preconditioned vectors z_j = V-cycle(v_j), classical Gram-Schmidt (one
// multi-dot pass, one multi-update pass), Hessenberg matrix, Givens rotations
// and the small least-squares solve per instance in FP64.
#define FG_MMAX 64

// partials of <w, V_i>, i < nv (V_i = V + i vstride), one slot per i
template <bool V4>
__global__ void k_fg_dots(int N, const float* __restrict__ w, const float* __restrict__ V, size_t vstride, int nv,
                          double* __restrict__ part) {
  const int b = blockIdx.y, B = gridDim.y;
  const size_t off = (size_t)b * N;
  const int n = V4 ? N >> 2 : N;
  for (int i = 0; i < nv; ++i) {
    const float* vi = V + i * vstride + off;
    float acc = 0.f;
    GRID_LOOP(q, n) {
      float4 a = vld<V4>(w + off, q), c = vld<V4>(vi, q);
      acc += a.x * c.x + a.y * c.y + a.z * c.z + a.w * c.w;
    }
    double s = block_sum((double)acc);
    if (threadIdx.x == 0) part[((size_t)i * B + b) * MPN_PMAX + blockIdx.x] = s;
  }
}

// w -= sum_i h_i V_i with h_i the summed partials of slot i; partials of |w|^2
template <bool V4>
__global__ void k_fg_orth(int N, float* __restrict__ w, const float* __restrict__ V, size_t vstride, int nv,
                          const double* __restrict__ part, int P, double* __restrict__ npart) {
  __shared__ float hs[FG_MMAX + 1];
  const int b = blockIdx.y, B = gridDim.y;
  for (int i = 0; i < nv; ++i) {
    double h = sum_partials(part + (size_t)i * B * MPN_PMAX, b, P);
    if (threadIdx.x == 0) hs[i] = (float)h;
  }
  __syncthreads();
  const size_t off = (size_t)b * N;
  const int n = V4 ? N >> 2 : N;
  float acc = 0.f;
  GRID_LOOP(q, n) {
    float4 a = vld<V4>(w + off, q);
    for (int i = 0; i < nv; ++i) a = a - hs[i] * vld<V4>(V + i * vstride + off, q);
    vst<V4>(w + off, q, a);
    acc += a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w;
  }
  double s = block_sum((double)acc);
  if (threadIdx.x == 0) npart[b * MPN_PMAX + blockIdx.x] = s;
}

// beta = |r|: g = beta e_0, hnext = beta (one warp per instance)
__global__ void k_fg_init(int m1, const double* __restrict__ part, int P, double* __restrict__ g,
                          double* __restrict__ hnext) {
  const int b = blockIdx.x;
  double beta = sqrt(sum_partials(part, b, P));
  for (int i = threadIdx.x; i < m1; i += blockDim.x) g[(size_t)b * m1 + i] = i == 0 ? beta : 0.0;
  if (threadIdx.x == 0) hnext[b] = beta;
}

// Column j of H from the dot partials, rotated by the previous Givens
// rotations; the new rotation zeroes h_{j+1,j} and updates g.  hnext keeps the
// unrotated h_{j+1,j} = |w| for normalising v_{j+1}.
__global__ void k_fg_hess(int j, int m, const double* __restrict__ part, int P, const double* __restrict__ npart,
                          double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn,
                          double* __restrict__ g, double* __restrict__ hnext) {
  __shared__ double h[FG_MMAX + 1];
  const int b = blockIdx.x, B = gridDim.x;
  for (int i = 0; i <= j; ++i) {
    double v = sum_partials(part + (size_t)i * B * MPN_PMAX, b, P);
    if (threadIdx.x == 0) h[i] = v;
  }
  double hn = sqrt(sum_partials(npart, b, P));
  if (threadIdx.x == 0) {
    double* c = cs + (size_t)b * m;
    double* s = sn + (size_t)b * m;
    double* gg = g + (size_t)b * (m + 1);
    for (int i = 0; i < j; ++i) {
      double a = c[i] * h[i] + s[i] * h[i + 1];
      h[i + 1] = -s[i] * h[i] + c[i] * h[i + 1];
      h[i] = a;
    }
    double r = sqrt(h[j] * h[j] + hn * hn);
    double cj = r > 0 ? h[j] / r : 1.0, sj = r > 0 ? hn / r : 0.0;
    c[j] = cj; s[j] = sj;
    h[j] = r;
    gg[j + 1] = -sj * gg[j];
    gg[j] = cj * gg[j];
    double* col = H + ((size_t)b * m + j) * (m + 1);
    for (int i = 0; i <= j; ++i) col[i] = h[i];
    hnext[b] = hn;
  }
}

// v = w / hnext (zero after a breakdown), also written to the preconditioner's input
template <bool V4>
__global__ void k_fg_scale(int N, const float* __restrict__ w, const double* __restrict__ hnext, float* __restrict__ v,
                           float* __restrict__ r_in) {
  const int b = blockIdx.y;
  const double h = hnext[b];
  const float inv = cta_scalar([&] { return h > 1e-300 ? (float)(1.0 / h) : 0.f; });
  const size_t off = (size_t)b * N;
  const int n = V4 ? N >> 2 : N;
  GRID_LOOP(q, n) {
    float4 a = inv * vld<V4>(w + off, q);
    vst<V4>(v + off, q, a);
    vst<V4>(r_in + off, q, a);
  }
}

// y = R^{-1} g over the first k columns (R upper triangular after the
// rotations); one thread per instance
__global__ void k_fg_ysolve(int B, int k, int m, const double* __restrict__ H, const double* __restrict__ g,
                            double* __restrict__ y) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const double* Hb = H + (size_t)b * m * (m + 1);
  const double* gb = g + (size_t)b * (m + 1);
  double* yb = y + (size_t)b * m;
  for (int i = k - 1; i >= 0; --i) {
    double s = gb[i];
    for (int c = i + 1; c < k; ++c) s -= Hb[(size_t)c * (m + 1) + i] * yb[c];
    const double d = Hb[(size_t)i * (m + 1) + i];
    yb[i] = d != 0.0 ? s / d : 0.0;
  }
}

// x = sum_j y_j Z_j
template <bool V4>
__global__ void k_fg_update(int N, const float* __restrict__ Z, size_t zstride, int k, int m, const double* __restrict__ y,
                            float* __restrict__ x) {
  __shared__ float ys[FG_MMAX];
  const int b = blockIdx.y;
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = (float)y[(size_t)b * m + i];
  __syncthreads();
  const size_t off = (size_t)b * N;
  const int n = V4 ? N >> 2 : N;
  GRID_LOOP(q, n) {
    float4 a = f4(0.f);
    for (int j = 0; j < k; ++j) a = a + ys[j] * vld<V4>(Z + j * zstride + off, q);
    vst<V4>(x + off, q, a);
  }
}

// out = g (FP64) with partials of |g|^2: the residual of a solve from zero.
__global__ void k_copy_norm64(int N, const double* __restrict__ g, double* __restrict__ out, double* __restrict__ part) {
  const int b = blockIdx.y;
  const size_t off = (size_t)b * N;
  double acc = 0;
  GRID_LOOP(p, N) {
    const double v = g[off + p];
    out[off + p] = v;
    acc += v * v;
  }
  double s = block_sum(acc);
  if (threadIdx.x == 0) part[b * MPN_PMAX + blockIdx.x] = s;
}

// With dinv set it also starts the finest level's smoother on r32 (the
// V-cycle that follows): d = e = inv_th D^-1 r32.
__global__ void k_to32(int N, const double* __restrict__ r64, const double* __restrict__ part, int P,
                       float* __restrict__ r32, double* __restrict__ scale, const float* __restrict__ dinv,
                       float inv_th, float* __restrict__ e, float* __restrict__ d) {
  int b = blockIdx.y;
  double nn = sqrt(sum_partials(part, b, P));
  if (blockIdx.x == 0 && threadIdx.x == 0) scale[b] = nn;
  double inv = nn > 0 ? 1.0 / nn : 0.0;
  size_t off = (size_t)b * N;
  GRID_LOOP(p, N) {
    const float r = (float)(r64[off + p] * inv);
    r32[off + p] = r;
    if (dinv) {
      const float v = inv_th * (dinv[off + p] * r);
      e[off + p] = v;
      if (d) d[off + p] = v;
    }
  }
}

// u += scale * x; partials ||scale x||^2 and ||u||^2
__global__ void k_update64(int N, const float* __restrict__ x, const double* __restrict__ scale,
                           double* __restrict__ u, double* __restrict__ part_du, double* __restrict__ part_u) {
  int b = blockIdx.y;
  double s = scale[b];
  size_t off = (size_t)b * N;
  double a1 = 0, a2 = 0;
  GRID_LOOP(p, N) {
    double du = s * (double)x[off + p];
    double un = u[off + p] + du;
    u[off + p] = un;
    a1 += du * du; a2 += un * un;
  }
  double s1 = block_sum(a1);
  double s2 = block_sum(a2);
  if (threadIdx.x == 0) { part_du[b * MPN_PMAX + blockIdx.x] = s1; part_u[b * MPN_PMAX + blockIdx.x] = s2; }
}

// out[k][b] = sum of partial slot k of instance b (k < nslots)
__global__ void k_collect(int B, int nslots, const double* __restrict__ part, int P, double* __restrict__ out) {
  int b = blockIdx.x;
  for (int k = 0; k < nslots; ++k) {
    double v = sum_partials(part + (size_t)k * B * MPN_PMAX, b, P);
    if (threadIdx.x == 0) out[k * B + b] = v;
  }
}

__global__ void k_set_u(int N, const float* __restrict__ u0, double* __restrict__ u) {
  size_t off = (size_t)blockIdx.y * N;
  GRID_LOOP(p, N) u[off + p] = u0 ? (double)u0[off + p] : 0.0;
}

// ----------------------------------------------- derivative unknowns and grads
// Every unknown of z at point p from u (FP64).  The derivative unknowns of
// point i minimise the rows owned by i; in scaled units w = (s u', s^2 u'')
// and with h_g = S^{-1} g_zeta (adjoint source; zero for the forward pass):
//   w = a(u) + W^{-1} h_g - rho E* W^{-1} beta,
//   E* = L u - bE + beta^T W^{-1} h_g,
// a(u) the difference forms of Eq. 5.  This form has no cancellation: E* is
// the (small) equation-row residual.  The duals follow from it:
// lambda_E = -rho E* (forward, bE = b) and d_lambda_E = -rho E* (adjoint).
// Returns rho E*.
// A point with a Neumann / mixed row B u + gamma^T w = omega (gamma = beta / s
// on the first derivative along its axis e) has two point rows: with
// E* = (E1*, E2*), E2* = B u - omE + gamma^T W^{-1} h_g, and R its 2x2 weight,
//   w = a(u) + W^{-1} h_g - W^{-1} (beta (R E*)_1 + gamma (R E*)_2),
// the duals of its equation and boundary rows are -(R E*)_1 and -(R E*)_2.
// Returns (R E*)_1 and writes (R E*)_2 to *rE2 (E2* itself, the Dirichlet
// residual u - omega, at other boundary points; 0 elsewhere).
template <int D, int MASK>
__device__ __forceinline__ double recover_point(const Grid& g, const Coef64<MASK>& C, int b, int p, const int pos[3],
                                                const double* __restrict__ u, double rho, double bE, double omE,
                                                const float* __restrict__ gz, double* zo, double* rE2) {
  constexpr int V = 1 + 2 * D;
  size_t off = (size_t)b * g.N;
  double uc = u[off + p];
  double Est = C.at(0, p) * uc - bE;
  double a[3][2], hw[3][2], qb[3][2], is[3][2];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    double a1 = 0, a2 = 0;
    if (!g.st64 && (g.per[d] || (pos[d] > 0 && pos[d] < g.n[d] - 1))) {
      const double um = u[off + nbr(g, p, pos, d, -1)], up = u[off + nbr(g, p, pos, d, 1)];
      a1 = 0.5 * (up - um); a2 = up - 2.0 * uc + um;
    } else {
#pragma unroll
      for (int o = -2; o <= 2; ++o) {
        double w1 = swt<double>(g, b, d, pos[d], 1, o), w2 = swt<double>(g, b, d, pos[d], 2, o);
        if (w1 == 0.0 && w2 == 0.0) continue;
        double xv = o == 0 ? uc : u[off + nbr(g, p, pos, d, o)];
        a1 += w1 * xv; a2 += w2 * xv;
      }
    }
    const double i1 = sis1<double>(g, b, d, pos[d]), i2 = sis2<double>(g, b, d, pos[d]);
    is[d][0] = i1; is[d][1] = i2;
    double b1 = C.at(1 + 2 * d, p) * i1;
    double b2 = C.at(2 + 2 * d, p) * i2;
    a[d][0] = a1; a[d][1] = a2;
    Est += b1 * a1 + b2 * a2;
    swinv<double>(g, b, d, pos[d], b1, b2, qb[d][0], qb[d][1]);    // W^{-1} beta
    hw[d][0] = hw[d][1] = 0;
    if (gz) {
      double g1 = (double)gz[((size_t)b * V + 1 + 2 * d) * g.N + p] * i1;
      double g2 = (double)gz[((size_t)b * V + 2 + 2 * d) * g.N + p] * i2;
      swinv<double>(g, b, d, pos[d], g1, g2, hw[d][0], hw[d][1]);  // W^{-1} h_g
      Est += b1 * hw[d][0] + b2 * hw[d][1];
    }
  }
  double rE = rho * Est;
  zo[0] = uc;
  const int e = mixed_axis(g, pos);
  if (e >= 1) {
    const double gm = g.bcb[e] * is[e][0];
    const double E2 = Brow<double>(g, b, p, pos, e, u + off) - omE + gm * hw[e][0];
    const double r12 = g.r12d[off + p], r22 = g.r22d[off + p];
    rE = rho * Est + r12 * E2;
    const double re2 = r12 * Est + r22 * E2;
    double qg1, qg2;
    swinv<double>(g, b, e, pos[e], gm, 0.0, qg1, qg2);   // W^{-1} gamma
    hw[e][0] -= re2 * qg1;
    hw[e][1] -= re2 * qg2;
    *rE2 = re2;
  } else {
    *rE2 = is_boundary(g, pos) ? uc - omE : 0.0;
  }
#pragma unroll
  for (int d = 0; d < D; ++d) {
    zo[1 + 2 * d] = (a[d][0] + hw[d][0] - rE * qb[d][0]) * is[d][0];
    zo[2 + 2 * d] = (a[d][1] + hw[d][1] - rE * qb[d][1]) * is[d][1];
  }
  return rE;
}

// z (FP32 and/or FP64) from u.
template <int D, int MASK>
__global__ void k_recover(Grid g, Coef cf, const double* __restrict__ rho64, const double* __restrict__ u,
                          const float* __restrict__ bE, const float* __restrict__ omE, const float* __restrict__ gz,
                          float* __restrict__ zf, double* __restrict__ zd) {
  int b = blockIdx.y;
  const Coef64<MASK> C(cf, b);
  constexpr int V = 1 + 2 * D;
  size_t off = (size_t)b * g.N;
  GRID_LOOP(p, g.N) {
    int pos[3]; decode_fast(g, p, pos);
    double zo[7], r2;
    recover_point<D, MASK>(g, C, b, p, pos, u, rho64[off + p], bE ? (double)bE[off + p] : 0.0,
                           omE ? (double)omE[off + p] : 0.0, gz, zo, &r2);
    size_t zb = (size_t)b * V * g.N;
    for (int v = 0; v < V; ++v) {
      if (zf) zf[zb + (size_t)v * g.N + p] = (float)zo[v];
      if (zd) zd[zb + (size_t)v * g.N + p] = zo[v];
    }
  }
}

// Gradients (formulas after Eq. 11) at every point from the forward u and the
// adjoint d_u (both FP64):
//   lambda_E = b - E z* = rho (b - L u)                       (closed form)
//   dlambda_E = -E d_z = -rho (L d_u + beta^T W^{-1} S^{-1} g_zeta)
//   dl/dc_v = dlambda_E z_v + lambda_E dz_v,  dl/db = -dlambda_E,
//   dl/domega = -d_lambda_B: d_u on Dirichlet points, (R E*)_2 of the adjoint
//   on Neumann / mixed points.
// z and d_z are recovered on the fly.  Field
// gradients sum over the unknowns sharing a field; scalar gradients are
// reduced per instance (partials in part[v]).
template <int D, int MASK>
__global__ void k_gradients(Grid g, Coef cf, const double* __restrict__ rho64, const float* __restrict__ rhs,
                            const float* __restrict__ omega,
                            const double* __restrict__ uf, const double* __restrict__ du, const float* __restrict__ gz,
                            float* __restrict__ dfields, float* __restrict__ drhs, float* __restrict__ domega,
                            float* __restrict__ dz_out, double* __restrict__ dz64_out, double* __restrict__ part) {
  int b = blockIdx.y;
  const Coef64<MASK> C(cf, b);
  constexpr int V = 1 + 2 * D;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  size_t off = (size_t)b * g.N;
  GRID_LOOP(p, g.N) {
    int pos[3]; decode_fast(g, p, pos);
    double zv[7], dv[7], r2, dr2;
    double r = rho64[off + p];
    double lam = -recover_point<D, MASK>(g, C, b, p, pos, uf, r, (double)rhs[off + p], (double)omega[off + p],
                                         nullptr, zv, &r2);
    double dlam = -recover_point<D, MASK>(g, C, b, p, pos, du, r, 0.0, 0.0, gz, dv, &dr2);
    double cv[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      cv[v] = dlam * zv[v] + lam * dv[v];
      if (cf.field_of[v] < 0) acc[v] += cv[v];
    }
#pragma unroll
    for (int f = 0; f < 7; ++f) {
      if (f >= cf.F) break;
      double s = 0;
#pragma unroll
      for (int v = 0; v < V; ++v) if (cf.field_of[v] == f) s += cv[v];
      dfields[((size_t)f * cf.B + b) * g.N + p] = (float)s;
    }
    drhs[off + p] = (float)(-dlam);
    domega[off + p] = is_boundary(g, pos) ? (float)dr2 : 0.f;
    if (dz_out) {
#pragma unroll
      for (int v = 0; v < V; ++v) dz_out[((size_t)b * V + v) * g.N + p] = (float)dv[v];
    }
    if (dz64_out) {
#pragma unroll
      for (int v = 0; v < V; ++v) dz64_out[((size_t)b * V + v) * g.N + p] = dv[v];
    }
  }
#pragma unroll
  for (int v = 0; v < V; ++v) {
    double s = block_sum(acc[v]);
    if (threadIdx.x == 0) part[((size_t)v * cf.B + b) * MPN_PMAX + blockIdx.x] = s;
  }
}

// Adjoint right-hand side, part 1: per point psi = (W + beta beta^T)^{-1} S^{-1} g_zeta
// and the coefficients of M_{u zeta} M_{zeta zeta}^{-1} g_zeta as a scatter through
// the difference forms: kap[0] = c_0 beta.psi (center), kap[1+2d], kap[2+2d] = -(W_d psi_d).
template <int D, int MASK>
__global__ void k_adj_kappa(Grid g, Coef cf, const float* __restrict__ gz, double* __restrict__ kap) {
  int b = blockIdx.y;
  const Coef64<MASK> C(cf, b);
  constexpr int V = 1 + 2 * D;
  GRID_LOOP(p, g.N) {
    int pos[3]; decode_fast(g, p, pos);
    double hw[3][2], be[3][2], bwh = 0, gam = 0;
    #pragma unroll
    for (int d = 0; d < D; ++d) {
      const double i1 = sis1<double>(g, b, d, pos[d]), i2 = sis2<double>(g, b, d, pos[d]);
      double b1 = C.at(1 + 2 * d, p) * i1;
      double b2 = C.at(2 + 2 * d, p) * i2;
      be[d][0] = b1; be[d][1] = b2;
      double h1 = (double)gz[((size_t)b * V + 1 + 2 * d) * g.N + p] * i1;
      double h2 = (double)gz[((size_t)b * V + 2 + 2 * d) * g.N + p] * i2;
      swinv<double>(g, b, d, pos[d], h1, h2, hw[d][0], hw[d][1]);
      double q1, q2; swinv<double>(g, b, d, pos[d], b1, b2, q1, q2);
      bwh += b1 * hw[d][0] + b2 * hw[d][1];
      gam += b1 * q1 + b2 * q2;
    }
    // (W + K K^T)^{-1} h = W^{-1} h - W^{-1} K (I + K^T W^{-1} K)^{-1} K^T W^{-1} h with
    // K = [beta] (one row) or [beta, gamma] at a Neumann / mixed point
    double fac = bwh / (1.0 + gam), fac2 = 0.0, gm = 0.0, qg1 = 0.0, qg2 = 0.0;
    const int e = mixed_axis(g, pos);
    if (e >= 1) {
      gm = g.bcb[e] * sis1<double>(g, b, e, pos[e]);
      swinv<double>(g, b, e, pos[e], gm, 0.0, qg1, qg2);
      const double hwg = gm * hw[e][0];
      const double g12 = be[e][0] * qg1 + be[e][1] * qg2, g22 = gm * qg1;
      const double idet = 1.0 / ((1.0 + gam) * (1.0 + g22) - g12 * g12);
      fac = ((1.0 + g22) * bwh - g12 * hwg) * idet;
      fac2 = ((1.0 + gam) * hwg - g12 * bwh) * idet;
    }
    double bpsi = 0, gpsi = 0;
    #pragma unroll
    for (int d = 0; d < D; ++d) {
      double q1, q2; swinv<double>(g, b, d, pos[d], be[d][0], be[d][1], q1, q2);
      double ps1 = hw[d][0] - q1 * fac, ps2 = hw[d][1] - q2 * fac;
      if (d == e) { ps1 -= qg1 * fac2; ps2 -= qg2 * fac2; gpsi = gm * ps1; }
      bpsi += be[d][0] * ps1 + be[d][1] * ps2;
      double w11, w12, w22; swmat(g, b, d, pos[d], w11, w12, w22);
      kap[((size_t)(1 + 2 * d) * gridDim.y + b) * g.N + p] = -(w11 * ps1 + w12 * ps2);
      kap[((size_t)(2 + 2 * d) * gridDim.y + b) * g.N + p] = -(w12 * ps1 + w22 * ps2);
    }
    // the boundary row's u part is alpha at the point itself
    kap[(size_t)b * g.N + p] = C.at(0, p) * bpsi + (e >= 1 ? g.bca[e] * gpsi : 0.0);
  }
}

// Adjoint right-hand side, part 2: rhs_u = g_u - scatter(kap)  (FP64).
template <int D>
__global__ void k_adj_rhs(Grid g, const float* __restrict__ gz, const double* __restrict__ kap,
                          double* __restrict__ out) {
  int b = blockIdx.y;
  int V = 1 + 2 * g.D, B = gridDim.y;
  GRID_LOOP(p, g.N) {
    int pos[3]; decode_fast(g, p, pos);
    double acc = kap[(size_t)b * g.N + p];
    #pragma unroll
    for (int d = 0; d < D; ++d)
      for (int o = -2; o <= 2; ++o) {
        int ip = pos[d] - o;
        if (g.per[d]) ip = wrap1(ip, g.n[d]);
        else if (ip < 0 || ip >= g.n[d]) continue;
        double w1 = swt<double>(g, b, d, ip, 1, o), w2 = swt<double>(g, b, d, ip, 2, o);
        if (w1 == 0.0 && w2 == 0.0) continue;
        int q = p + (ip - pos[d]) * g.stride[d];
        acc += w1 * kap[((size_t)(1 + 2 * d) * B + b) * g.N + q] + w2 * kap[((size_t)(2 + 2 * d) * B + b) * g.N + q];
      }
    out[(size_t)b * g.N + p] = (double)gz[(size_t)b * V * g.N + p] - acc;
  }
}

__global__ void k_scalar_grads(int V, int B, const int* __restrict__ field_of_dev, const double* __restrict__ part,
                               int P, float* __restrict__ dscalars) {
  int b = blockIdx.x;
  for (int v = 0; v < V; ++v) {
    double s = sum_partials(part + (size_t)v * B * MPN_PMAX, b, P);
    if (threadIdx.x == 0) dscalars[v * B + b] = field_of_dev[v] < 0 ? (float)s : 0.f;
  }
}

// g_z = d/dz of mean_{b,i} (u - target)^2
__global__ void k_mse_grad(int N, int V, int B, const float* __restrict__ z, const float* __restrict__ tgt,
                           float* __restrict__ gz) {
  int b = blockIdx.y;
  float sc = 2.f / ((float)N * (float)B);
  size_t zb = (size_t)b * V * N;
  GRID_LOOP(p, N) {
    gz[zb + p] = sc * (z[zb + p] - tgt[(size_t)b * N + p]);
    for (int v = 1; v < V; ++v) gz[zb + (size_t)v * N + p] = 0.f;
  }
}


// Partials of the size of z(u) and of the last correction measured on every
// unknown: u itself plus, per dimension, its first and second difference
// quotients (the derivative unknowns up to their small point-local
// correction).  Only a couple of digits are needed, so FP32.
__global__ void k_znorm(Grid g, const double* __restrict__ u, const float* __restrict__ x,
                        const double* __restrict__ scale, double* __restrict__ part_dz, double* __restrict__ part_z) {
  int b = blockIdx.y;
  float sc = (float)scale[b];
  size_t off = (size_t)b * g.N;
  const double* ub = u + off;
  const float* xb = x + off;
  float a1 = 0, a2 = 0;
  GRID_LOOP(p, g.N) {
    int pos[3]; decode_fast(g, p, pos);
    float uc = (float)ub[p], xc = sc * xb[p];
    a2 += uc * uc; a1 += xc * xc;
    const bool edge = any_edge(g, pos);
    for (int d = 0; d < g.D; ++d) {
      float u1 = 0, u2 = 0, x1 = 0, x2 = 0;
      if (!edge) {
        int qm = nbr(g, p, pos, d, -1), qp = nbr(g, p, pos, d, 1);
        float um = (float)ub[qm], up = (float)ub[qp], xm = sc * xb[qm], xp = sc * xb[qp];
        u1 = 0.5f * (up - um); u2 = up - 2.f * uc + um;
        x1 = 0.5f * (xp - xm); x2 = xp - 2.f * xc + xm;
      } else {
        for (int o = -2; o <= 2; ++o) {
          float w1 = swt<float>(g, b, d, pos[d], 1, o), w2 = swt<float>(g, b, d, pos[d], 2, o);
          if (w1 == 0.f && w2 == 0.f) continue;
          int q = o == 0 ? p : nbr(g, p, pos, d, o);
          float uv = (float)ub[q], xv = sc * xb[q];
          u1 += w1 * uv; u2 += w2 * uv; x1 += w1 * xv; x2 += w2 * xv;
        }
      }
      const float i1 = sis1<float>(g, b, d, pos[d]), i2 = sis2<float>(g, b, d, pos[d]);
      u1 *= i1; u2 *= i2; x1 *= i1; x2 *= i2;
      a2 += u1 * u1 + u2 * u2; a1 += x1 * x1 + x2 * x2;
    }
  }
  double s1 = block_sum((double)a1);
  double s2 = block_sum((double)a2);
  if (threadIdx.x == 0) { part_dz[b * MPN_PMAX + blockIdx.x] = s1; part_z[b * MPN_PMAX + blockIdx.x] = s2; }
}

// ------------------------------------------------- FP64 refinement residual
// Two passes so that every FP64 operation is done once per point (FP64
// throughput, not memory, bounds these):
//   k_res64_y:  y = rho (b - L u)              (b, u nullable => 0)
//   k_res64_q:  r = base + L^T y + theta 1_B (omega - u), partials of ||r||^2
// Points away from non-periodic edges use the central weights directly.  A
// point with a Neumann / mixed row takes (y, y2) = R (b - L u, omega - B u)
// and its boundary row adds B^T y2 (omega nullable => 0).
template <int D, int MASK>
__global__ void k_res64_y(Grid g, Coef cf, const double* __restrict__ rho64, const double* __restrict__ u,
                          const float* __restrict__ bsrc, const float* __restrict__ omega, double* __restrict__ y) {
  int b = blockIdx.y;
  size_t off = (size_t)b * g.N;
  const Coef64<MASK> C(cf, b);
  GRID_LOOP(p, g.N) {
    int pos[3]; decode_fast(g, p, pos);
    double Lu = 0;
    if (u) {
      double uc = u[off + p];
      if (!any_edge(g, pos)) {
        Lu = C.at(0, p) * uc;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          double um = u[off + nbr(g, p, pos, d, -1)], up = u[off + nbr(g, p, pos, d, 1)];
          Lu += C.at(1 + 2 * d, p) * (0.5 * g.ds1[d]) * (up - um) + C.at(2 + 2 * d, p) * g.ds2[d] * (up - 2.0 * uc + um);
        }
      } else {
        Lu = Lrow<double, D>(g, cf, b, p, pos, u + off, nullptr);
      }
    }
    double s = bsrc ? (double)bsrc[off + p] : 0.0;
    const int e = mixed_axis(g, pos);
    if (e >= 1) {
      const double eB = (omega ? (double)omega[off + p] : 0.0) - (u ? Brow<double>(g, b, p, pos, e, u + off) : 0.0);
      const double r12 = g.r12d[off + p];
      y[off + p] = rho64[off + p] * (s - Lu) + r12 * eB;
      g.y2d[off + p] = r12 * (s - Lu) + g.r22d[off + p] * eB;
      continue;
    }
    y[off + p] = rho64[off + p] * (s - Lu);
  }
}

template <int D, int MASK>
__global__ void k_res64_q(Grid g, Coef cf, const double* __restrict__ y, const double* __restrict__ base,
                          const float* __restrict__ omega, const double* __restrict__ u, double* __restrict__ out,
                          double* __restrict__ part) {
  int b = blockIdx.y;
  size_t off = (size_t)b * g.N;
  const Coef64<MASK> C(cf, b);
  double acc = 0;
  GRID_LOOP(p, g.N) {
    int pos[3]; decode_fast(g, p, pos);
    double q;
    const double* yb = y + off;
    if (!any_edge(g, pos)) {
      double yc = yb[p];
      q = C.at(0, p) * yc;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        int pm = nbr(g, p, pos, d, -1), pp = nbr(g, p, pos, d, 1);
        double ym = yb[pm], yp = yb[pp];
        const int v1 = 1 + 2 * d, v2 = 2 + 2 * d;
        if (Coef64<MASK>::scal(v1)) q += (0.5 * g.ds1[d] * C.sv[v1]) * (ym - yp);
        else q += 0.5 * g.ds1[d] * (C.at(v1, pm) * ym - C.at(v1, pp) * yp);
        if (Coef64<MASK>::scal(v2)) q += (g.ds2[d] * C.sv[v2]) * (ym - 2.0 * yc + yp);
        else q += g.ds2[d] * (C.at(v2, pm) * ym - 2.0 * C.at(v2, p) * yc + C.at(v2, pp) * yp);
      }
    } else {
      q = LTgather<double, D>(g, cf, b, p, pos, yb);
      if (g.mixed) q += BTgather<double>(g, b, p, pos, g.y2d + off);
    }
    if (base) q += base[off + p];
    if (is_boundary_t<D>(g, pos) && mixed_axis(g, pos) < 0)
      q += (double)g.theta * ((omega ? (double)omega[off + p] : 0.0) - (u ? u[off + p] : 0.0));
    out[off + p] = q;
    acc += q * q;
  }
  double s = block_sum(acc);
  if (threadIdx.x == 0) part[b * MPN_PMAX + blockIdx.x] = s;
}
