// Learned warm start: kernels of a small 3x3x3 convolutional network on the
// (t, x, y) grid, BF16 activations and weights with FP32 accumulation.
//
// Layout: activations channels-last [B][N][C] (C = 16 or 32, zero-padded
// channels), weights [27][Cout][Cin] (tap = (dt+1)*9 + (dx+1)*3 + (dy+1)),
// biases FP32 [Cout].  Time is zero-padded; x and y wrap when periodic and are
// zero-padded otherwise.
//
//   mpn_conv3d_forward        y = act(conv(x, W) + b)      tensor cores (mma.sync m16n8k16 bf16)
//   mpn_conv3d_backward_data  dx = conv^T(dy, W)            same kernel on flipped, transposed W
//   mpn_conv3d_backward_weights dW, db from dy and x       tensor cores per tap and chunk of points,
//                                                           then a fixed-order sum over the chunks
//   mpn_relu_mask             g = dx * (y > 0) -> BF16
//   mpn_adam_step             FP32 masters + BF16 copy
//   mpn_pack_inputs / mpn_mse_u  data plumbing of the net
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstring>
#include <cstdint>

#include "../../include/mpn.h"
#include "mpn_conv_tc.cuh"

namespace {

struct CGrid {
  int n[3], per[3], N;
};

CGrid make_cgrid(const mpn_conv_desc* d) {
  CGrid g;
  for (int k = 0; k < 3; ++k) { g.n[k] = d->n[k]; g.per[k] = d->periodic[k]; }
  g.N = d->n[0] * d->n[1] * d->n[2];
  return g;
}

__device__ __forceinline__ void cdecode(const CGrid& g, int p, int pos[3]) {
  pos[2] = p % g.n[2];
  int q = p / g.n[2];
  pos[1] = q % g.n[1];
  pos[0] = q / g.n[1];
}

// neighbour index of a point at offset (dt, dx, dy), or -1 (zero padding)
__device__ __forceinline__ int cnbr(const CGrid& g, const int pos[3], int dt, int dx, int dy) {
  int t = pos[0] + dt, x = pos[1] + dx, y = pos[2] + dy;
  if (t < 0 || t >= g.n[0]) return -1;
  if (x < 0 || x >= g.n[1]) { if (!g.per[1]) return -1; x = x < 0 ? x + g.n[1] : x - g.n[1]; }
  if (y < 0 || y >= g.n[2]) { if (!g.per[2]) return -1; y = y < 0 ? y + g.n[2] : y - g.n[2]; }
  return (t * g.n[1] + x) * g.n[2] + y;
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// Implicit-GEMM convolution: one warp computes 32 points x CO channels; the
// A fragments (points x input channels of one tap) are gathered from the
// channels-last input, the B fragments (input x output channels) from W.
// FLAGS: bit 0 ReLU, bit 1 FP32 output (else BF16), bit 2 add bias.
template <int CI, int CO, int FLAGS>
__global__ void __launch_bounds__(128) k_conv(CGrid g, const __nv_bfloat16* __restrict__ x,
                                              const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias,
                                              void* __restrict__ out) {
  constexpr int NT = CO / 8;   // n-tiles
  constexpr int KS = CI / 16;  // k-steps per tap
  extern __shared__ __align__(16) __nv_bfloat16 ws[];   // 27 * CO * CI weights
  for (int i = threadIdx.x; i < 27 * CO * CI / 2; i += blockDim.x)
    reinterpret_cast<uint32_t*>(ws)[i] = reinterpret_cast<const uint32_t*>(w)[i];
  __syncthreads();
  const int b = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const int base = (blockIdx.x * 4 + warp) * 32;
  const __nv_bfloat16* xb = x + (size_t)b * g.N * CI;
  // the four points of this thread: rows gid and gid+8 of m-tiles 0 and 1
  int pt[4], pos[4][3];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    pt[r] = base + (r >> 1) * 16 + (r & 1) * 8 + gid;
    if (pt[r] < g.N) cdecode(g, pt[r], pos[r]); else { pos[r][0] = -100; pos[r][1] = pos[r][2] = 0; }
  }
  float acc[2][NT][4];
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int n = 0; n < NT; ++n)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[m][n][k] = 0.f;
  for (int tap = 0; tap < 27; ++tap) {
    int dt = tap / 9 - 1, dx = (tap / 3) % 3 - 1, dy = tap % 3 - 1;
    int nb[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) nb[r] = pos[r][0] < 0 ? -1 : cnbr(g, pos[r], dt, dx, dy);
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      uint32_t a[2][4];
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        int r0 = nb[2 * m], r1 = nb[2 * m + 1];
        int c0 = ks * 16 + tig * 2;
        a[m][0] = r0 >= 0 ? ld_pair(xb + (size_t)r0 * CI + c0) : 0u;
        a[m][1] = r1 >= 0 ? ld_pair(xb + (size_t)r1 * CI + c0) : 0u;
        a[m][2] = r0 >= 0 ? ld_pair(xb + (size_t)r0 * CI + c0 + 8) : 0u;
        a[m][3] = r1 >= 0 ? ld_pair(xb + (size_t)r1 * CI + c0 + 8) : 0u;
      }
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        const __nv_bfloat16* wr = ws + ((size_t)tap * CO + n * 8 + gid) * CI + ks * 16 + tig * 2;
        uint32_t bb[2] = {ld_pair(wr), ld_pair(wr + 8)};
        mma_bf16(acc[0][n], a[0], bb);
        mma_bf16(acc[1][n], a[1], bb);
      }
    }
  }
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int p = pt[2 * m + h];
      if (p >= g.N) continue;
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        int co = n * 8 + tig * 2;
        float v0 = acc[m][n][2 * h], v1 = acc[m][n][2 * h + 1];
        if (FLAGS & 4) { v0 += bias[co]; v1 += bias[co + 1]; }
        if (FLAGS & 1) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
        size_t o = ((size_t)b * g.N + p) * CO + co;
        if (FLAGS & 2) {
          reinterpret_cast<float*>(out)[o] = v0;
          reinterpret_cast<float*>(out)[o + 1] = v1;
        } else {
          __nv_bfloat162 pr = __floats2bfloat162_rn(v0, v1);
          *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(out) + o) = pr;
        }
      }
    }
}

// W'[tap][ci][co] = W[26 - tap][co][ci]: weights of the transposed convolution
__global__ void k_flip_transpose(int CI, int CO, const __nv_bfloat16* __restrict__ w, __nv_bfloat16* __restrict__ wt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 27 * CI * CO) return;
  int ci = i % CI, co = (i / CI) % CO, tap = i / (CI * CO);
  wt[((size_t)(26 - tap) * CI + ci) * CO + co] = w[i];
}

// Weight gradient on the tensor cores, stage 1: for one tap (blockIdx.y) and
// one chunk of points (blockIdx.x),
//   dW_tap[co][ci] = sum_p g[p][co] x[nbr(p, tap)][ci],
// a GEMM with M = co, N = ci and K running over the points: sub-tiles of 64
// points are staged in shared memory as bf16 pairs packed along the point
// axis (G as [co][pair], the tap's gathered X as [ci][pair]), so every
// m16n8k16 fragment register is one 32-bit shared load; each of the 4 warps
// takes 16 points of a sub-tile.  The warps' accumulators are added in a
// fixed order; the centre tap's CTAs also sum g for db.  Deterministic.
template <int CI, int CO>
__global__ void __launch_bounds__(128) k_wgrad_mma(CGrid g, long long total, int chunk,
                                                   const __nv_bfloat16* __restrict__ gr,
                                                   const __nv_bfloat16* __restrict__ x, float* __restrict__ part,
                                                   float* __restrict__ bpart) {
  constexpr int PT = 64, PP = PT / 2 + 4;     // points per sub-tile; pair stride (padded)
  constexpr int MT = CO / 16, NT = CI / 8;
  __shared__ uint32_t gs[CO * PP];            // G^T, packed point pairs
  __shared__ uint32_t xs[CI * PP];            // X_tap^T, packed point pairs
  __shared__ float red[CO * CI];
  __shared__ float bred[32 * CO];
  const int tap = blockIdx.y;
  const int dt = tap / 9 - 1, dx = (tap / 3) % 3 - 1, dy = tap % 3 - 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  // staging role: point pair j (0..31), channel quarter q (0..3)
  const int j = threadIdx.x >> 2, q = threadIdx.x & 3;
  const long long p0 = (long long)blockIdx.x * chunk;
  const long long p1 = p0 + chunk < total ? p0 + chunk : total;
  float acc[MT][NT][4];
#pragma unroll
  for (int m = 0; m < MT; ++m)
#pragma unroll
    for (int n = 0; n < NT; ++n)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[m][n][k] = 0.f;
  float bacc[CO / 4];
#pragma unroll
  for (int k = 0; k < CO / 4; ++k) bacc[k] = 0.f;
  for (long long base = p0; base < p1; base += PT) {
    // stage the pair (2j, 2j+1): channels [q C/4, (q+1) C/4) of g and of x at the neighbour
    uint32_t ga[CO / 8], gb[CO / 8], xa[CI / 8], xb[CI / 8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long pp = base + 2 * j + h;
      uint32_t* gw = h ? gb : ga;
      uint32_t* xw = h ? xb : xa;
      int nb = -1;
      size_t row = 0;
      if (pp < p1) {
        const int b = (int)(pp / g.N), p = (int)(pp - (long long)b * g.N);
        int pos[3]; cdecode(g, p, pos);
        const int qn = cnbr(g, pos, dt, dx, dy);
        row = (size_t)b * g.N;
        nb = qn;
        const uint32_t* src = reinterpret_cast<const uint32_t*>(gr + (row + p) * CO + q * (CO / 4));
#pragma unroll
        for (int k = 0; k < CO / 8; ++k) gw[k] = src[k];
      } else {
#pragma unroll
        for (int k = 0; k < CO / 8; ++k) gw[k] = 0u;
      }
      if (nb >= 0) {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(x + (row + nb) * CI + q * (CI / 4));
#pragma unroll
        for (int k = 0; k < CI / 8; ++k) xw[k] = src[k];
      } else {
#pragma unroll
        for (int k = 0; k < CI / 8; ++k) xw[k] = 0u;
      }
    }
#pragma unroll
    for (int k = 0; k < CO / 8; ++k) {
      const int c = q * (CO / 4) + 2 * k;
      gs[c * PP + j] = __byte_perm(ga[k], gb[k], 0x5410);
      gs[(c + 1) * PP + j] = __byte_perm(ga[k], gb[k], 0x7632);
      if (tap == 13) {
        const __nv_bfloat162 a2 = *reinterpret_cast<const __nv_bfloat162*>(&ga[k]);
        const __nv_bfloat162 b2 = *reinterpret_cast<const __nv_bfloat162*>(&gb[k]);
        bacc[2 * k] += __bfloat162float(a2.x) + __bfloat162float(b2.x);
        bacc[2 * k + 1] += __bfloat162float(a2.y) + __bfloat162float(b2.y);
      }
    }
#pragma unroll
    for (int k = 0; k < CI / 8; ++k) {
      const int c = q * (CI / 4) + 2 * k;
      xs[c * PP + j] = __byte_perm(xa[k], xb[k], 0x5410);
      xs[(c + 1) * PP + j] = __byte_perm(xa[k], xb[k], 0x7632);
    }
    __syncthreads();
    const int k0 = warp * 8;                  // this warp's first pair (16 points)
    uint32_t a[MT][4], bf[NT][2];
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      a[m][0] = gs[(m * 16 + gid) * PP + k0 + tig];
      a[m][1] = gs[(m * 16 + gid + 8) * PP + k0 + tig];
      a[m][2] = gs[(m * 16 + gid) * PP + k0 + tig + 4];
      a[m][3] = gs[(m * 16 + gid + 8) * PP + k0 + tig + 4];
    }
#pragma unroll
    for (int n = 0; n < NT; ++n) {
      bf[n][0] = xs[(n * 8 + gid) * PP + k0 + tig];
      bf[n][1] = xs[(n * 8 + gid) * PP + k0 + tig + 4];
    }
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
      for (int n = 0; n < NT; ++n) mma_bf16(acc[m][n], a[m], bf[n]);
    __syncthreads();
  }
  // the four warps' sums, added in warp order
  for (int i = threadIdx.x; i < CO * CI; i += blockDim.x) red[i] = 0.f;
  __syncthreads();
  for (int w = 0; w < 4; ++w) {
    if (warp == w) {
#pragma unroll
      for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int n = 0; n < NT; ++n) {
          const int co = m * 16 + gid, ci = n * 8 + 2 * tig;
          red[co * CI + ci] += acc[m][n][0];
          red[co * CI + ci + 1] += acc[m][n][1];
          red[(co + 8) * CI + ci] += acc[m][n][2];
          red[(co + 8) * CI + ci + 1] += acc[m][n][3];
        }
    }
    __syncthreads();
  }
  float* o = part + ((size_t)blockIdx.x * 27 + tap) * CO * CI;
  for (int i = threadIdx.x; i < CO * CI; i += blockDim.x) o[i] = red[i];
  if (tap == 13) {
#pragma unroll
    for (int k = 0; k < CO / 4; ++k) bred[j * CO + q * (CO / 4) + k] = bacc[k];
    __syncthreads();
    for (int c = threadIdx.x; c < CO; c += blockDim.x) {
      float sacc = 0.f;
      for (int jj = 0; jj < 32; ++jj) sacc += bred[jj * CO + c];
      bpart[(size_t)blockIdx.x * CO + c] = sacc;
    }
  }
}

// stage 2: sum of the chunk partials in a fixed order
__global__ void k_wgrad_reduce(int nchunk, int n, const float* __restrict__ part, float* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int c = 0; c < nchunk; ++c) s += part[(size_t)c * n + i];
  out[i] = s;
}

__global__ void k_relu_mask(long long n, const float* __restrict__ g, const __nv_bfloat16* __restrict__ y,
                            __nv_bfloat16* __restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v = g[i];
  if (y && !(__bfloat162float(y[i]) > 0.f)) v = 0.f;
  out[i] = __float2bfloat16_rn(v);
}

__global__ void k_adam(long long n, float* __restrict__ w, const float* __restrict__ gr, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                       __nv_bfloat16* __restrict__ wb) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float g = gr[i];
  float mi = b1 * m[i] + (1.f - b1) * g;
  float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi; v[i] = vi;
  float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  w[i] = wi;
  if (wb) wb[i] = __float2bfloat16_rn(wi);
}

// x0[b][p][c] = channels (fields..., rhs) scaled, zero-padded to 16, BF16
__global__ void k_pack(int N, int F, const float* __restrict__ fields, const float* __restrict__ rhs,
                       const float* __restrict__ scale, __nv_bfloat16* __restrict__ x0, int B) {
  int b = blockIdx.y;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    __nv_bfloat16* o = x0 + ((size_t)b * N + p) * 16;
    for (int c = 0; c < 16; ++c) {
      float v = 0.f;
      if (c < F) v = fields[((size_t)c * B + b) * N + p] * scale[c];
      else if (c == F) v = rhs[(size_t)b * N + p] * scale[c];
      o[c] = __float2bfloat16_rn(v);
    }
  }
}

// Channel F + 1: the running sum over time planes of rhs at the same (x, y)
// (planes 0..t), times scale[F + 1]: the solution of a PDE that is first order
// in time depends on the right-hand side of every earlier plane, which the
// 3x3x3 stencils of a few layers cannot reach.  One thread per (b, x, y).
__global__ void k_pack_tsum(int nt, int plane, int F, const float* __restrict__ rhs, const float* __restrict__ scale,
                            __nv_bfloat16* __restrict__ x0, int B) {
  const int b = blockIdx.y;
  const float sc = scale[F + 1];
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < plane; c += gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int t = 0; t < nt; ++t) {
      const size_t p = (size_t)b * nt * plane + (size_t)t * plane + c;
      acc += rhs[p];
      x0[p * 16 + F + 1] = __float2bfloat16_rn(acc * sc);
    }
  }
}

// MSE on channel 0 of the FP32 output y [B][N][16] against target t [B][N]
// (already divided by the output scale): g = 2 (y - t) / (B N) on channel 0,
// and per-block partial losses.
__global__ void k_mse_u(int N, const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ g,
                        float* __restrict__ lpart, int B) {
  __shared__ float sh[256];
  int b = blockIdx.y;
  float acc = 0.f;
  float sc = 2.f / ((float)N * (float)B);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    size_t o = ((size_t)b * N + p) * 16;
    float r = y[o] - t[(size_t)b * N + p];
    acc += r * r;
    g[o] = sc * r;
    for (int c = 1; c < 16; ++c) g[o + c] = 0.f;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) lpart[(size_t)b * gridDim.x + blockIdx.x] = sh[0];
}

// u0[b][p] = scale * y[b][p][0]
__global__ void k_unpack_u(int N, const float* __restrict__ y, float scale, float* __restrict__ u0, int B) {
  int b = blockIdx.y;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x)
    u0[(size_t)b * N + p] = scale * y[((size_t)b * N + p) * 16];
}

int check(const mpn_conv_desc* d) {
  if (!d || d->batch < 1) return MPN_ERR_INVALID_ARG;
  for (int k = 0; k < 3; ++k) if (d->n[k] < 2) return MPN_ERR_INVALID_ARG;
  if (d->periodic[0]) return MPN_ERR_INVALID_ARG;
  if (!((d->cin == 16 && d->cout == 32) || (d->cin == 32 && (d->cout == 32 || d->cout == 16))))
    return MPN_ERR_UNSUPPORTED;
  return MPN_OK;
}

template <int CI, int CO, int FL>
void launch_conv1(const CGrid& g, int B, const __nv_bfloat16* x, const __nv_bfloat16* w, const float* bias, void* y,
                  cudaStream_t st) {
  const int smem = 27 * CI * CO * (int)sizeof(__nv_bfloat16);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_conv<CI, CO, FL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  dim3 gr((g.N + 127) / 128, B);
  k_conv<CI, CO, FL><<<gr, 128, smem, st>>>(g, x, w, bias, y);
}

template <int CI, int CO>
void launch_conv(const CGrid& g, int B, int flags, const __nv_bfloat16* x, const __nv_bfloat16* w, const float* bias,
                 void* y, cudaStream_t st) {
  switch (flags) {
    case 2: launch_conv1<CI, CO, 2>(g, B, x, w, bias, y, st); break;
    case 5: launch_conv1<CI, CO, 5>(g, B, x, w, bias, y, st); break;
    case 6: launch_conv1<CI, CO, 6>(g, B, x, w, bias, y, st); break;
    default: launch_conv1<CI, CO, 0>(g, B, x, w, bias, y, st); break;
  }
}

// Accumulator read-back: 32 lanes x N FP32 columns of this warp, one lane per
// thread (tcgen05.ld 32x32b), then the wait for the load.
template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[N]);
template <>
__device__ __forceinline__ void tmem_ld<32>(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// The same convolution as k_conv on the 5th-generation tensor cores (see
// mpn_conv_tc.cuh): persistent CTAs over tiles of 128 points, warp-specialised;
// err (nullable) is set when a bounded wait gives up.
template <int CI, int CO, int FLAGS>
__global__ void __launch_bounds__(tc::TPB) k_conv_tc(CGrid g, int B, const __nv_bfloat16* __restrict__ x,
                                                     const __nv_bfloat16* __restrict__ w,
                                                     const float* __restrict__ bias, void* __restrict__ out,
                                                     int* __restrict__ err) {
  constexpr int KS = tc::ks_of(CI), WOP = tc::op_bytes(CO), AOP = tc::op_bytes(tc::TM), ABUF = tc::a_bytes(CI);
  constexpr int S = tc::slots(CI);
  extern __shared__ __align__(1024) uint8_t csm[];
  uint8_t* ws = csm;
  uint8_t* as = csm + tc::w_bytes(CI, CO);
  uint64_t* full = reinterpret_cast<uint64_t*>(as + S * ABUF);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;
  uint64_t* acce = accf + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(acce + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the weights of every tap as B operands: row co, K chunk of 8 input channels
  for (int i = tid; i < 27 * CO * (CI / 8); i += tc::TPB) {
    const int c8 = i % (CI / 8), co = (i / (CI / 8)) % CO, tap = i / ((CI / 8) * CO);
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(w + ((size_t)tap * CO + co) * CI + c8 * 8));
    *reinterpret_cast<uint4*>(ws + (tap * KS + (c8 >> 1)) * WOP + tc::chunk_off(co, c8 & 1)) = v;
  }
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      tc::bar_init(&full[i], tc::TM);
      tc::bar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::bar_init(&accf[i], 1);
      tc::bar_init(&acce[i], tc::TM);
    }
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::s32(tslot)),
                 "n"(tc::tmem_cols(CO)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::fence_async_smem();
  tc::tc_before_sync();
  __syncthreads();
  tc::tc_after_sync();
  const uint32_t tmem = *tslot;
  const int tpi = (g.N + tc::TM - 1) / tc::TM, ntiles = B * tpi;
  bool ok = true;
  auto wait = [&](uint64_t* bar, uint32_t par) {
    if (!tc::bar_wait(bar, par, ok ? tc::WAIT_LIMIT : 1)) ok = false;
  };

  if (warp < 4) {
    // ---- gather: thread tid is row tid of every tile
    const uint32_t abase = tc::s32(as);
    int G = 0;   // taps copied by this CTA
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      const int bb = tile / tpi, pp = (tile - bb * tpi) * tc::TM + tid;
      const bool valid = pp < g.N;
      int pos[3] = {0, 0, 0};
      if (valid) cdecode(g, pp, pos);
      const __nv_bfloat16* xb = x + (size_t)bb * g.N * CI;
      for (int t0 = 0; t0 < 27; t0 += tc::TPS, ++G) {
        const int sl = G % S, use = G / S;
        if (use > 0) wait(&empty[sl], (use - 1) & 1);   // the MMAs of the slot's last use are done
#pragma unroll
        for (int j = 0; j < tc::TPS; ++j) {
          const int tap = t0 + j;
          const int nb = valid ? cnbr(g, pos, tap / 9 - 1, (tap / 3) % 3 - 1, tap % 3 - 1) : -1;
          const __nv_bfloat16* src = nb >= 0 ? xb + (size_t)nb * CI : xb;
          const uint32_t dst = abase + sl * ABUF + j * KS * AOP;
#pragma unroll
          for (int c8 = 0; c8 < CI / 8; ++c8)
            tc::cp16(dst + (c8 >> 1) * AOP + tc::chunk_off(tid, c8 & 1), src + c8 * 8, nb >= 0 ? 16u : 0u);
        }
        tc::cp_arrive(&full[sl]);
      }
    }
    // this thread's last copies have landed before it leaves
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp == 4) {
    // ---- MMA issue (one thread)
    if (lane == 0) {
      const uint32_t id = tc::idesc(tc::TM, CO);
      const uint32_t wbase = tc::s32(ws), abase = tc::s32(as);
      int G = 0, i = 0;
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
        const int acc = i & 1;
        if (i >= 2) wait(&acce[acc], ((i - 2) >> 1) & 1);   // the epilogue has read this accumulator
        tc::tc_after_sync();
        for (int t0 = 0; t0 < 27; t0 += tc::TPS, ++G) {
          const int sl = G % S;
          wait(&full[sl], (G / S) & 1);
          tc::fence_async_smem();   // the landed copies before the tensor core's reads
          tc::tc_after_sync();
#pragma unroll
          for (int j = 0; j < tc::TPS; ++j) {
            const int tap = t0 + j;
#pragma unroll
            for (int ks = 0; ks < KS; ++ks)
              tc::mma(tmem + (uint32_t)((acc * tc::NACC + tap % tc::NACC) * CO),
                      tc::sdesc(abase + sl * ABUF + (j * KS + ks) * AOP), tc::sdesc(wbase + (tap * KS + ks) * WOP), id,
                      (tap >= tc::NACC || ks > 0) ? 1u : 0u);
          }
          tc::commit(&empty[sl]);
        }
        tc::commit(&accf[acc]);
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32 (w mod 4) .. + 31
    const int q = warp & 3, m = 32 * q + lane;
    int i = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
      const int acc = i & 1;
      wait(&accf[acc], (i >> 1) & 1);
      tc::tc_after_sync();
      float v[CO];
      tmem_ld<CO>(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * tc::NACC * CO), v);
#pragma unroll
      for (int j = 1; j < tc::NACC; ++j) {
        float u[CO];
        tmem_ld<CO>(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((acc * tc::NACC + j) * CO), u);
#pragma unroll
        for (int c = 0; c < CO; ++c) v[c] += u[c];
      }
      tc::tc_before_sync();
      tc::bar_arrive(&acce[acc]);
      const int b = tile / tpi, p = (tile - b * tpi) * tc::TM + m;
      if (p < g.N) {
        const size_t o = ((size_t)b * g.N + p) * CO;
#pragma unroll
        for (int c = 0; c < CO; ++c) {
          if (FLAGS & 4) v[c] += __ldg(bias + c);
          if (FLAGS & 1) v[c] = fmaxf(v[c], 0.f);
        }
        if (FLAGS & 2) {
          float4* dst = reinterpret_cast<float4*>(reinterpret_cast<float*>(out) + o);
#pragma unroll
          for (int c = 0; c < CO / 4; ++c) dst[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
        } else {
          uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(out) + o);
#pragma unroll
          for (int c = 0; c < CO / 8; ++c) {
            uint32_t u[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const __nv_bfloat162 h = __floats2bfloat162_rn(v[8 * c + 2 * k], v[8 * c + 2 * k + 1]);
              u[k] = *reinterpret_cast<const uint32_t*>(&h);
            }
            dst[c] = make_uint4(u[0], u[1], u[2], u[3]);
          }
        }
      }
    }
  }
  if (!ok && err) atomicExch(err, 1);
  // every role is done (the epilogue waited for the last accumulator, so no
  // MMA is in flight) before the tensor memory is freed
  tc::tc_before_sync();
  __syncthreads();
  if (warp == 4) {
    tc::tc_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(tc::tmem_cols(CO)) : "memory");
  }
}

// The row-staged tcgen05 convolution (n_y % 128 == 0; see mpn_conv_tc.cuh):
// tiles of 128 consecutive y points of one (t, x) row, one ring slot per time
// plane holding the tile's three staged x rows, nine taps per commit.
template <int CI, int CO, int FLAGS>
__global__ void __launch_bounds__(tc::TPB) k_conv_tcr(CGrid g, int B, const __nv_bfloat16* __restrict__ x,
                                                      const __nv_bfloat16* __restrict__ w,
                                                      const float* __restrict__ bias, void* __restrict__ out,
                                                      int* __restrict__ err) {
  constexpr int KS = tc::ks_of(CI), KC = CI / 8, WOP = tc::op_bytes(CO);
  constexpr int RB = tc::rb_bytes(CI), SLOT = tc::rs_bytes(CI), S = tc::rslots(CI);
  constexpr uint32_t SBO_A = KC * 128;
  extern __shared__ __align__(1024) uint8_t csm[];
  uint8_t* ws = csm;
  uint8_t* as = csm + tc::w_bytes(CI, CO);
  uint64_t* full = reinterpret_cast<uint64_t*>(as + S * SLOT);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;
  uint64_t* acce = accf + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(acce + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < 27 * CO * (CI / 8); i += tc::TPB) {
    const int c8 = i % (CI / 8), co = (i / (CI / 8)) % CO, tap = i / ((CI / 8) * CO);
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(w + ((size_t)tap * CO + co) * CI + c8 * 8));
    *reinterpret_cast<uint4*>(ws + (tap * KS + (c8 >> 1)) * WOP + tc::chunk_off(co, c8 & 1)) = v;
  }
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      tc::bar_init(&full[i], tc::TM);
      tc::bar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::bar_init(&accf[i], 1);
      tc::bar_init(&acce[i], tc::TM);
    }
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::s32(tslot)),
                 "n"(tc::tmem_cols(CO)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::fence_async_smem();
  tc::tc_before_sync();
  __syncthreads();
  tc::tc_after_sync();
  const uint32_t tmem = *tslot;
  const int nyb = g.n[2] / tc::TM, rows = g.n[0] * g.n[1];
  const int ntiles = B * rows * nyb;
  bool ok = true;
  auto wait = [&](uint64_t* bar, uint32_t par) {
    if (!tc::bar_wait(bar, par, ok ? tc::WAIT_LIMIT : 1)) ok = false;
  };
  // tile -> instance, time plane, x row, first y
  auto tile_of = [&](int tile, int& bb, int& t, int& xr, int& y0) {
    bb = tile / (rows * nyb);
    const int q = tile - bb * rows * nyb, row = q / nyb;
    t = row / g.n[1];
    xr = row - t * g.n[1];
    y0 = (q - row * nyb) * tc::TM;
  };

  if (warp < 4) {
    // ---- staging: per time plane, the tile's three x rows (entry e = (row dx,
    //      core row c', chunk kc, row k) holds channels 8 kc.. of point y0 - 1 + c' + 16 k)
    constexpr int NE = 3 * 18 * KC * 8;
    const uint32_t abase = tc::s32(as);
    int G = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      int bb, t, xr, y0;
      tile_of(tile, bb, t, xr, y0);
      const __nv_bfloat16* xb = x + (size_t)bb * g.N * CI;
      for (int dt = 0; dt < 3; ++dt, ++G) {
        const int sl = G % S, use = G / S;
        if (use > 0) wait(&empty[sl], (use - 1) & 1);
        const int tt = t + dt - 1;
        const uint32_t dst0 = abase + sl * SLOT;
        for (int e = tid; e < NE; e += tc::TM) {
          const int k = e & 7, kc = (e >> 3) % KC, cp = (e / (8 * KC)) % 18, dx = e / (8 * KC * 18);
          int xx = xr + dx - 1, y = y0 - 1 + cp + 16 * k;
          bool in = tt >= 0 && tt < g.n[0];
          if (xx < 0 || xx >= g.n[1]) { if (g.per[1]) xx = xx < 0 ? xx + g.n[1] : xx - g.n[1]; else in = false; }
          if (y < 0 || y >= g.n[2]) { if (g.per[2]) y = y < 0 ? y + g.n[2] : y - g.n[2]; else in = false; }
          const __nv_bfloat16* src = in ? xb + ((size_t)(tt * g.n[1] + xx) * g.n[2] + y) * CI + kc * 8 : xb;
          tc::cp16(dst0 + dx * RB + cp * SBO_A + kc * 128 + k * 16, src, in ? 16u : 0u);
        }
        tc::cp_arrive(&full[sl]);
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp == 4) {
    // ---- MMA issue: per slot nine taps (dx, dy), one commit
    if (lane == 0) {
      const uint32_t id = tc::idesc(tc::TM, CO);
      const uint32_t wbase = tc::s32(ws), abase = tc::s32(as);
      int G = 0, i = 0;
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
        const int acc = i & 1;
        if (i >= 2) wait(&acce[acc], ((i - 2) >> 1) & 1);
        tc::tc_after_sync();
        for (int dt = 0; dt < 3; ++dt, ++G) {
          const int sl = G % S;
          wait(&full[sl], (G / S) & 1);
          tc::fence_async_smem();
          tc::tc_after_sync();
#pragma unroll
          for (int j = 0; j < 9; ++j) {
            const int dx = j / 3, dy = j % 3, tap = dt * 9 + j;
#pragma unroll
            for (int ks = 0; ks < KS; ++ks)
              tc::mma(tmem + (uint32_t)((acc * tc::NACC + tap % tc::NACC) * CO),
                      tc::sdesc(abase + sl * SLOT + dx * RB + dy * SBO_A + ks * 256, SBO_A),
                      tc::sdesc(wbase + (tap * KS + ks) * WOP), id, (tap >= tc::NACC || ks > 0) ? 1u : 0u);
          }
          tc::commit(&empty[sl]);
        }
        tc::commit(&accf[acc]);
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue: TMEM lane m is the point y0 + (m >> 3) + 16 (m & 7)
    const int q = warp & 3, m = 32 * q + lane;
    int i = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
      const int acc = i & 1;
      wait(&accf[acc], (i >> 1) & 1);
      tc::tc_after_sync();
      float v[CO];
      tmem_ld<CO>(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * tc::NACC * CO), v);
#pragma unroll
      for (int j = 1; j < tc::NACC; ++j) {
        float u[CO];
        tmem_ld<CO>(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((acc * tc::NACC + j) * CO), u);
#pragma unroll
        for (int c = 0; c < CO; ++c) v[c] += u[c];
      }
      tc::tc_before_sync();
      tc::bar_arrive(&acce[acc]);
      int bb, t, xr, y0;
      tile_of(tile, bb, t, xr, y0);
      const int p = (t * g.n[1] + xr) * g.n[2] + y0 + (m >> 3) + 16 * (m & 7);
      const size_t o = ((size_t)bb * g.N + p) * CO;
#pragma unroll
      for (int c = 0; c < CO; ++c) {
        if (FLAGS & 4) v[c] += __ldg(bias + c);
        if (FLAGS & 1) v[c] = fmaxf(v[c], 0.f);
      }
      if (FLAGS & 2) {
        float4* dst = reinterpret_cast<float4*>(reinterpret_cast<float*>(out) + o);
#pragma unroll
        for (int c = 0; c < CO / 4; ++c) dst[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
      } else {
        uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(out) + o);
#pragma unroll
        for (int c = 0; c < CO / 8; ++c) {
          uint32_t u4[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(v[8 * c + 2 * k], v[8 * c + 2 * k + 1]);
            u4[k] = *reinterpret_cast<const uint32_t*>(&h);
          }
          dst[c] = make_uint4(u4[0], u4[1], u4[2], u4[3]);
        }
      }
    }
  }
  if (!ok && err) atomicExch(err, 1);
  tc::tc_before_sync();
  __syncthreads();
  if (warp == 4) {
    tc::tc_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(tc::tmem_cols(CO)) : "memory");
  }
}

// Set by a tcgen05 convolution whose bounded wait gave up (read and cleared
// by mpn_conv_take_error).
__device__ int g_conv_err = 0;

int* conv_err_ptr() {
  int* p = nullptr;
  return cudaGetSymbolAddress((void**)&p, g_conv_err) == cudaSuccess ? p : nullptr;
}

// resident CTAs per SM of a tcgen05 convolution kernel with `smem` bytes of
// dynamic shared memory (the tensor memory bound included), times the SMs
template <class K>
int tc_ctas(K kern, int smem, int co_cols_ctas) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  int dev = 0, nsm = 148, smem_sm = 233472;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  // resident CTAs: shared memory (1 KB reserved per CTA) and tensor memory
  int per = smem_sm / (smem + 1024);
  per = per < 1 ? 1 : (per > co_cols_ctas ? co_cols_ctas : per);
  return nsm * per;
}

template <int CI, int CO, int FL>
void launch_conv_tc1(const CGrid& g, int B, const __nv_bfloat16* x, const __nv_bfloat16* w, const float* bias,
                     void* y, cudaStream_t st) {
  if (g.n[2] % tc::TM == 0) {
    // rows of whole 128-point tiles: the row-staged kernel
    constexpr int smem = tc::rsmem_bytes(CI, CO);
    static int nctas = 0;
    if (!nctas) nctas = tc_ctas(k_conv_tcr<CI, CO, FL>, smem, tc::tmem_ctas(CO));
    const int ntiles = B * g.n[0] * g.n[1] * (g.n[2] / tc::TM);
    k_conv_tcr<CI, CO, FL><<<ntiles < nctas ? ntiles : nctas, tc::TPB, smem, st>>>(g, B, x, w, bias, y,
                                                                                  conv_err_ptr());
    return;
  }
  constexpr int smem = tc::smem_bytes(CI, CO);
  static int nctas = 0;
  if (!nctas) nctas = tc_ctas(k_conv_tc<CI, CO, FL>, smem, tc::tmem_ctas(CO));
  const int ntiles = B * ((g.N + tc::TM - 1) / tc::TM);
  k_conv_tc<CI, CO, FL><<<ntiles < nctas ? ntiles : nctas, tc::TPB, smem, st>>>(g, B, x, w, bias, y,
                                                                               conv_err_ptr());
}

template <int CI, int CO>
void launch_conv_tc(const CGrid& g, int B, int flags, const __nv_bfloat16* x, const __nv_bfloat16* w,
                    const float* bias, void* y, cudaStream_t st) {
  switch (flags) {
    case 2: launch_conv_tc1<CI, CO, 2>(g, B, x, w, bias, y, st); break;
    case 5: launch_conv_tc1<CI, CO, 5>(g, B, x, w, bias, y, st); break;
    case 6: launch_conv_tc1<CI, CO, 6>(g, B, x, w, bias, y, st); break;
    default: launch_conv_tc1<CI, CO, 0>(g, B, x, w, bias, y, st); break;
  }
}

void conv_dispatch(const CGrid& g, int B, int ci, int co, int flags, bool tcore, const __nv_bfloat16* x,
                   const __nv_bfloat16* w, const float* bias, void* y, cudaStream_t st) {
  if (tcore) {
    if (ci == 16 && co == 32) launch_conv_tc<16, 32>(g, B, flags, x, w, bias, y, st);
    else if (ci == 32 && co == 32) launch_conv_tc<32, 32>(g, B, flags, x, w, bias, y, st);
    else if (ci == 32 && co == 16) launch_conv_tc<32, 16>(g, B, flags, x, w, bias, y, st);
    return;
  }
  if (ci == 16 && co == 32) launch_conv<16, 32>(g, B, flags, x, w, bias, y, st);
  else if (ci == 32 && co == 32) launch_conv<32, 32>(g, B, flags, x, w, bias, y, st);
  else if (ci == 32 && co == 16) launch_conv<32, 16>(g, B, flags, x, w, bias, y, st);
}

}  // namespace

// The kernels move activations and weights in 16-byte pieces (cp.async,
// uint4 loads, vector stores): every array argument must be 16-byte aligned.
static bool unaligned16(const void* a, const void* b = nullptr, const void* c = nullptr,
                        const void* d = nullptr) {
  return (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c | (uintptr_t)d) & 15) != 0;
}

extern "C" int mpn_conv_take_error(int* flag) {
  if (!flag) return MPN_ERR_INVALID_ARG;
  int* p = conv_err_ptr();
  if (!p) return MPN_ERR_CUDA;
  int v = 0;
  if (cudaMemcpy(&v, p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return MPN_ERR_CUDA;
  if (v && cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return MPN_ERR_CUDA;
  *flag = v;
  return MPN_OK;
}

extern "C" int mpn_conv3d_forward(const mpn_conv_desc* d, const void* x, const void* w, const float* bias, void* y,
                                  int flags, void* stream) {
  int s = check(d);
  if (s) return s;
  if (!x || !w || !y || ((flags & MPN_CONV_BIAS) && !bias)) return MPN_ERR_INVALID_ARG;
  if (unaligned16(x, w, y)) return MPN_ERR_INVALID_ARG;
  CGrid g = make_cgrid(d);
  conv_dispatch(g, d->batch, d->cin, d->cout, flags & 7, !(flags & MPN_CONV_MMA_SYNC), (const __nv_bfloat16*)x,
                (const __nv_bfloat16*)w, bias, y, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? MPN_OK : MPN_ERR_CUDA;
}

extern "C" int mpn_conv3d_backward_data(const mpn_conv_desc* d, const void* g_out, const void* w, void* wt_scratch,
                                        float* g_in, void* stream) {
  int s = check(d);
  if (s) return s;
  if (!g_out || !w || !wt_scratch || !g_in) return MPN_ERR_INVALID_ARG;
  if (unaligned16(g_out, w, wt_scratch, g_in)) return MPN_ERR_INVALID_ARG;
  if (d->cin != 32) return MPN_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  CGrid g = make_cgrid(d);
  int n = 27 * d->cin * d->cout;
  k_flip_transpose<<<(n + 255) / 256, 256, 0, st>>>(d->cin, d->cout, (const __nv_bfloat16*)w,
                                                    (__nv_bfloat16*)wt_scratch);
  // transposed convolution = convolution of g_out (channels cout) with W'
  if (d->cout == 32) launch_conv_tc<32, 32>(g, d->batch, MPN_CONV_F32, (const __nv_bfloat16*)g_out,
                                            (const __nv_bfloat16*)wt_scratch, nullptr, g_in, st);
  else launch_conv_tc<16, 32>(g, d->batch, MPN_CONV_F32, (const __nv_bfloat16*)g_out,
                              (const __nv_bfloat16*)wt_scratch, nullptr, g_in, st);
  return cudaGetLastError() == cudaSuccess ? MPN_OK : MPN_ERR_CUDA;
}

extern "C" size_t mpn_conv3d_wgrad_scratch_bytes(const mpn_conv_desc* d) {
  if (check(d)) return 0;
  long long total = (long long)d->batch * d->n[0] * d->n[1] * d->n[2];
  long long nchunk = (total + MPN_WGRAD_CHUNK - 1) / MPN_WGRAD_CHUNK;
  return (size_t)nchunk * (27 * d->cin * d->cout + d->cout) * sizeof(float);
}

extern "C" int mpn_conv3d_backward_weights(const mpn_conv_desc* d, const void* g_out, const void* x, float* scratch,
                                           float* dw, float* db, void* stream) {
  int s = check(d);
  if (s) return s;
  if (!g_out || !x || !scratch || !dw || !db) return MPN_ERR_INVALID_ARG;
  if (unaligned16(g_out, x, scratch)) return MPN_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CGrid g = make_cgrid(d);
  long long total = (long long)d->batch * g.N;
  int nchunk = (int)((total + MPN_WGRAD_CHUNK - 1) / MPN_WGRAD_CHUNK);
  int nw = 27 * d->cin * d->cout;
  float* part = scratch;
  float* bpart = scratch + (size_t)nchunk * nw;
  dim3 gr(nchunk, 27);
  const long long tot = (long long)d->batch * g.N;
  const __nv_bfloat16* go = (const __nv_bfloat16*)g_out;
  const __nv_bfloat16* xx = (const __nv_bfloat16*)x;
  if (d->cin == 16 && d->cout == 32) k_wgrad_mma<16, 32><<<gr, 128, 0, st>>>(g, tot, MPN_WGRAD_CHUNK, go, xx, part, bpart);
  else if (d->cin == 32 && d->cout == 32) k_wgrad_mma<32, 32><<<gr, 128, 0, st>>>(g, tot, MPN_WGRAD_CHUNK, go, xx, part, bpart);
  else if (d->cin == 32 && d->cout == 16) k_wgrad_mma<32, 16><<<gr, 128, 0, st>>>(g, tot, MPN_WGRAD_CHUNK, go, xx, part, bpart);
  else return MPN_ERR_UNSUPPORTED;
  k_wgrad_reduce<<<(nw + 255) / 256, 256, 0, st>>>(nchunk, nw, part, dw);
  k_wgrad_reduce<<<(d->cout + 255) / 256, 256, 0, st>>>(nchunk, d->cout, bpart, db);
  return cudaGetLastError() == cudaSuccess ? MPN_OK : MPN_ERR_CUDA;
}

extern "C" int mpn_relu_mask(long long n, const float* g, const void* y, void* out, void* stream) {
  if (!g || !out || n < 0) return MPN_ERR_INVALID_ARG;
  k_relu_mask<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, g, (const __nv_bfloat16*)y,
                                                                            (__nv_bfloat16*)out);
  return cudaGetLastError() == cudaSuccess ? MPN_OK : MPN_ERR_CUDA;
}

extern "C" int mpn_adam_step(long long n, float* w, const float* g, float* m, float* v, float lr, float beta1,
                             float beta2, float eps, int step, void* w_bf16, void* stream) {
  if (!w || !g || !m || !v || n < 0 || step < 1) return MPN_ERR_INVALID_ARG;
  float c1 = 1.f / (1.f - powf(beta1, (float)step)), c2 = 1.f / (1.f - powf(beta2, (float)step));
  k_adam<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, w, g, m, v, lr, beta1, beta2, eps, c1, c2,
                                                                       (__nv_bfloat16*)w_bf16);
  return cudaGetLastError() == cudaSuccess ? MPN_OK : MPN_ERR_CUDA;
}

extern "C" int mpn_pack_inputs(const mpn_conv_desc* d, int nfields, const float* fields, const float* rhs,
                               const float* scale, void* x0, void* stream) {
  if (!d || nfields < 0 || nfields > 14 || !rhs || !scale || !x0 || (nfields > 0 && !fields)) return MPN_ERR_INVALID_ARG;
  int N = d->n[0] * d->n[1] * d->n[2];
  dim3 gr((N + 255) / 256 < 1024 ? (N + 255) / 256 : 1024, d->batch);
  k_pack<<<gr, 256, 0, (cudaStream_t)stream>>>(N, nfields, fields, rhs, scale, (__nv_bfloat16*)x0, d->batch);
  const int plane = d->n[1] * d->n[2];
  dim3 gp((plane + 255) / 256 < 1024 ? (plane + 255) / 256 : 1024, d->batch);
  k_pack_tsum<<<gp, 256, 0, (cudaStream_t)stream>>>(d->n[0], plane, nfields, rhs, scale, (__nv_bfloat16*)x0, d->batch);
  return cudaGetLastError() == cudaSuccess ? MPN_OK : MPN_ERR_CUDA;
}

extern "C" int mpn_mse_u(const mpn_conv_desc* d, const float* y, const float* target, float* g, float* loss_part,
                         void* stream) {
  if (!d || !y || !target || !g || !loss_part) return MPN_ERR_INVALID_ARG;
  int N = d->n[0] * d->n[1] * d->n[2];
  dim3 gr(MPN_MSE_BLOCKS, d->batch);
  k_mse_u<<<gr, 256, 0, (cudaStream_t)stream>>>(N, y, target, g, loss_part, d->batch);
  return cudaGetLastError() == cudaSuccess ? MPN_OK : MPN_ERR_CUDA;
}

extern "C" int mpn_unpack_u(const mpn_conv_desc* d, const float* y, float scale, float* u0, void* stream) {
  if (!d || !y || !u0) return MPN_ERR_INVALID_ARG;
  int N = d->n[0] * d->n[1] * d->n[2];
  dim3 gr((N + 255) / 256 < 1024 ? (N + 255) / 256 : 1024, d->batch);
  k_unpack_u<<<gr, 256, 0, (cudaStream_t)stream>>>(N, y, scale, u0, d->batch);
  return cudaGetLastError() == cudaSuccess ? MPN_OK : MPN_ERR_CUDA;
}
