// Allocation-free variant of the reduced-operator apply (mpn_apply_reduced).
//
// Who needs it: callers that cannot allocate device memory — for instance a
// process whose device memory is owned by another allocator (a framework's
// caching allocator that has reserved the pool), or a code path where the
// failure or the implicit synchronisation of cudaMalloc / cudaFree is not
// acceptable (a real-time loop, a callback running inside another library).
// This entry point takes no problem object (creating one allocates its
// workspace) and allocates nothing: its only scratch, the intermediate
// y = -rho L u of the two-pass apply, lives in the file-scope device array
// below, of fixed size MPN_NOALLOC_MAX_POINTS floats, which every GPU that
// loads the library holds until the process exits.  The point weights rho
// are computed inline from the coefficients instead of being stored.
//
// The array is shared by every call: each call overwrites all of its first
// B*N entries before reading them, so nothing needs clearing, but calls that
// overlap on the GPU (e.g. on two streams) race on it.
#include <cuda_runtime.h>
#include <cstdio>
#include <cstring>

#include "../../include/mpn.h"
#include "mpn_device.cuh"

static __device__ __align__(256) float g_noalloc_y[MPN_NOALLOC_MAX_POINTS];

namespace {

// Device address of the scratch array on the current device.  The host-side
// name of a __device__ array is not a device address, so every call asks the
// runtime for it (a host-side lookup that allocates nothing; resolving it per
// call also stays correct after the device's context is re-created).
int scratch_ptr(float** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_y) != cudaSuccess || !p) return MPN_ERR_CUDA;
  *out = static_cast<float*>(p);
  return MPN_OK;
}

// y = -rho L u with rho computed from the coefficients at the point.
template <int D>
__global__ void k_na_Ly(Grid g, Coef cf, const float* __restrict__ u, float* __restrict__ y) {
  const int b = blockIdx.y;
  const size_t off = (size_t)b * g.N;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += gridDim.x * blockDim.x) {
    int pos[3]; decode_fast(g, p, pos);
    float Lx = Lrow<float, D>(g, cf, b, p, pos, u + off, nullptr);
    y[off + p] = -rho_point<float>(g, cf, b, p, pos) * Lx;
  }
}

// q = (L^T y)_j ... with the sign folded: q = S u = -(L^T y) + theta 1_B u.
template <int D>
__global__ void k_na_LTy(Grid g, Coef cf, const float* __restrict__ y, const float* __restrict__ u,
                         float* __restrict__ q) {
  const int b = blockIdx.y;
  const size_t off = (size_t)b * g.N;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < g.N; p += gridDim.x * blockDim.x) {
    int pos[3]; decode_fast(g, p, pos);
    float v = -LTgather<float, D>(g, cf, b, p, pos, y + off);
    if (is_boundary_t<D>(g, pos)) v += g.theta * u[off + p];
    q[off + p] = v;
  }
}

}  // namespace

extern "C" int mpn_apply_reduced_noalloc(const mpn_desc* desc, const float* fields, const float* scalars,
                                         const float* u, float* q, void* stream) {
  if (!desc || !scalars || !u || !q) return MPN_ERR_INVALID_ARG;
  const mpn_desc& d = *desc;
  if (d.ndim != 2 && d.ndim != 3) return MPN_ERR_INVALID_ARG;
  if (d.periodic[0] || d.batch < 1 || d.nfields < 0 || d.nfields > 7) return MPN_ERR_INVALID_ARG;
  if (d.stencil != 3) return d.stencil == 5 ? MPN_ERR_UNSUPPORTED : MPN_ERR_INVALID_ARG;
  // uniform steps and Dirichlet faces only: the kernels below apply that
  // operator, so per-interval steps or Neumann / mixed rows are refused
  // rather than silently treated as Dirichlet
  if (d.variable_steps) return MPN_ERR_UNSUPPORTED;
  for (int k = 1; k < d.ndim; ++k) {
    if (d.periodic[k]) continue;
    const double a = d.bc_alpha[k], bt = d.bc_beta[k];
    if (!(a == a) || !(bt == bt) || (a == 0.0 && bt == 0.0)) return MPN_ERR_INVALID_ARG;
    if (a != 1.0 || bt != 0.0) return MPN_ERR_UNSUPPORTED;
  }
  const int V = 1 + 2 * d.ndim;
  long long N = 1;
  for (int k = 0; k < d.ndim; ++k) {
    if (d.n[k] < 3 || !(d.step[k] > 0)) return MPN_ERR_INVALID_ARG;
    N *= d.n[k];
  }
  for (int v = 0; v < V; ++v)
    if (d.field_of[v] < -1 || d.field_of[v] >= d.nfields) return MPN_ERR_INVALID_ARG;
  if (d.nfields > 0 && !fields) return MPN_ERR_INVALID_ARG;
  if (N * d.batch > (long long)MPN_NOALLOC_MAX_POINTS) return MPN_ERR_UNSUPPORTED;  // scratch too small
  if (d.batch > 65535) return MPN_ERR_UNSUPPORTED;   // one grid row of CTAs per instance

  float* y = nullptr;
  int s = scratch_ptr(&y);
  if (s != MPN_OK) return s;

  Grid g;
  memset(&g, 0, sizeof(g));
  g.D = d.ndim;
  for (int k = 0; k < 3; ++k) {
    g.n[k] = k < d.ndim ? d.n[k] : 1;
    g.per[k] = k < d.ndim ? d.periodic[k] : 0;
    double sd = k < d.ndim ? d.step[k] : 1.0;
    g.ds1[k] = 1.0 / sd; g.ds2[k] = 1.0 / (sd * sd);
    g.is1[k] = (float)g.ds1[k]; g.is2[k] = (float)g.ds2[k];
  }
  g.stride[2] = 1; g.stride[1] = g.n[2]; g.stride[0] = g.n[1] * g.n[2];
  g.N = (int)N;
  g.final_rows = d.final_time_rows;
  g.theta = 1.f;
  grid_set_inverses(g);

  Coef cf;
  memset(&cf, 0, sizeof(cf));
  cf.V = V; cf.F = d.nfields; cf.B = d.batch;
  cf.fields = fields; cf.scalars = scalars;
  for (int v = 0; v < 7; ++v) {
    int f = v < V ? d.field_of[v] : -1;
    cf.field_of[v] = f;
    if (f >= 0) { cf.ptr[v] = fields + (size_t)f * d.batch * N; cf.bstride[v] = (int)N; cf.pstride[v] = 1; }
    else { cf.ptr[v] = scalars + (size_t)(v < V ? v : 0) * d.batch; cf.bstride[v] = 1; cf.pstride[v] = 0; }
    cf.ptr4[v] = nullptr; cf.bstride4[v] = 0;   // float4 scalar copies: not used here
  }

  cudaStream_t st = (cudaStream_t)stream;
  (void)cudaGetLastError();   // an earlier call's error is not this call's
  int nb = (int)((N + MPN_TPB - 1) / MPN_TPB);
  if (nb > 1024) nb = 1024;
  dim3 gr(nb, d.batch);
  if (d.ndim == 3) {
    k_na_Ly<3><<<gr, MPN_TPB, 0, st>>>(g, cf, u, y);
    k_na_LTy<3><<<gr, MPN_TPB, 0, st>>>(g, cf, y, u, q);
  } else {
    k_na_Ly<2><<<gr, MPN_TPB, 0, st>>>(g, cf, u, y);
    k_na_LTy<2><<<gr, MPN_TPB, 0, st>>>(g, cf, y, u, q);
  }
  if (cudaGetLastError() != cudaSuccess) return MPN_ERR_CUDA;
  return MPN_OK;
}
