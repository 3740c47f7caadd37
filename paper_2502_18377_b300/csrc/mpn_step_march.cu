// Instances and launcher of the t-marching fused operator step (k_march,
// mpn_march.cuh): columns of 16 or 8 x-rows x 64 y points, periodic x and y,
// the transport layout (fields on c_x, c_y) and reaction-diffusion with c_xx
// and c_yy one field; every mode but the direction-update apply.
#include "mpn_step.h"
#include "mpn_march.cuh"

bool march_has(const Grid& g, bool per1, bool per2, int layout, int mx) {
  return (mx == 16 || mx == 8) && per1 && per2 && (layout == SL_TR || layout == SL_RDI) && g.D == 3 &&
         g.n[1] % mx == 0 && g.n[2] % MS_Y == 0 && g.n[0] % MS_MIN_TC == 0;
}

size_t march_smem(int mx) { return sizeof(float) * (size_t)ms_floats(mx); }

int march_cols(const Grid& g, int mx) { return (g.n[1] / mx) * (g.n[2] / MS_Y); }

int march_ctas_per_sm(int mx) { return ms_ctas_per_sm(mx); }

int march_planes(const Grid& g, int B, int nsm, int mx) {
  // chunks of the time extent while the CTAs of all instances still fit in
  // one wave
  int nc = 1;
  const int cols = march_cols(g, mx) * B;
  while (g.n[0] % (2 * nc) == 0 && g.n[0] / (2 * nc) >= MS_MIN_TC && cols * 2 * nc <= ms_ctas_per_sm(mx) * nsm)
    nc *= 2;
  return g.n[0] / nc;
}

template <int MODE, int MK, int MX>
static cudaError_t attr1() {
  cudaError_t e = cudaFuncSetAttribute(k_march<MODE, MK, MX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)march_smem(MX));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_march<MODE, MK, MX>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  return e;
}
template <int MK, int MX>
static cudaError_t attr_modes() {
  cudaError_t e = attr1<SM_POST0, MK, MX>();
  if (e == cudaSuccess) e = attr1<SM_CHEB, MK, MX>();
  if (e == cudaSuccess) e = attr1<SM_RES, MK, MX>();
  if (e == cudaSuccess) e = attr1<SM_APPLY, MK, MX>();
  if (e == cudaSuccess) e = attr1<SM_CHEB_DOT, MK, MX>();
  return e;
}

int march_attrs() {
  cudaError_t e = attr_modes<FS_MASK_TR, 16>();
  if (e == cudaSuccess) e = attr_modes<FS_MASK_RDI, 16>();
  if (e == cudaSuccess) e = attr_modes<FS_MASK_TR, 8>();
  if (e == cudaSuccess) e = attr_modes<FS_MASK_RDI, 8>();
  return e == cudaSuccess ? 0 : 1;
}

template <int MK, int MX>
static void launch_m(int mode, dim3 gs, int tc, cudaStream_t st, const Grid& g, const Coef& cf, const float* rho,
                     const StepArgs& a) {
  const size_t sm = march_smem(MX);
  constexpr int T = ms_tpb(MX);
  switch (mode) {
    case SM_POST0: k_march<SM_POST0, MK, MX><<<gs, T, sm, st>>>(g, cf, rho, a, tc); break;
    case SM_CHEB: k_march<SM_CHEB, MK, MX><<<gs, T, sm, st>>>(g, cf, rho, a, tc); break;
    case SM_CHEB_DOT: k_march<SM_CHEB_DOT, MK, MX><<<gs, T, sm, st>>>(g, cf, rho, a, tc); break;
    case SM_RES: k_march<SM_RES, MK, MX><<<gs, T, sm, st>>>(g, cf, rho, a, tc); break;
    default: k_march<SM_APPLY, MK, MX><<<gs, T, sm, st>>>(g, cf, rho, a, tc); break;
  }
}

void march_launch(int mode, int layout, int B, int mx, int tc, cudaStream_t st, const Grid& g, const Coef& cf,
                  const float* rho, const StepArgs& a) {
  const dim3 gs(march_cols(g, mx) * (g.n[0] / tc), B);
  if (mx == 16) {
    if (layout == SL_TR) launch_m<FS_MASK_TR, 16>(mode, gs, tc, st, g, cf, rho, a);
    else launch_m<FS_MASK_RDI, 16>(mode, gs, tc, st, g, cf, rho, a);
  } else {
    if (layout == SL_TR) launch_m<FS_MASK_TR, 8>(mode, gs, tc, st, g, cf, rho, a);
    else launch_m<FS_MASK_RDI, 8>(mode, gs, tc, st, g, cf, rho, a);
  }
}
