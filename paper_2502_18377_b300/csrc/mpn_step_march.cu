// Instances and launcher of the t-marching fused operator step (k_march,
// mpn_march.cuh): columns of 16 x-rows x 64 y points, periodic x and y, the
// transport layout (fields on c_x, c_y) and reaction-diffusion with c_xx and
// c_yy one field; every mode but the direction-update apply.
#include "mpn_step.h"
#include "mpn_march.cuh"

bool march_has(const Grid& g, bool per1, bool per2, int layout) {
  return per1 && per2 && (layout == SL_TR || layout == SL_RDI) && g.D == 3 && g.n[1] % MS_X == 0 &&
         g.n[2] % MS_Y == 0 && g.n[0] % MS_MIN_TC == 0;
}

size_t march_smem() { return sizeof(float) * (size_t)ms_floats(); }

int march_cols(const Grid& g) { return (g.n[1] / MS_X) * (g.n[2] / MS_Y); }

int march_planes(const Grid& g, int B, int nsm) {
  // chunks of the time extent while the CTAs of all instances still fit in
  // one wave of two per SM
  int nc = 1;
  const int cols = march_cols(g) * B;
  while (g.n[0] % (2 * nc) == 0 && g.n[0] / (2 * nc) >= MS_MIN_TC && cols * 2 * nc <= 2 * nsm) nc *= 2;
  return g.n[0] / nc;
}

template <int MODE, int MK>
static cudaError_t attr1() {
  cudaError_t e = cudaFuncSetAttribute(k_march<MODE, MK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)march_smem());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_march<MODE, MK>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  return e;
}
template <int MK>
static cudaError_t attr_modes() {
  cudaError_t e = attr1<SM_POST0, MK>();
  if (e == cudaSuccess) e = attr1<SM_CHEB, MK>();
  if (e == cudaSuccess) e = attr1<SM_RES, MK>();
  if (e == cudaSuccess) e = attr1<SM_APPLY, MK>();
  if (e == cudaSuccess) e = attr1<SM_CHEB_DOT, MK>();
  return e;
}

int march_attrs() {
  cudaError_t e = attr_modes<FS_MASK_TR>();
  if (e == cudaSuccess) e = attr_modes<FS_MASK_RDI>();
  return e == cudaSuccess ? 0 : 1;
}

template <int MK>
static void launch_m(int mode, dim3 gs, int tc, cudaStream_t st, const Grid& g, const Coef& cf, const float* rho,
                     const StepArgs& a) {
  const size_t sm = march_smem();
  switch (mode) {
    case SM_POST0: k_march<SM_POST0, MK><<<gs, MS_TPB, sm, st>>>(g, cf, rho, a, tc); break;
    case SM_CHEB: k_march<SM_CHEB, MK><<<gs, MS_TPB, sm, st>>>(g, cf, rho, a, tc); break;
    case SM_CHEB_DOT: k_march<SM_CHEB_DOT, MK><<<gs, MS_TPB, sm, st>>>(g, cf, rho, a, tc); break;
    case SM_RES: k_march<SM_RES, MK><<<gs, MS_TPB, sm, st>>>(g, cf, rho, a, tc); break;
    default: k_march<SM_APPLY, MK><<<gs, MS_TPB, sm, st>>>(g, cf, rho, a, tc); break;
  }
}

void march_launch(int mode, int layout, int B, int tc, cudaStream_t st, const Grid& g, const Coef& cf,
                  const float* rho, const StepArgs& a) {
  const dim3 gs(march_cols(g) * (g.n[0] / tc), B);
  if (layout == SL_TR) launch_m<FS_MASK_TR>(mode, gs, tc, st, g, cf, rho, a);
  else launch_m<FS_MASK_RDI>(mode, gs, tc, st, g, cf, rho, a);
}
