// Instances and launcher of the fused operator step on tiles that split the
// y rows (k_step3y, mpn_fused_y.cuh): 8 time planes x 4 x-rows x 64 y points;
// the four periodicities of x and y with the layout read at run time, and
// the compile-time layouts of the reaction-diffusion and transport workloads
// with periodic x and y.
#include "mpn_step.h"
#include "mpn_fused_y.cuh"

#define FSY_TT 8
#define FSY_TY 64

bool step_y_has(int tt, int ty, bool per1, bool per2, int layout) {
  if (tt != FSY_TT || ty != FSY_TY) return false;
  return layout == SL_ANY || (per1 && per2);
}

template <int MODE, bool P1, bool P2, int MK>
static cudaError_t attr1() {
  return cudaFuncSetAttribute(k_step3y<MODE, FSY_TT, FSY_TY, P1, P2, MK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(sizeof(float) * fsy_floats(FSY_TT, FSY_TY)));
}
template <bool P1, bool P2, int MK>
static cudaError_t attr_modes() {
  cudaError_t e = attr1<SM_POST0, P1, P2, MK>();
  if (e == cudaSuccess) e = attr1<SM_CHEB, P1, P2, MK>();
  if (e == cudaSuccess) e = attr1<SM_RES, P1, P2, MK>();
  if (e == cudaSuccess) e = attr1<SM_APPLY, P1, P2, MK>();
  if (e == cudaSuccess) e = attr1<SM_CHEB_DOT, P1, P2, MK>();
  if (e == cudaSuccess) e = attr1<SM_APPLYP, P1, P2, MK>();
  return e;
}

int step_y_attrs() {
  cudaError_t e = attr_modes<true, true, FS_ANY>();
  if (e == cudaSuccess) e = attr_modes<true, false, FS_ANY>();
  if (e == cudaSuccess) e = attr_modes<false, true, FS_ANY>();
  if (e == cudaSuccess) e = attr_modes<false, false, FS_ANY>();
  if (e == cudaSuccess) e = attr_modes<true, true, FS_MASK_RD>();
  if (e == cudaSuccess) e = attr_modes<true, true, FS_MASK_RDI>();
  if (e == cudaSuccess) e = attr_modes<true, true, FS_MASK_TR>();
  return e == cudaSuccess ? 0 : 1;
}

template <bool P1, bool P2, int MK>
static void launch_m(int mode, dim3 gs, size_t sm, cudaStream_t st, const Grid& g, const Coef& cf, const float* rho,
                     const StepArgs& a) {
  constexpr int T = FSY_TT, Y = FSY_TY;
  switch (mode) {
    case SM_POST0: k_step3y<SM_POST0, T, Y, P1, P2, MK><<<gs, FS_TPB, sm, st>>>(g, cf, rho, a); break;
    case SM_CHEB: k_step3y<SM_CHEB, T, Y, P1, P2, MK><<<gs, FS_TPB, sm, st>>>(g, cf, rho, a); break;
    case SM_CHEB_DOT: k_step3y<SM_CHEB_DOT, T, Y, P1, P2, MK><<<gs, FS_TPB, sm, st>>>(g, cf, rho, a); break;
    case SM_APPLYP: k_step3y<SM_APPLYP, T, Y, P1, P2, MK><<<gs, FS_TPB, sm, st>>>(g, cf, rho, a); break;
    case SM_RES: k_step3y<SM_RES, T, Y, P1, P2, MK><<<gs, FS_TPB, sm, st>>>(g, cf, rho, a); break;
    default: k_step3y<SM_APPLY, T, Y, P1, P2, MK><<<gs, FS_TPB, sm, st>>>(g, cf, rho, a); break;
  }
}

void step_y_launch(int mode, int tt, int ty, bool per1, bool per2, int layout, int B, size_t smem, cudaStream_t st,
                   const Grid& g, const Coef& cf, const float* rho, const StepArgs& a) {
  (void)tt; (void)ty;
  const dim3 gs(step_ctas(StepTile{FSY_TT, FSY_TY}, g), B);
  if (per1 && per2 && layout == SL_RDI) launch_m<true, true, FS_MASK_RDI>(mode, gs, smem, st, g, cf, rho, a);
  else if (per1 && per2 && layout == SL_RD) launch_m<true, true, FS_MASK_RD>(mode, gs, smem, st, g, cf, rho, a);
  else if (per1 && per2 && layout == SL_TR) launch_m<true, true, FS_MASK_TR>(mode, gs, smem, st, g, cf, rho, a);
  else if (per1 && per2) launch_m<true, true, FS_ANY>(mode, gs, smem, st, g, cf, rho, a);
  else if (per1) launch_m<true, false, FS_ANY>(mode, gs, smem, st, g, cf, rho, a);
  else if (per2) launch_m<false, true, FS_ANY>(mode, gs, smem, st, g, cf, rho, a);
  else launch_m<false, false, FS_ANY>(mode, gs, smem, st, g, cf, rho, a);
}
