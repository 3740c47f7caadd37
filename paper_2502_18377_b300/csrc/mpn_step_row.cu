// Instances and launcher of the fused operator step on tiles of whole y rows
// (k_step3, mpn_fused.cuh): tile heights 8 and 4 time planes; the four
// periodicities of x and y with the layout read at run time, and the
// compile-time layouts of the reaction-diffusion (c_0, c_xx, c_yy fields, c_xx
// and c_yy shared or not) and transport (c_x, c_y fields) workloads with
// periodic x and y.
#include "mpn_step.h"
#include "mpn_fused.cuh"

// rows of at most this many points are kept whole
#define FS_ROW_MAX_NY 128

size_t step_smem(StepTile tile, int n2) {
  const int w = tile.ty ? tile.ty + 8 : n2;
  return sizeof(float) * (size_t)(fs_rows_x(tile.tt) + fs_rows_y(tile.tt)) * w;
}

int step_ctas(StepTile tile, const Grid& g) {
  return (g.n[0] / tile.tt) * (g.n[1] / FS_TX) * (tile.ty ? g.n[2] / tile.ty : 1);
}

bool step_row_has(int tt, bool per1, bool per2, int layout) {
  if (tt != 8 && tt != 4) return false;
  return layout == SL_ANY || (per1 && per2);
}

template <int MODE, int TT, bool P1, bool P2, int MK>
static cudaError_t attr1() {
  return cudaFuncSetAttribute(k_step3<MODE, TT, P1, P2, MK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)step_smem(StepTile{8, 0}, FS_ROW_MAX_NY));
}
template <int TT, bool P1, bool P2, int MK>
static cudaError_t attr_modes() {
  cudaError_t e = attr1<SM_POST0, TT, P1, P2, MK>();
  if (e == cudaSuccess) e = attr1<SM_CHEB, TT, P1, P2, MK>();
  if (e == cudaSuccess) e = attr1<SM_RES, TT, P1, P2, MK>();
  if (e == cudaSuccess) e = attr1<SM_APPLY, TT, P1, P2, MK>();
  if (e == cudaSuccess) e = attr1<SM_CHEB_DOT, TT, P1, P2, MK>();
  if (e == cudaSuccess) e = attr1<SM_APPLYP, TT, P1, P2, MK>();
  return e;
}
template <int TT>
static cudaError_t attr_tt() {
  cudaError_t e = attr_modes<TT, true, true, FS_ANY>();
  if (e == cudaSuccess) e = attr_modes<TT, true, false, FS_ANY>();
  if (e == cudaSuccess) e = attr_modes<TT, false, true, FS_ANY>();
  if (e == cudaSuccess) e = attr_modes<TT, false, false, FS_ANY>();
  if (e == cudaSuccess) e = attr_modes<TT, true, true, FS_MASK_RD>();
  if (e == cudaSuccess) e = attr_modes<TT, true, true, FS_MASK_RDI>();
  if (e == cudaSuccess) e = attr_modes<TT, true, true, FS_MASK_TR>();
  return e;
}

int step_row_attrs() {
  cudaError_t e = attr_tt<8>();
  if (e == cudaSuccess) e = attr_tt<4>();
  return e == cudaSuccess ? 0 : 1;
}

template <int TT, bool P1, bool P2, int MK>
static void launch_m(int mode, dim3 gs, size_t sm, cudaStream_t st, const Grid& g, const Coef& cf, const float* rho,
                     const StepArgs& a) {
  switch (mode) {
    case SM_POST0: k_step3<SM_POST0, TT, P1, P2, MK><<<gs, FS_TPB, sm, st>>>(g, cf, rho, a); break;
    case SM_CHEB: k_step3<SM_CHEB, TT, P1, P2, MK><<<gs, FS_TPB, sm, st>>>(g, cf, rho, a); break;
    case SM_CHEB_DOT: k_step3<SM_CHEB_DOT, TT, P1, P2, MK><<<gs, FS_TPB, sm, st>>>(g, cf, rho, a); break;
    case SM_APPLYP: k_step3<SM_APPLYP, TT, P1, P2, MK><<<gs, FS_TPB, sm, st>>>(g, cf, rho, a); break;
    case SM_RES: k_step3<SM_RES, TT, P1, P2, MK><<<gs, FS_TPB, sm, st>>>(g, cf, rho, a); break;
    default: k_step3<SM_APPLY, TT, P1, P2, MK><<<gs, FS_TPB, sm, st>>>(g, cf, rho, a); break;
  }
}
template <int TT>
static void launch_tt(int mode, bool per1, bool per2, int layout, dim3 gs, size_t sm, cudaStream_t st, const Grid& g,
                      const Coef& cf, const float* rho, const StepArgs& a) {
  if (per1 && per2 && layout == SL_RDI) launch_m<TT, true, true, FS_MASK_RDI>(mode, gs, sm, st, g, cf, rho, a);
  else if (per1 && per2 && layout == SL_RD) launch_m<TT, true, true, FS_MASK_RD>(mode, gs, sm, st, g, cf, rho, a);
  else if (per1 && per2 && layout == SL_TR) launch_m<TT, true, true, FS_MASK_TR>(mode, gs, sm, st, g, cf, rho, a);
  else if (per1 && per2) launch_m<TT, true, true, FS_ANY>(mode, gs, sm, st, g, cf, rho, a);
  else if (per1) launch_m<TT, true, false, FS_ANY>(mode, gs, sm, st, g, cf, rho, a);
  else if (per2) launch_m<TT, false, true, FS_ANY>(mode, gs, sm, st, g, cf, rho, a);
  else launch_m<TT, false, false, FS_ANY>(mode, gs, sm, st, g, cf, rho, a);
}

void step_row_launch(int mode, int tt, bool per1, bool per2, int layout, int B, size_t smem, cudaStream_t st,
                     const Grid& g, const Coef& cf, const float* rho, const StepArgs& a) {
  const dim3 gs(step_ctas(StepTile{tt, 0}, g), B);
  if (tt == 8) launch_tt<8>(mode, per1, per2, layout, gs, smem, st, g, cf, rho, a);
  else launch_tt<4>(mode, per1, per2, layout, gs, smem, st, g, cf, rho, a);
}
