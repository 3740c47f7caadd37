// Launchers of the fused operator step (internal to the library).
//
// The kernels (k_step3: tiles of whole y rows; k_step3y: tiles that split the
// y rows) are instantiated in their own translation units, one per tiling,
// for the tile heights, periodicities and compile-time coefficient layouts
// listed there; the solver picks a tiling per multigrid level.
#pragma once
#include <cuda_runtime.h>

#include "mpn_device.cuh"
#include "mpn_stepargs.cuh"

// Coefficient layouts the fused kernels are compiled for.
enum StepLayout { SL_ANY = 0, SL_RD = 1, SL_RDI = 2, SL_TR = 3 };

// Tile of a fused level: tt time planes x 4 x-rows x (ty y points, or the
// whole row when ty = 0).
struct StepTile { int tt, ty; };

// Opts every instance of one tiling into the dynamic shared memory of its
// largest tile (host call, once).
int step_row_attrs();
int step_y_attrs();
// Shared-memory bytes of a tile for rows of n2 points.
size_t step_smem(StepTile tile, int n2);
// CTAs per instance of a tiling on grid g.
int step_ctas(StepTile tile, const Grid& g);
// Whether a tiling is compiled for (tt, periodic x, periodic y, layout).
bool step_row_has(int tt, bool per1, bool per2, int layout);
bool step_y_has(int tt, int ty, bool per1, bool per2, int layout);
// Launches one fused step (mode SM_*) of a level on B instances.
void step_row_launch(int mode, int tt, bool per1, bool per2, int layout, int B, size_t smem, cudaStream_t st,
                     const Grid& g, const Coef& cf, const float* rho, const StepArgs& a);
void step_y_launch(int mode, int tt, int ty, bool per1, bool per2, int layout, int B, size_t smem, cudaStream_t st,
                   const Grid& g, const Coef& cf, const float* rho, const StepArgs& a);

// t-marching fused step (k_march) on columns of mx = 16 or 8 x-rows x 64 y
// points: whether a level qualifies (periodic x and y, n_x % mx == 0,
// n_y % 64 == 0, n_t % 8 == 0, the SL_TR or SL_RDI layout); its
// shared-memory bytes; columns per instance; resident CTAs per SM; planes per
// CTA for B instances on nsm SMs; the attributes (host call, once); one launch
// (any mode but SM_APPLYP) with tc planes per CTA.
bool march_has(const Grid& g, bool per1, bool per2, int layout, int mx);
size_t march_smem(int mx);
int march_cols(const Grid& g, int mx);
int march_ctas_per_sm(int mx);
int march_planes(const Grid& g, int B, int nsm, int mx);
int march_attrs();
void march_launch(int mode, int layout, int B, int mx, int tc, cudaStream_t st, const Grid& g, const Coef& cf,
                  const float* rho, const StepArgs& a);
