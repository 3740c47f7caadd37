// C ABI and host orchestration of the batched NeuRLP-PDE solver (sm_103a).
//
// Solve structure (forward and adjoint alike):
//   setup      coefficients copied into the problem, point weights rho,
//              hierarchy built by halving the spatial dimensions (time kept),
//              coefficient fields and rho carried down by full weighting,
//              Chebyshev-Jacobi scaling by a power-method lambda_max per level
//              and instance, coarsest system factorised and inverted.
//   refinement FP64 residual r = g - S u of the reduced normal equations
//              (Schur complement of A^T A, Eq. 9, onto u), normalised to FP32,
//              a fixed number of multigrid-preconditioned CG iterations in
//              FP32, u += correction in FP64; one device-to-host read of a few
//              scalars per sweep decides whether to stop.
//   recovery   every derivative unknown from u, point by point (FP64).
#include <cuda_runtime.h>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>

#include "../../include/mpn.h"
#include "mpn_kernels.cuh"
#include "mpn_stencil.cuh"
#include "mpn_tail.cuh"
#include "mpn_fused.cuh"
#include "mpn_step.h"
#include "mpn_steps.cuh"

#define MAXL 16

static thread_local char g_cuda_err[256] = "";

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      snprintf(g_cuda_err, sizeof(g_cuda_err), "%s at %s:%d", cudaGetErrorString(e_), \
               __FILE__, __LINE__);                                                    \
      return MPN_ERR_CUDA;                                                             \
    }                                                                                  \
  } while (0)
#define CKL() CK(cudaGetLastError())
#define TRY(x) do { int s_ = (x); if (s_ != MPN_OK) return s_; } while (0)

struct Level {
  Grid g;
  int vec4 = 0;        // float4 stencil kernels apply (D = 3, n_y % 4 == 0)
  int vec2 = 0;        // float4 stencil kernels of 1-D + t grids apply (D = 2, n_x % 4 == 0)
  int papply = 0;      // partial sums per instance written by an operator apply
  int cz[3];           // dims halved from this level to the next
  int fs_tt = 0;       // > 0: operator steps as one fused kernel with TT-plane tiles
  int fs_ty = 0;       // fused tiles of fs_ty y points (k_step3y), or of whole y rows when 0 (k_step3)
  int fs_layout = SL_ANY;  // compile-time coefficient layout of the fused kernels
  int ms_tc = 0;       // > 0: the t-marching fused step (k_march) with this many planes per CTA, for
                       // every mode but the direction-update apply
  int ms_mx = 16;      // x rows of its columns
  float* e2 = nullptr; // second iterate buffer of the fused smoother (the operand is read with a halo)
  float* fields = nullptr;  // [F][B][N]
  float *rho = nullptr, *dinv = nullptr;
  float *r = nullptr, *e = nullptr, *d = nullptr, *y = nullptr, *t = nullptr;
  float *r12 = nullptr, *r22 = nullptr, *y2 = nullptr;   // Neumann / mixed rows (see Grid)
};

struct mpn_problem {
  mpn_desc desc;
  int D, V, F, B;
  int L;
  Level lv[MAXL];
  int M, bw;           // coarsest system size and band width
  float *Kband = nullptr, *Kinv = nullptr;
  int* ferr = nullptr;
  int* kerr = nullptr;     // device word a kernel sets when a bounded wait gives up (cleared per solve)
  int* dbg = nullptr;      // bounds-checked build: first out-of-range index code (see dbg_index)
  int inject_wait = 0;     // host-side fault injection: the next solve sets kerr itself
  float *scalars = nullptr, *rhs = nullptr, *omega = nullptr;
  float* scal4 = nullptr;  // scalars replicated 4 times, [V][B][4]
  int field_mask = 0;      // bit v: c_v is a field
  bool band_smem = true;   // coarsest band factorised in shared memory
  // FGMRES workspace: basis V[mk + 1], preconditioned Z[mk], dot partials,
  // Hessenberg / rotations / rhs / solution per instance
  int mk = 0;
  float *fgV = nullptr, *fgZ = nullptr;
  double *fgpart = nullptr, *fgH = nullptr, *fgc = nullptr, *fgs = nullptr, *fgg = nullptr, *fgy = nullptr, *fgh = nullptr;
  int* field_of_dev = nullptr;
  float *x = nullptr, *pv = nullptr, *q = nullptr, *z = nullptr;
  float* pv2 = nullptr;    // second PCG direction buffer (fused direction update)
  double *u64 = nullptr, *r64 = nullptr, *y64 = nullptr, *g64 = nullptr;
  double* rho64 = nullptr;  // finest-level point weights in FP64 (refinement residual)
  double *kap = nullptr;
  double *uf64 = nullptr;  // FP64 u of the last forward (the adjoint's lambda*)
  double *part = nullptr;  // partial-sum slots [NSLOT][B][PMAX]
  int* pcnt = nullptr;     // [2][B] CTA counters of the fused steps that finish <r, z> and <p, S p>
  double* ptot = nullptr;  // [2][B] their finished sums
  double *dscal = nullptr; // device scalars: scale[B], rz_old[B], out[8][B]
  float* lam = nullptr;    // lambda_max per level and instance [L][B]
  double* hbuf = nullptr;  // pinned host buffer
  // per-interval steps (variable_steps): intervals [L][B][3][stn] (level 0
  // from mpn_set_steps, the others built by the setup), step records
  // [L][B][3][stn][ST_REC] in FP64 and FP32, the step check word
  int stn = 0;
  double* hlev = nullptr;
  double* st64 = nullptr;
  float* st32 = nullptr;
  int* sterr = nullptr;
  bool steps_set = false;
  // Neumann / mixed boundary rows: per-level R12, R22 and second pass-1
  // output (FP32 [L][B][N] each) and their finest-level FP64 copies
  bool mixed = false;
  double *r12d = nullptr, *r22d = nullptr, *y2d = nullptr;
  size_t bytes = 0;
  bool setup_ok = false;
  bool zd_valid = false;   // uf64 holds the FP64 u of the last forward
  long long gen = 0;       // forward solves completed on this problem
  const void* fwd_in[4] = {nullptr, nullptr, nullptr, nullptr};   // fields, scalars, rhs, omega of the last forward
  float cheb_c1[32], cheb_c2[32], cheb_inv_th;
  // fused coarse end of the V-cycle: first level (-1: none), cluster size,
  // dynamic shared memory per CTA, kernel arguments
  int tail_k0 = -1, tail_cs = 0;
  size_t tail_smem = 0;
  TailArgs tail;
  std::vector<void*> allocs;
  // live timing of the finest-level smoothing step (events on the solve stream)
  int prof_on = 0;
  std::vector<cudaEvent_t> prof_ev;
  double prof_ms = 0, prof_bytes = 0;
  long long prof_n = 0;
  long long nlaunch = 0;   // kernels launched since the last mpn_profile reset
  int prof_next = 0;       // next free event of the pool (graphs keep theirs)
  // one CUDA graph per (solve kind, inner iterations, profiling): a whole
  // refinement sweep, replayed on an internal stream
  struct SweepGraph { int adjoint, iters, prof; bool from_zero; cudaGraphExec_t exec; long long kernels; int ev0, ev1; };
  std::vector<SweepGraph> graphs;
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_user = nullptr;
  // the setup after the input copies, as one CUDA graph (its buffers are the
  // problem's own, so one capture serves every call)
  cudaGraphExec_t setup_exec = nullptr;
  long long setup_kernels = 0;
  cudaEvent_t ev_setup = nullptr;
  // setup: one stream per level for the independent power iterations
  cudaStream_t aux[MAXL] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[MAXL] = {};
};

enum { S_RZ = 0, S_PQ, S_RN, S_DU, S_UN, S_PW, S_GN, S_GR0, S_PW0 = S_GR0 + 8, S_PW1 = S_PW0 + MAXL, NSLOT = S_PW1 + MAXL };

static inline double* slot(mpn_problem* p, int k) { return p->part + (size_t)k * p->B * MPN_PMAX; }
// CTAs per instance of the grid-stride kernels (FP64 refinement, recovery
// and gradient passes, setup, and the reductions their consumers sum): enough
// that the FP64 kernels keep warps in flight to hide the FP64 pipe's latency
// (one wave of 8 CTAs on each of 148 SMs over the batch, 64 to 512 per
// instance: every consumer CTA of a reduction sums its partials again, so no
// more than that)
static int nblk_cap(int B) { int c = 148 * 8 / (B > 0 ? B : 1); return c < 64 ? 64 : (c > 512 ? 512 : c); }
static int nblk(const mpn_problem* p, int N) {
  const int b = (N + MPN_TPB - 1) / MPN_TPB, c = nblk_cap(p->B);
  return b < 1 ? 1 : (b > c ? c : b);
}

static int sblk(int N) { int b = (N + MPN_TPB - 1) / MPN_TPB; return b < 1 ? 1 : (b > 512 ? 512 : b); }
// PCG vector kernels: one float4 group (or one value) per thread, up to
// MPN_PMAX blocks per instance (each block writes one partial sum).
static bool vec4_len(int N) { return N % 4 == 0; }
static int vgrid(int N) {
  int n = vec4_len(N) ? N / 4 : N;
  int b = (n + MPN_TPB - 1) / MPN_TPB;
  return b < 1 ? 1 : (b > MPN_PMAX ? MPN_PMAX : b);
}

static int dalloc(mpn_problem* p, void** ptr, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    snprintf(g_cuda_err, sizeof(g_cuda_err), "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MPN_ERR_NO_MEMORY : MPN_ERR_CUDA;
  }
  p->allocs.push_back(*ptr);
  p->bytes += bytes;
  return MPN_OK;
}
template <class T>
static int dalloc_t(mpn_problem* p, T** ptr, size_t n) { return dalloc(p, (void**)ptr, n * sizeof(T)); }

static Grid make_grid(int D, const int n[3], const double s[3], const int per[3], int final_rows, float theta) {
  Grid g;
  memset(&g, 0, sizeof(g));
  g.D = D;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = d < D ? n[d] : 1;
    g.per[d] = d < D ? per[d] : 0;
    double sd = d < D ? s[d] : 1.0;
    g.ds1[d] = 1.0 / sd; g.ds2[d] = 1.0 / (sd * sd);
    g.is1[d] = (float)g.ds1[d]; g.is2[d] = (float)g.ds2[d];
  }
  g.stride[2] = 1; g.stride[1] = g.n[2]; g.stride[0] = g.n[1] * g.n[2];
  g.N = g.n[0] * g.n[1] * g.n[2];
  g.final_rows = final_rows;
  g.theta = theta;
  grid_set_inverses(g);
  return g;
}

static Coef make_coef(const mpn_problem* p, const float* fields) {
  Coef c;
  c.V = p->V; c.F = p->F; c.B = p->B;
  for (int v = 0; v < 7; ++v) c.field_of[v] = v < p->V ? p->desc.field_of[v] : -1;
  c.fields = fields;
  c.scalars = p->scalars;
  // per-level point count from the field pointer's level (fields are [F][B][N])
  int N = 0;
  for (int k = 0; k < p->L; ++k) if (p->lv[k].fields == fields) N = p->lv[k].g.N;
  for (int v = 0; v < 7; ++v) {
    int f = v < p->V ? p->desc.field_of[v] : -1;
    if (f >= 0) {
      c.ptr[v] = c.ptr4[v] = fields + (size_t)f * p->B * N;
      c.bstride[v] = c.bstride4[v] = N; c.pstride[v] = 1;
    } else {
      c.ptr[v] = p->scalars + (size_t)(v < p->V ? v : 0) * p->B; c.bstride[v] = 1; c.pstride[v] = 0;
      c.ptr4[v] = p->scal4 + (size_t)(v < p->V ? v : 0) * p->B * 4; c.bstride4[v] = 4;
    }
  }
  return c;
}

extern "C" int mpn_default_desc(mpn_desc* d) {
  if (!d) return MPN_ERR_INVALID_ARG;
  memset(d, 0, sizeof(*d));
  d->ndim = 2;
  d->n[0] = d->n[1] = 32; d->n[2] = 1;
  d->step[0] = d->step[1] = d->step[2] = 1.0;
  d->stencil = 3;
  d->batch = 1;
  for (int v = 0; v < 7; ++v) d->field_of[v] = -1;
  d->tol = 1e-7;
  d->max_refine = 12;
  d->inner_iters = 5;
  d->cheb_degree = 5;
  d->coarse_min = 4;
  d->max_coarse = 2048;
  d->fused_coarse = 1;
  d->fused_step = 3;
  d->krylov = MPN_KRYLOV_CG;
  d->coarsen_time = 0;
  d->direct = 0;
  d->variable_steps = 0;
  d->adj_inner_iters = 0;
  for (int k = 0; k < 3; ++k) { d->bc_alpha[k] = 1.0; d->bc_beta[k] = 0.0; }
  return MPN_OK;
}

extern "C" const char* mpn_strerror(int s) {
  switch (s) {
    case MPN_OK: return "ok";
    case MPN_ERR_INVALID_ARG: return "invalid argument";
    case MPN_ERR_UNSUPPORTED: return "unsupported configuration";
    case MPN_ERR_NOT_CONVERGED: return "refinement did not reach the tolerance";
    case MPN_ERR_NONFINITE: return "non-finite value in inputs or iterates";
    case MPN_ERR_DIVERGED: return "refinement correction grew";
    case MPN_ERR_CUDA: return "CUDA error";
    case MPN_ERR_NO_MEMORY: return "out of device memory";
  }
  return "unknown status";
}

extern "C" const char* mpn_last_cuda_error(void) { return g_cuda_err; }

extern "C" void mpn_destroy(mpn_problem* p) {
  if (!p) return;
  for (auto& g : p->graphs) cudaGraphExecDestroy(g.exec);
  if (p->setup_exec) cudaGraphExecDestroy(p->setup_exec);
  if (p->ev_setup) cudaEventDestroy(p->ev_setup);
  if (p->gstream) cudaStreamDestroy(p->gstream);
  if (p->ev_user) cudaEventDestroy(p->ev_user);
  for (int k = 0; k < MAXL; ++k) {
    if (p->aux[k]) cudaStreamDestroy(p->aux[k]);
    if (p->ev_join[k]) cudaEventDestroy(p->ev_join[k]);
  }
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  for (cudaEvent_t e : p->prof_ev) cudaEventDestroy(e);
  for (void* a : p->allocs) cudaFree(a);
  if (p->hbuf) cudaFreeHost(p->hbuf);
  delete p;
}

extern "C" size_t mpn_workspace_bytes(const mpn_problem* p) { return p ? p->bytes : 0; }

extern "C" int mpn_levels(const mpn_problem* p, int* nl, int* shapes) {
  if (!p || !nl) return MPN_ERR_INVALID_ARG;
  *nl = p->L;
  if (shapes)
    for (int k = 0; k < p->L; ++k)
      for (int d = 0; d < 3; ++d) shapes[3 * k + d] = p->lv[k].g.n[d];
  return MPN_OK;
}

// rows of at most this many points stay whole in a fused tile; wider rows
// (a multiple of 64, >= 128) are split into 64-point y segments
#define FS_MAX_NY 128
// Lower end of the Chebyshev smoothing interval, as a fraction of the
// estimated lambda_max of D^-1 S
#ifndef MPN_CHEB_LO
#define MPN_CHEB_LO 0.1
#endif
// CTAs of one fused step below which a level's tiles are made thinner in time
// (148 SMs x 4 resident CTAs)
#ifndef FS_MIN_CTAS
#define FS_MIN_CTAS 592
#endif
// largest whole-problem system of the direct path (unknowns per instance)
#define MPN_DIRECT_MAX 4096
// shared memory of the coarsest-inverse kernel (floats)
#define INV_SMEM_FLOATS (224 * 1024 / 4)
// Opt the fused step kernels into the shared memory of their largest tile.
static int fs_set_smem() {
  return (step_row_attrs() == 0 && step_y_attrs() == 0 && march_attrs() == 0) ? MPN_OK : MPN_ERR_CUDA;
}

// Compile-time coefficient layout of the FP64 kernels and the fused coarse
// end: FS_MASK_RDI (c_xx and c_yy one field), FS_MASK_RD, FS_MASK_TR, or 0
// (layout read at run time).
static int fp64_layout(const mpn_problem* p) {
  if (p->field_mask == FS_MASK_TR) return FS_MASK_TR;
  if (p->field_mask != FS_MASK_RD) return 0;
  return p->desc.field_of[4] == p->desc.field_of[6] ? FS_MASK_RDI : FS_MASK_RD;
}
// Instantiation of the fused coarse end for this problem's dimension and
// coefficient layout.
static const void* tail_fn(const mpn_problem* p) {
  if (p->D == 3 && fp64_layout(p) == FS_MASK_RDI) return (const void*)k_vtail<3, FS_MASK_RDI>;
  if (p->D == 3 && fp64_layout(p) == FS_MASK_TR) return (const void*)k_vtail<3, FS_MASK_TR>;
  if (p->D == 3) return p->field_mask == FS_MASK_RD ? (const void*)k_vtail<3, FS_MASK_RD> : (const void*)k_vtail<3, FS_ANY>;
  return (const void*)k_vtail<2, FS_ANY>;
}

// Fused coarse end (mpn_tail.cuh): the finest level k0 with at most two
// points per thread and CTA from which all coarser levels fit, per CTA, in
// shared memory, with the cluster size and the shared-memory layout.  Left at -1 when fewer than two levels would be fused
// or the cluster cannot be resident on this device.
static void plan_tail(mpn_problem* p) {
  p->tail_k0 = -1;
  if (!p->desc.fused_coarse || p->L < 2 || p->desc.variable_steps || p->mixed) return;
  const int n0 = p->lv[0].g.n[0];
  // cluster size: 4 CTAs per instance, more (up to TAIL_MAX_CLUSTER) while
  // the batch gives fewer than TAIL_TARGET_CTAS CTAs in all; smaller sizes
  // are tried when a larger one finds no plan
  int cs_want = 4;
  while (cs_want < TAIL_MAX_CLUSTER && p->B * cs_want < TAIL_TARGET_CTAS) cs_want *= 2;
  for (int cs_try = cs_want; cs_try >= 1; cs_try /= 2) {
  int cs = 1;
  while (cs * 2 <= std::min(cs_try, n0)) cs *= 2;
  const int P = (n0 + cs - 1) / cs;
  const size_t budget = 200 * 1024;
  for (int k0 = 0; k0 + 1 < p->L; ++k0) {
    if (p->L - k0 > TAIL_MAXL) continue;
    // every fused level keeps the time planes (transfers stay inside a CTA)
    bool keeps_t = true;
    for (int k = k0; k + 1 < p->L; ++k) keeps_t = keeps_t && !p->lv[k].cz[0];
    if (!keeps_t) continue;
    // a level with more than TAIL_MAX_PPT points per thread and CTA runs
    // better pass by pass over the whole GPU (vectorised kernels, full occupancy)
    if ((size_t)P * p->lv[k0].g.n[1] * p->lv[k0].g.n[2] > TAIL_MAX_PPT * TAIL_TPB) continue;
    TailArgs& ta = p->tail;
    memset(&ta, 0, sizeof(ta));
    size_t off = 0;
    for (int k = k0; k < p->L; ++k) {
      const Level& l = p->lv[k];
      TailLevel& T = ta.lv[k - k0];
      T.g = l.g;
      for (int d = 0; d < 3; ++d) T.cz[d] = l.cz[d];
      T.plane = l.g.n[1] * l.g.n[2];
      T.cap = P * T.plane;
      T.fields = l.fields; T.rho = l.rho; T.dinv = l.dinv;
      const int c = T.cap;
      T.o_r = (int)off; T.o_e = (int)off + c;
      if (k + 1 < p->L) {
        T.o_d = (int)off + 2 * c; T.o_y = (int)off + 3 * c; T.o_rho = (int)off + 4 * c; T.o_dinv = (int)off + 5 * c;
        T.o_f = (int)off + 6 * c;
        off += (size_t)(6 + p->F) * c;
      } else {
        T.o_d = T.o_y = T.o_rho = T.o_dinv = T.o_f = T.o_r;
        off += (size_t)2 * c;
      }
      off = (off + 3) & ~(size_t)3;
    }
    ta.o_g = (int)off;
    off += (size_t)p->M;
    ta.o_tw = (int)off;
    off += (size_t)P * TW_STRIDE;
    const size_t smem = off * sizeof(float);
    if (smem > budget) continue;
    ta.nl = p->L - k0;
    ta.V = p->V; ta.F = p->F; ta.B = p->B; ta.M = p->M; ta.m = p->desc.cheb_degree; ta.P = P;
    ta.invP = 1.f / (float)P;
    for (int v = 0; v < 7; ++v) ta.field_of[v] = v < p->V ? p->desc.field_of[v] : -1;
    ta.scalars = p->scalars;
    for (int k = 0; k < 32; ++k) { ta.c1[k] = p->cheb_c1[k]; ta.c2[k] = p->cheb_c2[k]; }
    ta.inv_th = p->cheb_inv_th;
    ta.Kinv = p->Kinv;
    ta.rin = p->lv[k0].r;
    ta.eout = p->lv[k0].e;
    const void* fn = tail_fn(p);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        (cs > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
      (void)cudaGetLastError();
      break;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, p->B);
    cfg.blockDim = dim3(TAIL_TPB);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
    cfg.attrs = at; cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, fn, &cfg) != cudaSuccess || ncl < 1) {
      (void)cudaGetLastError();
      break;
    }
    p->tail_k0 = k0; p->tail_cs = cs; p->tail_smem = smem;
    return;
  }
  }
}

static void launch_tail(mpn_problem* p, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p->tail_cs, p->B);
  cfg.blockDim = dim3(TAIL_TPB);
  cfg.dynamicSmemBytes = p->tail_smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = p->tail_cs; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
  cfg.attrs = at; cfg.numAttrs = 1;
  ++p->nlaunch;
  void* args[] = {&p->tail};
  cudaLaunchKernelExC(&cfg, tail_fn(p), args);
}

extern "C" int mpn_fused_level(const mpn_problem* p) { return p ? p->tail_k0 : -1; }

extern "C" int mpn_create(const mpn_desc* desc, mpn_problem** out) {
  if (!desc || !out) return MPN_ERR_INVALID_ARG;
  *out = nullptr;
  const mpn_desc& d = *desc;
  if (d.ndim != 2 && d.ndim != 3) return MPN_ERR_INVALID_ARG;
  if (d.batch < 1 || d.nfields < 0 || d.nfields > 7) return MPN_ERR_INVALID_ARG;
  if (d.batch > 65535) return MPN_ERR_UNSUPPORTED;   // instances are the grid's y (or z) extent
  if (d.periodic[0]) return MPN_ERR_INVALID_ARG;
  if (d.stencil == 5) return MPN_ERR_UNSUPPORTED;
  if (d.stencil != 3) return MPN_ERR_INVALID_ARG;
  if (d.inner_iters < 1 || d.max_refine < 1 || d.cheb_degree < 1 || d.cheb_degree > 30) return MPN_ERR_INVALID_ARG;
  if (d.adj_inner_iters < 0) return MPN_ERR_INVALID_ARG;
  if (d.coarse_min < 3 || !(d.tol > 0)) return MPN_ERR_INVALID_ARG;
  if (d.krylov != MPN_KRYLOV_CG && d.krylov != MPN_KRYLOV_FGMRES) return MPN_ERR_INVALID_ARG;
  if (d.fused_step < 0 || d.fused_step > 4) return MPN_ERR_INVALID_ARG;
  if (d.variable_steps != 0 && d.variable_steps != 1) return MPN_ERR_INVALID_ARG;
  bool mixed = false;
  for (int k = 1; k < d.ndim; ++k) {
    if (d.periodic[k]) continue;
    const double a = d.bc_alpha[k], bt = d.bc_beta[k];
    if (!std::isfinite(a) || !std::isfinite(bt) || (a == 0.0 && bt == 0.0)) return MPN_ERR_INVALID_ARG;
    mixed = mixed || a != 1.0 || bt != 0.0;
  }
  int V = 1 + 2 * d.ndim;
  for (int k = 0; k < d.ndim; ++k) {
    if (d.n[k] < 3 || !(d.variable_steps || d.step[k] > 0)) return MPN_ERR_INVALID_ARG;
  }
  if (d.ndim == 2 && d.n[2] != 1 && d.n[2] != 0) return MPN_ERR_INVALID_ARG;
  for (int v = 0; v < V; ++v)
    if (d.field_of[v] < -1 || d.field_of[v] >= d.nfields) return MPN_ERR_INVALID_ARG;
  long long Nfine = 1;
  for (int k = 0; k < d.ndim; ++k) Nfine *= d.n[k];
  if (Nfine * V * d.batch > (1LL << 31)) return MPN_ERR_UNSUPPORTED;

  mpn_problem* p = new mpn_problem();
  p->desc = d;
  p->mixed = mixed;
  p->D = d.ndim; p->V = V; p->F = d.nfields; p->B = d.batch;
  for (int v = 0; v < V; ++v) if (d.field_of[v] >= 0) p->field_mask |= 1 << v;
  if (p->D == 2) p->desc.n[2] = 1;

  // hierarchy: halve spatial dims (t kept unless coarsen_time) while the half is >= coarse_min
  int n[3] = {p->desc.n[0], p->desc.n[1], p->desc.n[2]};
  // (per-interval steps: the uniform steps of the levels are unused)
  double s[3] = {d.variable_steps ? 1.0 : d.step[0], d.variable_steps ? 1.0 : d.step[1],
                 p->D == 3 && !d.variable_steps ? d.step[2] : 1.0};
  int per[3] = {0, d.periodic[1], p->D == 3 ? d.periodic[2] : 0};
  float theta = 1.f;
  p->L = 0;
  while (true) {
    Level& l = p->lv[p->L];
    l.g = make_grid(p->D, n, s, per, d.final_time_rows, theta);
    int nd = 0;
    for (int k = 0; k < 3; ++k) {
      l.cz[k] = (!d.direct && (k >= 1 || d.coarsen_time) && k < p->D && n[k] % 2 == 0 && n[k] / 2 >= d.coarse_min) ? 1 : 0;
      nd += l.cz[k];
    }
    p->L++;
    if (nd == 0 || p->L == MAXL) { for (int k = 0; k < 3; ++k) l.cz[k] = 0; break; }
    // periodic dims: nested halving (step doubled); non-periodic dims: the
    // coarse points span the same interval (both Dirichlet faces kept)
    for (int k = 0; k < 3; ++k)
      if (l.cz[k]) {
        int nc = n[k] / 2;
        s[k] = per[k] ? 2.0 * s[k] : s[k] * (double)(n[k] - 1) / (double)(nc - 1);
        n[k] = nc;
      }
    theta *= (float)(1 << nd);
  }
  int nsm = 148, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  for (int k = 0; k < p->L; ++k) {
    Level& l = p->lv[k];
    // per-interval steps, Neumann / mixed rows: the general (scalar) kernels only
    l.vec4 = (p->D == 3 && l.g.n[2] % 4 == 0 && l.g.n[2] >= 8 && !d.variable_steps && !mixed) ? 1 : 0;
    l.vec2 = (p->D == 2 && l.g.n[1] % 4 == 0 && l.g.n[1] >= 8 && !d.variable_steps && !mixed) ? 1 : 0;
    l.papply = (l.vec4 || l.vec2) ? sblk(l.g.N / 4) : sblk(l.g.N);
    // fused operator step: tiles that divide the t and x extents, with whole
    // y rows of at most FS_MAX_NY points, or 64-point y segments of wider rows
    // (or of rows >= 128 with fused_step = 2)
    if (d.fused_step && l.vec4 && l.g.n[1] % FS_TX == 0) {
      const int n0 = l.g.n[0], n2 = l.g.n[2];
      const bool per1 = l.g.per[1], per2 = l.g.per[2];
      const bool rd = p->field_mask == FS_MASK_RD;
      l.fs_layout = !(per1 && per2) ? SL_ANY
                    : rd ? (d.field_of[4] == d.field_of[6] ? SL_RDI : SL_RD)
                    : p->field_mask == FS_MASK_TR ? SL_TR : SL_ANY;
      int tt = n0 % 8 == 0 ? 8 : (n0 % 4 == 0 ? 4 : 0);
      // whole-row levels with rows of >= 64 points that 8-plane tiles would
      // leave short of one wave of CTAs on the device take 4-plane tiles
      if (tt == 8 && n2 >= 64 && (n0 / 8) * (l.g.n[1] / FS_TX) * p->B < FS_MIN_CTAS) tt = 4;
      const bool split_ok = n2 % 64 == 0 && n2 >= 128 && step_y_has(8, 64, per1, per2, l.fs_layout) && n0 % 8 == 0;
      const bool whole_ok = tt && n2 <= FS_MAX_NY && step_row_has(tt, per1, per2, l.fs_layout);
      if (split_ok && (d.fused_step == 2 || !whole_ok)) { l.fs_tt = 8; l.fs_ty = 64; }
      else if (whole_ok) { l.fs_tt = tt; l.fs_ty = 0; }
      if (l.fs_tt) {
        l.papply = step_ctas(StepTile{l.fs_tt, l.fs_ty}, l.g);
        if (l.papply > MPN_PMAX) l.fs_tt = l.fs_ty = 0;   // too many partial sums per instance
      }
      if (!l.fs_tt) l.papply = sblk(l.g.N / 4);
      // t-marching columns where they apply: with fused_step = 3 on levels
      // whose columns of 16 rows fill the SMs' resident CTAs over the batch,
      // with 4 on all (16 rows where they divide n_x, else 8)
      if (l.fs_tt && d.fused_step >= 3) {
        for (int mx : {16, 8}) {
          if (!march_has(l.g, per1, per2, l.fs_layout, mx)) continue;
          // (8-row columns measured slower than the whole-row tiles on the
          // levels they would serve: used with fused_step = 4 only)
          if (d.fused_step == 3 && (mx != 16 || march_ctas_per_sm(mx) * march_cols(l.g, mx) * p->B < nsm)) continue;
          const int tc = march_planes(l.g, p->B, nsm, mx);
          const int pm = march_cols(l.g, mx) * (n0 / tc);
          if (pm > MPN_PMAX) continue;
          l.ms_tc = tc; l.ms_mx = mx; l.papply = pm;
          break;
        }
      }
    }
  }
  Level& lc = p->lv[p->L - 1];
  p->M = lc.g.N;
  int plane = lc.g.n[1] * lc.g.n[2];
  p->bw = std::min(p->M - 1, 3 * plane - 1);
  // the coarsest band is factorised in shared memory when it fits, else in
  // global memory (the direct path's whole-problem systems)
  p->band_smem = ((size_t)p->M * (p->bw + 1) + p->bw) * sizeof(float) <= 200 * 1024;
  const int mmax = d.direct ? MPN_DIRECT_MAX : d.max_coarse;
  if (p->M > mmax || p->bw >= 256 || (!d.direct && !p->band_smem)) {
    delete p;
    return MPN_ERR_UNSUPPORTED;
  }

  int B = p->B, F = p->F;
  int rc = MPN_OK;
#define AL(ptr, n) do { rc = dalloc_t(p, &(ptr), (size_t)(n)); if (rc) { mpn_destroy(p); return rc; } } while (0)
  for (int k = 0; k < p->L; ++k) {
    Level& l = p->lv[k];
    size_t N = (size_t)l.g.N * B;
    AL(l.fields, (size_t)std::max(F, 1) * N);
    AL(l.rho, N); AL(l.dinv, N);
    AL(l.r, N); AL(l.e, N); AL(l.d, N); AL(l.y, N); AL(l.t, N);
    if (l.fs_tt) AL(l.e2, N);
  }
  size_t N0 = (size_t)p->lv[0].g.N * B;
  AL(p->Kband, (size_t)B * p->M * (p->bw + 1));
  AL(p->Kinv, (size_t)B * p->M * p->M);
  AL(p->ferr, B);
  AL(p->kerr, 1);
#ifdef MPN_DEBUG
  AL(p->dbg, 1);
  if (cudaMemset(p->dbg, 0, sizeof(int)) != cudaSuccess) { mpn_destroy(p); return MPN_ERR_CUDA; }
  for (int k = 0; k < p->L; ++k) p->lv[k].g.dbg = p->dbg;
#endif
  AL(p->scalars, (size_t)V * B);
  AL(p->scal4, (size_t)V * B * 4);
  AL(p->rhs, N0); AL(p->omega, N0);
  AL(p->field_of_dev, 8);
  AL(p->x, N0); AL(p->pv, N0); AL(p->q, N0); AL(p->z, N0);
  if (p->lv[0].fs_tt) AL(p->pv2, N0);
  AL(p->u64, N0); AL(p->r64, N0); AL(p->y64, N0); AL(p->g64, N0); AL(p->rho64, N0);
  AL(p->uf64, N0); AL(p->kap, N0 * V);
  AL(p->part, (size_t)NSLOT * B * MPN_PMAX);
  AL(p->pcnt, (size_t)2 * B);
  AL(p->ptot, (size_t)2 * B);
  AL(p->dscal, (size_t)16 * B);
  AL(p->lam, (size_t)MAXL * B);
  if (d.variable_steps) {
    p->stn = std::max(p->desc.n[0], std::max(p->desc.n[1], p->desc.n[2]));
    const size_t per_level = (size_t)B * 3 * p->stn;
    AL(p->hlev, per_level * p->L);
    AL(p->st64, per_level * p->L * ST_REC);
    AL(p->st32, per_level * p->L * ST_REC);
    AL(p->sterr, 1);
    for (int k = 0; k < p->L; ++k) {
      Grid& g = p->lv[k].g;
      g.st64 = p->st64 + per_level * k * ST_REC;
      g.st32 = p->st32 + per_level * k * ST_REC;
      g.stn = p->stn;
    }
  }
  if (mixed) {
    AL(p->r12d, N0); AL(p->r22d, N0); AL(p->y2d, N0);
    for (int k = 0; k < p->L; ++k) {
      Level& l = p->lv[k];
      const size_t N = (size_t)l.g.N * B;
      AL(l.r12, N); AL(l.r22, N); AL(l.y2, N);
      Grid& g = l.g;
      g.mixed = 1;
      for (int e = 0; e < 3; ++e) {
        const bool on = e >= 1 && e < p->D && !d.periodic[e] && (d.bc_alpha[e] != 1.0 || d.bc_beta[e] != 0.0);
        g.bcm[e] = on ? 1 : 0;
        g.bca[e] = on ? (float)d.bc_alpha[e] : 1.f;
        g.bcb[e] = on ? (float)d.bc_beta[e] : 0.f;
      }
      g.r12 = l.r12; g.r22 = l.r22; g.y2 = l.y2;
      if (k == 0) { g.r12d = p->r12d; g.r22d = p->r22d; g.y2d = p->y2d; }
    }
  }
  if (d.krylov == MPN_KRYLOV_FGMRES) {
    p->mk = std::min(FG_MMAX, 8 * std::max(d.inner_iters, d.adj_inner_iters));
    const int mk = p->mk;
    AL(p->fgV, (size_t)(mk + 1) * N0);
    AL(p->fgZ, (size_t)mk * N0);
    AL(p->fgpart, (size_t)(mk + 2) * B * MPN_PMAX);
    AL(p->fgH, (size_t)B * mk * (mk + 1));
    AL(p->fgc, (size_t)B * mk); AL(p->fgs, (size_t)B * mk); AL(p->fgy, (size_t)B * mk);
    AL(p->fgg, (size_t)B * (mk + 1)); AL(p->fgh, (size_t)B);
  }
#undef AL
  int fo[8];
  for (int v = 0; v < 8; ++v) fo[v] = v < V ? d.field_of[v] : -1;
  if (cudaMemcpy(p->field_of_dev, fo, sizeof(fo), cudaMemcpyHostToDevice) != cudaSuccess) { mpn_destroy(p); return MPN_ERR_CUDA; }
  if (cudaMemset(p->kerr, 0, sizeof(int)) != cudaSuccess) { mpn_destroy(p); return MPN_ERR_CUDA; }
  if (cudaMemset(p->pcnt, 0, sizeof(int) * 2 * B) != cudaSuccess) { mpn_destroy(p); return MPN_ERR_CUDA; }
  if (cudaMallocHost((void**)&p->hbuf, sizeof(double) * 16 * B) != cudaSuccess) { mpn_destroy(p); return MPN_ERR_CUDA; }

  // Chebyshev coefficients on [lo, 1] for Dinv scaled by 1 / lambda_max
  const double lo = MPN_CHEB_LO, th = (1.0 + lo) / 2, de = (1.0 - lo) / 2, sg = th / de;
  p->cheb_inv_th = (float)(1.0 / th);
  double r0 = 1.0 / sg;
  for (int k = 1; k < d.cheb_degree && k < 32; ++k) {
    double r1 = 1.0 / (2 * sg - r0);
    p->cheb_c1[k] = (float)(r1 * r0);
    p->cheb_c2[k] = (float)(2 * r1 / de);
    r0 = r1;
  }
  if (fs_set_smem() != MPN_OK) { mpn_destroy(p); return MPN_ERR_CUDA; }
  plan_tail(p);
  *out = p;
  return MPN_OK;
}

// ------------------------------------------------------------------ pieces
#define PROF_PAIRS 1024
// Events are recorded only while a sweep graph is being captured; each graph
// owns the range of the pool it recorded into.
static void prof_mark(mpn_problem* p, cudaStream_t st) {
  if (!p->prof_on || p->prof_next >= 2 * PROF_PAIRS) return;
  // inside stream capture a timing event must be an external event-record node
  if (cudaEventRecordWithFlags(p->prof_ev[p->prof_next], st, cudaEventRecordExternal) == cudaSuccess)
    ++p->prof_next;
  else
    (void)cudaGetLastError();
}
// Accumulates the (start, end) pairs of events [e0, e1); the graph that
// recorded them has completed.
static void prof_flush(mpn_problem* p, int e0, int e1) {
  if (!p->prof_on) return;
  const Level& l = p->lv[0];
  // algorithmic bytes of the bracketed smoothing step on the finest grid
  // (FP32): read e, r, dinv, rho and the F coefficient fields once, and either
  // the previous iterate (fused step, no direction array) or the direction d,
  // write e (and d)
  double bytes = 4.0 * (l.fs_tt ? 6 + p->F : 7 + p->F) * (double)l.g.N * p->B;
  for (int k = e0; k + 1 < e1; k += 2) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p->prof_ev[k], p->prof_ev[k + 1]) == cudaSuccess) {
      p->prof_ms += ms; p->prof_n += 1; p->prof_bytes += bytes;
    }
  }
}
// One operator pass pair at level k: y = -rho L x, then the mode's update.
static void stencil(mpn_problem* p, int k, StepArgs a, int mode, cudaStream_t st) {
  Level& l = p->lv[k];
  Coef cf = make_coef(p, l.fields);
  a.y = l.y;
  if (!a.dinv) a.dinv = l.dinv;
  if (!a.err) a.err = p->kerr;
  if (l.ms_tc && mode != SM_APPLYP) {
    ++p->nlaunch;
    march_launch(mode, l.fs_layout, p->B, l.ms_mx, l.ms_tc, st, l.g, cf, l.rho, a);
    return;
  }
  if (l.fs_tt) {
    const size_t sm = step_smem(StepTile{l.fs_tt, l.fs_ty}, l.g.n[2]);
    ++p->nlaunch;
    if (l.fs_ty) step_y_launch(mode, l.fs_tt, l.fs_ty, l.g.per[1], l.g.per[2], l.fs_layout, p->B, sm, st, l.g, cf, l.rho, a);
    else step_row_launch(mode, l.fs_tt, l.g.per[1], l.g.per[2], l.fs_layout, p->B, sm, st, l.g, cf, l.rho, a);
    return;
  }
  if (l.vec4) {
    dim3 g4(sblk(l.g.N / 4), p->B);
    ++p->nlaunch, k_Ly4<<<g4, MPN_TPB, 0, st>>>(l.g, cf, l.rho, a.x, l.y);
    switch (mode) {
      case SM_POST0: ++p->nlaunch, k_LTy4<SM_POST0><<<g4, MPN_TPB, 0, st>>>(l.g, cf, a); break;
      case SM_CHEB: ++p->nlaunch, k_LTy4<SM_CHEB><<<g4, MPN_TPB, 0, st>>>(l.g, cf, a); break;
      case SM_RES: ++p->nlaunch, k_LTy4<SM_RES><<<g4, MPN_TPB, 0, st>>>(l.g, cf, a); break;
      default: ++p->nlaunch, k_LTy4<SM_APPLY><<<g4, MPN_TPB, 0, st>>>(l.g, cf, a); break;
    }
    return;
  }
  if (l.vec2) {
    dim3 g4(sblk(l.g.N / 4), p->B);
    ++p->nlaunch, k_Ly4_2<<<g4, MPN_TPB, 0, st>>>(l.g, cf, l.rho, a.x, l.y);
    switch (mode) {
      case SM_POST0: ++p->nlaunch, k_LTy4_2<SM_POST0><<<g4, MPN_TPB, 0, st>>>(l.g, cf, a); break;
      case SM_CHEB: ++p->nlaunch, k_LTy4_2<SM_CHEB><<<g4, MPN_TPB, 0, st>>>(l.g, cf, a); break;
      case SM_RES: ++p->nlaunch, k_LTy4_2<SM_RES><<<g4, MPN_TPB, 0, st>>>(l.g, cf, a); break;
      default: ++p->nlaunch, k_LTy4_2<SM_APPLY><<<g4, MPN_TPB, 0, st>>>(l.g, cf, a); break;
    }
    return;
  }
  dim3 gr(sblk(l.g.N), p->B);
#define LTY(DD, MM) ++p->nlaunch, k_LTy<DD, MM><<<gr, MPN_TPB, 0, st>>>(l.g, cf, a)
#define LTY_D(DD)                                   \
  switch (mode) {                                   \
    case SM_POST0: LTY(DD, SM_POST0); break;        \
    case SM_CHEB: LTY(DD, SM_CHEB); break;          \
    case SM_RES: LTY(DD, SM_RES); break;            \
    default: LTY(DD, SM_APPLY); break;              \
  }
  if (p->D == 3) {
    ++p->nlaunch, k_Ly<3><<<gr, MPN_TPB, 0, st>>>(l.g, cf, l.rho, a.x, l.y);
    LTY_D(3)
  } else {
    ++p->nlaunch, k_Ly<2><<<gr, MPN_TPB, 0, st>>>(l.g, cf, l.rho, a.x, l.y);
    LTY_D(2)
  }
#undef LTY_D
#undef LTY
}

// q = S x at level k (FP32), optional <x, q> partials into `part` (sblk per instance).
static int apply_S(mpn_problem* p, int k, const float* x, float* q, double* part, cudaStream_t st) {
  StepArgs a;
  memset(&a, 0, sizeof(a));
  a.x = x; a.out = q; a.part = part;
  stencil(p, k, a, SM_APPLY, st);
  CKL();
  return MPN_OK;
}

// Streams and events of the setup and of the sweep graphs (created once).
static int ensure_streams(mpn_problem* p) {
  if (!p->gstream) {
    CK(cudaStreamCreateWithFlags(&p->gstream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&p->ev_user, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&p->ev_setup, cudaEventDisableTiming));
  }
  if (!p->ev_fork) {
    CK(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
    for (int k = 0; k < MAXL; ++k) {
      CK(cudaStreamCreateWithFlags(&p->aux[k], cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&p->ev_join[k], cudaEventDisableTiming));
    }
  }
  return MPN_OK;
}

// Shared-memory sizes of the coarsest factorisation and inverse, and the
// inverse's warps per CTA.
static size_t coarse_factor_smem(const mpn_problem* p) { return sizeof(float) * ((size_t)p->M * (p->bw + 1) + p->bw); }
static int coarse_inverse_warps(const mpn_problem* p) {
  const size_t fixed = (p->band_smem ? (size_t)p->M * (p->bw + 1) : 0) + p->M;
  return (int)std::min<size_t>(32, (INV_SMEM_FLOATS - fixed) / p->M);
}
static size_t coarse_inverse_smem(const mpn_problem* p) {
  const size_t fixed = (p->band_smem ? (size_t)p->M * (p->bw + 1) : 0) + p->M;
  return sizeof(float) * (fixed + (size_t)coarse_inverse_warps(p) * p->M);
}
// Opts the coarsest-level kernels of this problem into their shared memory
// (host calls, kept out of the captured setup).
static int coarse_attrs(mpn_problem* p) {
  if (p->band_smem) {
    CK(cudaFuncSetAttribute(k_coarse_factor<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)coarse_factor_smem(p)));
    CK(cudaFuncSetAttribute(k_coarse_factor1<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)coarse_factor_smem(p)));
  }
  const int sm = (int)coarse_inverse_smem(p);
#define INV_ATTR(NW) \
  CK(cudaFuncSetAttribute(p->band_smem ? (const void*)k_coarse_inverse<NW, true> : (const void*)k_coarse_inverse<NW, false>, \
                          cudaFuncAttributeMaxDynamicSharedMemorySize, sm))
  if (p->bw < 32) INV_ATTR(1);
  else if (p->bw < 64) INV_ATTR(2);
  else if (p->bw < 128) INV_ATTR(4);
  else INV_ATTR(8);
#undef INV_ATTR
  return MPN_OK;
}

// The setup after the input copies: coefficients and weights of every level,
// Jacobi diagonals, lambda_max estimates, the coarsest factorisation and
// inverse.  Reads only the problem's own buffers.
static int setup_body(mpn_problem* p, cudaStream_t st) {
  int B = p->B, F = p->F, V = p->V;
  Level& l0 = p->lv[0];
  if (p->desc.variable_steps) {
    // intervals of every level, then the step records of every level
    const size_t per_level = (size_t)B * 3 * p->stn;
    const int nrec = (int)per_level;
    for (int k = 0; k < p->L; ++k) {
      if (k > 0) {
        const Level& lf = p->lv[k - 1];
        ++p->nlaunch, k_level_steps<<<(B * p->D + 63) / 64, 64, 0, st>>>(
            lf.g, p->lv[k].g, lf.cz[0], lf.cz[1], lf.cz[2], p->hlev + per_level * (k - 1), p->hlev + per_level * k, B);
      }
      ++p->nlaunch, k_step_table<<<(nrec + 127) / 128, 128, 0, st>>>(
          p->lv[k].g, p->hlev + per_level * k, p->st64 + per_level * k * ST_REC, p->st32 + per_level * k * ST_REC, B,
          p->sterr);
    }
    CKL();
  }
  ++p->nlaunch, k_rep4<<<(V * B + MPN_TPB - 1) / MPN_TPB, MPN_TPB, 0, st>>>(V * B, p->scalars, p->scal4);
  {
    Coef cf = make_coef(p, l0.fields);
    if (p->D == 3) ++p->nlaunch, k_rho_fine<3><<<dim3(nblk(p, l0.g.N), B), MPN_TPB, 0, st>>>(l0.g, cf, l0.rho, p->rho64);
    else ++p->nlaunch, k_rho_fine<2><<<dim3(nblk(p, l0.g.N), B), MPN_TPB, 0, st>>>(l0.g, cf, l0.rho, p->rho64);
    if (p->mixed)
      ++p->nlaunch, k_mixed_weights<<<dim3(nblk(p, l0.g.N), B), MPN_TPB, 0, st>>>(l0.g, cf, l0.rho, l0.r12, l0.r22, p->rho64,
                                                                          p->r12d, p->r22d);
    CKL();
  }
  for (int k = 1; k < p->L; ++k) {
    Level& lf = p->lv[k - 1];
    Level& lc = p->lv[k];
    int nd = lf.cz[0] + lf.cz[1] + lf.cz[2];
    dim3 gf(nblk(p, lc.g.N), F * B);
    if (F > 0)
      ++p->nlaunch, k_restrict_field<<<gf, MPN_TPB, 0, st>>>(lf.g, lc.g, lf.cz[0], lf.cz[1], lf.cz[2], lf.fields, lc.fields, 1.f);
    ++p->nlaunch, k_restrict_field<<<dim3(nblk(p, lc.g.N), B), MPN_TPB, 0, st>>>(lf.g, lc.g, lf.cz[0], lf.cz[1], lf.cz[2], lf.rho,
                                                               lc.rho, (float)(1 << nd));
    if (p->mixed) {
      Coef cfc = make_coef(p, lc.fields);
      ++p->nlaunch, k_mixed_weights<<<dim3(nblk(p, lc.g.N), B), MPN_TPB, 0, st>>>(lc.g, cfc, lc.rho, lc.r12, lc.r22, nullptr,
                                                                          nullptr, nullptr);
    }
    CKL();
  }
  // Jacobi diagonals and lambda_max(Dinv S) per level: the levels are
  // independent, so each runs its power iteration on a stream of its own
  // while the coarsest system is factorised on st.
  CK(cudaEventRecord(p->ev_fork, st));
  // the coarsest level first: its factorisation and inverse are the longest
  // dependent chain of the setup, so st starts on it while the host is still
  // launching the power iterations
  {
    Level& l = p->lv[p->L - 1];
    Coef cf = make_coef(p, l.fields);
    ++p->nlaunch, k_diag_inv<<<dim3(nblk(p, l.g.N), B), MPN_TPB, 0, st>>>(l.g, cf, l.rho, l.dinv);
    CKL();
  }
  // coarsest: banded assembly, Cholesky, explicit inverse
  Level& lc = p->lv[p->L - 1];
  Coef cfc = make_coef(p, lc.fields);
  CK(cudaMemsetAsync(p->ferr, 0, sizeof(int) * B, st));
  ++p->nlaunch, k_coarse_assemble<<<dim3(nblk(p, p->M), B), MPN_TPB, 0, st>>>(lc.g, cfc, lc.rho, p->bw, p->Kband);
  // bands up to FACT1_MAXBW: one barrier per column step (k_coarse_factor1)
  const bool f1 = p->bw <= FACT1_MAXBW;
  if (p->band_smem) {
    if (f1) ++p->nlaunch, k_coarse_factor1<true><<<B, 512, coarse_factor_smem(p), st>>>(p->M, p->bw, p->Kband, p->ferr);
    else ++p->nlaunch, k_coarse_factor<true><<<B, 512, coarse_factor_smem(p), st>>>(p->M, p->bw, p->Kband, p->ferr);
  } else {
    if (f1) ++p->nlaunch, k_coarse_factor1<false><<<B, 512, 0, st>>>(p->M, p->bw, p->Kband, p->ferr);
    else ++p->nlaunch, k_coarse_factor<false><<<B, 512, sizeof(float) * p->bw, st>>>(p->M, p->bw, p->Kband, p->ferr);
  }
  // one warp per column of the inverse; the CTA stages the band, the
  // reciprocal diagonal and one forward-solution vector per warp
  {
    const int nwarps = coarse_inverse_warps(p);
    dim3 gi(((p->M + nwarps - 1) / nwarps) * B);
    const size_t sm = coarse_inverse_smem(p);
#define INV_LAUNCH2(NW, SM) \
  ++p->nlaunch, k_coarse_inverse<NW, SM><<<gi, 32 * nwarps, sm, st>>>(p->M, p->bw, p->Kband, p->Kinv)
#define INV_LAUNCH(NW) do { if (p->band_smem) INV_LAUNCH2(NW, true); else INV_LAUNCH2(NW, false); } while (0)
    if (p->bw < 32) INV_LAUNCH(1);
    else if (p->bw < 64) INV_LAUNCH(2);
    else if (p->bw < 128) INV_LAUNCH(4);
    else INV_LAUNCH(8);
#undef INV_LAUNCH2
#undef INV_LAUNCH
  }

  CKL();
  for (int k = 0; k + 1 < p->L; ++k) {
    Level& l = p->lv[k];
    Coef cf = make_coef(p, l.fields);
    dim3 gr(nblk(p, l.g.N), B);
    cudaStream_t sk = p->aux[k];
    CK(cudaStreamWaitEvent(sk, p->ev_fork, 0));
    ++p->nlaunch, k_diag_inv<<<gr, MPN_TPB, 0, sk>>>(l.g, cf, l.rho, l.dinv);
    CKL();
    // power method for lambda_max(Dinv S)
    // x_{k+1} = Dinv S x_k / ||x_k||: the norms are read from the partial
    // sums of the previous step (two slots, alternating), so no separate
    // normalisation pass
    double* pw[2] = {slot(p, S_PW0 + k), slot(p, S_PW1 + k)};
    ++p->nlaunch, k_fill_hash<<<gr, MPN_TPB, 0, sk>>>(l.g.N, l.t, pw[0]);
    const int nit = 12;
    for (int it = 0; it < nit; ++it) {
      TRY(apply_S(p, k, l.t, l.d, nullptr, sk));
      ++p->nlaunch, k_power_w<<<gr, MPN_TPB, 0, sk>>>(l.g.N, l.dinv, l.d, pw[it & 1], gr.x, l.t, pw[(it + 1) & 1]);
    }
    ++p->nlaunch, k_scale_dinv<<<gr, MPN_TPB, 0, sk>>>(l.g.N, l.dinv, pw[nit & 1], gr.x, 1.1f, p->lam + k * B);
    CKL();
    CK(cudaEventRecord(p->ev_join[k], sk));
  }
  CKL();
  for (int k = 0; k + 1 < p->L; ++k) CK(cudaStreamWaitEvent(st, p->ev_join[k], 0));
  return MPN_OK;
}

// Setup for new coefficients: copies them in on st, then replays the
// captured setup graph on the internal stream, ordered after st and before
// st's next work.
static int setup(mpn_problem* p, const float* fields, const float* scalars, cudaStream_t st) {
  int B = p->B, F = p->F, V = p->V;
  p->setup_ok = false;
  p->zd_valid = false;
  Level& l0 = p->lv[0];
  if (F > 0) CK(cudaMemcpyAsync(l0.fields, fields, sizeof(float) * (size_t)F * B * l0.g.N, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(p->scalars, scalars, sizeof(float) * (size_t)V * B, cudaMemcpyDeviceToDevice, st));
  TRY(ensure_streams(p));
  if (!p->setup_exec) {
    TRY(coarse_attrs(p));
    long long nl0 = p->nlaunch;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(p->gstream, cudaStreamCaptureModeThreadLocal));
    int s = setup_body(p, p->gstream);
    cudaError_t ec = cudaStreamEndCapture(p->gstream, &graph);
    if (s != MPN_OK) { if (graph) cudaGraphDestroy(graph); return s; }
    CK(ec);
    cudaError_t ei = cudaGraphInstantiate(&p->setup_exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(ei);
    p->setup_kernels = p->nlaunch - nl0;
    p->nlaunch = nl0;
  }
  CK(cudaEventRecord(p->ev_user, st));
  CK(cudaStreamWaitEvent(p->gstream, p->ev_user, 0));
  CK(cudaGraphLaunch(p->setup_exec, p->gstream));
  p->nlaunch += p->setup_kernels;
  CK(cudaEventRecord(p->ev_setup, p->gstream));
  CK(cudaStreamWaitEvent(st, p->ev_setup, 0));
  p->setup_ok = true;
  return MPN_OK;
}

// One V-cycle at level k: e_k ~ S_k^{-1} r_k (result in l.e).
// started: the restriction into this level already started its smoother
// (d = e = inv_th D^-1 r in the iterate buffer the pre-smoothing begins in).
// zdot (fused level 0 only): its last smoothing step writes the partials of
// <e, r> of the V-cycle's result there.
static int vcycle(mpn_problem* p, int k, cudaStream_t st, bool started = false, double* zdot = nullptr) {
  Level& l = p->lv[k];
  int B = p->B;
  dim3 gr(nblk(p, l.g.N), B);
  if (k == p->tail_k0) {
    launch_tail(p, st);
    CKL();
    return MPN_OK;
  }
  if (k == p->L - 1) {
    ++p->nlaunch, k_coarse_solve<<<dim3((p->M * 32 + MPN_TPB - 1) / MPN_TPB, B), MPN_TPB, 0, st>>>(p->M, p->Kinv, l.r, l.e);
    CKL();
    return MPN_OK;
  }
  int m = p->desc.cheb_degree;
  bool prof = (k == 0);
  // Iterate buffers: a fused level reads the operand with a halo and writes
  // the updated iterate to the other buffer.  The 2m - 1 halo-reading updates
  // of a V-cycle flip the buffer an odd number of times, so starting in e2
  // ends in e.
  float* cur = l.fs_tt ? l.e2 : l.e;
  auto other = [&](float* e) { return !l.fs_tt ? e : (e == l.e ? l.e2 : l.e); };
  // A fused level keeps no direction array: its Chebyshev steps read the
  // previous iterate (the other buffer, null after a start from zero).
  float* ddir = l.fs_tt ? nullptr : l.d;
  auto prev = [&](float* e, bool zero) -> float* { return !l.fs_tt ? l.d : (zero ? nullptr : other(e)); };
  StepArgs a;
  memset(&a, 0, sizeof(a));
  a.r = l.r;
  // pre-smoothing from e = 0: d = Dinv r / th, e = d
  if (!started) {
    if (vec4_len(l.g.N))
      ++p->nlaunch, k_cheb_init<true><<<dim3(vgrid(l.g.N), B), MPN_TPB, 0, st>>>(l.g.N, l.r, l.dinv, p->cheb_inv_th, cur, ddir);
    else
      ++p->nlaunch, k_cheb_init<false><<<dim3(vgrid(l.g.N), B), MPN_TPB, 0, st>>>(l.g.N, l.r, l.dinv, p->cheb_inv_th, cur, ddir);
  }
  // profiling brackets one smoothing step per V-cycle (each event is a graph
  // node of its own, so bracketing every step would slow the sweep): the
  // second, the first that reads a previous iterate
  const int prof_s = m >= 3 ? 2 : 1;
  for (int s = 1; s < m; ++s) {
    a.c1 = p->cheb_c1[s]; a.c2 = p->cheb_c2[s];
    a.x = cur; a.e = other(cur); a.d = prev(cur, s == 1);
    if (prof && s == prof_s) prof_mark(p, st);
    stencil(p, k, a, SM_CHEB, st);
    if (prof && s == prof_s) prof_mark(p, st);
    cur = other(cur);
  }
  // residual, restricted to the coarse level
  a.x = cur; a.e = cur;
  a.out = l.t;
  stencil(p, k, a, SM_RES, st);
  Level& lc = p->lv[k + 1];
  const bool vec4r = !l.cz[0] && l.cz[1] && l.cz[2] && l.g.per[1] && l.g.per[2] && l.g.n[2] % 8 == 0;
  // the float4 restriction also starts the coarse level's smoother, unless
  // that level is the fused coarse end or the coarsest solve
  const bool start_c = vec4r && k + 1 != p->tail_k0 && k + 1 != p->L - 1;
  if (vec4r)
    ++p->nlaunch, k_restrict_vec4<<<dim3(sblk(lc.g.N / 4), B), MPN_TPB, 0, st>>>(
        l.g, lc.g, l.t, lc.r, start_c ? lc.dinv : nullptr, p->cheb_inv_th, lc.fs_tt ? lc.e2 : lc.e,
        lc.fs_tt ? nullptr : lc.d);
  else
    ++p->nlaunch, k_restrict_vec<<<dim3(nblk(p, lc.g.N), B), MPN_TPB, 0, st>>>(l.g, lc.g, l.cz[0], l.cz[1], l.cz[2], l.t, lc.r);
  CKL();
  TRY(vcycle(p, k + 1, st, start_c));
  if (!l.cz[0] && l.cz[1] && l.cz[2] && l.g.per[1] && l.g.per[2] && l.g.n[2] % 4 == 0)
    ++p->nlaunch, k_prolong_add4<<<dim3(sblk(l.g.N / 4), B), MPN_TPB, 0, st>>>(l.g, lc.g, lc.e, cur);
  else
    ++p->nlaunch, k_prolong_add<<<gr, MPN_TPB, 0, st>>>(l.g, lc.g, l.cz[0], l.cz[1], l.cz[2], lc.e, nullptr, cur);
  // post-smoothing
  a.c1 = 0.f; a.c2 = p->cheb_inv_th;
  a.x = cur; a.e = other(cur); a.d = ddir;
  stencil(p, k, a, SM_POST0, st);
  cur = other(cur);
  for (int s = 1; s < m; ++s) {
    a.c1 = p->cheb_c1[s]; a.c2 = p->cheb_c2[s];
    a.x = cur; a.e = other(cur); a.d = prev(cur, false);
    const bool dot = zdot && s == m - 1;
    a.part = dot ? zdot : nullptr;
    // the step's last CTA per instance also finishes <e', r> (PCG's <r, z>)
    a.cnt = dot ? p->pcnt : nullptr;
    a.tot = dot ? p->ptot : nullptr;
    stencil(p, k, a, dot ? SM_CHEB_DOT : SM_CHEB, st);
    cur = other(cur);
  }
  CKL();
  return MPN_OK;
}

// z = V(r) at the finest level with partial <r, z> in slot S_RZ.
// started: the kernel that wrote lv[0].r also started the smoother.
// zin_e: z is the V-cycle's result lv[0].e itself, the partials of <r, z>
// written by its last smoothing step (see z_in_e()); else z is copied out.
static int precond(mpn_problem* p, cudaStream_t st, bool started = false, bool zin_e = false) {
  Level& l = p->lv[0];
  TRY(vcycle(p, 0, st, started, zin_e ? slot(p, S_RZ) : nullptr));
  if (zin_e) return MPN_OK;
  dim3 gv(vgrid(l.g.N), p->B);
  if (vec4_len(l.g.N)) ++p->nlaunch, k_final_z<true><<<gv, MPN_TPB, 0, st>>>(l.g.N, l.e, l.r, p->z, slot(p, S_RZ));
  else ++p->nlaunch, k_final_z<false><<<gv, MPN_TPB, 0, st>>>(l.g.N, l.e, l.r, p->z, slot(p, S_RZ));
  CKL();
  return MPN_OK;
}

// PCG may take z from the finest level's iterate buffer (the V-cycle ends in
// lv[0].e, which nothing overwrites before z is consumed) when that level runs
// the fused step's smoothing through the V-cycle's end.
static bool z_in_e(const mpn_problem* p) {
  return p->lv[0].fs_tt && p->tail_k0 != 0 && p->L > 1 && p->desc.cheb_degree >= 2;
}

// Inner FP32 PCG on S x = r (r = lv[0].r), fixed iteration count, x = p->x.
// started: the kernel that wrote r also started the first V-cycle's smoother;
// the residual updates start the following ones.
static int pcg(mpn_problem* p, int iters, cudaStream_t st, bool started) {
  Level& l = p->lv[0];
  float* cur0 = l.fs_tt ? l.e2 : l.e;       // the iterate buffer the V-cycle's pre-smoothing begins in
  float* ddir0 = l.fs_tt ? nullptr : l.d;   // its direction array (none on a fused level)
  const int N = l.g.N;
  dim3 gv(vgrid(N), p->B);
  const int P = gv.x;
  const bool ze = z_in_e(p);
  float* zv = ze ? l.e : p->z;
  const int Prz = ze ? l.papply : P;         // partials of <r, z>
  const bool v4 = vec4_len(N);
  double* rz_old = p->dscal + p->B;
  TRY(precond(p, st, started, ze));
  if (l.fs_tt) {
    // the direction update rides on the operator apply (mode SM_APPLYP):
    // p = z, then p = z + beta p, written to the other direction buffer
    CK(cudaMemsetAsync(p->x, 0, sizeof(float) * (size_t)N * p->B, st));
    float* pb[2] = {p->pv, p->pv2};
    int c = 0;
    for (int it = 0; it < iters; ++it) {
      StepArgs a;
      memset(&a, 0, sizeof(a));
      a.x = zv; a.out = p->q; a.part = slot(p, S_PQ);
      a.cnt = p->pcnt + p->B; a.tot = p->ptot + p->B;   // <p, S p> finished by the step's last CTAs
      if (l.ms_tc) {
        // on the t-marching step: p = z + beta p_old by a vector pass, then the apply
        float* pn = it == 0 ? pb[c] : pb[c ^ 1];
        if (v4)
          ++p->nlaunch, k_pcg_pd<true><<<gv, MPN_TPB, 0, st>>>(N, ze ? p->ptot : nullptr, slot(p, S_RZ), Prz, rz_old,
                                                               zv, it == 0 ? nullptr : pb[c], pn);
        else
          ++p->nlaunch, k_pcg_pd<false><<<gv, MPN_TPB, 0, st>>>(N, ze ? p->ptot : nullptr, slot(p, S_RZ), Prz, rz_old,
                                                                zv, it == 0 ? nullptr : pb[c], pn);
        CKL();
        if (it > 0) c ^= 1;
        a.x = pn;
        stencil(p, 0, a, SM_APPLY, st);
      } else {
        if (it == 0) {
          a.e = pb[c];
        } else {
          a.d = pb[c]; a.e = pb[c ^ 1];
          a.rz = slot(p, S_RZ); a.nrz = Prz; a.rz_old = rz_old;
          a.rz_tot = ze ? p->ptot : nullptr;
          c ^= 1;
        }
        stencil(p, 0, a, SM_APPLYP, st);
      }
      const float* dst = it < iters - 1 ? l.dinv : nullptr;   // a V-cycle follows
      if (v4)
        ++p->nlaunch, k_pcg_xr<true><<<gv, MPN_TPB, 0, st>>>(N, slot(p, S_RZ), slot(p, S_PQ), l.papply, Prz, pb[c], p->q,
                                                              p->x, l.r, rz_old, dst, p->cheb_inv_th, cur0, ddir0,
                                                              ze ? p->ptot : nullptr, p->ptot + p->B);
      else
        ++p->nlaunch, k_pcg_xr<false><<<gv, MPN_TPB, 0, st>>>(N, slot(p, S_RZ), slot(p, S_PQ), l.papply, Prz, pb[c], p->q,
                                                               p->x, l.r, rz_old, dst, p->cheb_inv_th, cur0, ddir0,
                                                               ze ? p->ptot : nullptr, p->ptot + p->B);
      CKL();
      if (it == iters - 1) break;
      TRY(precond(p, st, true, ze));
    }
    return MPN_OK;
  }
  if (v4) ++p->nlaunch, k_pcg_init<true><<<gv, MPN_TPB, 0, st>>>(N, zv, p->x, p->pv);
  else ++p->nlaunch, k_pcg_init<false><<<gv, MPN_TPB, 0, st>>>(N, zv, p->x, p->pv);
  for (int it = 0; it < iters; ++it) {
    TRY(apply_S(p, 0, p->pv, p->q, slot(p, S_PQ), st));
    const float* dst = it < iters - 1 ? l.dinv : nullptr;   // a V-cycle follows
    if (v4)
      ++p->nlaunch, k_pcg_xr<true><<<gv, MPN_TPB, 0, st>>>(N, slot(p, S_RZ), slot(p, S_PQ), l.papply, Prz, p->pv, p->q,
                                                            p->x, l.r, rz_old, dst, p->cheb_inv_th, cur0, ddir0,
                                                            nullptr, nullptr);
    else
      ++p->nlaunch, k_pcg_xr<false><<<gv, MPN_TPB, 0, st>>>(N, slot(p, S_RZ), slot(p, S_PQ), l.papply, Prz, p->pv, p->q,
                                                             p->x, l.r, rz_old, dst, p->cheb_inv_th, cur0, ddir0,
                                                             nullptr, nullptr);
    CKL();
    if (it == iters - 1) break;
    TRY(precond(p, st, true, ze));
    if (v4) ++p->nlaunch, k_pcg_p<true><<<gv, MPN_TPB, 0, st>>>(N, slot(p, S_RZ), Prz, rz_old, zv, p->pv);
    else ++p->nlaunch, k_pcg_p<false><<<gv, MPN_TPB, 0, st>>>(N, slot(p, S_RZ), Prz, rz_old, zv, p->pv);
    CKL();
  }
  return MPN_OK;
}

// Inner FP32 FGMRES(m) on S x = r (r = lv[0].r, overwritten by the basis
// vectors), m = iters capped at the workspace, x = p->x.  The V-cycle reads
// its right-hand side from lv[0].r and leaves z_j in lv[0].e.
static int fgmres(mpn_problem* p, int iters, cudaStream_t st) {
  Level& l = p->lv[0];
  const int N = l.g.N, B = p->B;
  const int m = std::min(iters, p->mk);
  const size_t vs = (size_t)N * B;          // vector stride
  dim3 gv(vgrid(N), B);
  const int P = gv.x;
  const bool v4 = vec4_len(N);
  double* dots = p->fgpart;                 // slots 0..m
  double* nrm = p->fgpart + (size_t)(p->mk + 1) * B * MPN_PMAX;
#define FG_V4(K, ...) do { if (v4) ++p->nlaunch, K<true><<<gv, MPN_TPB, 0, st>>>(__VA_ARGS__); \
                           else ++p->nlaunch, K<false><<<gv, MPN_TPB, 0, st>>>(__VA_ARGS__); } while (0)
  // beta = |r|, v_0 = r / beta
  FG_V4(k_fg_dots, N, l.r, l.r, (size_t)0, 1, dots);
  ++p->nlaunch, k_fg_init<<<B, 32, 0, st>>>(p->mk + 1, dots, P, p->fgg, p->fgh);
  FG_V4(k_fg_scale, N, l.r, p->fgh, p->fgV, l.r);
  CKL();
  for (int j = 0; j < m; ++j) {
    TRY(vcycle(p, 0, st));                                        // z_j in lv[0].e
    CK(cudaMemcpyAsync(p->fgZ + j * vs, l.e, sizeof(float) * vs, cudaMemcpyDeviceToDevice, st));
    TRY(apply_S(p, 0, l.e, p->q, nullptr, st));                   // w = S z_j
    FG_V4(k_fg_dots, N, p->q, p->fgV, vs, j + 1, dots);
    FG_V4(k_fg_orth, N, p->q, p->fgV, vs, j + 1, dots, P, nrm);
    ++p->nlaunch, k_fg_hess<<<B, 32, 0, st>>>(j, p->mk, dots, P, nrm, p->fgH, p->fgc, p->fgs, p->fgg, p->fgh);
    if (j + 1 < m) FG_V4(k_fg_scale, N, p->q, p->fgh, p->fgV + (j + 1) * vs, l.r);
    CKL();
  }
  ++p->nlaunch, k_fg_ysolve<<<(B + 63) / 64, 64, 0, st>>>(B, m, p->mk, p->fgH, p->fgg, p->fgy);
  FG_V4(k_fg_update, N, p->fgZ, vs, m, p->mk, p->fgy, p->x);
#undef FG_V4
  CKL();
  return MPN_OK;
}

// FP64 residual out = rhs_vec - S u (u nullable => 0) where rhs_vec is either
// the forward right-hand side L^T rho b + theta 1_B omega (g_adj null) or
// g_adj; partials of ||out||^2 into `part` (one per tile).
static int residual64(mpn_problem* p, const double* u, const double* g_adj, double* out, double* part,
                      cudaStream_t st) {
  Level& l = p->lv[0];
  Coef cf = make_coef(p, l.fields);
  dim3 gr(nblk(p, l.g.N), p->B);   // partial count per instance = nblk (as every refinement reduction)
  const float* src = g_adj ? nullptr : p->rhs;
  const float* om = g_adj ? nullptr : p->omega;
  if (!u && g_adj) {   // adjoint from zero: the residual is the right-hand side
    ++p->nlaunch, k_copy_norm64<<<gr, MPN_TPB, 0, st>>>(l.g.N, g_adj, out, part);
    CKL();
    return MPN_OK;
  }
  if (p->D == 3 && fp64_layout(p) == FS_MASK_RDI) {
    ++p->nlaunch, k_res64_y<3, FS_MASK_RDI><<<gr, MPN_TPB, 0, st>>>(l.g, cf, p->rho64, u, src, om, p->y64);
    ++p->nlaunch, k_res64_q<3, FS_MASK_RDI><<<gr, MPN_TPB, 0, st>>>(l.g, cf, p->y64, g_adj, om, u, out, part);
  } else if (p->D == 3 && fp64_layout(p) == FS_MASK_RD) {
    ++p->nlaunch, k_res64_y<3, FS_MASK_RD><<<gr, MPN_TPB, 0, st>>>(l.g, cf, p->rho64, u, src, om, p->y64);
    ++p->nlaunch, k_res64_q<3, FS_MASK_RD><<<gr, MPN_TPB, 0, st>>>(l.g, cf, p->y64, g_adj, om, u, out, part);
  } else if (p->D == 3 && fp64_layout(p) == FS_MASK_TR) {
    ++p->nlaunch, k_res64_y<3, FS_MASK_TR><<<gr, MPN_TPB, 0, st>>>(l.g, cf, p->rho64, u, src, om, p->y64);
    ++p->nlaunch, k_res64_q<3, FS_MASK_TR><<<gr, MPN_TPB, 0, st>>>(l.g, cf, p->y64, g_adj, om, u, out, part);
  } else if (p->D == 3) {
    ++p->nlaunch, k_res64_y<3, RES_ANY><<<gr, MPN_TPB, 0, st>>>(l.g, cf, p->rho64, u, src, om, p->y64);
    ++p->nlaunch, k_res64_q<3, RES_ANY><<<gr, MPN_TPB, 0, st>>>(l.g, cf, p->y64, g_adj, om, u, out, part);
  } else {
    ++p->nlaunch, k_res64_y<2, RES_ANY><<<gr, MPN_TPB, 0, st>>>(l.g, cf, p->rho64, u, src, om, p->y64);
    ++p->nlaunch, k_res64_q<2, RES_ANY><<<gr, MPN_TPB, 0, st>>>(l.g, cf, p->y64, g_adj, om, u, out, part);
  }
  CKL();
  return MPN_OK;
}

// The work of one refinement sweep on stream `st`: FP64 residual, inner PCG,
// FP64 update, the sizes the stop rule needs, and their copy to the host.
static int sweep_body(mpn_problem* p, const double* g_adj, int iters, int P, bool from_zero, cudaStream_t st) {
  Level& l = p->lv[0];
  int B = p->B, N = l.g.N;
  dim3 gr(P, B);
  double* scale = p->dscal;
  double* outv = p->dscal + 2 * B;  // [slots][B]
  // from a zero iterate the residual needs no operator apply on u
  TRY(residual64(p, from_zero ? nullptr : p->u64, g_adj, p->r64, slot(p, S_RN), st));
  // CG's first V-cycle runs on this r: its smoother starts here
  const bool cg = p->desc.krylov != MPN_KRYLOV_FGMRES;
  ++p->nlaunch, k_to32<<<gr, MPN_TPB, 0, st>>>(N, p->r64, slot(p, S_RN), P, l.r, scale, cg ? l.dinv : nullptr,
                                                p->cheb_inv_th, l.fs_tt ? l.e2 : l.e, l.fs_tt ? nullptr : l.d);
  CKL();
  if (p->desc.krylov == MPN_KRYLOV_FGMRES) TRY(fgmres(p, iters, st));
  else TRY(pcg(p, iters, st, true));
  ++p->nlaunch, k_update64<<<gr, MPN_TPB, 0, st>>>(N, p->x, scale, p->u64, slot(p, S_DU), slot(p, S_UN));
  // correction and solution sizes measured on every unknown of z
  ++p->nlaunch, k_znorm<<<gr, MPN_TPB, 0, st>>>(l.g, p->u64, p->x, scale, slot(p, S_DU), slot(p, S_UN));
  // slots S_RN, S_DU, S_UN, (S_PW unused), S_GN -> outv
  ++p->nlaunch, k_collect<<<B, 64, 0, st>>>(B, 5, slot(p, S_RN), P, outv);
  CKL();
  CK(cudaMemcpyAsync(p->hbuf, outv, sizeof(double) * 5 * B, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(p->hbuf + 5 * B, p->kerr, sizeof(int), cudaMemcpyDeviceToHost, st));
  return MPN_OK;
}

// One refinement sweep, as a CUDA graph replayed on the problem's internal
// stream (captured on first use for this solve kind, inner-iteration count and
// profiling state).  Ordered after the caller's stream; returns once the
// sweep's scalars are on the host.
static int run_sweep(mpn_problem* p, const double* g_adj, int iters, int P, bool from_zero, cudaStream_t st) {
  TRY(ensure_streams(p));
  int adj = g_adj ? 1 : 0;
  mpn_problem::SweepGraph* g = nullptr;
  for (auto& x : p->graphs)
    if (x.adjoint == adj && x.iters == iters && x.prof == p->prof_on && x.from_zero == from_zero) g = &x;
  if (!g) {
    long long nl0 = p->nlaunch;
    int ev0 = p->prof_next;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(p->gstream, cudaStreamCaptureModeThreadLocal));
    int s = sweep_body(p, g_adj, iters, P, from_zero, p->gstream);
    cudaError_t ec = cudaStreamEndCapture(p->gstream, &graph);
    if (s != MPN_OK) { if (graph) cudaGraphDestroy(graph); return s; }
    CK(ec);
    cudaGraphExec_t exec = nullptr;
    cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(ei);
    p->graphs.push_back({adj, iters, p->prof_on, from_zero, exec, p->nlaunch - nl0, ev0, p->prof_next});
    p->nlaunch = nl0;
    g = &p->graphs.back();
  }
  CK(cudaEventRecord(p->ev_user, st));
  CK(cudaStreamWaitEvent(p->gstream, p->ev_user, 0));
  CK(cudaGraphLaunch(g->exec, p->gstream));
  p->nlaunch += g->kernels;
  CK(cudaStreamSynchronize(p->gstream));
  prof_flush(p, g->ev0, g->ev1);
  return MPN_OK;
}

// Solve S u = rhs (forward: g_adj null; adjoint: the FP64 rhs g_adj) by FP64
// refinement around FP32 MG-PCG.  u64 holds the initial guess on entry.
static int refine_solve(mpn_problem* p, const double* g_adj, bool zero_start, mpn_stats* stats, cudaStream_t st) {
  Level& l = p->lv[0];
  int B = p->B, N = l.g.N;
  int P = nblk(p, N);          // partials per instance of every refinement-level reduction
  std::vector<double> prev_upd(B, 1.0), prev_q(B, 0.0);
  mpn_stats sres;
  memset(&sres, 0, sizeof(sres));
  int status = MPN_ERR_NOT_CONVERGED;
  // the device error word starts clear (or, under injection, set as a kernel
  // whose bounded wait gave up would set it)
  CK(cudaMemsetAsync(p->kerr, p->inject_wait ? 1 : 0, sizeof(int), st));
  p->inject_wait = 0;
  // ||rhs|| for the relative residual: the first residual when starting from 0
  if (!zero_start) TRY(residual64(p, nullptr, g_adj, p->r64, slot(p, S_GN), st));
  // first sweep whose predicted error can end the refinement: from a zero
  // start the first update is the whole solution, so the contraction is
  // measured from the second ratio on (third sweep); from a warm start the
  // first update is already a correction (second sweep)
  const int first = zero_start ? 2 : 1;
  std::vector<double> gnorm(B, 0.0);
  const int base_iters = (g_adj && p->desc.adj_inner_iters > 0) ? p->desc.adj_inner_iters : p->desc.inner_iters;
  int iters = p->desc.direct ? 1 : base_iters, total_iters = 0;
  const bool trace = getenv("MPN_TRACE") != nullptr;
  for (int sweep = 0; sweep < p->desc.max_refine; ++sweep) {
    TRY(run_sweep(p, g_adj, iters, P, zero_start && sweep == 0, st));
    total_iters += iters;
    const double* h = p->hbuf;
    if (*(const int*)(h + 5 * B)) {   // a kernel's bounded wait gave up
      snprintf(g_cuda_err, sizeof(g_cuda_err), "a kernel's bounded wait for its asynchronous copies gave up");
      status = MPN_ERR_CUDA;
      break;
    }
    double maxpred = 0, maxupd = 0, maxres = 0, maxrate = 0, maxq = 0;
    bool bad = false, grew = false;
    for (int b = 0; b < B; ++b) {
      double rn = sqrt(h[0 * B + b]), du = sqrt(h[1 * B + b]), un = sqrt(h[2 * B + b]);
      if (sweep == 0) gnorm[b] = zero_start ? rn : sqrt(h[4 * B + b]);
      if (!std::isfinite(rn) || !std::isfinite(du) || !std::isfinite(un)) bad = true;
      double upd = un > 0 ? du / un : (du > 0 ? 1.0 : 0.0);
      // the first update is the whole solution; contraction is measured from
      // sweep 2 on, as the larger of the last two update ratios (a single
      // lucky sweep of an erratic inner solve does not end the refinement),
      // and the remaining error is the geometric tail of the next
      // corrections: upd (q + q^2 + ...) = upd q / (1 - q)
      const double q1 = upd / std::max(prev_upd[b], 1e-300);
      if (sweep >= 1) maxq = std::max(maxq, q1);
      const double q = sweep >= 1 ? std::max(q1, prev_q[b]) : q1;
      if (sweep >= 1) prev_q[b] = q1;
      double pred = sweep < first ? upd : (q < 1.0 ? upd * q / (1.0 - q) : HUGE_VAL);
      if (sweep >= 2 && upd > 10.0 * prev_upd[b] && upd > 1e-3) grew = true;
      if (sweep >= 2) maxrate = std::max(maxrate, upd / std::max(prev_upd[b], 1e-300));
      prev_upd[b] = upd;
      maxpred = std::max(maxpred, pred);
      maxupd = std::max(maxupd, upd);
      maxres = std::max(maxres, gnorm[b] > 0 ? rn / gnorm[b] : 0.0);
    }
    sres.sweeps = sweep + 1;
    sres.pcg_iters = total_iters;
    sres.rel_update = maxupd;
    sres.pred_error = maxpred;
    sres.rel_residual = maxres;
    if (bad) { status = MPN_ERR_NONFINITE; break; }
    if (grew) { status = MPN_ERR_DIVERGED; break; }
    if ((sweep >= first && maxpred <= p->desc.tol) || (sweep >= 1 && maxupd <= p->desc.tol * 0.1)) { status = MPN_OK; break; }
    const int done_iters = iters;
    // a sweep that gained less than a digit: lengthen the inner solve
    if (!p->desc.direct && sweep >= 1 && maxrate > 0.1 && iters < 8 * base_iters) iters *= 2;
    if (trace)
      fprintf(stderr, "[mpn] %s sweep %d: %d inner iterations, update %.3e, residual %.3e, predicted error %.3e, "
                      "gain %.3e -> next %d\n", g_adj ? "adjoint" : "forward", sweep, done_iters, maxupd, maxres,
              maxpred, maxq, iters);
  }
  if (stats) *stats = sres;
  return status;
}

static int check_ptrs(const void* a, const void* b) { return (a && b) ? MPN_OK : MPN_ERR_INVALID_ARG; }

static int forward_impl(mpn_problem* p, const float* fields, const float* scalars, const float* rhs,
                        const float* omega, const float* u0, float* z, double* z64, mpn_stats* stats,
                        cudaStream_t st) {
  Level& l = p->lv[0];
  int B = p->B;
  size_t N0 = (size_t)l.g.N * B;
  TRY(setup(p, fields, scalars, st));
  CK(cudaMemcpyAsync(p->rhs, rhs, sizeof(float) * N0, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(p->omega, omega, sizeof(float) * N0, cudaMemcpyDeviceToDevice, st));
  dim3 gr(nblk(p, l.g.N), B);
  ++p->nlaunch, k_set_u<<<gr, MPN_TPB, 0, st>>>(l.g.N, u0, p->u64);
  CKL();
  p->zd_valid = false;
  int status = refine_solve(p, nullptr, u0 == nullptr, stats, st);
  if (status != MPN_OK && status != MPN_ERR_NOT_CONVERGED) return status;
  Coef cf = make_coef(p, l.fields);
  if (p->D == 3 && fp64_layout(p) == FS_MASK_RDI)
    ++p->nlaunch, k_recover<3, FS_MASK_RDI><<<gr, MPN_TPB, 0, st>>>(l.g, cf, p->rho64, p->u64, p->rhs, p->omega, nullptr, z, z64);
  else if (p->D == 3 && fp64_layout(p) == FS_MASK_RD)
    ++p->nlaunch, k_recover<3, FS_MASK_RD><<<gr, MPN_TPB, 0, st>>>(l.g, cf, p->rho64, p->u64, p->rhs, p->omega, nullptr, z, z64);
  else if (p->D == 3 && fp64_layout(p) == FS_MASK_TR)
    ++p->nlaunch, k_recover<3, FS_MASK_TR><<<gr, MPN_TPB, 0, st>>>(l.g, cf, p->rho64, p->u64, p->rhs, p->omega, nullptr, z, z64);
  else if (p->D == 3)
    ++p->nlaunch, k_recover<3, RES_ANY><<<gr, MPN_TPB, 0, st>>>(l.g, cf, p->rho64, p->u64, p->rhs, p->omega, nullptr, z, z64);
  else
    ++p->nlaunch, k_recover<2, RES_ANY><<<gr, MPN_TPB, 0, st>>>(l.g, cf, p->rho64, p->u64, p->rhs, p->omega, nullptr, z, z64);
  CKL();
  CK(cudaMemcpyAsync(p->uf64, p->u64, sizeof(double) * N0, cudaMemcpyDeviceToDevice, st));
  p->zd_valid = true;
  ++p->gen;
  p->fwd_in[0] = fields; p->fwd_in[1] = scalars; p->fwd_in[2] = rhs; p->fwd_in[3] = omega;
  CK(cudaStreamSynchronize(st));
  return status;
}

extern "C" int mpn_forward(mpn_problem* p, const float* fields, const float* scalars, const float* rhs,
                           const float* omega, const float* u0, float* z, double* z64, mpn_stats* stats,
                           void* stream) {
  if (!p || (p->desc.variable_steps && !p->steps_set)) return MPN_ERR_INVALID_ARG;
  TRY(check_ptrs(scalars, rhs));
  if (!omega || (!z && !z64)) return MPN_ERR_INVALID_ARG;
  if (p->F > 0 && !fields) return MPN_ERR_INVALID_ARG;
  return forward_impl(p, fields, scalars, rhs, omega, u0, z, z64, stats, (cudaStream_t)stream);
}

extern "C" int mpn_adjoint(mpn_problem* p, const float* fields, const float* scalars, const float* rhs,
                           const float* omega, const float* z, const float* g_z, float* dfields, float* dscalars,
                           float* drhs, float* domega, float* dz, double* dz64, int flags, mpn_stats* stats,
                           void* stream) {
  if (!p || (p->desc.variable_steps && !p->steps_set)) return MPN_ERR_INVALID_ARG;
  TRY(check_ptrs(scalars, rhs));
  TRY(check_ptrs(omega, g_z));
  TRY(check_ptrs(dscalars, drhs));
  if (!domega) return MPN_ERR_INVALID_ARG;
  if (p->F > 0 && (!fields || !dfields)) return MPN_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  Level& l = p->lv[0];
  int B = p->B, V = p->V;
  dim3 gr(nblk(p, l.g.N), B);
  (void)z;
  // the kept forward state serves only the buffers that forward read
  const bool same_inputs = p->fwd_in[0] == (const void*)fields && p->fwd_in[1] == (const void*)scalars &&
                           p->fwd_in[2] == (const void*)rhs && p->fwd_in[3] == (const void*)omega;
  if (!((flags & MPN_REUSE_SETUP) && p->setup_ok && p->zd_valid && same_inputs)) {
    // no kept forward state for these data: recompute the forward solution
    int s = forward_impl(p, fields, scalars, rhs, omega, nullptr, nullptr, nullptr, nullptr, st);
    if (s != MPN_OK && s != MPN_ERR_NOT_CONVERGED) return s;
  }
  Coef cf = make_coef(p, l.fields);
  // reduced right-hand side g_u - M_{u zeta} M_{zeta zeta}^{-1} g_zeta (FP64)
  if (p->D == 3) {
    if (fp64_layout(p) == FS_MASK_RDI) ++p->nlaunch, k_adj_kappa<3, FS_MASK_RDI><<<gr, MPN_TPB, 0, st>>>(l.g, cf, g_z, p->kap);
    else if (fp64_layout(p) == FS_MASK_RD) ++p->nlaunch, k_adj_kappa<3, FS_MASK_RD><<<gr, MPN_TPB, 0, st>>>(l.g, cf, g_z, p->kap);
    else if (fp64_layout(p) == FS_MASK_TR) ++p->nlaunch, k_adj_kappa<3, FS_MASK_TR><<<gr, MPN_TPB, 0, st>>>(l.g, cf, g_z, p->kap);
    else ++p->nlaunch, k_adj_kappa<3, RES_ANY><<<gr, MPN_TPB, 0, st>>>(l.g, cf, g_z, p->kap);
    ++p->nlaunch, k_adj_rhs<3><<<gr, MPN_TPB, 0, st>>>(l.g, g_z, p->kap, p->g64);
  } else {
    ++p->nlaunch, k_adj_kappa<2, RES_ANY><<<gr, MPN_TPB, 0, st>>>(l.g, cf, g_z, p->kap);
    ++p->nlaunch, k_adj_rhs<2><<<gr, MPN_TPB, 0, st>>>(l.g, g_z, p->kap, p->g64);
  }
  ++p->nlaunch, k_set_u<<<gr, MPN_TPB, 0, st>>>(l.g.N, nullptr, p->u64);
  CKL();
  int status = refine_solve(p, p->g64, true, stats, st);
  if (status != MPN_OK && status != MPN_ERR_NOT_CONVERGED) return status;
  double* gp = slot(p, S_GR0);
#define GRAD_LAUNCH(DD, MK)                                                                              \
  ++p->nlaunch, k_gradients<DD, MK><<<gr, MPN_TPB, 0, st>>>(l.g, cf, p->rho64, p->rhs, p->omega, p->uf64, p->u64, g_z, dfields, \
                                                           drhs, domega, dz, dz64, gp)
  if (p->D == 3 && fp64_layout(p) == FS_MASK_RDI) GRAD_LAUNCH(3, FS_MASK_RDI);
  else if (p->D == 3 && fp64_layout(p) == FS_MASK_RD) GRAD_LAUNCH(3, FS_MASK_RD);
  else if (p->D == 3 && fp64_layout(p) == FS_MASK_TR) GRAD_LAUNCH(3, FS_MASK_TR);
  else if (p->D == 3) GRAD_LAUNCH(3, RES_ANY);
  else GRAD_LAUNCH(2, RES_ANY);
#undef GRAD_LAUNCH
  ++p->nlaunch, k_scalar_grads<<<B, 64, 0, st>>>(V, B, p->field_of_dev, gp, gr.x, dscalars);
  CKL();
  CK(cudaStreamSynchronize(st));
  return status;
}

extern "C" int mpn_set_steps(mpn_problem* p, const float* steps, void* stream) {
  if (!p || !steps || !p->desc.variable_steps) return MPN_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  // the kept setup and forward state belong to the old steps
  p->steps_set = false;
  p->setup_ok = false;
  p->zd_valid = false;
  const int nrec = p->B * 3 * p->stn;
  CK(cudaMemsetAsync(p->sterr, 0, sizeof(int), st));
  ++p->nlaunch, k_steps_in<<<(nrec + 127) / 128, 128, 0, st>>>(p->lv[0].g, steps, p->hlev, p->B, p->sterr);
  CKL();
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, p->sterr, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (bad) return MPN_ERR_INVALID_ARG;
  p->steps_set = true;
  return MPN_OK;
}

extern "C" int mpn_step_grads(mpn_problem* p, const double* z64, const double* dz64, float* dsteps, void* stream) {
  if (!p || !z64 || !dz64 || !dsteps || !p->desc.variable_steps || !p->steps_set) return MPN_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  ++p->nlaunch, k_step_grads<<<dim3(p->stn, p->D, p->B), MPN_TPB, 0, st>>>(p->lv[0].g, p->hlev, z64, dz64, dsteps, p->B);
  CKL();
  return MPN_OK;
}

extern "C" int mpn_debug_take(mpn_problem* p, int* code) {
  if (!p || !code) return MPN_ERR_INVALID_ARG;
#ifdef MPN_DEBUG
  CK(cudaDeviceSynchronize());
  int v = 0;
  CK(cudaMemcpy(&v, p->dbg, sizeof(int), cudaMemcpyDeviceToHost));
  if (v) CK(cudaMemset(p->dbg, 0, sizeof(int)));
  *code = v;
  return MPN_OK;
#else
  *code = 0;
  return MPN_ERR_UNSUPPORTED;
#endif
}

extern "C" long long mpn_generation(const mpn_problem* p) { return p ? p->gen : -1; }

extern "C" int mpn_inject_wait_failure(mpn_problem* p) {
  if (!p) return MPN_ERR_INVALID_ARG;
  p->inject_wait = 1;
  return MPN_OK;
}

extern "C" int mpn_mse_grad(mpn_problem* p, const float* z, const float* target, float* g_z, void* stream) {
  if (!p || !z || !target || !g_z) return MPN_ERR_INVALID_ARG;
  Level& l = p->lv[0];
  ++p->nlaunch, k_mse_grad<<<dim3(nblk(p, l.g.N), p->B), MPN_TPB, 0, (cudaStream_t)stream>>>(l.g.N, p->V, p->B, z, target, g_z);
  CKL();
  return MPN_OK;
}

extern "C" int mpn_apply_reduced(mpn_problem* p, const float* fields, const float* scalars, const float* u, float* q,
                                 void* stream) {
  if (!p || !scalars || !u || !q) return MPN_ERR_INVALID_ARG;
  // u and q go to the operator kernels as they are, and those read and write
  // float4 groups: 16-byte alignment is checked here, before p is touched
  if (((uintptr_t)u | (uintptr_t)q) & 15) return MPN_ERR_INVALID_ARG;
  if (p->F > 0 && !fields) return MPN_ERR_INVALID_ARG;
  if (p->desc.variable_steps && !p->steps_set) return MPN_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  TRY(setup(p, fields, scalars, st));
  TRY(apply_S(p, 0, u, q, nullptr, st));
  CK(cudaStreamSynchronize(st));
  return MPN_OK;
}

extern "C" int mpn_profile(mpn_problem* p, int enable, double* ms_total, long long* launches, double* bytes,
                           long long* kernels) {
  if (!p) return MPN_ERR_INVALID_ARG;
  if (ms_total) *ms_total = p->prof_ms;
  if (launches) *launches = p->prof_n;
  if (bytes) *bytes = p->prof_bytes;
  if (kernels) *kernels = p->nlaunch;
  if (enable >= 0) {
    if (enable && p->prof_ev.empty()) {
      p->prof_ev.resize(2 * PROF_PAIRS);
      for (auto& e : p->prof_ev) CK(cudaEventCreate(&e));
    }
    p->prof_on = enable;
    p->prof_ms = 0; p->prof_n = 0; p->prof_bytes = 0;
    p->nlaunch = 0;
  }
  return MPN_OK;
}
