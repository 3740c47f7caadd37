// Arguments and modes of one operator step (y = -rho L x, then L^T y and a
// mode-specific update), shared by the two-pass kernels and the fused step.
#pragma once

enum { SM_POST0 = 0, SM_CHEB = 1, SM_RES = 2, SM_APPLY = 3,
       SM_CHEB_DOT = 4,     // fused step only: a Chebyshev step that also sums <e', r>
       SM_APPLYP = 5 };     // fused step only: apply to p = x + beta d, p also written to e

struct StepArgs {
  const float* x;     // operand of S (pass 1 and the theta 1_B term)
  const float* y;     // pass-1 output
  const float* r;     // right-hand side at this level
  const float* dinv;  // Chebyshev-scaled inverse diagonal
  float* e;           // iterate (modes 0, 1: updated in place; it is x; fused step: the new iterate)
  float* d;           // direction (modes 0, 1); fused step, modes 1, 4: the previous iterate (null = 0),
                      // which may be the buffer e writes: each point is read once, by the thread that
                      // owns it, before that thread stores the new iterate there
  float* out;         // mode 2: r - S x;  mode 3: S x
  double* part;       // mode 3: partials of <x, S x>; mode 4: of <e', r> (nullable)
  int* err;           // set when a bounded wait gives up (fused step; nullable)
  float c1, c2;
  // mode 5: beta = sum(rz partials, nrz of them) / rz_old[b] (0 when d is null);
  // rz_tot (nullable): the finished sums of those partials, read instead
  const double* rz;
  const double* rz_old;
  int nrz;
  const double* rz_tot;
  // fused step: with cnt set, the last CTA of an instance also sums the
  // partials it wrote (part) into tot[b] (counter cnt[b], reset after use)
  int* cnt;
  double* tot;
};

