"""CPU FP64 oracle for the NeuRLP-PDE least-squares solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package;
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may call it.  It shares no code with the CUDA path: it assembles
the sparse constraint matrix A and vector d row by row as Section 3 of the
paper defines them (Eqs. 3-8), solves the least-squares problem exactly through
the saddle-point system of Eq. 10 with a sparse LU factorisation, and computes
parameter gradients from the saddle-point system of Eq. 11 and the gradient
formulas that follow it.

Modules
  assemble      rows of A and d (Eqs. 3-8), boundary set, row counts
  solve         least-squares solve via Eq. 10 (and via Eq. 9 as a cross-check)
  grad          adjoint solve (Eq. 11) and dL/dc, dL/db, dL/domega
  manufactured  data whose least-squares solution is known exactly at any grid
                size (consistent equation and boundary data for any u; adjoint
                sources on u with their exact solution), for full-size checks
  conv          the warm-start network's 3x3x3 convolution, written plainly
  nonuniform    per-interval steps (three-point forms through unequal
                intervals), Neumann / mixed boundary rows, dl/dsteps through
                the entries of A
"""
