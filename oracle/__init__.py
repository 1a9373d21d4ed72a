"""CPU oracle for the HPS skeleton solver -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 / complex128 restatement of the method of
"Towards a Multigrid Preconditioner Interpretation of Hierarchical
Poincare-Steklov Solvers" (arXiv 2511.00735), written from the paper's
equations, in the paper's order and notation.  Only `tests/`, the smoke check
in `__graft_entry__.py` and the CPU-baseline leg of `bench.py` may import it.
The CUDA library shares no code with it and never calls it.

Modules
  gll       1D Gauss-Lobatto-Legendre rule, D, M, K           (section 3.1)
  leaf      element operator L, impedance operators, T and H  (section 3.1, eq. ItIOperator)
  skeleton  mesh, faces, dense skeleton system M g = RHS      (section 3.2, eqs. localiti, faceequations)
  hps       pair merges, nested dissection, direct HPS,
            multigrid preconditioner MG(M)                    (section 4, eqs. localfacesystem,
                                                               globalfacesystem, block-inverse identity)
  krylov    GMRES with a fixed number of steps, flexible GMRES (section 4.3)

Readings of the paper that the text leaves open or prints garbled are listed
in each function's docstring (sign of the c-term, the missing i in the
impedance operators, the transmission sign, the T_pair/H_pair signs).

Parity status of each function is stated in its docstring; every function
here is pinned by a `-m "not gpu"` test in tests/test_oracle_*.py except the
iteration counts of the multigrid-preconditioned FGMRES, which the paper only
reports for a problem whose wavenumber and mesh it does not state
(parity unpinned in absolute terms; only the monotone trends of Table 1 are
checked).
"""
