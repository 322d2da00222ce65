"""Plain, slow FP64 CPU oracle for the scaled-stencil P1 operators of
Drzisga, Ruede, Wohlmuth, "Stencil scaling for vector-valued PDEs on hybrid
grids with applications to generalized Newtonian fluids" (arXiv 1908.08666).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library: it refines the macro mesh by its own recursive
red refinement (Bey's rule), integrates every element's local stiffness by
quadrature, and builds each operator from its definition in the paper:

* nodal integration a_h .......................... Sec. 2, eq. (nodalintegration)
* physical scaling  \\hat a_h (patch mean, reflected elements, correction R)
                                                   Sec. 2, Lemma 2.1, eqs. (patchmean),
                                                   (corrtermgeneral)
* unphysical scaling \\tilde a_h .................. Sec. 2, eq. (stencilscalingwithoutcorr)
* interface rows (symmetric / practical) ......... Sec. 2.2, the two interface definitions
* Stokes blocks B, B^T and the stabilisation C ... Sec. 5.2, stabilised P1-P1
* nodal strain-rate least squares and Carreau ..... Sec. 3, eq. (minimization_problem);
                                                   Sec. 5.2.2, eq. (carreau)
* inexact Uzawa multigrid for the saddle system .... Sec. 5.2 (the library's variant, step
                                                   by step)
* learned preconditioner (not in the paper) ...... its conv net, features, training pairs
                                                   and combination rule

Modules: ``mesh`` (refinement, node classification, transfer parents),
``fem`` (quadrature and element matrices), ``operators`` (global sparse
operators), ``rows`` (one operator row at any level by local refinement),
``solvers`` (Dirichlet handling, PCG, Chebyshev, V-cycle, MINRES, iterative
refinement), ``stokes`` (saddle operator, inexact Uzawa multigrid), ``carreau``,
``learned``.
"""
