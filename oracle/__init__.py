"""Plain FP64 CPU oracle for the matrix-free H(div) saddle-point solver.

TEST INFRASTRUCTURE ONLY. Nothing in the product path (the CUDA library and its
Python binding) may import, call or link anything in this package; only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.

Everything here is written from the paper (Pazner, Kolev, Vassilevski,
"Matrix-free GPU-accelerated saddle-point solvers for high-order problems in
H(div)", arXiv 2304.12387) as plainly as possible: element matrices by full
Gauss-Legendre quadrature, global matrices assembled as scipy CSR, the L2 mass
inverse by dense per-element inverses, the approximate Schur complement by its
defining sparse product, and MINRES in FP64. It shares no code with the CUDA path.

Modules
  basis1d   1D Gauss-Lobatto / Gauss-Legendre points, Lagrange interpolation and
            histopolation bases (Sec. 2.1).
  lattice   global numbering of the refined (subcell) lattice, the 24 element
            rotations, the signed element-to-dof maps, essential dofs and the
            divergence by Algorithm 1.
  element   reference RT/L2 bases, trilinear geometry, Piola maps and element
            matrices M_e, W_e, B_e by full quadrature (Eq. matrices).
  assembly  global CSR M, D, W^{-1}; the transformed block operator (Eq.
            transformed-system and its Darcy form).
  precond   diag(M), diag(W), the approximate Schur complement (Eq. approx-schur)
            and the geometric V-cycle spec that stands in for AMG.
  minres    preconditioned MINRES (Paige & Saunders 1975) in FP64.
  gmres     restarted right-preconditioned GMRES (Saad & Schultz 1986) for the
            block-triangular preconditioner of the remark in Sec. 2.3.
  conditioning  condition numbers on single elements: the diagonally scaled L2 mass
            in three bases (Sec. 2.5) and the transformed versus the untransformed
            Schur complement.
  sampled   single rows of the block operator at any mesh size (element-local).
  conv      reference 3D convolution forward/backward for the learned Schur
            preconditioner.
"""
