"""Plain FP64 CPU oracle for BDDC-SO (Badia, Martin, Nguyen, arXiv 2001.07289).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the tests, the smoke check and the bench's CPU-baseline / reference leg
do.  It shares no code with the CUDA library; both sides read their inputs
from paper_2001_07289_gb300.inputs, which holds no method arithmetic.

The oracle is written from the paper's definitions, slow and direct:

  fem.py        Q1 element matrix (tensor-product definition), global
                assembly, load vector (Section 2, eq. weakform; Remark 1).
  partition.py  the partition Theta and the sub-partition Theta-hat
                (Section 3, first two paragraphs and the remark on local
                subdivision).
  objects.py    classification of interface DOFs into (sub)objects by the set
                of sub-subdomains containing them, selection vef / ve / f
                (Section 3; Table 1 variants).
  multilevel.py the second level of multilevel BDDC-SO (BDDC on the coarse
                problem, Section 6).
  paths.py      the acceptable-path check of a selection (remark after
                Theorem 1).
  weights.py    the weighting E of eq. (W) and the rho-weighting of Remark 1.
  bddc.py       the multispace BDDC preconditioner of Definition 1 with
                V1 = U_I, Q1 = I, V2 = W-tilde, Q2 = (I - P)E (Section 3, last
                paragraph), solved on W-tilde directly as a constrained
                problem; the local coarse basis by its energy-minimisation
                definition; PCG stopped on the 2-norm residual reduction
                (Section 5); Lanczos eigenvalue estimates; adjoint gradient.

Pins (tests/test_oracle_*.py, run with -m "not gpu"): closed-form element
matrix and stencil, quadrature route to the element matrix, sparse direct
solves, O(h^2) convergence to a manufactured solution, Table 1 coarse sizes,
the Figure 1 weight 2/3, partition of unity, C_i Phi_i = I, Phi_i 1 = 1,
symmetry of B, B = A^{-1} when every interface DOF is primal, lambda_min >= 1,
the Euler identity of the gradient and finite differences.
"""
