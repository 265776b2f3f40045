"""FP64 CPU oracle for the hp space-time multigrid of arXiv 2502.09159.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may import this package.  The product path
(paper_2502_09159_gb300) never imports it and shares no code with it.

A plain, slow, obviously correct restatement of what the method computes, written
from the paper's definitions:

* fe.py      - quadrature rules, 1D Lagrange/Legendre bases, temporal matrices
               K, M, C (Eq. DefKMC), spatial matrices M_h, A_h, B_h (Eq. DefMAB)
               assembled from element matrices computed by full d-dimensional
               Gauss quadrature.
* stokes.py  - slab operator (Eq. InAlg / DefDtauh), right-hand side (Eq. DefFn),
               slab coupling (Eq. AlgSysTMS), transfer operators (App. A),
               hierarchy (Alg. 2/3), Vanka smoothers (Eq. vanka0, vanka), the
               V-cycle (Alg. 1, App. B), FGMRES, time marching, error norms.
* warmstart.py - cell tensors of slab vectors, temporal extrapolation of the DG(k)
               polynomial, and the convolutional network of the learned initial
               guess (forward, backward, loss, Adam); no counterpart in the paper.

Everything is float64 (numpy / scipy.sparse).  Functions whose result has no pin
independent of the oracle itself say "parity unpinned" in their docstring.
"""
