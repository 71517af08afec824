"""CPU FP64 oracle for the fractional SEM system (TEST INFRASTRUCTURE ONLY).

Plain, slow, obviously correct numpy code that computes what the solver
computes, written from the paper (Li, Mao, Song, Wang, Karniadakis,
"A fast solver for spectral element approximation applied to fractional
differential equations using hierarchical matrix approximation"):

  basis.py      Legendre recurrence, bubble/hat basis, mesh (Sec. 2.2)
  quadrature.py Gauss-Legendre / Gauss-Jacobi rules (Golub-Welsch)
  assemble.py   dense stiffness S_l, S_r, mass M, A = rho M + S (eq. (lsys))
  load.py       load vector G
  solve.py      exact discrete solution X* = A^{-1} G (dense LU + refinement)
  hmatrix.py    cluster/block tree, admissibility (eq. (admis)), Taylor
                low-rank blocks (eq. (eqn:Lexpan), Sec. 3.2), dense H-matrix
                approximation A~ (eq. (approxsys))

Only the tests, __graft_entry__.smoke() and bench.py's cpu_baseline /
reference arm may import this package.  It shares no code with the CUDA
library and never imports it; the library never calls back into it.
"""
