"""CPU oracle for the posterior-mean system of the CMB source-separation model (FP64).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import or run anything here; the solver library never does and shares no
code with it.

What it computes (all in float64, unknowns stored as X with shape (k, n), so that
``X.reshape(-1)`` is the column-stacked vec(X) of the n x k matrix of Sec. 3.1):

* ``model``: power-law mixing a_cj = (nu_c / 100)^beta_j; the graph Laplacian rebuilt from
  the grid definition; prior blocks Q_j = tau_j (kappa_j^2 W + L) (the SPD Matern-type form of
  the Gaussian-field prior of Sec. 2.1 / App. C); the assembled Kronecker-sum matrix
  G = sum_j (e_j e_j^T) kron Q_j + sum_c (a_c a_c^T) kron D_c, which is Q + B^T C B of
  eq. Q* with C generalised to per-channel per-pixel maps; the right-hand side
  b = vec(sum_c D_c y_c a_c^T) = B^T C Y of eq. mu*; a matrix-free apply following the block
  mapping of eq. block-vector-mapping-matvec.
* ``solve``: sparse direct and dense solves of G x = b; textbook CG (Algorithm 2) and the same
  CG with a pixel-block Jacobi preconditioner.
* ``closed_form``: exact solutions of special cases that do not use the assembled matrix
  (Fourier-diagonalised lattice, latitude-only noise on the sphere, the Sylvester form
  eq. Axb-Sylv, the scalar case).
* ``gradient``: derivatives of a loss on the posterior mean with respect to tau_j, kappa_j and
  beta_j through one adjoint solve, and central finite differences of the direct solve.
* ``physical_mixing``: the physical mixing matrix of App. B (CMB, synchrotron, dust, free-free).
* ``variance``: the posterior variances diag(G^{-1}) (exact, and the probe estimator of Bekas,
  Kokiopoulou and Saad), with the lattice closed form.
* ``sylvester``: the block-Lanczos solver of the Sylvester form eq. Axb-Sylv for separable noise
  and a common prior shape (Algorithms 4 and 5, Sec. 3.3).
"""
