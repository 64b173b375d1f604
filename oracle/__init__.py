"""CPU oracle for the NFFT-based fast summation of the graph Laplacian.

This package is TEST INFRASTRUCTURE.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import, call, link or run anything in it.  The
product path (``paper_1808_04580_gb300``) never touches it, and this package
never imports the product path: the two share no code.

Everything here is plain, slow and written to be checked against the paper
by eye (Alfke, Potts, Stoll, Volkmer, "NFFT meets Krylov methods", 2018):

* ``direct``   -- O1, the ground truth: dense FP64 sums with the Gaussian
                  weights of Sec. 2, eq. (W_gaussian), zero diagonal; the degree
                  vector, ``A = D^{-1/2} W D^{-1/2}`` and ``L_s = I - A``
                  (Sec. 2, eq. (nomlap)).  A plain-C twin (``direct.c``) sums
                  selected rows over all sources for large n.
* ``kernel``   -- the Gaussian, its regularization ``K_R`` (Sec. 3) and the
                  trapezoidal-rule Fourier coefficients ``b_l`` (Sec. 3,
                  eq. (b_l::K_RF)).
* ``nfft``     -- Kaiser-Bessel window, adjoint NFFT and NFFT with
                  oversampling 2, plus the direct NDFT sums they approximate.
* ``fastsum``  -- O2 (exact trigonometric-polynomial sum, eq. (K_RF)) and
                  O3 (Alg. 1 and Alg. 2 step by step).
* ``spectral`` -- O4/O5: dense symmetric eigendecomposition and dense solves
                  for the Lanczos (Sec. 4) and CG (Sec. 6.2.2, eq.
                  (ssl::system)) checks.
* ``apps``     -- the consumers of the eigenpairs in Sec. 6.2: spectral
                  clustering (k-means on normalized eigenvector rows) and
                  phase-field SSL (the Allen-Cahn convexity-splitting step).

Parity status of each function is stated in its module docstring.
"""
