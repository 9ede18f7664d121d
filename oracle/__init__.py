"""CPU FP64 oracle for the lattice SIGW hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library (no kernels, headers, tables or helpers); the two
sides meet only through the parameter sets in ``workloads.py``, which hold none
of the method's arithmetic.

Every function follows a passage of the paper (arXiv 2605.27231, "A Fast Method
to Compute Scalar Induced Gravitational Waves on a Lattice with Primordial
Non-Gaussianities") and cites it by section / equation label.  The code is a
plain, slow restatement: library FFTs and ``numpy.linalg.eigh`` are used as
steps, with no blocking, fusion or reordering beyond what the definitions say.

Modules
-------
philox          Philox4x32-10 counter-based generator (Salmon et al., SC'11)
kernels         analytic time-integral kernels I_s, I_c (Eq. eq_kernels)
decomposition   u-grid (Eq. eq_grid_density), C matrix (Eq. eq_C_matrix_discrete),
                eigen-truncation (Eq. eq_diagonalization)
synth           Gaussian curvature field, non-Gaussian maps, Phi = 2 zeta / 3
sigw            FFT-convolution envelopes (Eq. eq_final_envelopes), TT projection,
                shell binning and Omega_GW (Sec. sec_envelope_obs)
brute           direct O(N^6) lattice sum (Eqs. eq_naive_A / eq_naive_B)
wick            exact Gaussian expectation of the lattice estimator
semi_analytic   Gaussian Omega_GW quadrature (Eq. eq_semi_anal)
"""
