"""FP64 CPU oracle for the space-time GW hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct numpy code that writes out the definitions of
Liu, Kaltak, Klimes and Kresse, "Cubic scaling GW" (arXiv:1607.02859) on the
same discretisation the GPU path uses.  Only the tests, the smoke check and the
CPU-baseline leg of the benchmark may import it; the product path never does.
It shares no code with the CUDA library: its only common dependency is the
seeded input generator ``paper_1607_02859_gb300.inputs``.

Modules (each function cites the passage it follows):
  grids   -- CT/ST weights (Eqs. CT_FFT, cos_error_function, ST_FFT,
             sin_error_function, INV_CT_FFT)
  gvec    -- G set, FFT index map, Coulomb kernel (Eq. bareV)
  green   -- G_occ, G_unocc (Eqs. Green_occ, Green_unocc)
  chi     -- chi(r,r',tau) (Eqs. chi_GG, chi_rr), spatial transform (Eqs.
             FFTX1, FFTX2), the pair route (Eq. CHI_g_it), CT (Eq. CTX)
  screen  -- W~ (Eqs. W_tot, bareV, die, W_correlated), inverse CT (Eq. CT_W),
             W~(r,r') (Eq. FFTW)
  sigma   -- Sigma_nn(tau) (Eqs. Sigma_occ, Sigma_rr, Sigma_occ_reduce first
             term), even/odd split and CT+ST (Eqs. cos_sin_sigma*,
             sigma_r_w), pair route; the full matrix Sigma_nm by both routes
  thiele  -- Thiele reciprocal differences (Eqs. pade1, pade2) and the
             derivative of the continued fraction
  qp      -- linearised QP energies and spectral functions (Eqs. QP, GWQP,
             Z, A)
  pipeline-- the chain chi0(i omega) -> W~ -> Sigma_nn(i omega) -> Sigma_nn(omega)

Parity pins live in tests/test_oracle_*.py.  No function here is "parity
unpinned" except where its docstring says so.
"""
