"""CPU oracle for the spectral hyper-viscosity Navier-Stokes solver.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement
of what the paper defines (Rohner & Mishra, "Efficient Computation of
Large-Scale Statistical Solutions to Incompressible Fluid Flows", PASC'24):
the spectral hyper-viscosity discretisation (eq. shv_disc, section 2.2), the
Fourier-space evolution with the pressure eliminated (section 2.3), Algorithm 2
(pad, inverse transform, product, forward transform, remove the upper third,
time derivative), the SSP-RK3 integrator (section 2.3) and the writers'
statistics (section 2.4).  It shares no code with the CUDA library and never
imports it.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.

Modules
-------
fft      own mixed-radix FFT (radix 2, 3, 5, 7, direct DFT otherwise)
solver   parameters, wavenumbers, dissipation, padded transforms, RHS in three
         equivalent nonlinear forms, Leray projection, SSP-RK3, CFL time step
stats    ensemble statistics (mean, second moments, energy spectrum, second
         order structure function, Monte Carlo standard errors, Chan merge)
adjoint  tangent-linear RHS, its adjoint, the discrete adjoint of one RK3 step
         and the band-energy gradient with checkpoint/recompute (not in the
         paper; built on its RHS and RK3)

Parity pins for every function live in ``tests/test_oracle_*.py``.  The
paper fixes no prefactors for m_N and eps_N: "matches the paper's constants"
is parity unpinned (both sides take the same parameters).
"""
