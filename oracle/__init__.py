"""FP64 CPU oracle for the adjoint particle-mesh method (arXiv:2211.09815).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The CUDA library in ``paper_2211_09815_gb300`` never imports, links or calls anything
here, and nothing here imports that package: the two share no code.  Inputs (the
white-noise field and the cosmological parameters) are passed in as arrays.

The oracle is a plain, slow, obviously correct restatement of the paper in float64:

* ``oracle.cosmo`` -- linear power spectrum (Sec. 2.1, Eq. 7), Eisenstein & Hu no-wiggle
  transfer function, growth ODE (App. A, Eqs. 52-58) and the FastPM drift/kick factors
  (Sec. 2.3, Eqs. 13-15).
* ``oracle.pm`` -- Zel'dovich initial conditions (Sec. 2.1, Eqs. 2-6), CIC scatter and
  gather (Sec. 2.2, Eq. 10), the FFT Poisson force (Sec. 2.2, Eq. 11), the
  kick-drift-kick leapfrog (Sec. 2.3, Eq. 16), the density MSE objective (Sec. 2.4,
  Eq. 17) and the discrete adjoint with reverse time integration (Sec. 3.6,
  Eqs. 49-51).

Library primitives used as single steps: ``numpy.fft.rfftn/irfftn`` (the DFT),
``numpy.bincount`` (a sum of weights per mesh cell).  No blocking, fusion or reordering
beyond what the equations state.

Parity status (each function's docstring repeats it):

* T(k) (Eisenstein & Hu no-wiggle) is pinned by its limits (T -> 1 as k -> 0, monotone
  decrease), the zero-baryon form against the independent BBKS fit, the sound-horizon fit
  against Planck 2018's r_drag and, through P_lin, sigma_8 against Planck 2018; the f_b^2
  coefficient of alpha_Gamma moves none of these by more than 0.2% and stays **parity
  unpinned**.  Every other function is pinned by a test in ``tests/test_oracle_*.py``
  against a closed form, an invariant, a brute-force evaluation or central finite
  differences.
"""
