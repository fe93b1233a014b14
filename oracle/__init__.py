"""FP64 CPU oracle for the phase-shift-dealiased pseudo-spectral Navier-Stokes step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The product path (the CUDA library and its Python binding) never imports, links or runs
anything here, and nothing here imports the product path.

The oracle is plain, slow and written to be checked against the paper by eye:
NumPy in float64, ``numpy.fft`` as the only library primitive (or ``scipy.fft``, the same
pocketfft transforms on several threads, see ``spectral.set_fft_workers``), no blocking or
fusion.
Every function cites the passage of the paper it follows ("Lambert, Reneuve & Augier,
Aliasing and phase shifting in pseudo-spectral simulations of the incompressible
Navier-Stokes equations").

Array conventions (shared by value, not by code, with the CUDA path):

* physical fields ``u[c, z, y, x]`` (C order, x fastest), grid x_j = 2*pi*j/N;
* spectral fields ``uh[c, kz, ky, kx]`` with kz, ky in FFT order (0..N/2-1, -N/2..-1)
  and kx = 0..N/2-1 (the real-to-complex half spectrum without its Nyquist plane,
  which every admissible truncation zeroes).

Modules:

* :mod:`oracle.spectral`    DFT convention, wavenumbers, truncation masks, projection,
  phase shifts (pinned);
* :mod:`oracle.nonlinear`   the nonlinear term with a phase shift, the brute-force
  classified convolution and the 3/2-padded alias-free product (pinned);
* :mod:`oracle.schemes`     RK2, RK4, RK2 phase-shift exact / approx / random / split
  (pinned);
* :mod:`oracle.forcing`     time-correlated random forcing at constant injection rate
  (pinned only by its injection-rate invariant: "parity unpinned" against the paper,
  which does not specify the mechanics);
* :mod:`oracle.diagnostics` energy, dissipation, spectra, spectral error index (pinned);
* :mod:`oracle.rng`         splitmix64 counter generator and the random shifts (pinned);
* :mod:`oracle.adjoint`     transposed (adjoint) step for gradients (pinned by
  dot-product and finite-difference tests);
* :mod:`oracle.nl1d`        the 1D quadratic model of Section 3.3 (pinned by its closed-form
  first evaluation, the Taylor expansion of one step and the exact solution).
"""
