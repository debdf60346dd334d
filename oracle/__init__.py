"""Plain, slow FP64 CPU oracle for the exponential-integrator Fourier
pseudospectral scheme for periodic 3D Maxwell (Wang & Jiang, arXiv 2210.06232).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
or run anything in this package.  The product library never calls it, and it
shares no code with the CUDA path: it uses numpy only (its own mixed-radix
FFT in ``fft``, ``numpy.linalg.eigh`` for the brute-force check; no library
transform).

Modules
-------
``fft``          The 1D and 3D DFT of Sec. 2.3 by a recursive mixed-radix (2, 3,
                 5) Cooley-Tukey FFT, other prime factors by the definition.
``scheme``       Alg. 1 (initial values) and Alg. 2 (fully discrete scheme) of
                 Sec. 2.4-2.5, in the paper's order and notation: wavenumber
                 vectors a_w, b_w, Psi, the coefficients r1, r2, c11..c33,
                 s12, s13, s23, the scaled update and the inverse transform.
``invariants``   The discrete invariants of Sec. 4 (Thm 4.1, 4.3, 4.4, 4.6),
                 evaluated in physical space with the spectral differentiation
                 matrices D_w built from their cot formula (Sec. 2.2).
``bruteforce``   The semi-discrete system (eq. maxreformFD) assembled as a
                 dense 3 N_S x 3 N_S matrix D and its exact flow via an
                 eigendecomposition (Prop. 2.1), for tiny grids.
``closed_form``  Exact solutions: the standing wave of Sec. 5.1, the
                 travelling wave of Sec. 5.2, sums of plane waves.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
against closed forms, brute force, textbook identities or values the paper
prints; none is "parity unpinned".
"""
