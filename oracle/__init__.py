"""FP64 CPU oracle of the truncated-Green's-function volume-potential method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may use it.  It shares no code, tables or constants with the
CUDA library under ``paper_1604_03155_gb300/csrc``.

It is a plain, slow, obviously correct restatement of what the method computes
(Vico, Greengard & Ferrando, "Fast convolution with free-space Green's
functions", arXiv:1604.03155), in float64 with numpy/scipy:

* ``fft``            its own mixed-radix FFT and a direct DFT (no numpy.fft);
* ``spectrum``       the truncated spectra G^L(s) of Tables 1-2 (Section 3) and
                     the defining radial integrals of Section 2;
* ``kernel``         the discrete kernel T of Section 4 (inverse 4N transform of
                     G^L), derivative kernels, and the (2N)^d multipliers;
* ``apply``          the volume potential phi_i = sum_i' T(i-i') f_i' by brute
                     force, by the (2N)^d FFT and by the un-precomputed 4N form;
* ``closed_forms``   Gaussian-source potentials of Section 5.1.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, quadrature, brute force or textbook routines, except where its
docstring says "parity unpinned".
"""
