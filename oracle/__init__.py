"""Independent FP64 CPU oracle for FFT-based homogenization with higher-order terms.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or link
anything in this package: only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

The oracle restates the method of Dietrich, Merkert and Simeon, "Derivation of
higher-order terms in FFT-based numerical homogenization" (arXiv:1712.05145), in
plain numpy FP64, following the paper's equations in its own notation:

* ``fourier``              -- its own radix-2 FFT and naive DFT (Sec. 2, Eq. of the
                              periodic Lippmann-Schwinger equation: Fourier series over xi)
* ``tensors``              -- Mandel vectors, Hooke's law (Sec. 2), reference C0
* ``lippmann_schwinger``   -- Green operator Gamma0_hat (Sec. 2, four-index formula),
                              polarization, the Lippmann-Schwinger step, the Basic
                              Scheme and its CG form (Algorithm 1, Eq. cg_form)
* ``hierarchy``            -- the order-alpha problems of Sec. 3 (p_alpha, g_alpha,
                              theta_alpha) and the higher-order effective tensors
* ``closed_forms``         -- laminate, Voigt/Reuss and Hashin-Shtrikman formulas used
                              to pin the oracle

It shares no code with the CUDA path; the only common inputs are the seeded
microstructures from ``paper_1712_05145_gb300.synthetic``, which callers pass in
as plain arrays (this package imports none of the product package).

Parity status per function is listed in each module header.  The paper prints no
value for the higher-order tensors.  Their builders are pinned by symmetry and linearity
checks, and by a laminate whose higher-order problems have closed solutions, to which the
oracle's D_1 .. D_6 converge.
"""
