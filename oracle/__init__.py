"""FP64 CPU oracle of the averaged-Yee Maxwell step (arXiv:1907.13088).

TEST INFRASTRUCTURE ONLY.  ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers; the product package
never imports it and shares no code with it.

* ``oracle.core``     -- ctypes front end of the stencil oracle (plain C).
* ``oracle.spectral`` -- per-wavevector form of the same step and the paper's
                         closed forms (dispersion, CFL, phase speed).
* ``oracle.nci``      -- NCI resonance curves and asymptotic growth rate
                         (Sec. 3, App. E).
"""
