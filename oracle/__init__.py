"""FP64 CPU oracle for the abc set-projection iteration (test infrastructure).

This package is the plain, slow, obviously correct reference that the CUDA
path is checked against.  It is TEST INFRASTRUCTURE ONLY: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The product path (the C-ABI library and
its Python binding) never imports, calls or links anything here, and this
package imports nothing from the product path.

Modules
-------
dft      the unnormalised 2-D DFT as dense matrix products (no FFT library)
abc      relaxed projections and the generic abc driver, the named presets
ptycho   divide (Fourier modulus) and concur (overlap) projections,
         re-split, one abc iteration over all exit waves
metrics  Fourier error and the phase-ramp-corrected object error
toy      the three-circle product-space example
sp       sequential projections (the non-product-space alternative)

Paper: W. Mei, A. M. Maiden, "Set projection algorithms for blind
ptychographic phase retrieval" (arXiv 2311.11466).  Citations name the
paper's section, figure or displayed equation.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, brute force or library routines the oracle
does not call.  Two quantities are "parity unpinned" beyond the oracle
itself: the values of the error curves after many iterations (the paper's
Figs. 7 and 8 are not recoverable), which are compared GPU-vs-oracle only.
"""
