"""Plain, slow FP64 CPU oracle for the REXII time step (arXiv 2008.11607).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code, table or constant generator with the CUDA library under
``paper_2008_11607_gb300/``; each side transcribes the paper on its own.

Modules
-------
coeffs     Table A constants, Gaussian sum (Step 1), rational fit (Step 2),
           REXII single sum (Step 3, eq. modifiedRexi), pole-count rule
           (eq. matrixAccuracyBound, Appendix B), single-shift poles.
operator   Staggered C-grid linear rotating shallow-water operator as a
           scipy.sparse matrix (Section 4, with variable depth).
rexi       Matrix REXII by one sparse direct solve pair per term, in the order
           of the per-term solve sequence of Section 4 (eq.
           modifiedRexiMatrixReducedSum), plus the same chain on a single
           Fourier mode for sampled checks of large grids.
exact      Reference exponentials: closed-form per-wavenumber e^{tau B(k)} and
           dense scipy.linalg.expm for tiny grids.

Every function cites the passage of the paper it follows.  Functions without
an independent pin say "parity unpinned" in their docstring.
"""
