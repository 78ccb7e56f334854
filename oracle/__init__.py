"""FP64 CPU oracle for the hybrid wave-particle / FFT height-field synthesis
of "Real-Time Interactive Hybrid Ocean: Spectrum-Consistent Wave
Particle-FFT Coupling" (arXiv 2511.02852).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call,
link or execute anything in this package: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` use it.  It shares no code, headers, tables or
generators with the CUDA library in ``paper_2511_02852_gb300/csrc``.

The oracle is a plain, slow restatement of the method, step by step, in the
paper's order and notation, in float64 (integers where the method's state is
integer).  Each function cites the paper passage it follows (section,
equation).  Where the paper is silent or ambiguous the oracle implements the
reading recorded in the repository's design notes; every such reading is
marked "reading" in the docstring.

Pinned by the ``-m "not gpu"`` tests (closed forms, normalisation
conditions, brute-force DFTs, single-particle closed forms, invariants).
Parity unpinned: the steady-state variance of the wave-particle field against
the background's (the paper never measures it).

Modules
-------
philox      Philox4x32-10 counter-based generator (Salmon et al., SC'11).
spectrum    JONSWAP / Phillips spectra, spreading, dispersion, buckets,
            amplitudes (Sec. 3.1 Eqs. 1-6, Sec. 3.2 Eq. A, Sec. 3.3 Eqs. 7-8).
background  FFT background: h0(k), h(k,t), inverse 2-D DFT (Sec. 4.1).
particles   Fixed-point particle state, injection counts (Eqs. 9-17),
            spawn, advection, expiry, wake emission (Sec. 4.3), binning.
synth       Bump-kernel synthesis, displacement, blend (Sec. 4.2), and the
            layered splat + separable-filter variant (Sec. 4.2).
scene       A whole scene stepped frame by frame.
"""
