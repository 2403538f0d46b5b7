"""FP64 CPU oracle for the natively periodic FMM (Gnedin, arXiv:2011.07099).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of what the paper defines, used to prove the CUDA path right.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The product library never calls it and it never
calls the product library: the two share no code, tables or constants.

Modules
-------
green   Green's functions G_0, G_K, G_X and G_S1 (Sec. 1, Sec. 3 ansatz,
        Sec. 4 eq. gfs1) and the cell self-term reading.
pm      Brute-force periodic convolution and the FFT particle-mesh solution
        (Sec. 1; Sec. 3 eq. pmconv).
fmm     The FMM-HPM solve step by step: masses, gridlet multipoles by the
        Vandermonde system (Sec. 2), M2M / M2L / L2L (Sec. 3 eqs. fmm1-fmm3),
        L2P and the near-zone direct sum (Sec. 2).

Every function is FP64.  Parity status of each function is stated in its
docstring ("pinned by ..." or "parity unpinned").
"""
