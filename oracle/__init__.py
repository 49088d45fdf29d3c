"""CPU oracle for the TT-SVD hot path -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, obviously correct FP64 restatement of what the
paper "Performance of the low-rank tensor-train SVD (TT-SVD) for large dense
tensors on modern multi-core CPUs" (Roehrig-Zoellner, Thies, Basermann)
computes.  It exists to check the CUDA path, never to stand in for it:

* only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
  ``--impl reference`` legs of ``bench.py`` may import it;
* it shares no code with the CUDA library (``paper_2102_00104_gb300``) and
  imports nothing from it; both sides only share the seeded input generator
  module ``paper_2102_00104_gb300.inputs``, which holds no TT-SVD arithmetic.

Modules
-------
``tt_svd_oracle``  Alg. 1 (original TT-SVD, Sec. 3.1.1) with explicit
                   unfoldings and a full LAPACK SVD; the truncation rule;
                   TT reconstruction; brute-force unfolding spectra.
``householder``    Alg. 6 (Q-less Householder QR of a rectangle stacked on a
                   triangle, Sec. 3.2) and the flat-tree TSQR built from it.
``tt_svd_tsqr``    Alg. 2 (TSQR TT-SVD, Sec. 3.1.2) built from ``householder``
                   and a LAPACK SVD of R; used to pin Alg. 1 == Alg. 2.
``model``          the performance model of Sec. 4 (Eqs. for TSQR/TSMM flops
                   and bytes, Eq. TT-SVD_data_volume, Eq. TT-SVD_operations).
``thick_bounds``   Alg. 3 (thick-bounds TT-SVD, Sec. 3.1.3): combined right-most
                   dimensions, TT-SVD of the reshaped tensor, recovery of the
                   combined cores from a TT-SVD of the last core.
``two_sided``      Alg. 4 (two-sided TT-SVD, Sec. 3.1.3): cores alternately at the
                   right and the left end, middle core last.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, library routines, brute force or values printed in the
paper; none is "parity unpinned".  ``tests/test_oracle_mutants.py`` plants one
plausible mistake at a time in a copy of these modules and checks that a pin fails.
"""
