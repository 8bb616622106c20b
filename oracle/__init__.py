"""The oracle: a plain, slow, obviously correct CPU restatement of the REXI
method of Rittich & Speck, "Time-parallel simulation of the Schroedinger
equation" (arXiv:1912.03312), in complex FP64 (numpy) with the pole/weight
construction in arbitrary precision (mpmath).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package.
It shares no code with the CUDA library (``paper_1912_03312_gb300``) and
imports nothing from it; the seeded input generators in ``workloads`` are the
only common module, and they hold none of the method's arithmetic.

Modules:
  fcf      -- Algorithm 1 (CF) and Algorithm 2 (FaberCF), Eq. (7)-(9)
  tables   -- FCF poles/weights per (K, R1), cached as text written by
              ``oracle/make_tables.py`` (mpmath is absent on some hosts)
  plan     -- spectral enclosure, substeps (Eq. (10)), physical poles (Eq. (5))
  operator -- finite-difference H of Eq. (1), periodic, second order
  gmres    -- textbook restarted GMRES(m), MGS, Givens
  step     -- Eq. (5) step, substeps, adjoint and gradient, dense references
"""
