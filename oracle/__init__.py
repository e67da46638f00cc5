"""CPU oracle for the Matérn log-likelihood path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct float64 implementations of what the CUDA path
computes, written from the paper (eq. 1 likelihood, eqs. 2-4 kriging, eq. 5
Matérn covariance, Sec. V tile low-rank approximation).  Only the test suite,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` may import anything here; the product path never does, and the
oracle never imports the product package (only its seeded input generators in
``paper_1804_09137_gb300.inputs``, which hold no method arithmetic).

Modules
-------
matern : eq. 5 and its parameter derivatives (scipy.special based).
dense  : exact dense-Cholesky likelihood, gradient, kriging, z = L e.
tlr    : CPU tile low-rank reference (truncated SVD + right-looking TLR Cholesky).

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``
(closed forms, brute force, invariants); see each module's header.
"""
