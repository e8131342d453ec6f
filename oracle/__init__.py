"""FP64 CPU oracle for groupwise-Tucker SINR evaluation (arXiv 2401.09792).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
NumPy (complex128) restatement of the paper's method, written to check the
CUDA library against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product library never imports, links or calls anything here, and this
package imports nothing from the product except the seeded input generators
(``paper_2401_09792_gb300.synth``), which hold no step of the method.

Modules:
  tucker   -- tensor algebra of Section 2.3, HOSVD (Algorithm 1), the
              groupwise fit (eq. 16-22, Algorithm 2), storage (Table 1, eq. 29)
  sinr     -- channel rebuild (eq. 9, eq. 15), SVD precoding (eq. 7, eq. 23),
              covariance (eq. 4, eq. 25), MMSE filter and SINR (eq. 3, 5, 6,
              26-28), the stable SINR form, and the error metric e_c (eq. 30)
  adjoint  -- gradients of the Tucker-form SINR (float64 PyTorch autograd on
              CPU) and a central finite-difference helper

Every function in ``tucker`` and ``sinr`` is pinned by ``tests/test_oracle_*``
against closed forms, library routines or brute force; none is marked
"parity unpinned".
"""
