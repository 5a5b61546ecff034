"""CPU oracle for the MPO Lindblad solver of Landa & Misguich (2022).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may call it.  It shares no code with
the CUDA path: every formula here is written again, independently, from the
paper (model, Sec. 2.1; MPO representation, App. A; SVD compression, App. B).

Plain, slow, FP64 code:

* ``model``    - the Lindbladian of Eq. (dtrho) with Eq. (H0), Eq. (K_def),
                 Eqs. (D0)-(D2), as 2^N x 2^N operators (dense oracle) and as
                 local superoperators in the normalised Pauli basis of
                 Eq. (mpo_def) built by explicit traces.
* ``schedule`` - the two-site op list of one 2nd-order Trotter step (even
                 bonds, odd bonds, long-range bonds through swap chains).
* ``dense``    - exact evolution of the full density matrix (sparse
                 expm-multiply of the vectorised Liouvillian) and the dense
                 Trotter product on the 4^N Pauli-coefficient vector.
* ``svd``      - one-sided (Hestenes) Jacobi SVD in plain C (``jacobi.c``).
* ``tebd``     - MPO time evolution with two-site gates and SVD truncation
                 (App. B's rule: the more severe of cut_off_rho and
                 max_dim_rho), trace forcing and Pauli observables.

Every function that has no independent pin says "parity unpinned" in its
docstring; all others are pinned by ``tests/test_oracle_*.py``.
"""
