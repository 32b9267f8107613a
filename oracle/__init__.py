"""Plain FP64 CPU oracle for the deflated Arnoldi sign function.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import or run it. It shares no
code, constants or tables with the CUDA library; the only inputs both sides
see come from the seeded generators in ``paper_0710_0341_gb300.synth``.

Bloch, Wettig, Frommer, Lang, "An iterative method to compute the overlap
Dirac operator at nonzero chemical potential" (Lattice 2007, arXiv:0710.0341).

Modules and what they restate:

* ``dirac``    -- the Wilson-Dirac operator D_w(mu) of Eq. 2 and
                  H_w(mu) = gamma5 D_w(mu) as a scipy sparse matrix (Sec. 1).
* ``matfunc``  -- the scalar sign of Eq. 5 and the matrix sign by the
                  spectral definition (Eqs. 4 and 6); a dense scaled Newton
                  iteration (the matrix iterations cited in Sec. 2) kept only
                  as an independent second route for the tests.
* ``freefield``-- the closed-form sign of H_w(mu) on the free field U = 1 in
                  momentum space (derived from Eq. 2).
* ``overlap``  -- the overlap operator D_ov(mu) = 1 + gamma5 sgn(H_w(mu)) of
                  Eq. 1 and its adjoint via sgn(H_w(-mu)); LR data of the adjoint.
* ``krylov``   -- Arnoldi (Eq. 7) with classical Gram-Schmidt plus one
                  reorthogonalisation, the approximation of Eq. 11, the Schur
                  deflation of Eqs. 13-19 (with the Sylvester equation, Eq. 18),
                  the LR deflation of Eqs. 20-22 and the Hermitian deflation of
                  Eq. 12.
* ``eigen``    -- the m critical eigenpairs (smallest |Re lambda|, Sec. 5) from
                  a dense eigendecomposition, Schur vectors for Eq. 13 and
                  normalised left/right pairs for Eq. 20.

Every function is pinned by a ``-m "not gpu"`` test against closed forms,
invariants or brute force (``tests/test_oracle_*.py``); none is "parity
unpinned".
"""
