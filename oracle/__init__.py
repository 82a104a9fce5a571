"""CPU oracle for accelerated cyclic reduction (ACR) -- test infrastructure only.

A plain, slow, FP64 NumPy restatement of what the GPU path computes, written
from the paper (Chavez, Turkiyyah, Zampini, Keyes, "Parallel accelerated
cyclic reduction preconditioner for three-dimensional elliptic PDEs with
variable coefficients", JCAM 2017):

* ``assembly``   -- 7-point operators of Sec. 6 (Eq. poissonEquation, harmonic
                    face averages) and Sec. 7 (Eq. codi, first-order upwind).
* ``hstructure`` -- index set, cluster tree, block cluster tree and the
                    admissibility condition of Sec. 3.1 (Eq. admis).
* ``hformat``    -- H-format projection with blockwise SVD truncation at
                    H_eps (Sec. 3.1.5, Sec. 4.3), formatted products and the
                    recursive 2x2 H-inverse.
* ``cr``         -- exact block cyclic reduction with dense blocks and the
                    ACR variant with every plane block in H-format (Sec. 4.1,
                    Sec. 4.2): setup (elimination) and apply (substitution).
* ``krylov``     -- FP64 preconditioned CG and right-preconditioned GMRES(m)
                    (Sec. 5.3, Sec. 7).
* ``adjoint``    -- dL/dkappa of a Poisson solve by the adjoint of the Sec. 6
                    assembly (no counterpart in the paper).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library
and its Python binding) never calls it and has no CPU fallback.

Parity status of each part is stated in the module headers; every function
here is pinned by ``tests/test_oracle_*.py`` against closed forms, dense
direct solves, DST-I, constructed spectra or brute force, except where a
header says "parity unpinned".
"""
