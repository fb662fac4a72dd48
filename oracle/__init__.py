"""Plain, slow FP64 CPU oracle for the butterfly-accelerated manifold harmonic transform.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports, links or runs this package;
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may.
It shares no code with the CUDA path: the only common module is ``workloads`` (seeded
input shapes, none of the method's arithmetic).

Contents, each following the paper's statement of the result:

* ``harmonics`` -- the transform matrix Phi for closed-form manifolds: complex
  exponentials on the flat periodic square (Eq. ``2D-DFT``) and orthonormal real
  spherical harmonics on the unit sphere (Sec. 1);
* ``fem`` -- cotangent stiffness and lumped mass on a triangle mesh and the lowest
  generalized eigenpairs of the Laplace-Beltrami eigenproblem (Eq. ``eigenproblem``);
* ``dense`` -- the transform by direct summation, ``f = Phi c`` (Eq. ``MHT-sum``) and its
  weighted adjoint ``c = Phi^H diag(w) f``;
* ``butterfly`` -- an independent row-wise butterfly factorization with interpolative
  decompositions (Sec. 2, Algorithm 1), Fiedler trees (Sec. 3, Algorithm 2), the
  apply of a factorization in both directions, and the apply of factors handed in as
  plain arrays.

Pins (``tests/test_oracle_*.py``, run with ``-m "not gpu"``) tie every function to
something other than itself: FFTs, library spherical harmonics, quadrature identities,
exact mesh invariants, brute force on tiny inputs and the paper's error claim.
"""
