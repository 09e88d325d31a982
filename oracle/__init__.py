"""Plain, slow FP64 CPU oracle for twisted-mass DD-alpha-AMG (arXiv:1610.02370).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s measurements
around the product (the CPU-baseline timings: the ``cpu_baseline`` leg, the
reference arm and ``--study oracle``; and the residual check of the timed
solutions, after the timed region) use it.  It shares no code with the CUDA
library; both sides only receive the same seeded inputs.

Conventions (fixed here, used by every module of the oracle):

* A fine field lives on a T x Z x Y x X lattice stored as a numpy array whose
  leading axes are ``(T, Z, Y, X)`` (x fastest, the canonical site order
  ``((t*Lz + z)*Ly + y)*Lx + x``).  Direction mu = 0, 1, 2, 3 is t, x, y, z
  (Sec. 2: x_0 is the temporal coordinate).  ``AXIS[mu]`` is the array axis
  that carries direction mu.
* Gauge field ``U``: complex128, shape ``(T, Z, Y, X, 4, 3, 3)``,
  ``U[..., mu, a, b]`` is the (row a, column b) entry of U_mu(x).
* Spinor: complex128, shape ``(T, Z, Y, X, 4, 3)`` = [spin][colour] per site.
  Several right-hand sides carry an extra leading axis.
* Complex inner product <a, b> = sum conj(a) * b.

Modules:
  dirac        -- gamma matrices, clover leaves, site term, D(mu) (Sec. 2.1)
  sap          -- red-black SAP with block MR, full and even-odd blocks (Sec. 2.4)
  aggregation  -- Gamma5-compatible aggregation, P and R = P^dagger (Sec. 2.3)
  coarse       -- Galerkin coarse operator and its stencil (Sec. 2.3)
  krylov       -- GMRES, even-odd GMRES on the coarsest level, FGMRES (Sec. 2.5)
  mg           -- K-cycle preconditioner, adaptive setup, outer solve (Sec. 2.2, 2.6)
"""

from . import dirac, sap, aggregation, coarse, krylov, mg  # noqa: F401
