"""Oracle: DD-alpha-AMG preconditioner (K-cycle), adaptive setup and outer solve.

TEST INFRASTRUCTURE ONLY.  Written from Sec. 2.2 (error propagation with j
pre- and k post-smoothing steps, coarse correction psi <- psi + P D_c^-1 R r,
K-cycle recursion), Sec. 2.4 (SAP smoother with block size = aggregate size),
Sec. 2.5 (FGMRES outer and K-cycle solver, even-odd GMRES on the coarsest
level, relaxed inner tolerances), Sec. 2.6 (setup by inverse iteration) and
Table 1 (defaults).

Readings where the paper is silent:
* no pre-smoothing (Table 1 lists only post-smoothing steps); one
  preconditioner application on level l is  x = P D_{l+1}^-1 R v  followed by
  ``post_smooth`` SAP cycles on D_l x = v started from that x;
* only the coarsest level uses the shifted twist delta*mu (Table 1:
  mu_coarse = 5.2 mu); every other level uses mu; a twist that differs on even
  and odd sites is shifted on both parities alike;
* setup iteration k = 1 runs the SAP smoother (``post_smooth`` cycles) on each
  test vector as right-hand side, iterations k >= 2 run one preconditioner
  application per test vector; after every iteration each vector is normalised
  and P, D_c are rebuilt.  Deeper levels (three-level hierarchies) repeat the
  same procedure on the level above, right after it was rebuilt, starting from
  their own random vectors.
"""

from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

from . import aggregation, coarse, krylov, sap
from .operators import scale_twist


@dataclass
class Params:
    """Table 1 defaults."""
    nlevels: int = 3
    n_setup: int = 5
    nv: List[int] = field(default_factory=lambda: [28, 28])
    bdims: List[Tuple[int, int, int, int]] = field(default_factory=lambda: [(4, 4, 4, 4), (2, 2, 2, 2)])
    post_smooth: int = 4
    nmr: int = 3
    sap_eo: bool = True
    kcycle_restart: int = 5
    kcycle_max_restarts: int = 2
    kcycle_tol: float = 1e-1
    coarse_restart: int = 100
    coarse_max_restarts: int = 5
    coarse_tol: float = 1e-1
    delta: float = 5.2
    outer_restart: int = 30
    outer_max_restarts: int = 50
    outer_tol: float = 1e-10


class Hierarchy:
    """ops[l] is the operator of level l (ops[0] the fine D), W[l] the P of l -> l+1."""

    def __init__(self, fine_op, params):
        self.p = params
        self.ops = [fine_op]
        self.W = []
        self.coarse_iters = 0

    @property
    def L(self):
        return self.p.nlevels

    def mu_at(self, level, mu):
        """The coarsest level uses delta times the twist (both parities of a pair)."""
        return scale_twist(mu, self.p.delta) if level == self.L - 1 else mu

    def rebuild(self, level, v):
        """Normalise test vectors v of level ``level``, build P and D_{level+1}."""
        v = np.array([t / np.linalg.norm(t) for t in v])
        W = aggregation.build_P(self.ops[level], v, self.p.bdims[level])
        cop = coarse.build_coarse_operator(self.ops[level], W, self.p.bdims[level])
        if len(self.W) > level:
            self.W[level] = W
            self.ops[level + 1] = cop
        else:
            self.W.append(W)
            self.ops.append(cop)
        return v

    def coarse_solve(self, level, c, mu):
        """Approximate D_level^-1 c for level >= 1."""
        p = self.p
        op = self.ops[level]
        if level == self.L - 1:
            x, info = krylov.eo_gmres(op, c, self.mu_at(level, mu), p.coarse_restart,
                                      p.coarse_max_restarts, p.coarse_tol)
            self.coarse_iters += info['iters']
            return x
        x, _ = krylov.fgmres(lambda v: op.apply(v, mu), c, lambda v: self.precondition(level, v, mu),
                             p.kcycle_restart, p.kcycle_max_restarts, p.kcycle_tol)
        return x

    def precondition(self, level, v, mu):
        """One K-cycle preconditioner application M_level v (level < L-1)."""
        p = self.p
        op = self.ops[level]
        bd = p.bdims[level]
        c = aggregation.restrict(self.W[level], v, op.lat, bd)
        e = self.coarse_solve(level + 1, c, mu)
        x = aggregation.prolong(self.W[level], e, op.lat, bd)
        return sap.sap(op, v, mu, bd, p.post_smooth, p.nmr, x0=x, eo=p.sap_eo)


def setup(fine_op, params, mu, tv0):
    """Adaptive setup (Sec. 2.6).  tv0[l] holds the random start vectors of level l,
    shape (Nv_l,) + lat_l + dof_l.  Returns the Hierarchy."""
    h = Hierarchy(fine_op, params)
    p = params
    vs = []
    for level in range(p.nlevels - 1):  # k = 1: SAP only, level by level
        op = h.ops[level]
        v = np.array([sap.sap(op, t, mu, p.bdims[level], p.post_smooth, p.nmr, eo=p.sap_eo)
                      for t in tv0[level]])
        vs.append(h.rebuild(level, v))
    for _k in range(2, p.n_setup + 1):
        for level in range(p.nlevels - 1):
            v = np.array([h.precondition(level, t, mu) for t in vs[level]])
            vs[level] = h.rebuild(level, v)
    h.test_vectors = vs
    return h


def hierarchy_from_vectors(fine_op, params, vs):
    """Hierarchy with P built from given test vectors (no inverse iteration)."""
    h = Hierarchy(fine_op, params)
    for level in range(params.nlevels - 1):
        h.rebuild(level, vs[level])
    return h


def solve(h, b, mu):
    """Outer FGMRES(restart) on D(mu) x = b preconditioned by the K-cycle (Sec. 2.5)."""
    p = h.p
    op = h.ops[0]
    h.coarse_iters = 0
    x, info = krylov.fgmres(lambda v: op.apply(v, mu), b, lambda v: h.precondition(0, v, mu),
                            p.outer_restart, p.outer_max_restarts, p.outer_tol)
    info['coarse_iters'] = h.coarse_iters
    return x, info
