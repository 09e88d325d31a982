"""Oracle: D(mu) psi evaluated at chosen sites only (Sec. 2.1), for parity checks on lattices too large
for a full oracle application.

TEST INFRASTRUCTURE ONLY.  The operator is local: (D psi)(x) needs psi and the links within one hop of
x, and the clover term at x needs the links of the four plaquette leaves around x in every plane.  Each
requested site is evaluated on its own with explicit coordinate arithmetic (periodic wrap, a sign on
hops that wrap in t for antiperiodic boundaries, exp(+-i theta_mu) on hops that wrap in direction mu for
twisted ones), from the same formulas as ``dirac.py``:

  (D psi)(x) = S(x) psi(x) + i mu gamma5 psi(x)
               - 1/2 sum_mu [(I - gamma_mu) U_mu(x) psi(x + mu) + (I + gamma_mu) U_mu(x - mu)^dagger psi(x - mu)],
  S(x) = (m + 4) I - c_sw/32 sum_{mu != nu} (gamma_mu gamma_nu) x (Q_mu_nu(x) - Q_nu_mu(x)),

with Q_mu_nu(x) the sum of the four equally oriented plaquette leaves in the mu-nu plane at x.
Arrays are (T, Z, Y, X, ...) as everywhere in the oracle; a site is given as (t, x, y, z).
"""

import numpy as np

from .dirac import gamma_matrices


def _link(U, L, c, d):
    t, x, y, z = (c[k] % L[k] for k in range(4))
    return U[t, z, y, x, d]


def _step(c, d, s):
    c = list(c)
    c[d] += s
    return c


def _leaves(U, L, c, a, b):
    dag = lambda A: A.conj().T
    xa, xb = _step(c, a, 1), _step(c, b, 1)
    xma, xmb = _step(c, a, -1), _step(c, b, -1)
    xmab = _step(xma, b, -1)
    q = _link(U, L, c, a) @ _link(U, L, xa, b) @ dag(_link(U, L, xb, a)) @ dag(_link(U, L, c, b))
    q = q + _link(U, L, c, b) @ dag(_link(U, L, _step(xma, b, 1), a)) @ dag(_link(U, L, xma, b)) @ _link(U, L, xma, a)
    q = q + dag(_link(U, L, xma, a)) @ dag(_link(U, L, xmab, b)) @ _link(U, L, xmab, a) @ _link(U, L, xmb, b)
    q = q + dag(_link(U, L, xmb, b)) @ _link(U, L, xmb, a) @ _link(U, L, _step(xmb, a, 1), b) @ dag(_link(U, L, c, a))
    return q


def site_term_at(U, kappa, c_sw, c):
    """The clover site term S(x) (without the twist) as a 12 x 12 matrix at site c = (t, x, y, z)."""
    T, Z, Y, X = U.shape[:4]
    L = (T, X, Y, Z)
    g, _ = gamma_matrices()
    S = (1.0 / (2.0 * kappa)) * np.eye(12, dtype=complex)  # m + 4 = 1 / (2 kappa)
    for a in range(4):
        for b in range(4):
            if a != b:
                Q = _leaves(U, L, c, a, b)
                S -= c_sw / 32.0 * np.kron(g[a] @ g[b], Q - Q.conj().T)
    return S


def apply_D_at_sites(U, kappa, c_sw, psi, mu, sites, bc_t=0, theta=None):
    """(D(mu) psi)(x) for each x in ``sites`` (a list of (t, x, y, z)); returns (len(sites), 4, 3)."""
    T, Z, Y, X = U.shape[:4]
    L = (T, X, Y, Z)
    g, g5 = gamma_matrices()
    i4 = np.eye(4)

    def spinor(c):
        t, x, y, z = (c[k] % L[k] for k in range(4))
        return psi[t, z, y, x].reshape(12)

    out = np.zeros((len(sites), 12), dtype=complex)
    for n, c in enumerate(sites):
        c = list(c)
        v = (site_term_at(U, kappa, c_sw, c) + 1j * mu * np.kron(g5, np.eye(3))) @ spinor(c)
        for d in range(4):
            fwd, bwd = _step(c, d, 1), _step(c, d, -1)
            ff = fb = 1.0 + 0j
            if c[d] == L[d] - 1:  # the forward hop wraps
                ff *= -1.0 if (d == 0 and bc_t == 1) else 1.0
                ff *= np.exp(1j * theta[d]) if theta is not None else 1.0
            if c[d] == 0:  # the backward hop wraps
                fb *= -1.0 if (d == 0 and bc_t == 1) else 1.0
                fb *= np.exp(-1j * theta[d]) if theta is not None else 1.0
            v = v - 0.5 * ff * (np.kron(i4 - g[d], _link(U, L, c, d)) @ spinor(fwd))
            v = v - 0.5 * fb * (np.kron(i4 + g[d], _link(U, L, bwd, d).conj().T) @ spinor(bwd))
        out[n] = v
    return out.reshape(len(sites), 4, 3)
