"""Oracle: D(mu) psi evaluated at chosen sites only (Sec. 2.1), one red-black SAP cycle (Sec. 2.4) and
the Galerkin coarse operator (Sec. 2.3) evaluated at chosen blocks, for parity checks on lattices too
large for a whole-lattice oracle run.

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

from . import aggregation
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


# ---- one red-black SAP cycle (Sec. 2.4) at chosen blocks, for parity on lattices too large for the
# whole-lattice oracle.  From x = 0, the red blocks' result depends only on b in the block; a black
# block's residual needs the red solutions of its neighbouring blocks, whose hops reach it.

def block_sites(bdims, bcoord):
    """Sites (t, x, y, z) of the block at block coordinates bcoord, in lexical order."""
    o = [bcoord[k] * bdims[k] for k in range(4)]
    return [(o[0] + t, o[1] + x, o[2] + y, o[3] + z)
            for t in range(bdims[0]) for x in range(bdims[1]) for y in range(bdims[2]) for z in range(bdims[3])]


def block_matrix(U, kappa, c_sw, mu, sites):
    """Dense matrix of the block operator D_BB + i mu Gamma5: the site terms and the hops between sites
    of the block; hops that leave the block are dropped (Dirichlet block boundaries, Sec. 2.4).  A block
    never wraps around the lattice, so no boundary phase enters."""
    T, Z, Y, X = U.shape[:4]
    L = (T, X, Y, Z)
    g, g5 = gamma_matrices()
    i4 = np.eye(4)
    index = {s: i for i, s in enumerate(sites)}
    n = 12 * len(sites)
    A = np.zeros((n, n), dtype=complex)
    tw = 1j * mu * np.kron(g5, np.eye(3))
    for i, s in enumerate(sites):
        A[12 * i:12 * i + 12, 12 * i:12 * i + 12] = site_term_at(U, kappa, c_sw, s) + tw
        for d in range(4):
            fwd, bwd = tuple(_step(s, d, 1)), tuple(_step(s, d, -1))
            if fwd in index:
                j = index[fwd]
                A[12 * i:12 * i + 12, 12 * j:12 * j + 12] += -0.5 * np.kron(i4 - g[d], _link(U, L, s, d))
            if bwd in index:
                j = index[bwd]
                A[12 * i:12 * i + 12, 12 * j:12 * j + 12] += -0.5 * np.kron(i4 + g[d], _link(U, L, bwd, d).conj().T)
    return A


def eo_block_mr(A, r, sites, nmr):
    """The even-odd block solve of the SAP smoother (Sec. 2.4, 2.5) on the dense block matrix: nmr
    minimal-residual steps from 0 on A_hat e_o = r_o - A_oe A_ee^-1 r_e with
    A_hat = A_oo - A_oe A_ee^-1 A_eo, then e_e = A_ee^-1 (r_e - A_eo e_o).  A_ee is site-local."""
    par = np.repeat([sum(s) % 2 for s in sites], 12)
    E, O = np.flatnonzero(par == 0), np.flatnonzero(par == 1)
    Aee_inv = np.zeros((len(E), len(E)), dtype=complex)
    for k in range(0, len(E), 12):
        Aee_inv[k:k + 12, k:k + 12] = np.linalg.inv(A[np.ix_(E[k:k + 12], E[k:k + 12])])
    Aeo, Aoe, Aoo = A[np.ix_(E, O)], A[np.ix_(O, E)], A[np.ix_(O, O)]
    Ahat = Aoo - Aoe @ Aee_inv @ Aeo
    rho = r[O] - Aoe @ (Aee_inv @ r[E])
    eo = np.zeros_like(rho)
    for _ in range(nmr):
        p = Ahat @ rho
        den = np.vdot(p, p).real
        al = np.vdot(p, rho) / den if den > 0 else 0.0
        eo = eo + al * rho
        rho = rho - al * p
    e = np.zeros_like(r)
    e[O] = eo
    e[E] = Aee_inv @ (r[E] - Aeo @ eo)
    return e


def sap_cycle_at_block(U, kappa, c_sw, b, mu, bdims, bcoord, nmr, bc_t=0):
    """x on the block at bcoord after one SAP cycle from x = 0 (red blocks, block colour
    sum(bcoord) mod 2 = 0, then black), each block solved by eo_block_mr; returns (nsites, 4, 3)."""
    T, Z, Y, X = U.shape[:4]
    NB = (T // bdims[0], X // bdims[1], Y // bdims[2], Z // bdims[3])

    def spinors(sites, field):
        return np.concatenate([field[t, z, y, x].reshape(12) for (t, x, y, z) in sites])

    def red_solve(bc):
        sites = block_sites(bdims, bc)
        return sites, eo_block_mr(block_matrix(U, kappa, c_sw, mu, sites), spinors(sites, b), sites, nmr)

    sites = block_sites(bdims, bcoord)
    if sum(bcoord) % 2 == 0:
        return red_solve(bcoord)[1].reshape(len(sites), 4, 3)
    # black: r_B = b_B - (D x_red)_B with x_red the red solutions on the neighbouring blocks
    neighbours = set()
    for d in range(4):
        for s in (1, -1):
            bc = list(bcoord)
            bc[d] = (bc[d] + s) % NB[d]
            neighbours.add(tuple(bc))
    x = np.zeros_like(b)
    for bc in neighbours:
        rs, e = red_solve(bc)
        for k, (t, xx, y, z) in enumerate(rs):
            x[t, z, y, xx] = e[12 * k:12 * k + 12].reshape(4, 3)
    r = spinors(sites, b) - apply_D_at_sites(U, kappa, c_sw, x, mu, sites, bc_t).reshape(-1)
    e = eo_block_mr(block_matrix(U, kappa, c_sw, mu, sites), r, sites, nmr)
    return e.reshape(len(sites), 4, 3)


# ---- the Galerkin coarse operator (Sec. 2.3) at chosen aggregates -------------------------------------

class _Aggregate:
    """The lattice of one aggregate, for aggregation.build_P on that aggregate alone (the
    orthonormalisation acts per aggregate half, so the result is that of the whole lattice there)."""

    def __init__(self, lat):
        self.lat = lat
        self.dof = (4, 3)

    def chirality_mask(self, s):
        m = np.zeros(self.dof, dtype=bool)
        m[2 * s:2 * s + 2, :] = True
        return m


def block_slices(bdims, bcoord):
    """Array slices (t, z, y, x) of the block at bcoord in a (T, Z, Y, X, ...) field."""
    o = [bcoord[k] * bdims[k] for k in range(4)]
    return (slice(o[0], o[0] + bdims[0]), slice(o[3], o[3] + bdims[3]), slice(o[2], o[2] + bdims[2]),
            slice(o[1], o[1] + bdims[1]))


def prolongator_at_block(vb, bdims, bcoord):
    """Columns of P on the aggregate at bcoord as a (12 Vb) x (2 Nv) matrix: rows in the order of
    block_sites and spin-colour, columns (s, i) -> s Nv + i.  vb: the test vectors on the aggregate,
    (Nv, bt, bz, by, bx, 4, 3) (a block_slices cut of the whole vectors)."""
    t0, x0, y0, z0 = (bcoord[k] * bdims[k] for k in range(4))
    W = aggregation.build_P(_Aggregate(vb.shape[1:5]), vb, bdims)  # (2, Nv, bt, bz, by, bx, 4, 3)
    nv = vb.shape[0]
    cols = []
    for s in range(2):
        for i in range(nv):
            cols.append(np.concatenate([W[s, i, t - t0, z - z0, y - y0, x - x0].reshape(12)
                                        for (t, x, y, z) in block_sites(bdims, bcoord)]))
    return np.stack(cols, axis=1)


def _coupling(U, rows, cols, bc_t, L):
    """Hopping part of D from the sites `cols` to the sites `rows` (rows never equal cols): the hops
    x -> x +- mu_hat with periodic wrap, a sign -1 on hops that wrap in t when bc_t = 1."""
    g, _ = gamma_matrices()
    i4 = np.eye(4)
    index = {s: j for j, s in enumerate(cols)}
    H = np.zeros((12 * len(rows), 12 * len(cols)), dtype=complex)
    for i, s in enumerate(rows):
        for d in range(4):
            for sign in (1, -1):
                n = list(s)
                n[d] += sign
                wraps = n[d] < 0 or n[d] >= L[d]
                n[d] %= L[d]
                j = index.get(tuple(n))
                if j is None:
                    continue
                f = -1.0 if (wraps and d == 0 and bc_t == 1) else 1.0
                if sign > 0:
                    blk = np.kron(i4 - g[d], _link(U, L, s, d))
                else:
                    blk = np.kron(i4 + g[d], _link(U, L, n, d).conj().T)
                H[12 * i:12 * i + 12, 12 * j:12 * j + 12] += -0.5 * f * blk
    return H


def coarse_columns_at_block(U, kappa, c_sw, v_at, mu, bdims, bcoord, bc_t=0):
    """D_c(mu) e_(A, r) for the 2 Nv unit vectors of the coarse site A = bcoord, restricted to A and its
    8 neighbouring coarse sites: {A: P_A^dagger (D + i mu Gamma5)_AA P_A,
    B: P_B^dagger D_BA P_A for each neighbouring aggregate B}, each (2 Nv) x (2 Nv), column r for e_(A, r).
    v_at(bc) returns the test vectors on the aggregate bc, (Nv, bt, bz, by, bx, 4, 3).  Every aggregate
    lies inside the lattice (no wrap), so the self block needs no boundary phase; the couplings to
    neighbours do (_coupling)."""
    T, Z, Y, X = U.shape[:4]
    L = (T, X, Y, Z)
    NB = tuple(L[k] // bdims[k] for k in range(4))
    sites_A = block_sites(bdims, bcoord)
    P_A = prolongator_at_block(v_at(tuple(bcoord)), bdims, bcoord)
    out = {tuple(bcoord): P_A.conj().T @ block_matrix(U, kappa, c_sw, mu, sites_A) @ P_A}
    for d in range(4):
        for sign in (1, -1):
            bc = list(bcoord)
            bc[d] = (bc[d] + sign) % NB[d]
            bc = tuple(bc)
            sites_B = block_sites(bdims, bc)
            P_B = prolongator_at_block(v_at(bc), bdims, bc)
            out[bc] = out.get(bc, 0) + P_B.conj().T @ _coupling(U, sites_B, sites_A, bc_t, L) @ P_A
    return out
