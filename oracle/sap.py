"""Oracle: red-black multiplicative Schwarz Alternating Procedure (Sec. 2.4).

TEST INFRASTRUCTURE ONLY.  One SAP cycle applies the block inverses of the red
blocks, then those of the black blocks, each on the freshly recomputed residual;
its error propagator is (I - B_bb D)(I - B_rr D) read right to left, i.e. red
first (our reading: the paper prints the product E_SAP in Sec. 2.4 and calls
the method red-black; ``order`` switches the colour order).

Each block system (D_BB + i mu Gamma5) e = r_B, with the hops that leave the
block dropped (Dirichlet block boundaries, Sec. 2.4), is solved approximately
by ``nmr`` steps of the Minimal Residual method started from e = 0
(Sec. 2.4 names MR; Table 1 lists its step count).  By default the block
system is first reduced to its odd sites (Sec. 2.5 uses even-odd inside the
smoother blocks too):

    A_hat = A_oo - A_oe A_ee^-1 A_eo,   A_hat e_o = r_o - A_oe A_ee^-1 r_e,
    e_e = A_ee^-1 (r_e - A_eo e_o),

where A_ee, A_oo are the site-local parts.  ``eo=False`` runs MR on the full
block instead.

All blocks of one colour are handled at once: blocks of one colour never touch
(``blocks.check_colouring``), so masking a field to one colour and applying the
operator restricted to the same mask is exactly the block-diagonal D_rr or D_bb.
"""

import numpy as np

from . import blocks
from .dirac import parity


def _ndof(op):
    return len(op.dof)


def _mr_blocks(apply_A, rhs, nmr, lat, bdims, nd):
    """nmr MR steps per block from e = 0:  p = A rho, alpha = <p, rho>/<p, p>,
    e += alpha rho, rho -= alpha p (Saad's minimal residual iteration)."""
    e = np.zeros_like(rhs)
    rho = rhs.copy()
    for _ in range(nmr):
        p = apply_A(rho)
        num = blocks.block_sum(np.conj(p) * rho, lat, bdims)
        den = blocks.block_sum(np.abs(p) ** 2, lat, bdims).real
        alpha = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
        a = blocks.broadcast(alpha, lat, bdims, nd)
        e = e + a * rho
        rho = rho - a * p
    return e


def block_solve(op, r, mu, bdims, colour, nmr, eo=True):
    """Approximate block inverses B_cc(mu) r for every block of one colour.

    r is a full field; the result is supported on the blocks of ``colour``.
    """
    lat = op.lat
    nd = _ndof(op)
    cmask = (blocks.block_colour(lat, bdims) == colour).reshape(lat + (1,) * nd)
    rc = r * cmask

    def hop_c(v):
        return cmask * op.hop(cmask * v)

    if not eo:
        def A(v):
            return op.site(v, mu) + hop_c(v)
        return _mr_blocks(A, rc, nmr, lat, bdims, nd)

    par = parity(lat).reshape(lat + (1,) * nd)
    even, odd = (par == 0), (par == 1)
    r_e, r_o = rc * even, rc * odd

    def A_hat(v_o):
        t = even * hop_c(v_o)             # A_eo v_o
        t = op.site_inv(t, mu) * even     # A_ee^-1 A_eo v_o
        return odd * op.site(v_o, mu) - odd * hop_c(t)

    rhat = r_o - odd * hop_c(op.site_inv(r_e, mu) * even)
    e_o = _mr_blocks(A_hat, rhat, nmr, lat, bdims, nd)
    e_e = op.site_inv(r_e - even * hop_c(e_o), mu) * even
    return e_o + e_e


def sap(op, b, mu, bdims, ncycles, nmr, x0=None, eo=True, order=(0, 1)):
    """ncycles red-black SAP cycles for D(mu) x = b, started from x0 (default 0)."""
    blocks.check_colouring(op.lat, bdims)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    for _ in range(ncycles):
        for colour in order:
            r = b - op.apply(x, mu)
            x = x + block_solve(op, r, mu, bdims, colour, nmr, eo)
    return x
