"""Oracle: Krylov solvers of Sec. 2.5 -- GMRES, even-odd GMRES, flexible GMRES.

TEST INFRASTRUCTURE ONLY.  Textbook (Saad) algorithms in FP64: Arnoldi with
modified Gram-Schmidt, Givens rotations on the Hessenberg matrix, the
least-squares residual |g_{j+1}| as the in-cycle estimate, zero initial guess.
Stopping is relative to ||b|| of the system solved.

FGMRES is right preconditioned and flexible (it stores Z_j = M v_j and updates
x with Z), as Sec. 2.5 requires because the multigrid preconditioner is not a
fixed linear map.

Even-odd GMRES (coarsest level, Sec. 2.5) solves the Schur complement onto the
odd sites,  D_hat phi_o = eta_o - D_oe D_ee^-1 eta_e  with
D_hat = D_oo - D_oe D_ee^-1 D_eo,  and retrieves
phi_e = D_ee^-1 (eta_e - D_eo phi_o).  (Our reading: the printed retrieval has
phi_e on both sides, and Sec. 2.1 reduces onto the other parity; both are
garbled forms of this Schur complement.)

Even-odd CG (the baseline of Sec. 3.1.2): conjugate gradients need a
Hermitian positive definite matrix, so the even-odd reduced system of the fine
operator is squared, D_hat^dagger D_hat x_o = D_hat^dagger rhat with the same
Schur complement and retrieval as above; textbook CG (Hestenes-Stiefel) from
x_o = 0, stopped on the recursively updated residual of the squared system.
"""

import numpy as np

from .dirac import parity
from .operators import negate_twist


def _dot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def _norm(a):
    return float(np.sqrt(np.real(_dot(a, a))))


def fgmres(A, b, M=None, restart=30, max_restarts=100, tol=1e-10):
    """Flexible GMRES(restart) for A x = b with right preconditioner M (identity if None).

    Each cycle runs Arnoldi until the Givens estimate |g_{j+1}|/||b|| <= tol or
    the restart length is reached, updates x += Z y, and recomputes the true
    residual b - A x, which decides convergence and starts the next cycle.
    The rotation for column j is G = [[conj(c), conj(s)], [-s, c]] with
    c = H_jj / rho, s = H_{j+1,j} / rho, rho = sqrt(|H_jj|^2 + |H_{j+1,j}|^2).

    Returns (x, info) with info = dict(iters, restarts, relres, converged).
    """
    bn = _norm(b)
    x = np.zeros_like(b)
    info = dict(iters=0, restarts=0, relres=1.0, converged=False)
    if bn == 0.0:
        info.update(relres=0.0, converged=True)
        return x, info
    r = b.copy()
    for cyc in range(max_restarts + 1):
        beta = _norm(r)
        info['relres'] = beta / bn
        if beta / bn <= tol:
            info['converged'] = True
            return x, info
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart), dtype=complex)
        cs = np.zeros(restart, dtype=complex)
        sn = np.zeros(restart, dtype=complex)
        g = np.zeros(restart + 1, dtype=complex)
        g[0] = beta
        k = 0
        for j in range(restart):
            z = V[j] if M is None else M(V[j])
            Z.append(z)
            w = A(z)
            for i in range(j + 1):  # modified Gram-Schmidt
                H[i, j] = _dot(V[i], w)
                w = w - H[i, j] * V[i]
            hn = _norm(w)
            H[j + 1, j] = hn
            for i in range(j):  # earlier rotations on the new column
                t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            rho = np.sqrt(abs(H[j, j]) ** 2 + abs(H[j + 1, j]) ** 2)
            cs[j] = H[j, j] / rho
            sn[j] = H[j + 1, j] / rho
            H[j, j] = rho
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            k = j + 1
            info['iters'] += 1
            if abs(g[j + 1]) / bn <= tol or hn == 0.0:
                break
            V.append(w / hn)
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        for i in range(k):
            x = x + y[i] * Z[i]
        info['restarts'] = cyc
        r = b - A(x)
    info['relres'] = _norm(r) / bn
    info['converged'] = info['relres'] <= tol
    return x, info


def gmres(A, b, restart, max_restarts, tol):
    """Restarted GMRES(restart): FGMRES with no preconditioner, estimate-based restarts,
    true residual checked at the end of every cycle."""
    return fgmres(A, b, None, restart, max_restarts, tol)


def eo_gmres(cop, eta, mu, restart=100, max_restarts=5, tol=1e-1):
    """Even-odd preconditioned GMRES for the coarse system D_c(mu) phi = eta (Sec. 2.5).

    ``cop`` is an operator object with site / site_inv / hop on its lattice;
    coarse parity is the sum of coarse coordinates mod 2 (0 = even).
    Returns (phi, info); info['relres'] refers to the reduced odd system.
    """
    lat = cop.lat
    nd = len(cop.dof)
    par = parity(lat).reshape(lat + (1,) * nd)
    even, odd = (par == 0), (par == 1)

    def D_ee_inv(v):
        return cop.site_inv(v * even, mu) * even

    def D_oe(v_e):
        return odd * cop.hop(v_e * even)

    def D_eo(v_o):
        return even * cop.hop(v_o * odd)

    def D_hat(v_o):
        return odd * cop.site(v_o * odd, mu) - D_oe(D_ee_inv(D_eo(v_o)))

    eta_e, eta_o = eta * even, eta * odd
    rhs = eta_o - D_oe(D_ee_inv(eta_e))
    phi_o, info = gmres(D_hat, rhs, restart, max_restarts, tol)
    phi_o = phi_o * odd
    phi_e = D_ee_inv(eta_e - D_eo(phi_o))
    return phi_e + phi_o, info


def eo_cg(op, b, mu, tol=1e-10, max_iter=100000):
    """Even-odd reduced CG on D_hat^dagger D_hat (Sec. 3.1.2) for D(mu) x = b on the
    lattice of ``op`` (site / site_inv / hop / gamma5 on its lattice).  D_hat^dagger is
    applied as Gamma5 D_hat(-mu) Gamma5 (Gamma5-hermiticity of every piece).  Stops when
    ||r_k|| <= tol ||D_hat^dagger rhat|| for the residual r_k of the squared system.
    Returns (x, info) with info['iters'] and info['residuals'] (the ||r_k|| sequence)."""
    lat = op.lat
    nd = len(op.dof)
    par = parity(lat).reshape(lat + (1,) * nd)
    even, odd = (par == 0), (par == 1)

    def d_hat(v_o, m):
        t = op.site_inv(even * op.hop(v_o * odd), m) * even
        return odd * op.site(v_o * odd, m) - odd * op.hop(t)

    def d_hat_dag(v_o):
        return op.gamma5(d_hat(op.gamma5(v_o), negate_twist(mu)))

    b_e, b_o = b * even, b * odd
    rhat = b_o - odd * op.hop(op.site_inv(b_e, mu) * even)
    rhs = d_hat_dag(rhat)
    x = np.zeros_like(b)
    r = rhs.copy()
    p = r.copy()
    rr = _dot(r, r).real
    stop = tol * np.sqrt(rr)
    res = [np.sqrt(rr)]
    it = 0
    while np.sqrt(rr) > stop and it < max_iter:
        q = d_hat_dag(d_hat(p, mu))
        alpha = rr / _dot(p, q).real
        x = x + alpha * p
        r = r - alpha * q
        rr_new = _dot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
        res.append(np.sqrt(rr))
    x_o = x * odd
    x_e = op.site_inv(b_e - even * op.hop(x_o), mu) * even
    return x_e + x_o, {"iters": it, "residuals": res, "converged": np.sqrt(rr) <= stop}
