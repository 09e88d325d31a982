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
"""

import numpy as np

from .dirac import parity


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
