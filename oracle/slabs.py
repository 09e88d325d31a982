"""Oracle: D(mu) psi on a large lattice, evaluated slab by slab in t (Sec. 2.1).

TEST INFRASTRUCTURE ONLY.  D is local: (D psi)(x) needs psi and the links within one hop of x, and
the clover site term at x needs the links within one hop of x in every plane.  So the operator on
the t-slab [t0, t1) is the whole-lattice oracle (``operators.FineOperator``, unchanged) applied to
the sub-lattice [t0 - 1, t1 + 1) cut out of the periodic lattice, keeping only its interior layers:
the extra layer on each side absorbs the (wrong) wrap of the sub-lattice.  With antiperiodic t
boundaries the fermion layers taken across the global t boundary carry the sign -1 (the links never
do).  Slabs are independent, so they run in a pool of processes (started with ``spawn``), which
makes whole-lattice residuals of the 32^3 x 64 workload affordable on the host.
"""

import multiprocessing as mp

import numpy as np

from .operators import FineOperator

HALO = 1


def _extended(a, t0, t1, T):
    """Layers t0 - HALO .. t1 + HALO - 1 (periodic wrap) of an array whose axis 0 is t."""
    idx = np.arange(t0 - HALO, t1 + HALO) % T
    return a[idx]


def _wrap_sign(t0, t1, T, bc_t):
    """-1 on the extended layers that come from across the global t boundary (antiperiodic), else 1."""
    raw = np.arange(t0 - HALO, t1 + HALO)
    s = np.ones(raw.shape)
    if bc_t == 1:
        s[(raw < 0) | (raw >= T)] = -1.0
    return s


def _slab_apply(args):
    U_ext, kappa, c_sw, psis_ext, sign, mu = args
    op = FineOperator(U_ext, kappa, c_sw, 0)
    out = []
    for p in psis_ext:
        p = p * sign.reshape((-1,) + (1,) * (p.ndim - 1))
        out.append(op.apply(p, mu)[HALO:-HALO])
    return out


def apply_D_slabs(U, kappa, c_sw, psis, mu, bc_t=0, slab=4, workers=None):
    """[D(mu) psi for psi in psis] on the whole lattice, computed per t-slab of ``slab`` layers.

    U: (T, Z, Y, X, 4, 3, 3); psis: sequence of (T, Z, Y, X, 4, 3) spinors (or an array with a leading
    right-hand-side axis).  ``workers`` processes (None: one per slab up to the CPU count; 0: in this
    process)."""
    T = U.shape[0]
    if T % slab:
        raise ValueError("slab must divide T")
    jobs = []
    for t0 in range(0, T, slab):
        t1 = t0 + slab
        jobs.append((_extended(U, t0, t1, T), kappa, c_sw, [_extended(p, t0, t1, T) for p in psis],
                     _wrap_sign(t0, t1, T, bc_t), mu))
    if workers == 0:
        parts = [_slab_apply(j) for j in jobs]
    else:
        n = min(len(jobs), workers or mp.cpu_count() or 1)
        with mp.get_context("spawn").Pool(n) as pool:
            parts = pool.map(_slab_apply, jobs, chunksize=1)
    return [np.concatenate([parts[j][r] for j in range(len(jobs))], axis=0) for r in range(len(psis))]


def relative_residuals(U, kappa, c_sw, b, x, mu, bc_t=0, slab=4, workers=None):
    """||b_r - D(mu) x_r|| / ||b_r|| for every right-hand side r, with the oracle's FP64 D."""
    Dx = apply_D_slabs(U, kappa, c_sw, x, mu, bc_t, slab, workers)
    return [float(np.linalg.norm(b[r] - Dx[r]) / np.linalg.norm(b[r])) for r in range(len(Dx))]
