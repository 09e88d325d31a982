"""Seeded synthetic inputs: gauge fields, right-hand sides and special fields.

This module holds no arithmetic of the solver; it only draws inputs.  Both the
CUDA library (through the binding) and the CPU oracle receive what it
produces.  Layout of everything returned (torch tensors, complex128):

* gauge field: (T, Z, Y, X, 4, 3, 3), U[t, z, y, x, mu, a, b] with mu = 0:t,
  1:x, 2:y, 3:z -- the canonical site order ((t*Lz + z)*Ly + y)*Lx + x;
* spinor: (T, Z, Y, X, 4, 3) [spin][colour], with a leading rhs axis for
  several right-hand sides.

Random gauge links follow U = exp(i eps H) with H = (A + A^dagger)/2 - tr/3,
A having i.i.d. complex entries with N(0,1) real and imaginary parts; the
exponential is a scaled-and-squared Taylor series (unitary to rounding).  The draws come from
a torch generator seeded with ``seed`` on ``device``, so a CPU and a CUDA field
of the same seed differ; tests always hand the same tensor to both sides.
"""

import math

import torch


def _lat(dims):
    T, X, Y, Z = dims
    return (T, Z, Y, X)


def _gen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def expm_i_hermitian(H, eps):
    """exp(i eps H) for a batch of Hermitian 3x3 matrices by Taylor series with
    scaling and squaring (Moler and Van Loan): A = i eps H / 2^s with
    ||A||_F <= 1/2, 20 Taylor terms (remainder below 1e-20), then s squarings."""
    A = 1j * eps * H
    nrm = float(torch.linalg.matrix_norm(A).max()) if A.numel() else 0.0
    s = max(0, int(math.ceil(math.log2(nrm / 0.5)))) if nrm > 0.5 else 0
    A = A / (2.0 ** s)
    eye = torch.eye(3, dtype=A.dtype, device=A.device)
    term = eye.expand(A.shape).clone()
    out = term.clone()
    for k in range(1, 21):
        term = term @ A / k
        out = out + term
    for _ in range(s):
        out = out @ out
    return out


def random_hermitian_exp(shape, eps, seed, device="cpu"):
    """exp(i eps H) for a batch of traceless Hermitian Gaussian 3x3 H."""
    g = _gen(seed, device)
    a = torch.randn(shape + (3, 3, 2), generator=g, dtype=torch.float64, device=device)
    A = torch.complex(a[..., 0], a[..., 1])
    H = 0.5 * (A + A.mH)
    tr = torch.diagonal(H, dim1=-2, dim2=-1).sum(-1)
    H = H - (tr / 3.0)[..., None, None] * torch.eye(3, dtype=H.dtype, device=device)
    return expm_i_hermitian(H, eps)


def gauge_field(dims, eps, seed=0, device="cpu", chunk_sites=1 << 20):
    """Random SU(3) gauge field U_mu(x) = exp(i eps H_mu(x)) on a T x X x Y x Z lattice."""
    lat = _lat(dims)
    V = math.prod(lat)
    if V <= chunk_sites:
        return random_hermitian_exp(lat + (4,), eps, seed, device)
    # large lattices: draw in slabs of t so that eigh never sees a huge batch
    out = torch.empty(lat + (4, 3, 3), dtype=torch.complex128, device=device)
    per_t = V // lat[0]
    step = max(1, chunk_sites // per_t)
    for t0 in range(0, lat[0], step):
        t1 = min(lat[0], t0 + step)
        out[t0:t1] = random_hermitian_exp((t1 - t0,) + lat[1:] + (4,), eps, seed * 1000003 + t0, device)
    return out


def unit_gauge(dims, device="cpu"):
    """Free field U_mu(x) = 1."""
    lat = _lat(dims)
    return torch.eye(3, dtype=torch.complex128, device=device).expand(lat + (4, 3, 3)).clone()


def gaussian_spinor(dims, seed=1, nrhs=None, device="cpu"):
    """Complex Gaussian spinor field(s) with N(0,1) real and imaginary parts."""
    lat = _lat(dims)
    shape = lat + (4, 3) if nrhs is None else (nrhs,) + lat + (4, 3)
    g = _gen(seed, device)
    a = torch.randn(shape + (2,), generator=g, dtype=torch.float64, device=device)
    return torch.complex(a[..., 0], a[..., 1])


def point_sources(dims, site=(0, 0, 0, 0), device="cpu"):
    """The 12 spin-colour point sources e_{site, s, c}; rhs index 3*s + c.

    ``site`` is (t, x, y, z)."""
    lat = _lat(dims)
    b = torch.zeros((12,) + lat + (4, 3), dtype=torch.complex128, device=device)
    t, x, y, z = site
    for s in range(4):
        for c in range(3):
            b[3 * s + c, t, z, y, x, s, c] = 1.0
    return b


def random_gauge_transform(dims, seed=7, device="cpu"):
    """A random SU(3) matrix g(x) per site, shape (T, Z, Y, X, 3, 3)."""
    return random_hermitian_exp(_lat(dims), 1.0, seed, device)


def gaussian_vectors(shape, seed, device="cpu"):
    """Complex Gaussian array of an arbitrary shape (e.g. coarse fields, test vectors)."""
    g = _gen(seed, device)
    a = torch.randn(tuple(shape) + (2,), generator=g, dtype=torch.float64, device=device)
    return torch.complex(a[..., 0], a[..., 1])
