"""Oracle: lattice blocks V_j = T_j x Z_j x Y_j x X_j (Sec. 2.3) and per-block reductions.

TEST INFRASTRUCTURE ONLY.  ``bdims`` is given per direction mu = (t, x, y, z);
every lattice extent must be a multiple of its block extent.  Blocks are
coloured red (0) / black (1) by the parity of the sum of their block
coordinates (Sec. 2.4, checkerboard of blocks).
"""

import numpy as np

from .dirac import AXIS


def axis_blocks(lat, bdims):
    """Block extents in array-axis order (T, Z, Y, X)."""
    b = [0, 0, 0, 0]
    for mu in range(4):
        b[AXIS[mu]] = bdims[mu]
    for n, e in zip(lat, b):
        if n % e:
            raise ValueError("lattice extent %d not divisible by block extent %d" % (n, e))
    return tuple(b)


def coarse_lat(lat, bdims):
    b = axis_blocks(lat, bdims)
    return tuple(n // e for n, e in zip(lat, b))


def block_sum(f, lat, bdims):
    """Sum of f over the sites of each block and over every trailing axis.

    f has shape lat + rest; returns an array of shape coarse_lat.
    """
    b = axis_blocks(lat, bdims)
    shp = []
    for n, e in zip(lat, b):
        shp += [n // e, e]
    g = f.reshape(tuple(shp) + (-1,))
    return g.sum(axis=(1, 3, 5, 7, 8))


def block_sum_keep(f, lat, bdims, nkeep):
    """Per-block sum over sites and over the trailing axes beyond the first ``nkeep``
    leading (non-lattice) axes.  f has shape keep + lat + rest."""
    keep = f.shape[:nkeep]
    b = axis_blocks(lat, bdims)
    shp = []
    for n, e in zip(lat, b):
        shp += [n // e, e]
    g = f.reshape(keep + tuple(shp) + (-1,))
    ax = tuple(nkeep + a for a in (1, 3, 5, 7, 8))
    return g.sum(axis=ax)


def broadcast(c, lat, bdims, dofdims=0):
    """Expand a per-block array (coarse_lat + extra) to sites (lat + extra), then add
    ``dofdims`` singleton axes so it multiplies a field."""
    b = axis_blocks(lat, bdims)
    out = c
    for ax, e in enumerate(b):
        out = np.repeat(out, e, axis=ax)
    return out.reshape(out.shape + (1,) * dofdims)


def block_colour(lat, bdims):
    """Colour (0 red, 1 black) of the block containing each site."""
    cl = coarse_lat(lat, bdims)
    g = np.indices(cl).sum(axis=0) % 2
    return broadcast(g, lat, bdims)


def crossing_mask(lat, bdims, d, sign):
    """True where the hop x -> x + sign*d_hat leaves the block of x."""
    b = axis_blocks(lat, bdims)[AXIS[d]]
    n = lat[AXIS[d]]
    coord = np.arange(n) % b
    edge = (coord == b - 1) if sign > 0 else (coord == 0)
    shp = [1, 1, 1, 1]
    shp[AXIS[d]] = n
    return np.broadcast_to(edge.reshape(shp), lat)


def check_colouring(lat, bdims):
    """Red-black SAP needs an even number (>= 2) of blocks in every direction, so that
    two blocks of one colour never touch."""
    for n in coarse_lat(lat, bdims):
        if n < 2 or n % 2:
            raise ValueError("red-black block colouring needs an even number of blocks per direction")
