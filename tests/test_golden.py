"""Pins against values the paper prints (fixtures under tests/golden/, each citing its source).

* Table 1 (Sec. 3.1): the parameter set of the method.  The oracle's defaults are that set; the
  library's defaults are that set too, except the number of levels (this library's validated solver
  runs two levels; three are the oracle's default).
* Sec. 2.1: gamma5 = gamma0 gamma1 gamma2 gamma3 is diagonal with the printed diagonal; together with
  the anticommutation relation this fixes the chiral basis that Gamma5 and the spin-chirality split of
  the aggregates (Sec. 2.3) rely on.
"""

import os

import numpy as np

from oracle import dirac, mg

HERE = os.path.join(os.path.dirname(__file__), "golden")


def lines(name):
    """The non-comment lines of a fixture, split into tokens."""
    with open(os.path.join(HERE, name)) as f:
        return [ln.split("#", 1)[0].split() for ln in f if ln.split("#", 1)[0].strip()]


def read_fixture(name):
    """name value(s) per line -> {name: [values]}."""
    return {ln[0]: [float(v) for v in ln[1:]] for ln in lines(name)}


def test_table1_is_the_oracles_default():
    t = read_fixture("table1_parameters.txt")
    p = mg.Params()
    assert p.nlevels == t["n_levels"][0]
    assert p.n_setup == t["n_setup"][0]
    assert p.nv == [t["nv_level1"][0], t["nv_level2"][0]]
    assert list(p.bdims[0]) == t["aggregate_block_level1"] == t["sap_block_level1"]
    assert list(p.bdims[1]) == t["aggregate_block_level2"] == t["sap_block_level2"]
    assert (p.post_smooth, p.nmr) == (t["post_smoothing_steps"][0], t["mr_steps"][0])
    assert (p.kcycle_restart, p.kcycle_max_restarts, p.kcycle_tol) == (
        t["kcycle_restart"][0], t["kcycle_max_restarts"][0], t["kcycle_tol"][0])
    assert (p.coarse_restart, p.coarse_max_restarts, p.coarse_tol, p.delta) == (
        t["coarse_restart"][0], t["coarse_max_restarts"][0], t["coarse_tol"][0], t["coarse_mu_factor"][0])


def test_table1_is_the_librarys_default():
    from paper_1610_02370_gb300 import build
    build.build()  # no-op when the library is current
    from paper_1610_02370_gb300 import ddtm
    t = read_fixture("table1_parameters.txt")
    p = ddtm.ddtm_default_params()
    assert p.n_setup == t["n_setup"][0]
    assert (p.nv[0], p.nv[1]) == (t["nv_level1"][0], t["nv_level2"][0])
    assert list(p.block[0]) == t["aggregate_block_level1"] and list(p.block[1]) == t["aggregate_block_level2"]
    assert (p.post_smooth, p.nmr) == (t["post_smoothing_steps"][0], t["mr_steps"][0])
    assert (p.kcycle_restart, p.kcycle_max_restarts, p.kcycle_tol) == (
        t["kcycle_restart"][0], t["kcycle_max_restarts"][0], t["kcycle_tol"][0])
    assert (p.coarse_restart, p.coarse_max_restarts, p.coarse_tol, p.delta) == (
        t["coarse_restart"][0], t["coarse_max_restarts"][0], t["coarse_tol"][0], t["coarse_mu_factor"][0])
    assert p.restart_tol == t["outer_restart_tol"][0]


def test_gamma5_is_the_printed_diagonal():
    (row,) = lines("gamma5.txt")
    diag = np.array([float(v) for v in row])
    g, g5 = dirac.gamma_matrices()
    assert np.array_equal(g5, np.diag(diag))
    assert np.allclose(g[0] @ g[1] @ g[2] @ g[3], np.diag(diag), atol=1e-15)
    for a in range(4):
        for b in range(4):
            assert np.allclose(g[a] @ g[b] + g[b] @ g[a], 2.0 * np.eye(4) * (a == b), atol=1e-15)
    assert np.array_equal(dirac.apply_Gamma5(np.ones((1, 1, 1, 1, 4, 3), dtype=complex))[0, 0, 0, 0, :, 0], diag)
