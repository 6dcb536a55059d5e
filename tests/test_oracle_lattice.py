"""Pins of the oracle's lattice constants and equilibrium (Sect. 2.2).

The velocity set is compared with Table 1 as printed; the weights and the
equilibrium are checked against the moment identities that define a D3Q19
lattice with c_s^2 = 1/3 (isotropy up to fourth order, and the Maxwellian's
density, momentum and momentum-flux moments that Eq. 9 is the second-order
expansion of), not against a retyped formula.
"""
import numpy as np
import pytest

import oracle


def test_tables_match_table1(d3q19):
    c_paper, w_paper = d3q19
    c, w, opp = oracle.tables()
    assert np.array_equal(c, c_paper)
    assert np.allclose(w, w_paper, rtol=0, atol=1e-17)


def test_opposites_are_i_plus_9(d3q19):
    c, _, opp = oracle.tables()
    for i in range(1, 10):
        assert opp[i] == i + 9 and opp[i + 9] == i
        assert np.array_equal(c[opp[i]], -c[i])
    assert opp[0] == 0


def test_weight_isotropy(d3q19):
    c, w = d3q19
    c = c.astype(float)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w @ c, 0.0, atol=1e-16)
    second = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(second, np.eye(3) / 3.0, atol=1e-16)
    third = np.einsum("i,ia,ib,ic->abc", w, c, c, c)
    assert np.allclose(third, 0.0, atol=1e-16)
    fourth = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(fourth, iso, atol=1e-16)


@pytest.mark.parametrize("rho,u", [(1.0, (0.0, 0.0, 0.0)), (1.03, (0.04, -0.02, 0.01)),
                                   (0.97, (-0.05, 0.03, 0.07))])
def test_equilibrium_moments(d3q19, rho, u):
    c, _ = d3q19
    c = c.astype(float)
    u = np.array(u)
    f = oracle.feq(rho, u)
    assert abs(f.sum() - rho) < 1e-14
    assert np.allclose(f @ c, rho * u, atol=1e-15)
    flux = np.einsum("i,ia,ib->ab", f, c, c)
    assert np.allclose(flux, rho * (np.eye(3) / 3.0 + np.outer(u, u)), atol=1e-15)


def test_rest_equilibrium_is_the_weights(d3q19):
    _, w = d3q19
    f = oracle.feq(1.0, np.zeros(3))
    assert np.array_equal(f, oracle.tables()[1])
    assert np.allclose(f, w, rtol=0, atol=1e-17)


def test_equilibrium_galilean_pair_identity(d3q19):
    """f^eq_i(u) - f^eq_opp(i)(u) = 6 w_i c_i.u at rho = 1: the quadratic terms
    are even in c, which is what makes the moving-wall term of Eq. (21) exact
    for a boundary moving with a uniform flow."""
    c, w = d3q19
    _, _, opp = oracle.tables()
    u = np.array([0.03, -0.015, 0.02])
    f = oracle.feq(1.0, u)
    for i in range(19):
        assert abs(f[i] - f[opp[i]] - 6 * w[i] * (c[i] @ u)) < 1e-16
