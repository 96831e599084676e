"""Pins of the oracle's equilibrium and forcing terms (Eqs. feq, f, rho, v).

Each check is a property the mathematics fixes, not a re-typed formula:
the moments an incompressible equilibrium must reproduce and the moments
of the Guo forcing term.
"""
import numpy as np
import pytest

import oracle

CS2 = 1.0 / 3.0


def test_weights_and_isotropy(d3q19):
    # f^eq at rest with P = c_s^2 returns the weights: sum 1, second moment c_s^2 I,
    # fourth moment c_s^4 (d_ab d_cd + d_ac d_bd + d_ad d_bc)
    w = oracle.feq(CS2, [0.0, 0.0, 0.0])
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(w[0], 1 / 3) and np.allclose(w[1:7], 1 / 18) and np.allclose(w[7:], 1 / 36)
    m2 = np.einsum("i,ia,ib->ab", w, d3q19, d3q19)
    assert np.allclose(m2, CS2 * np.eye(3), atol=1e-16)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, d3q19, d3q19, d3q19, d3q19)
    d = np.eye(3)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(m4, iso, atol=1e-16)
    # odd moments vanish
    assert np.allclose(np.einsum("i,ia->a", w, d3q19), 0.0, atol=1e-17)


@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments(d3q19, seed):
    rng = np.random.default_rng(seed)
    P = CS2 * (1 + 0.05 * rng.standard_normal())
    v = 0.05 * rng.standard_normal(3)
    f = oracle.feq(P, v)
    # Eq. rho: P = c_s^2 sum f ; Eq. v (no force): rho0 v = sum e f
    assert f.sum() * CS2 == pytest.approx(P, rel=1e-15)
    assert np.allclose(d3q19.T @ f, v, rtol=1e-14, atol=1e-17)
    # momentum flux of the incompressible model: P d_ab + rho0 v_a v_b
    m2 = np.einsum("i,ia,ib->ab", f, d3q19, d3q19)
    assert np.allclose(m2, P * np.eye(3) + np.outer(v, v), rtol=1e-13, atol=1e-17)


@pytest.mark.parametrize("tau", [0.55, 0.8, 1.3])
def test_forcing_moments(d3q19, tau):
    rng = np.random.default_rng(int(tau * 100))
    v = 0.05 * rng.standard_normal(3)
    b = 1e-3 * rng.standard_normal(3)
    F = oracle.forcing(tau, v, b)
    k = 1.0 - 1.0 / (2.0 * tau)
    # zeroth moment 0, first moment (1 - 1/2tau) b,
    # second moment (1 - 1/2tau)(v b + b v)
    assert abs(F.sum()) < 1e-18
    assert np.allclose(d3q19.T @ F, k * b, rtol=1e-13, atol=1e-19)
    m2 = np.einsum("i,ia,ib->ab", F, d3q19, d3q19)
    assert np.allclose(m2, k * (np.outer(v, b) + np.outer(b, v)), rtol=1e-12, atol=1e-19)


def test_forcing_linear_in_b():
    v = [0.01, -0.02, 0.03]
    F1 = oracle.forcing(0.8, v, [1e-3, 0, 0])
    F2 = oracle.forcing(0.8, v, [0, 2e-3, 0])
    F12 = oracle.forcing(0.8, v, [1e-3, 2e-3, 0])
    assert np.allclose(F1 + F2, F12, atol=1e-19)
    assert np.allclose(oracle.forcing(0.8, v, [0, 0, 0]), 0.0)
