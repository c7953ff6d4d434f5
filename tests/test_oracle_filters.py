"""Pins of the oracle's filter functions (Sec. 2.1 and Sec. 4).

Each check compares the oracle with something other than itself: the B3
two-scale relation, the wavelet of eq. splinewl cut along an axis, eq. QU by
numerical quadrature, the compensation condition eq. comp, and values the
paper prints (tests/golden/paper_facts.json).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def test_phi_samples_and_support():
    # B3-spline knots: 2/3 at 0, 1/6 at +-1, 0 at +-2 and beyond (Sec. 4.2).
    assert oracle.phi_b3(0.0) == pytest.approx(2.0 / 3.0, abs=1e-15)
    for x in (1.0, -1.0):
        assert oracle.phi_b3(x) == pytest.approx(1.0 / 6.0, abs=1e-15)
    for x in (2.0, -2.0, 2.5, -3.7, 10.0):
        assert oracle.phi_b3(x) == pytest.approx(0.0, abs=1e-14)
    total, _ = integrate.quad(oracle.phi_b3, -2, 2, points=[-1, 0, 1])
    assert total == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("x", [0.0, 0.3, 1.0, 1.7, 2.5, -0.9, 3.3])
def test_two_scale_relation_fixes_h(x):
    # phi(x/2)/2 = sum_k h_k phi(x - k), k = -2..2, with the oracle's taps.
    h = oracle.starlet_taps()
    rhs = sum(h[k + 2] * oracle.phi_b3(x - k) for k in range(-2, 3))
    assert 0.5 * oracle.phi_b3(x / 2.0) == pytest.approx(rhs, abs=1e-14)


def test_taps_sum_to_one_and_symmetric():
    h = oracle.starlet_taps()
    assert h.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(h, h[::-1])


@pytest.mark.parametrize("eta", np.linspace(0.0, 2.6, 27))
def test_u_starlet_is_axis_cut_of_splinewl(eta):
    # eq. splinewl along y = 0: psi(eta, 0) = 4 phi(0) [phi(2 eta) - phi(eta)/4].
    psi = 4.0 * oracle.phi_b3(0.0) * (oracle.phi_b3(2 * eta) - 0.25 * oracle.phi_b3(eta))
    assert oracle.u_starlet(eta) == pytest.approx(psi, abs=1e-13)


def _q_from_u(u, v):
    # eq. QU: Q(v) = (2 / v^2) int_0^v v' U(v') dv' - U(v)
    kinks = [p for p in (0.5, 1.0, 2.0) if p < v] or None  # knots of the starlet U in eta
    integral, _ = integrate.quad(lambda t: t * u(t), 0.0, v, points=kinks, limit=200, epsabs=1e-14, epsrel=1e-12)
    return 2.0 / (v * v) * integral - u(v)


@pytest.mark.parametrize("eta", [0.05, 0.1, 0.25, 0.5, 0.75, 1.0, 1.3, 1.5, 1.9, 2.0, 2.4, 3.0])
def test_q_starlet_matches_eq_QU(eta):
    # U from the splinewl cut (independent of the printed U and Q).
    def u(t):
        return 4.0 * oracle.phi_b3(0.0) * (oracle.phi_b3(2 * t) - 0.25 * oracle.phi_b3(t))

    assert oracle.q_starlet(eta) == pytest.approx(_q_from_u(u, eta), abs=2e-11)


def test_starlet_compensated_within_two_theta():
    # Sec. 4.3: the starlet U is compensated within 2 theta, and Q vanishes there.
    val, _ = integrate.quad(lambda t: t * oracle.u_starlet(t), 0, 2, points=[0.5, 1.0], epsabs=1e-15)
    assert abs(val) < 1e-13
    for eta in (2.0, 2.2, 3.0, 5.0):
        assert abs(oracle.q_starlet(eta)) < 1e-12
        assert abs(oracle.u_starlet(eta)) < 1e-12


@pytest.mark.parametrize("ell", [1, 3])
@pytest.mark.parametrize("theta", [2.0, 8.0])
def test_s98_compensation_and_QU(ell, theta):
    # eq. comp: int_0^theta v U dv = 0; eq. QU links U and Q (eq. sch).
    val, _ = integrate.quad(lambda v: v * oracle.u_s98(v, theta, ell), 0, theta, epsabs=1e-15)
    assert abs(val) < 1e-13
    for frac in (0.1, 0.4, 0.7, 0.95):
        v = frac * theta
        assert oracle.q_s98(v, theta, ell) == pytest.approx(
            _q_from_u(lambda t: oracle.u_s98(t, theta, ell), v), rel=1e-9, abs=1e-13)
    assert oracle.q_s98(1.01 * theta, theta, ell) == 0.0


@pytest.mark.parametrize("b", [0.5, 4.0])
def test_gauss_QU_and_printed_peak(b):
    theta = 4.0
    for v in (0.5, 2.0, 5.0, 9.0):
        assert oracle.q_gauss(v, theta, b) == pytest.approx(
            _q_from_u(lambda t: oracle.u_gauss(t, theta, b), v), rel=1e-9, abs=1e-14)
    if b == 0.5:
        # Sec. 4.1 prints the position of the JBJ04 Q peak: sqrt(2) theta.
        peak = _golden()["jbj04_q_peak_over_theta"]["value"]
        vs = np.linspace(0.01, 5 * theta, 200001)
        q = np.array([oracle.q_gauss(v, theta, b) for v in vs[::100]])
        vmax = vs[::100][int(np.argmax(q))]
        assert vmax / theta == pytest.approx(peak, abs=2e-3)


def test_golden_supports_match_filters():
    g = _golden()
    # starlet U compensated within 2 theta, S98 within theta (Sec. 4.3).
    assert oracle.default_cut(oracle.STARLET_Q) == g["starlet_compensation_radius_over_theta"]["value"]
    assert oracle.default_cut(oracle.S98) == g["s98_compensation_radius_over_theta"]["value"]
    # theta = 2^j pixels for band j (Sec. 3); J = j_max + 1 (Sec. 5.1).
    for theta, J in zip(g["timing_thetas_px"]["value"], g["timing_J"]["value"]):
        assert theta == 2 ** (J - 1)
