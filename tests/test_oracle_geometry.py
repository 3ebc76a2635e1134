"""Pins of the oracle's closest-point geometry (Sec. 3.1, Eq. signed_distance)
against brute force and closed forms."""

import math
import os

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

import oracle as O
from paper_2609_10165_b300 import inputs as I


def _check_foot(body, X, psi, n):
    S = X + psi[:, None] * n
    # S lies on the boundary: the closest point of S to the body is S itself
    psi2, _ = O.closest_point(body, S)
    assert np.max(np.abs(psi2)) < 1e-12
    # unit normal
    assert np.allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-14)


def test_circle_closed_form():
    body = O.Body.from_dict(I.circle(0.1, -0.2, 0.5))
    rng = np.random.default_rng(0)
    X = rng.uniform(-1, 1, size=(500, 2))
    psi, n = O.closest_point(body, X)
    rho = np.hypot(X[:, 0] - 0.1, X[:, 1] + 0.2)
    assert np.allclose(psi, 0.5 - rho, atol=1e-15)
    assert np.array_equal(O.inside(body, X), psi >= 0)
    _check_foot(body, X, psi, n)


def test_sphere_closed_form():
    body = O.Body.from_dict(I.sphere(0.0, 0.1, 0.0, 0.5))
    rng = np.random.default_rng(1)
    X = rng.uniform(-1, 1, size=(500, 3))
    psi, n = O.closest_point(body, X)
    rho = np.linalg.norm(X - np.array([0.0, 0.1, 0.0]), axis=1)
    assert np.allclose(psi, 0.5 - rho, atol=1e-15)
    _check_foot(body, X, psi, n)


def _ellipse_brute(a, b, q):
    # minimise the distance over the ellipse angle: dense grid then bounded refine
    th = np.linspace(0, 2 * math.pi, 20001)
    d2 = (a * np.cos(th) - q[0]) ** 2 + (b * np.sin(th) - q[1]) ** 2
    k = int(np.argmin(d2))
    res = minimize_scalar(lambda t: (a * math.cos(t) - q[0]) ** 2 + (b * math.sin(t) - q[1]) ** 2,
                          bounds=(th[max(k - 1, 0)], th[min(k + 1, th.size - 1)]), method="bounded",
                          options={"xatol": 1e-14})
    return math.sqrt(res.fun)


def test_ellipse_vs_brute_force():
    rng = np.random.default_rng(2)
    for trial in range(4):
        a, b = rng.uniform(0.2, 0.8, size=2)
        ang = rng.uniform(0, math.pi)
        body = O.Body.from_dict(I.ellipse(0.03, -0.02, a, b, ang))
        X = rng.uniform(-1, 1, size=(60, 2))
        psi, n = O.closest_point(body, X)
        R = np.array(I.rot2(ang)).reshape(3, 3)[:2, :2]
        for k in range(X.shape[0]):
            q = R.T @ (X[k] - np.array([0.03, -0.02]))
            dist = _ellipse_brute(a, b, q)
            assert abs(abs(psi[k]) - dist) < 1e-9, (abs(psi[k]), dist)
        _check_foot(body, X, psi, n)


def _airfoil_dist_brute(t, c, q, M=1_000_000):
    u = np.linspace(0.0, 1.0, M + 1)
    x = c * u * u
    a0, a1, a2, a3, a4 = 0.2969, -0.1260, -0.3516, 0.2843, -0.1015
    y = 5 * t * c * (a0 * u + a1 * u ** 2 + a2 * u ** 4 + a3 * u ** 6 + a4 * u ** 8)
    qy = abs(q[1])
    d_up = np.min((x - q[0]) ** 2 + (y - qy) ** 2)
    yte = y[-1]
    d_base = (q[0] - c) ** 2 + (qy - min(qy, yte)) ** 2
    return math.sqrt(min(d_up, d_base))


def test_airfoil_vs_brute_force():
    rng = np.random.default_rng(3)
    bd = I.airfoil(0.0, 0.0, 0.12, 1.0, 5.0)
    body = O.Body.from_dict(bd)
    R = np.array(bd["rot"]).reshape(3, 3)[:2, :2]
    # points near the surface (the band where psi matters) plus a few far ones
    qs = []
    for _ in range(40):
        u = rng.uniform(0, 1)
        xb = u * u
        yt = O.geometry.airfoil_half_thickness(0.12, 1.0, xb)
        sgn = rng.choice([-1, 1])
        qs.append([xb + rng.normal() * 0.004, sgn * yt + rng.normal() * 0.004])
    qs += [[1.003, 0.0021], [1.002, -0.004], [-0.003, 0.0005], [0.5, 0.0], [1.2, 0.3]]
    qs = np.array(qs)
    X = (R @ qs.T).T
    psi, n = O.closest_point(body, X)
    for k in range(qs.shape[0]):
        dist = _airfoil_dist_brute(0.12, 1.0, qs[k])
        # sampling resolution of the brute force (du = 1e-6) bounds its own error
        assert abs(abs(psi[k]) - dist) < 1e-8, (k, abs(psi[k]), dist)
        assert abs(psi[k]) <= dist + 1e-15
    assert np.array_equal(O.inside(body, X), psi >= 0)
    _check_foot(body, X, psi, n)


def test_airfoil_is_convex_and_trailing_edge():
    # y_t'' < 0 on (0, 1]: the closed section is convex (needed for acyclic levels)
    x = np.linspace(1e-4, 1.0, 10001)
    y = O.geometry.airfoil_half_thickness(0.12, 1.0, x)
    d2 = np.diff(y, 2)
    assert np.all(d2 < 0)
    # open trailing edge half-thickness of the standard coefficients
    assert abs(O.geometry.airfoil_half_thickness(0.12, 1.0, 1.0) - 0.00126) < 1e-5
