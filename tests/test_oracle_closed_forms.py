"""Pins of the oracle's closed forms (Secs. 4-5) against the Appendix A
Vandermonde system solved directly, and against the properties the paper
states for the weights."""

import numpy as np
import pytest

import oracle as O
from oracle.reconstruct import ghost_weights, vandermonde_ghost_value, ghost_value


def _random_geometry(rng, d, placement="HGC"):
    h = rng.uniform(0.5, 2.0, size=d)
    n = rng.normal(size=d)
    n /= np.linalg.norm(n)
    e = np.where(n >= 0, 1, -1)
    r = np.ones(d, dtype=int) if placement != "ES" else rng.integers(1, 3, size=d)
    # |psi| small enough that every alpha_i stays well away from 1
    psi = rng.uniform(-0.45, 0.45) * min(h)
    return h, psi, n, e, r


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("bc", [O.DIRICHLET, O.NEUMANN])
@pytest.mark.parametrize("pl", ["HGC", "ES"])
def test_closed_form_equals_vandermonde(d, bc, pl):
    rng = np.random.default_rng(10 * d + bc)
    K = 3 if d == 2 else 7
    for _ in range(200):
        h, psi, n, e, r = _random_geometry(rng, d, pl)
        phi = rng.uniform(-1, 1, size=K)
        datum = rng.uniform(-1, 1)
        a = ghost_value(h, psi, n, e, r, bc, phi, datum)
        b = vandermonde_ghost_value(h, psi, n, e, r, bc, phi, datum)
        assert abs(a - b) <= 1e-12 * (1 + np.abs(phi).sum() + abs(datum)), (a, b)


@pytest.mark.parametrize("d", [2, 3])
def test_neumann_weights_sum_to_one(d):
    # Neumann: the weights on the stencil values sum to 1 (constants are
    # reproduced with zero normal derivative), Eqs. phi_G_Neu_2d / _3d.
    rng = np.random.default_rng(5 + d)
    for _ in range(200):
        h, psi, n, e, r = _random_geometry(rng, d)
        w, ws = ghost_weights(h, psi, n, e, r, O.NEUMANN)
        assert abs(w.sum() - 1.0) < 1e-13


@pytest.mark.parametrize("d", [2, 3])
def test_dirichlet_weights_with_ws_sum_to_one(d):
    rng = np.random.default_rng(7 + d)
    for _ in range(200):
        h, psi, n, e, r = _random_geometry(rng, d)
        w, ws = ghost_weights(h, psi, n, e, r, O.DIRICHLET)
        assert abs(w.sum() + ws - 1.0) < 1e-12


@pytest.mark.parametrize("d", [2, 3])
def test_neumann_weights_independent_of_normal_sense(d):
    # Sec. 5: "The reconstruction weights are independent of the sense of the
    # surface-normal vector": flipping n (same stencil) keeps w_1..w_K and
    # flips w_s, which multiplies dphi/dn (also flipped).
    rng = np.random.default_rng(11 + d)
    for _ in range(100):
        h, psi, n, e, r = _random_geometry(rng, d)
        w1, s1 = ghost_weights(h, psi, n, e, r, O.NEUMANN)
        # same boundary point S = G + psi n, reversed normal: psi -> -psi, n -> -n
        w2, s2 = ghost_weights(h, -psi, -n, e, r, O.NEUMANN)
        assert np.allclose(w1, w2, rtol=0, atol=1e-13)
        assert abs(s1 + s2) < 1e-13 * (1 + abs(s1))


def test_2d_zero_normal_component_special_cases():
    # Sec. 4 note: n_x = 0 gives x_s = x_1, w1 = 0, w2 = 1 (Neumann); n_y = 0
    # gives w1 = 1, w2 = 0.  Dirichlet: the weights of x-offset members vanish.
    h = (1.0, 1.0)
    w, ws = ghost_weights(h, 0.3, np.array([0.0, 1.0]), np.array([1, 1]), np.array([1, 1]), O.NEUMANN)
    assert w[0] == 0.0 and w[1] == 1.0 and w[2] == 0.0
    w, ws = ghost_weights(h, 0.3, np.array([1.0, 0.0]), np.array([1, 1]), np.array([1, 1]), O.NEUMANN)
    assert w[0] == 1.0 and w[1] == 0.0 and w[2] == 0.0
    w, ws = ghost_weights(h, 0.3, np.array([0.0, -1.0]), np.array([1, -1]), np.array([1, 1]), O.DIRICHLET)
    assert w[0] == 0.0 and w[2] == 0.0


def test_3d_zero_normal_component_removes_offset_members():
    h = (1.0, 1.0, 1.0)
    n = np.array([0.0, 0.6, 0.8])
    for bc in (O.DIRICHLET, O.NEUMANN):
        w, ws = ghost_weights(h, 0.25, n, np.array([1, 1, 1]), np.array([1, 1, 1]), bc)
        offs = O.stencil_offsets(3)
        for k, o in enumerate(offs):
            if o[0] == 1:
                assert w[k] == 0.0, (bc, k, w)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("bc", [O.DIRICHLET, O.NEUMANN])
def test_multilinear_exactness_single_ghost(d, bc):
    # Secs. 4-5: the reconstruction is exact for phi = C0 + C1 x + ... (bi/tri-linear).
    rng = np.random.default_rng(3 + d + 10 * bc)
    offs = O.stencil_offsets(d)
    for _ in range(100):
        h, psi, n, e, r = _random_geometry(rng, d, "ES")
        C = rng.uniform(-1, 1, size=4 if d == 2 else 8)

        def phi(p):
            if d == 2:
                x, y = p
                return C[0] + C[1] * x + C[2] * y + C[3] * x * y
            x, y, z = p
            return C[0] + C[1] * x + C[2] * y + C[3] * z + C[4] * x * y + C[5] * y * z + C[6] * x * z + C[7] * x * y * z

        def grad(p):
            if d == 2:
                x, y = p
                return np.array([C[1] + C[3] * y, C[2] + C[3] * x])
            x, y, z = p
            return np.array([C[1] + C[4] * y + C[6] * z + C[7] * y * z,
                             C[2] + C[4] * x + C[5] * z + C[7] * x * z,
                             C[3] + C[5] * y + C[6] * x + C[7] * x * y])

        x2 = np.array([r[a] * e[a] * h[a] for a in range(d)])
        S = psi * n
        members = [phi(np.array(o) * x2) for o in offs]
        datum = phi(S) if bc == O.DIRICHLET else float(grad(S) @ n)
        val = ghost_value(h, psi, n, e, r, bc, members, datum)
        assert abs(val - phi(np.zeros(d))) < 1e-12 * (1 + np.abs(C).sum())
