"""Host side of the moving-body consumer: the prescribed rigid motion moves
the reference point by u t and turns the body frame by omega t (no GPU)."""

import math

import numpy as np

import oracle as O
from paper_2609_10165_b300 import inputs as I
from paper_2609_10165_b300.moving import RigidMotion


def test_rigid_motion_moves_and_turns_the_body():
    m = RigidMotion(I.ellipse(0.1, -0.2, 0.5, 0.3, 0.4), velocity=(0.2, 0.1, 0.0), omega=0.5)
    b = m.at(2.0)
    assert np.allclose(b["centre"][:2], [0.5, 0.0])
    # the turned body is the original one rotated by omega t about its centre
    want = I.ellipse(0.5, 0.0, 0.5, 0.3, 0.4 + 1.0)
    assert np.allclose(b["rot"], want["rot"], atol=1e-15)
    # a point of the boundary stays on the boundary under the motion
    body0 = O.Body.from_dict(m.at(0.0))
    body1 = O.Body.from_dict(b)
    th = 1.0
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    X0 = np.array([[0.1 + 0.5 * math.cos(0.4), -0.2 + 0.5 * math.sin(0.4)]])   # end of the major axis
    X1 = (R @ (X0[0] - np.array([0.1, -0.2])) + np.array([0.5, 0.0]))[None, :]
    assert abs(O.closest_point(body0, X0)[0][0]) < 1e-12
    assert abs(O.closest_point(body1, X1)[0][0]) < 1e-12
