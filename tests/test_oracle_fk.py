"""Pins of the oracle's forward kinematics (Sec. II-A, Eqs. 1-2) against hand
derivations, the textbook planar chain, the DH convention written as a product
of elementary transforms, and invariants of rigid links."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_06451_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fk_closed_form.json")


def _val(x):
    if isinstance(x, str):
        return {"pi/2": math.pi / 2, "-pi/2": -math.pi / 2, "0": 0.0}[x]
    return float(x)


def _chain_from_golden(g):
    dh = np.array([[_val(l["a"]), _val(l["alpha"]), _val(l["d"]), 0.0, 0.0] for l in g["chain"]])
    return dh


def test_closed_form_origins():
    g = json.load(open(GOLDEN))
    dh = _chain_from_golden(g)
    for case in g["cases"]:
        q = np.array([_val(v) for v in case["q"]])
        T = O.frames(dh, np.eye(4), q)
        np.testing.assert_allclose(T[:, :3, 3], np.array(case["origins"]), atol=1e-12)


def test_planar_chain_matches_textbook():
    # all twists zero: x = sum a_i cos(theta_1 + .. + theta_i), y likewise, z = sum d_i
    rng = np.random.default_rng(1)
    D = 5
    dh = np.zeros((D, 5))
    dh[:, 0] = rng.uniform(0.1, 0.5, D)
    dh[:, 2] = rng.uniform(0.0, 0.2, D)
    for _ in range(20):
        q = rng.uniform(-math.pi, math.pi, D)
        T = O.frames(dh, np.eye(4), q)
        cum = np.cumsum(q)
        x = np.cumsum(dh[:, 0] * np.cos(cum))
        y = np.cumsum(dh[:, 0] * np.sin(cum))
        z = np.cumsum(dh[:, 2])
        np.testing.assert_allclose(T[1:, 0, 3], x, atol=1e-13)
        np.testing.assert_allclose(T[1:, 1, 3], y, atol=1e-13)
        np.testing.assert_allclose(T[1:, 2, 3], z, atol=1e-13)


def _rz(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[c, -s, 0, 0], [s, c, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1.0]])


def _rx(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[1, 0, 0, 0], [0, c, -s, 0], [0, s, c, 0], [0, 0, 0, 1.0]])


def _tz(d):
    m = np.eye(4)
    m[2, 3] = d
    return m


def _tx(a):
    m = np.eye(4)
    m[0, 3] = a
    return m


@pytest.mark.parametrize("arm_fn", [synth.arm_3dof, synth.arm_7dof])
def test_dh_equals_elementary_product(arm_fn):
    # standard DH: i-1 A_i = Rz(theta) Tz(d) Tx(a) Rx(alpha)
    arm = arm_fn(7)
    base = np.eye(4)
    base[:3, 3] = [0.1, -0.2, 0.3]
    base[:3, :3] = _rz(0.4)[:3, :3] @ _rx(-0.3)[:3, :3]
    q = synth.uniform_configs(11, 25, arm.D, arm.qlim).astype(np.float64)
    for k in range(q.shape[0]):
        T = O.frames(arm.dh, base, q[k])
        W = base.copy()
        for i in range(arm.D):
            a, al, d, th0, _ = arm.dh[i]
            W = W @ _rz(q[k, i] + th0) @ _tz(d) @ _tx(a) @ _rx(al)
            np.testing.assert_allclose(T[i + 1], W, atol=1e-13)


def test_joint_offsets_add_to_the_joint_values():
    # theta = q + theta0 (Eq. 1): one link of length 1 with theta0 = pi/2
    # points along y at q = 0 and along x at q = -pi/2
    dh = np.array([[1.0, 0.0, 0.0, math.pi / 2, 0.0]])
    np.testing.assert_allclose(O.frames(dh, np.eye(4), np.array([0.0]))[1, :3, 3], [0, 1, 0], atol=1e-15)
    np.testing.assert_allclose(O.frames(dh, np.eye(4), np.array([-math.pi / 2]))[1, :3, 3], [1, 0, 0], atol=1e-15)
    # and every frame of a twisted chain with offsets is the elementary product
    arm = synth.arm_7dof(5)
    dh = arm.dh.copy()
    dh[:, 3] = np.random.default_rng(3).uniform(-math.pi, math.pi, arm.D)
    q = synth.uniform_configs(12, 10, arm.D, arm.qlim).astype(np.float64)
    for k in range(q.shape[0]):
        T = O.frames(dh, np.eye(4), q[k])
        W = np.eye(4)
        for i in range(arm.D):
            a, al, d, th0, _ = dh[i]
            W = W @ _rz(q[k, i] + th0) @ _tz(d) @ _tx(a) @ _rx(al)
            np.testing.assert_allclose(T[i + 1], W, atol=1e-13)


def test_link_length_invariant():
    arm = synth.arm_7dof(3)
    q = synth.uniform_configs(5, 200, arm.D, arm.qlim).astype(np.float64)
    L = np.hypot(arm.dh[:, 0], arm.dh[:, 2])
    for k in range(q.shape[0]):
        o = O.frames(arm.dh, arm.base, q[k])[:, :3, 3]
        np.testing.assert_allclose(np.linalg.norm(np.diff(o, axis=0), axis=1), L, rtol=0, atol=1e-14)


def test_control_points_with_offsets():
    # FK_m(x) = pos(wA_{j_m} T_m) with T_m a translation (Eq. 2)
    arm = synth.arm_7dof(4)
    rng = np.random.default_rng(2)
    cj = np.array([0, 2, 5, 7, 7], dtype=np.int32)
    co = rng.uniform(-0.2, 0.2, (5, 3))
    arm2 = synth.Arm(arm.dh, arm.base, cj, co, arm.qlim)
    q = synth.uniform_configs(6, 10, arm.D, arm.qlim).astype(np.float64)
    cp = O.fk_points(arm2, q)
    for k in range(q.shape[0]):
        T = O.frames(arm.dh, arm.base, q[k])
        for m in range(5):
            np.testing.assert_allclose(cp[k, m], T[cj[m], :3, :3] @ co[m] + T[cj[m], :3, 3], atol=1e-14)


def test_prismatic_joint_slides_along_z():
    dh = np.array([[0.0, 0.0, 0.5, 0.0, 1.0], [0.3, 0.0, 0.0, 0.0, 0.0]])
    T0 = O.frames(dh, np.eye(4), np.array([0.0, 0.0]))
    T1 = O.frames(dh, np.eye(4), np.array([0.25, 0.0]))
    np.testing.assert_allclose(T1[1, :3, 3] - T0[1, :3, 3], [0, 0, 0.25], atol=1e-15)
    np.testing.assert_allclose(T1[2, :3, 3], [0.3, 0.0, 0.75], atol=1e-15)


def test_invalid_control_point_frame_rejected():
    arm = synth.arm_3dof(0)
    bad = synth.Arm(arm.dh, arm.base, np.array([0, 4], dtype=np.int32), np.zeros((2, 3)), arm.qlim)
    with pytest.raises(ValueError):
        O.fk_points(bad, np.zeros((1, 3)))
