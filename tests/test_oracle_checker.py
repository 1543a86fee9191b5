"""Pins of the oracle's geometric checker (sphere-swept links vs boxes, the
stand-in for the paper's geometric collision detector, Sec. IV) and of the
correctness metrics (Eqs. 10-12)."""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1910_06451_gb300 import synth


def _point_box_dist(p, lo, hi):
    return float(np.linalg.norm(np.maximum(np.maximum(lo - p, 0.0), p - hi)))


def test_segment_box_closed_forms():
    lo, hi = np.array([0.0, 0.0, 0.0]), np.array([1.0, 1.0, 1.0])
    # parallel to the top face at height 1.3: distance 0.3 everywhere over the box
    assert O.seg_box_dist2([0.2, 0.5, 1.3], [0.8, 0.5, 1.3], lo, hi) == pytest.approx(0.09, rel=1e-14)
    # passes through the box
    assert O.seg_box_dist2([-1.0, 0.5, 0.5], [2.0, 0.5, 0.5], lo, hi) == 0.0
    # degenerate segment = point
    assert O.seg_box_dist2([2.0, 3.0, 1.0], [2.0, 3.0, 1.0], lo, hi) == pytest.approx(1.0 + 4.0, rel=1e-14)
    # skew segment passing an edge: closest approach computed by hand.  The
    # segment (2, t, -1) .. (2, t, 3) for t fixed misses the edge x=1,z in [0,1]
    assert O.seg_box_dist2([2.0, 0.5, -1.0], [2.0, 0.5, 3.0], lo, hi) == pytest.approx(1.0, rel=1e-14)
    # diagonal towards a corner: from (2,2,2) to (3,3,3); nearest point (2,2,2) -> corner (1,1,1)
    assert O.seg_box_dist2([2.0, 2.0, 2.0], [3.0, 3.0, 3.0], lo, hi) == pytest.approx(3.0, rel=1e-14)


def test_segment_box_against_dense_sampling():
    # the distance is a minimum over the segment of a 1-Lipschitz function, so
    # sampling at spacing h overestimates it by at most h |seg| / 2
    rng = np.random.default_rng(0)
    for _ in range(300):
        p0, p1 = rng.uniform(-1.5, 1.5, 3), rng.uniform(-1.5, 1.5, 3)
        c = rng.uniform(-0.5, 0.5, 3)
        h = rng.uniform(0.05, 0.4, 3)
        lo, hi = c - h, c + h
        d = math.sqrt(O.seg_box_dist2(p0, p1, lo, hi))
        ts = np.linspace(0.0, 1.0, 2001)
        ds = min(_point_box_dist(p0 + t * (p1 - p0), lo, hi) for t in ts)
        L = np.linalg.norm(p1 - p0)
        assert d <= ds + 1e-12
        assert ds - d <= 0.5 * L / 2000 + 1e-12


def _brute_labels(scene, q, spacing=0.002):
    """Brute force: sample points along every link and test point-box distance."""
    arm = scene.arm
    out = []
    for k in range(q.shape[0]):
        o = O.frames(arm.dh, arm.base, q[k])[:, :3, 3]
        dmin = np.inf
        for i in range(1, arm.D + 1):
            L = np.linalg.norm(o[i] - o[i - 1])
            ts = np.linspace(0, 1, max(2, int(L / spacing) + 2))
            pts = o[i - 1] + ts[:, None] * (o[i] - o[i - 1])
            for b in scene.boxes:
                gap = np.maximum(np.maximum(b[:3] - pts, 0.0), pts - b[3:])
                dmin = min(dmin, float(np.min(np.linalg.norm(gap, axis=1))))
        out.append(dmin)
    return np.array(out)


@pytest.mark.parametrize("D", [2, 3])
def test_labels_agree_with_brute_force_on_a_grid(D):
    # full joint grid of a 2- or 3-DOF arm; agreement required outside the
    # sampling band of half a spacing
    arm = synth.arm_3dof(5)
    if D == 2:
        arm = synth.Arm(arm.dh[:2], arm.base, np.arange(3, dtype=np.int32), np.zeros((3, 3)), arm.qlim)
    scene = synth.Scene(arm, synth.random_boxes(5, 6), 0.03)
    g = np.linspace(-math.pi, math.pi, 13 if D == 3 else 40)
    q = np.array(list(itertools.product(g, repeat=D)))
    y = O.check(scene, q)
    spacing = 0.002
    dmin = _brute_labels(scene, q, spacing)
    sure_hit = dmin <= scene.radius
    sure_free = dmin > scene.radius + spacing / 2
    assert np.all(y[sure_hit] == 1)
    assert np.all(y[sure_free] == -1)
    assert 0 < np.sum(y == 1) < len(y)


def test_special_cases():
    arm = synth.arm_3dof(2)
    q = synth.uniform_configs(3, 50, arm.D, arm.qlim).astype(np.float64)
    # a box around the tip of the arm: always a collision
    for k in range(10):
        tip = O.frames(arm.dh, arm.base, q[k])[-1, :3, 3]
        sc = synth.Scene(arm, np.concatenate([tip - 0.01, tip + 0.01])[None], 0.03)
        assert O.check(sc, q[k:k + 1])[0] == 1
    # a box beyond the reach plus the radius: never
    reach = float(np.sum(np.hypot(arm.dh[:, 0], arm.dh[:, 2])))
    far = np.array([[reach + 0.1, -1, -1, reach + 1, 1, 1]])
    assert np.all(O.check(synth.Scene(arm, far, 0.03), q) == -1)
    # touching counts: a box whose face is exactly the radius away from the base link's start
    touch = np.array([[-0.5, -0.5, 0.03, 0.5, 0.5, 0.5]])
    assert O.check(synth.Scene(arm, touch, 0.03), q[:1])[0] == 1


def test_touching_the_first_link_is_a_collision():
    # one link from the origin to (1, 0, 0) (a = 1, q = 0) and a box whose
    # lower y face lies 0.25 from it: at radius 0.25 the swept link touches
    # the box (distance equal to the radius counts), at 0.2499 it does not
    box = np.array([[0.2, 0.25, -1.0, 0.8, 1.0, 1.0]])
    one = synth.Arm(np.array([[1.0, 0.0, 0.0, 0.0, 0.0]]), np.eye(4), np.array([1], dtype=np.int32),
                    np.zeros((1, 3)), math.pi)
    q1 = np.zeros((1, 1))
    assert O.check(synth.Scene(one, box, 0.25), q1)[0] == 1
    assert O.check(synth.Scene(one, box, 0.2499), q1)[0] == -1
    # a second link turned away (to (1, -1, 0)) stays clear, so the first
    # link alone decides
    two = synth.Arm(np.array([[1.0, 0.0, 0.0, 0.0, 0.0]] * 2), np.eye(4), np.array([2], dtype=np.int32),
                    np.zeros((1, 3)), math.pi)
    q2 = np.array([[0.0, -math.pi / 2]])
    assert O.check(synth.Scene(two, box, 0.25), q2)[0] == 1
    assert O.check(synth.Scene(two, box, 0.2499), q2)[0] == -1


def test_metrics_identities():
    yt = np.array([1, 1, 1, -1, -1, -1, -1, 1])
    yp = np.array([1, -1, 1, -1, 1, -1, -1, 1])
    m = O.metrics(yt, yp)
    assert (m["tp"], m["fn"], m["tn"], m["fp"]) == (3, 1, 3, 1)
    assert m["accuracy"] == 6 / 8 and m["tpr"] == 3 / 4 and m["tnr"] == 3 / 4
    # an unbalanced matrix (tp 1, fn 2, fp 1, tn 3) separates every ratio:
    # TPR = tp / (tp + fn), TNR = tn / (tn + fp) (Sec. IV)
    m = O.metrics(np.array([1, 1, 1, -1, -1, -1, -1]), np.array([1, -1, -1, 1, -1, -1, -1]))
    assert (m["tp"], m["fn"], m["tn"], m["fp"]) == (1, 2, 3, 1)
    assert m["accuracy"] == 4 / 7 and m["tpr"] == 1 / 3 and m["tnr"] == 3 / 4
