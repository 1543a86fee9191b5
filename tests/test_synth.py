"""The seeded generator: SplitMix64 reference outputs, determinism, and the
shapes and ranges of the synthetic workloads."""
import math

import numpy as np

from paper_1910_06451_gb300 import synth


def test_splitmix64_reference_values():
    # SplitMix64 from state 0: the first outputs of the published generator
    z = synth.splitmix64(0, np.arange(3, dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF
    assert int(z[1]) == 0x6E789E6AA1B965F4
    assert int(z[2]) == 0x06C45D188009454F


def test_stream_is_counter_based():
    a = synth.Stream(42)
    x = np.concatenate([a.u64(5), a.u64(7)])
    y = synth.Stream(42).u64(12)
    assert np.array_equal(x, y)
    u = synth.Stream(1).uniform(100000)
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01


def test_canonical_values_are_fp32():
    for name in ("arm3-n1000", "arm7-n5000"):
        w = synth.workload(name)
        arm = w.scene.arm
        for arr in (arm.dh[:, :4], w.scene.boxes):
            assert np.array_equal(arr, arr.astype(np.float32).astype(np.float64))
        q = w.train_configs()
        assert q.dtype == np.float32 and q.shape == (w.n_train, arm.D)
        assert np.all(np.abs(q) <= arm.qlim)


def test_workload_shapes():
    w3 = synth.workload("arm3-n1000")
    assert w3.scene.arm.D == 3 and w3.scene.arm.M == 4 and w3.scene.boxes.shape == (6, 6)
    assert np.all((w3.scene.arm.dh[:, 0] >= 0.2) & (w3.scene.arm.dh[:, 0] <= 0.5))
    w7 = synth.workload("arm7-n5000")
    assert w7.scene.arm.D == 7 and w7.scene.arm.M == 8 and w7.scene.boxes.shape == (10, 6)
    assert w7.scene.arm.qlim == np.float32(math.radians(170))
    for w in (w3, w7):
        b = w.scene.boxes
        half = (b[:, 3:] - b[:, :3]) / 2
        assert np.all(half > 0.049) and np.all(half < 0.151)
        gap = np.maximum(np.maximum(b[:, :3], -b[:, 3:]), 0.0)
        assert np.all(np.linalg.norm(gap, axis=1) > 0.1)
    assert np.array_equal(synth.workload("arm7-n5000").query_configs(100), w7.query_configs(100))


def test_twelve_control_point_arm_adds_link_midpoints():
    from oracle import oracle as O
    arm = synth.arm_7dof_m12(4000)
    assert arm.M == 12 and list(arm.cp_joint[:8]) == list(range(8))
    length = np.hypot(arm.dh[:, 0], arm.dh[:, 2])
    assert sorted(arm.cp_joint[8:] - 1) == sorted(np.argsort(-length)[:4])
    q = synth.uniform_configs(7, 50, arm.D, arm.qlim).astype(np.float64)
    cp = O.fk_points(arm, q)
    for m in range(8, 12):
        j = int(arm.cp_joint[m])
        mid = 0.5 * (cp[:, j - 1] + cp[:, j])  # frame origins j-1 and j are control points j-1 and j
        np.testing.assert_allclose(cp[:, m], mid, atol=1e-7)


def test_moving_boxes_stay_in_bounds_and_move_slowly():
    w = synth.workload("arm7m12-n65536")
    b = synth.moving_boxes(w.seed, w.scene.boxes, 100)
    assert b.shape == (100, 10, 6)
    np.testing.assert_array_equal(b[0], w.scene.boxes)
    c = 0.5 * (b[..., :3] + b[..., 3:])
    h = b[..., 3:] - b[..., :3]
    step = np.linalg.norm(np.diff(c, axis=0), axis=2)
    assert step.max() <= 0.05 * 1.0001 and step.max() > 0.01
    np.testing.assert_allclose(h, h[0:1].repeat(100, axis=0), atol=1e-6)  # sizes fixed
    assert np.all(np.abs(c) <= 0.8 + 1e-6)
    gap = np.maximum(np.maximum(b[..., :3], -b[..., 3:]), 0.0)
    assert np.all(np.linalg.norm(gap, axis=2) > 0.1)
    np.testing.assert_array_equal(b, synth.moving_boxes(w.seed, w.scene.boxes, 100))
