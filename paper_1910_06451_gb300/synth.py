"""Seeded synthetic inputs: robot arms, box obstacles and joint configurations.

This module is the only code shared by the CUDA path and the FP64 oracle.  It
draws numbers and nothing else: it holds no forward kinematics, no kernel, no
Fastron arithmetic and no collision test.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: draw ``k`` of stream ``seed`` is the SplitMix64 finaliser applied to
``seed + (k + 1) * 0x9E3779B97F4A7C15``.  Uniform doubles take the top 53 bits.
Every value is drawn in FP64 and rounded to FP32 once; the FP32 value (widened
back to FP64 where FP64 is needed) is the canonical input both sides consume.

The shapes follow the workloads of the paper's evaluation (Sec. IV): serial
revolute arms described by standard Denavit-Hartenberg parameters (Eq. 1) with
control points at the joint-frame origins (Sec. III-A), random axis-aligned box
obstacles, and configurations drawn uniformly inside the joint limits.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_MASK = (1 << 64) - 1
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counter: np.ndarray) -> np.ndarray:
    """SplitMix64 outputs for the given draw indices of stream ``seed``."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + (c + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


class Stream:
    """Sequential reader over one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = int(seed) & _MASK
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        out = splitmix64(self.seed, np.arange(self.pos, self.pos + n, dtype=np.uint64))
        self.pos += n
        return out

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * u


def _f32(x) -> np.ndarray:
    """Round once to FP32 and widen back: the canonical value of a draw."""
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


REVOLUTE = 0
PRISMATIC = 1


@dataclasses.dataclass
class Arm:
    """A serial chain in standard DH form plus its control points.

    ``dh`` rows are ``(a, alpha, d, theta0, type)`` (Eq. 1; ``theta0`` is the
    joint-angle offset, ``type`` 0 = revolute, 1 = prismatic).  ``base`` is the
    world-from-frame-0 transform.  Control point ``m`` sits at offset
    ``cp_off[m]`` in frame ``cp_joint[m]`` (Eq. 2, ``T_m`` a pure translation).
    """

    dh: np.ndarray
    base: np.ndarray
    cp_joint: np.ndarray
    cp_off: np.ndarray
    qlim: float

    @property
    def D(self) -> int:
        return int(self.dh.shape[0])

    @property
    def M(self) -> int:
        return int(self.cp_joint.shape[0])


@dataclasses.dataclass
class Scene:
    arm: Arm
    boxes: np.ndarray   # (nb, 6): lo_x, lo_y, lo_z, hi_x, hi_y, hi_z
    radius: float       # radius of the sphere swept along each link


def frame_origin_cps(D: int) -> tuple[np.ndarray, np.ndarray]:
    """Control points at the origins of frames 0..D (offset zero)."""
    return np.arange(D + 1, dtype=np.int32), np.zeros((D + 1, 3))


def random_arm(seed: int, D: int, a_range, d_range, qlim: float) -> Arm:
    """Random revolute arm: twist +-pi/2 with a random sign, theta0 = 0, base = I."""
    st = Stream(seed)
    a = _f32(st.uniform(D, *a_range))
    d = _f32(st.uniform(D, *d_range)) if d_range is not None else np.zeros(D)
    sign = np.where(st.uniform(D) < 0.5, -1.0, 1.0)
    alpha = _f32(sign * (math.pi / 2))
    dh = np.zeros((D, 5))
    dh[:, 0], dh[:, 1], dh[:, 2] = a, alpha, d
    cj, co = frame_origin_cps(D)
    return Arm(dh=dh, base=np.eye(4), cp_joint=cj, cp_off=co, qlim=float(_f32(qlim)))


def arm_3dof(seed: int) -> Arm:
    """3-DOF spatial arm: a ~ U[0.2, 0.5] m, d = 0, limits +-pi, 4 control points."""
    return random_arm(seed, 3, (0.2, 0.5), None, math.pi)


def arm_7dof(seed: int) -> Arm:
    """7-DOF arm: a ~ U[0.1, 0.4] m, d ~ U[0, 0.1] m, limits +-170 deg, 8 control points."""
    return random_arm(seed, 7, (0.1, 0.4), (0.0, 0.1), math.radians(170.0))


def arm_7dof_m12(seed: int) -> Arm:
    """The 7-DOF arm of ``arm_7dof(seed)`` with 12 control points: the origins
    of frames 0..7 and the midpoints of the four links with the largest
    sqrt(a^2 + d^2).  Link j joins the origins of frames j-1 and j; in frame j
    its midpoint sits at the constant offset -(a_j, d_j sin alpha_j,
    d_j cos alpha_j) / 2 (the DH step of Eq. 1 walked back by half), rounded
    to FP32 like every other input."""
    arm = arm_7dof(seed)
    a, al, d = arm.dh[:, 0], arm.dh[:, 1], arm.dh[:, 2]
    length = np.sqrt(a * a + d * d)
    longest = np.sort(np.argsort(-length, kind="stable")[:4])  # DH rows, ascending
    cj = list(arm.cp_joint)
    co = [row for row in arm.cp_off]
    for r in longest:
        cj.append(int(r) + 1)
        co.append(_f32(-0.5 * np.array([a[r], d[r] * math.sin(al[r]), d[r] * math.cos(al[r])])))
    return dataclasses.replace(arm, cp_joint=np.array(cj, dtype=np.int32), cp_off=np.array(co))


def random_boxes(seed: int, nb: int, centre=(-0.8, 0.8), half=(0.05, 0.15),
                 keep_clear: float = 0.1) -> np.ndarray:
    """Axis-aligned boxes; a draw whose box comes within ``keep_clear`` of the
    base origin is rejected and redrawn (otherwise every configuration collides)."""
    st = Stream(seed ^ 0x5DEECE66D)
    out = []
    while len(out) < nb:
        c = st.uniform(3, *centre)
        h = st.uniform(3, *half)
        lo, hi = _f32(c - h), _f32(c + h)
        gap = np.maximum(np.maximum(lo, -hi), 0.0)      # per-axis gap from the origin
        if math.sqrt(float(np.sum(gap * gap))) <= keep_clear:
            continue
        out.append(np.concatenate([lo, hi]))
    return np.array(out)


def moving_boxes(seed: int, boxes0: np.ndarray, n_frames: int, vmax: float = 0.05, region=(-0.8, 0.8),
                 keep_clear: float = 0.1) -> np.ndarray:
    """Box positions over n_frames frames, shape (n_frames, nb, 6); frame 0 is
    boxes0.  Each box moves along a straight line at a constant speed drawn
    uniformly in [0, vmax] per frame, in a direction uniform on the sphere;
    its centre is reflected at the faces of the region cube, and a step that
    would bring the box within keep_clear of the base origin is undone and the
    velocity reversed.  Positions are tracked in FP64 and each frame's box is
    rounded to FP32."""
    st = Stream(seed ^ 0x30B1E5)
    b0 = np.asarray(boxes0, dtype=np.float64)
    nb = b0.shape[0]
    c = 0.5 * (b0[:, :3] + b0[:, 3:])
    h = 0.5 * (b0[:, 3:] - b0[:, :3])
    z = st.uniform(nb, -1.0, 1.0)
    phi = st.uniform(nb, 0.0, 2.0 * math.pi)
    speed = st.uniform(nb, 0.0, vmax)
    r = np.sqrt(np.maximum(1.0 - z * z, 0.0))
    v = (speed * np.stack([r * np.cos(phi), r * np.sin(phi), z])).T
    lo_r, hi_r = region
    out = np.empty((n_frames, nb, 6))
    out[0] = b0
    for k in range(1, n_frames):
        nxt = c + v
        for ax in range(3):
            over = nxt[:, ax] > hi_r
            under = nxt[:, ax] < lo_r
            nxt[over, ax] = 2 * hi_r - nxt[over, ax]
            nxt[under, ax] = 2 * lo_r - nxt[under, ax]
            v[over | under, ax] *= -1.0
        lo, hi = nxt - h, nxt + h
        gap = np.maximum(np.maximum(lo, -hi), 0.0)
        near = np.sqrt(np.sum(gap * gap, axis=1)) <= keep_clear
        nxt[near] = c[near]
        v[near] *= -1.0
        c = nxt
        out[k] = np.concatenate([_f32(c - h), _f32(c + h)], axis=1)
    return out


def uniform_configs(seed: int, n: int, D: int, qlim: float) -> np.ndarray:
    """n configurations uniform in [-qlim, qlim]^D, canonical FP32, shape (n, D)."""
    st = Stream(seed)
    return st.uniform(n * D, -qlim, qlim).astype(np.float32).reshape(n, D)


@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    gamma: float
    beta: float
    n_train: int
    n_query: int
    iter_max: int
    s_max: int
    seed: int

    def train_configs(self) -> np.ndarray:
        return uniform_configs(self.seed + 1, self.n_train, self.scene.arm.D, self.scene.arm.qlim)

    def query_configs(self, n: int | None = None) -> np.ndarray:
        return uniform_configs(self.seed + 2, self.n_query if n is None else n,
                               self.scene.arm.D, self.scene.arm.qlim)


def workload(name: str, trial: int = 0, **over) -> Workload:
    """Named workloads.  Scene seed s, training seed s+1, query seed s+2.

    ``arm3-n1000``: 3-DOF arm, 4 control points, 6 boxes, N = 1000 training
    configurations, 10,000 queries, gamma = 10, up to 5000 iterations.
    ``arm7-n5000``: 7-DOF arm, 8 control points, 10 boxes, N = 5000, 4M
    queries, gamma = 40 (the paper picks its kernel parameters by grid search,
    Sec. IV; 40 gave the best held-out accuracy of 5, 10, 20, 40, 80, 160).
    ``arm7m12-n65536``: the changing environment: 7-DOF arm with 12 control
    points (``arm_7dof_m12``), 10 boxes that move (``moving_boxes``, up to
    0.05 m per frame), N = 65,536 training configurations, 16,777,216 queries
    per frame, gamma = 40, S_max = 20,000, up to 100,000 iterations.
    """
    if name == "arm3-n1000":
        s = 1000 * 0 + trial
        sc = Scene(arm_3dof(s), random_boxes(s, 6), 0.03)
        w = Workload(name, sc, 10.0, 1.0, 1000, 10_000, 5000, 1000, s)
    elif name == "arm7-n5000":
        s = 1000 * 1 + trial
        sc = Scene(arm_7dof(s), random_boxes(s, 10), 0.03)
        w = Workload(name, sc, 40.0, 1.0, 5000, 4_000_000, 5000, 5000, s)
    elif name == "arm7m12-n65536":
        s = 1000 * 4 + trial
        sc = Scene(arm_7dof_m12(s), random_boxes(s, 10), 0.03)
        w = Workload(name, sc, 40.0, 1.0, 65_536, 16_777_216, 100_000, 20_000, s)
    else:
        raise KeyError(name)
    return dataclasses.replace(w, **over)


@dataclasses.dataclass
class BatchScene:
    scene: Scene
    support: np.ndarray   # (ns, D) FP32 support configurations
    alpha: np.ndarray     # (ns,) weights
    queries: np.ndarray   # (nq, D) FP32 queries
    gamma: float


def _log_uniform_int(st: Stream, lo: int, hi: int) -> int:
    return int(round(math.exp(st.uniform(1, math.log(lo), math.log(hi))[0])))


def batch_scenes(seed: int, n_scenes: int, support=(200, 6000), queries=(1000, 65536), boxes=(4, 20),
                 gamma: float = 40.0) -> list[BatchScene]:
    """Independent 7-DOF scenes with uneven sizes: support-set and query-batch
    sizes log-uniform in the given ranges, 4-20 boxes.  The support sets are
    random configurations with normal weights (scale 5, like the trained
    7-DOF model's): the scoring work and its parity do not depend on how the
    weights were found."""
    st = Stream(seed ^ 0xB47C4)
    out = []
    for i in range(n_scenes):
        s = seed * 1000 + i
        arm = arm_7dof(s)
        nb = int(st.uniform(1, boxes[0], boxes[1] + 1)[0])
        ns = _log_uniform_int(st, *support)
        nq = _log_uniform_int(st, *queries)
        sc = Scene(arm, random_boxes(s, nb), 0.03)
        sup = uniform_configs(s + 11, ns, arm.D, arm.qlim)
        alpha = Stream(s + 13).uniform(ns, -1.0, 1.0)
        alpha = _f32(np.sign(alpha) * (0.5 + 5.0 * np.abs(alpha)))
        q = uniform_configs(s + 17, nq, arm.D, arm.qlim)
        out.append(BatchScene(sc, sup, alpha, q, gamma))
    return out
