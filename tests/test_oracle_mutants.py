"""Mutation check of the oracle's pins.

Each mutant below plants one plausible mistake in a copy of the oracle: a
dropped term, a wrong sign, index or power, a transposed operand, a wrong tie
or boundary rule.  The pin suite (tests/test_oracle_*.py: closed forms,
invariants, brute force) must fail on every mutant, and must pass on the
unmodified copy.  Mistakes are planted in the CPU oracle only, in a
temporary directory; the copy is compiled and loaded by a child process.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = [os.path.join("tests", f"test_oracle_{n}.py") for n in ("fk", "kernel", "fastron", "checker", "gauss", "mlp")]
ORACLE_FILES = ("__init__.py", "oracle.py", "mlp.py", "fk_oracle.c")
C, PY, MLP = "fk_oracle.c", "oracle.py", "mlp.py"

# (name, file, text, replacement): the text occurs exactly once in the file.
MUTANTS = [
    # forward kinematics, Eqs. 1-2
    ("dh rotation sign", C, "ct, -ca * st,  sa * st, a * ct,", "ct,  ca * st,  sa * st, a * ct,"),
    ("dh translation uses cos twice", C, "st,  ca * ct, -sa * ct, a * st,", "st,  ca * ct, -sa * ct, a * ct,"),
    ("dh offset d dropped", C, "0.0,      sa,       ca,      d,", "0.0,      sa,       ca,    0.0,"),
    ("dh theta0 ignored", C, "theta += q;", "theta = q;"),
    ("prismatic joint sign", C, "        d += q;", "        d -= q;"),
    ("chain product transposed", C, "mat4_mul(T + 16 * (i - 1), A, T + 16 * i);",
     "mat4_mul(A, T + 16 * (i - 1), T + 16 * i);"),
    ("control-point offset by the transposed rotation", C,
     "W[4 * c + 0] * t[0] + W[4 * c + 1] * t[1] + W[4 * c + 2] * t[2]",
     "W[4 * 0 + c] * t[0] + W[4 * 1 + c] * t[1] + W[4 * 2 + c] * t[2]"),
    ("control point on the previous frame", C, "const double *W = T + 16 * cp_joint[m];",
     "const double *W = T + 16 * (cp_joint[m] > 0 ? cp_joint[m] - 1 : 0);"),
    # RQ kernel (Eq. 3), FK kernel (Eq. 4), Gaussian summand
    ("rq gamma for gamma/2", C, "double t = 1.0 + 0.5 * gamma * d2;", "double t = 1.0 + gamma * d2;"),
    ("rq first power", C, "return 1.0 / (t * t);", "return 1.0 / t;"),
    ("rq distance not squared", C, "        d2 += dc * dc;\n    }\n    double t = 1.0",
     "        d2 += fabs(dc);\n    }\n    double t = 1.0"),
    ("fk kernel sum instead of mean", C, "return s / M;", "return s;"),
    ("fk kernel skips the first control point", C, "for (int m = 0; m < M; ++m)\n        s += summand(",
     "for (int m = 1; m < M; ++m)\n        s += summand("),
    ("gauss gamma for gamma/2", C, "return exp(-0.5 * gamma * d2);", "return exp(-gamma * d2);"),
    ("gauss summand never selected", C, "return kind == 1 ? orc_k_gauss(", "return kind == 2 ? orc_k_gauss("),
    # kernel matrix and model value (Sec. II-B, III-B)
    ("kernel matrix stored transposed", C, "K[i * nb + j] = orc_k_fk_s(", "K[j * na + i] = orc_k_fk_s("),
    ("score sign", C, "f += j->alpha[s] * orc_k_fk_s(", "f -= j->alpha[s] * orc_k_fk_s("),
    ("score drops the first support point", C, "for (int64_t s = 0; s < j->ns; ++s)",
     "for (int64_t s = 1; s < j->ns; ++s)"),
    ("label of f = 0", PY, "np.where(np.asarray(f) >= 0.0, 1, -1)", "np.where(np.asarray(f) > 0.0, 1, -1)"),
    # Algorithm 1, Eqs. 6-8
    ("beta on the wrong class", C, "double b = y[i] > 0 ? beta : 1.0;", "double b = y[i] > 0 ? 1.0 : beta;"),
    ("delta sign of F", C, "double delta = b * y[i] - F[i];", "double delta = b * y[i] + F[i];"),
    ("argmin ties to the highest index", C, "if (m < mmin) {", "if (m <= mmin) {"),
    ("strict misclassification test", C, "if (i >= 0 && mmin <= 0.0) {", "if (i >= 0 && mmin < 0.0) {"),
    ("s_max off by one", C, "if (nnz < s_max || alpha[i] != 0.0) {", "if (nnz <= s_max || alpha[i] != 0.0) {"),
    ("s_max blocks adjusting a support point", C, "if (nnz < s_max || alpha[i] != 0.0) {",
     "if (nnz < s_max) {"),
    ("add uses the wrong column", C, "kernel_column(&pool, i);", "kernel_column(&pool, 0);"),
    ("removal margin keeps the point's own weight", C, "double m = y[j] * (F[j] - alpha[j]);",
     "double m = y[j] * F[j];"),
    ("removal update sign", C, "F[j] = fma(-a, col[j], F[j]);", "F[j] = fma(a, col[j], F[j]);"),
    ("removal at zero margin", C, "if (r >= 0 && mmax > 0.0) {", "if (r >= 0 && mmax >= 0.0) {"),
    ("removal ties to the highest index", C, "if (m > mmax) {", "if (m >= mmax) {"),
    ("removed weight kept in part", C, "alpha[r] = 0.0;", "alpha[r] *= 0.5;"),
    ("fp32 storage ignored in training", C, "p->col[j] = p->store32 ? (double)(float)k : k;", "p->col[j] = k;"),
    ("carried margins drop the first point", C, "for (int64_t s = 0; s < ns; ++s) {",
     "for (int64_t s = 1; s < ns; ++s) {"),
    ("carried margins ignore fp32 storage", C, "k = (double)(float)k;", "k = k + 0.0;"),
    ("active samples not clipped", PY, "v = np.clip(S + near[c], -qlim, qlim)", "v = S + near[c]"),
    ("active samples drawn point-major", PY,
     "near = st.uniform(k_near * ns * D, -sigma, sigma).reshape(k_near, ns, D)",
     "near = st.uniform(k_near * ns * D, -sigma, sigma).reshape(ns, k_near, D).transpose(1, 0, 2)"),
    ("active samples rounded after the clip only for copies", PY,
     "out.append(v.astype(np.float32).astype(np.float64))", "out.append(v)"),
    ("uniform samples over half the limits", PY, "uni = st.uniform(n_uniform * D, -qlim, qlim)",
     "uni = st.uniform(n_uniform * D, 0.0, qlim)"),
    # capsule-box checker and metrics (Sec. IV, Eqs. 10-12)
    ("touching is free", C, "boxes + 6 * b + 3) <= r2)", "boxes + 6 * b + 3) < r2)"),
    ("radius not squared", C, "double r2 = radius * radius;", "double r2 = radius;"),
    ("first link skipped", C, "for (int i = 1; i <= D && !hit; ++i) {", "for (int i = 2; i <= D && !hit; ++i) {"),
    ("segment minimiser sign", C, "t = -sab / sbb;", "t = sab / sbb;"),
    ("slab breakpoints dropped", C, "if (t > 0.0 && t < 1.0)\n                ts[nt++] = t;",
     "if (t > 0.0 && t < 0.0)\n                ts[nt++] = t;"),
    ("point-box distance to the wrong face", C, "e = p[c] - hi[c];", "e = p[c] - lo[c];"),
    ("segment interior ignored", C, "double g = point_box_dist2(p, lo, hi);", "double g = INFINITY;"),
    ("tpr over predicted positives", PY, '"tpr": tp / (tp + fn) if tp + fn else',
     '"tpr": tp / (tp + fp) if tp + fp else'),
    ("tnr over actual positives", PY, '"tnr": tn / (tn + fp) if tn + fp else',
     '"tnr": tn / (tn + fn) if tn + fn else'),
    # surrogate: features, network, loss, Adam, bfloat16 rounding
    ("feature sin of the wrong joint", MLP, "out[:, col + 5] = np.sin(qq[:, j + 1])",
     "out[:, col + 5] = np.sin(qq[:, j])"),
    ("feature position of the wrong point", MLP, "out[:, col:col + 3] = cp[:, m]",
     "out[:, col:col + 3] = cp[:, max(m - 1, 0)]"),
    ("forward drops a relu", MLP, "h2 = np.maximum(z2, 0.0)", "h2 = z2"),
    ("backward mask of the wrong layer", MLP, 'd2 = (d3 @ p["W3"]) * (h2 > 0)', 'd2 = (d3 @ p["W3"]) * (h3 > 0)'),
    ("backward transposed weight gradient", MLP, 'd2 = (d3 @ p["W3"]) * (h2 > 0)\n    g["W2"] = d2.T @ h1',
     'd2 = (d3 @ p["W3"]) * (h2 > 0)\n    g["W2"] = h1.T @ d2'),
    ("mse gradient without the factor 2", MLP,
     '    dout = 2.0 * (out - target) / B\n    g = {"w4": h3.T @ dout, "b4": np.array([dout.sum()])}\n'
     '    d3 = np.outer(dout, p["w4"]) * (h3 > 0)',
     '    dout = (out - target) / B\n    g = {"w4": h3.T @ dout, "b4": np.array([dout.sum()])}\n'
     '    d3 = np.outer(dout, p["w4"]) * (h3 > 0)'),
    ("adam without bias correction", MLP, "mh = m / (1 - beta1 ** t)", "mh = m"),
    ("adam without the square root", MLP, "np.sqrt(vh) + eps", "vh + eps"),
    ("bf16 truncates", MLP, "b = (b + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)",
     "b = b & np.uint64(0xFFFF0000)"),
    ("bf16 ties away from zero", MLP, "(b + np.uint64(0x7FFF) + lsb)", "(b + np.uint64(0x8000))"),
]


def _make_copy(dst, mutant=None):
    """A copy of the oracle package under dst/oracle, with one mutant applied."""
    pkg = os.path.join(dst, "oracle")
    os.makedirs(pkg)
    for f in ORACLE_FILES:
        shutil.copy(os.path.join(ROOT, "oracle", f), os.path.join(pkg, f))
    if mutant is not None:
        _, fname, old, new = mutant
        path = os.path.join(pkg, fname)
        with open(path) as fh:
            src = fh.read()
        assert src.count(old) == 1, f"mutant text must occur once in {fname}: {old!r}"
        with open(path, "w") as fh:
            fh.write(src.replace(old, new))


def _run_pins(dst):
    """Run the pin suite in a child process that imports the oracle from dst
    (first on sys.path, before the repository root).  Returns (exit code,
    tail of the output): 0 all pins pass, 1 some pin failed."""
    code = ("import sys; sys.path[:0] = [%r, %r]; import pytest; "
            "sys.exit(pytest.main(['-x', '-q', '-p', 'no:cacheprovider', '-m', 'not gpu'] + %r))"
            % (dst, ROOT, PINS))
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    return r.returncode, (r.stdout + r.stderr)[-1500:]


def test_every_mutant_text_occurs_once():
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)
    for name, fname, old, new in MUTANTS:
        assert old != new, name
        with open(os.path.join(ROOT, "oracle", fname)) as fh:
            assert fh.read().count(old) == 1, f"{name}: text not found exactly once in {fname}"


def test_unmodified_copy_passes_the_pins(tmp_path):
    _make_copy(str(tmp_path))
    rc, out = _run_pins(str(tmp_path))
    assert rc == 0, out


def test_every_mutant_fails_a_pin(tmp_path):
    jobs = []
    for k, m in enumerate(MUTANTS):
        dst = str(tmp_path / f"m{k:02d}")
        _make_copy(dst, m)
        jobs.append((m[0], dst))
    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(lambda j: (j[0],) + _run_pins(j[1]), jobs))
    survivors = [(name, out) for name, rc, out in results if rc == 0]
    broken = [(name, rc, out) for name, rc, out in results if rc not in (0, 1)]
    assert not broken, "pin runs that neither passed nor failed: " + repr(broken[:3])
    assert not survivors, "mutants no pin catches: " + ", ".join(n for n, _ in survivors)
