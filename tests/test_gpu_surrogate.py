"""The learned surrogate on the tensor cores against the FP64 MLP oracle:
forward values, gradients of every parameter tensor, Adam steps,
training plus inference with fallback to the exact score, and what the
trained network gains over the exact path.

Forward values and gradients are compared element by element with the FP64
oracle that rounds where the kernels do (features, hidden activations and
deltas stored in bfloat16; oracle/mlp.py backward_bf16_storage), on the
BF16 weights both sides use.  Each element has its own tolerance: 8 units of
BF16 roundoff (2^-9) times the sum of the absolute products that form it
(|h3| |w4| for an output, |delta| |h| over the batch for a weight gradient,
|delta| for a bias).  This is a test tolerance, not a proven bound: a
rigorous worst case through three layers of BF16 storage lets every hidden
unit straddle a rounding boundary and gives bounds larger than the values.
The GPU differs from this oracle only by its FP32 accumulation order and the
one-ulp BF16 differences it causes on stored values that sit on a rounding
boundary (measured below 10% of the tolerance); a plausible mistake (a sign,
an index, a transposed operand) moves an element by about its own size, which
exceeds its tolerance on nearly every element that does not cancel to noise
(tests/test_oracle_mlp.py plants such mistakes in the oracle)."""
import numpy as np
import pytest
import torch

from oracle import mlp as L
from paper_1910_06451_gb300 import synth
from tests._surrogate_ref import elementwise_reference

pytestmark = pytest.mark.gpu

ORDER = [("W1", (256, 64)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)), ("W3", (256, 256)), ("b3", (256,)),
         ("w4", (256,)), ("b4", (1,))]


def _flat(p):
    return np.concatenate([np.asarray(p[k], dtype=np.float64).reshape(-1) for k, _ in ORDER]).astype(np.float32)


def _unflat(v):
    out, o = {}, 0
    for k, shp in ORDER:
        n = int(np.prod(shp))
        out[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def _bf16(x):
    return torch.from_numpy(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).double().numpy()


@pytest.fixture(scope="module")
def setup(fk):
    w = synth.workload("arm7-n5000")
    chain = fk.chain_from_arm(w.scene.arm)
    s = fk.surrogate_create(chain, seed=1)
    yield w, chain, s
    fk.surrogate_destroy(s)
    fk.fk_chain_destroy(chain)


def _params(seed):
    rng = np.random.default_rng(seed)
    p = L.init_params(rng)
    for k in ("b1", "b2", "b3", "b4"):
        p[k] = rng.normal(size=p[k].shape) * 0.05
    return p


def _oracle_with_bf16(p, w, q):
    """The oracle's parameters with the BF16-rounded weights the GPU uses, and
    the FP64 features (rounded to BF16 inside elementwise_reference)."""
    pb = dict(p)
    for k in ("W1", "W2", "W3"):
        pb[k] = _bf16(p[k])
    return pb, L.features(w.scene.arm, q.astype(np.float64))


def test_forward_matches_oracle(fk, setup):
    w, chain, s = setup
    p = _params(3)
    fk.surrogate_set_params(s, _flat(p))
    q = w.query_configs(1000)
    out = torch.empty(1000, dtype=torch.float32, device="cuda")
    fk.surrogate_forward(s, torch.from_numpy(q).cuda(), out)
    pb, X = _oracle_with_bf16(_unflat(_flat(p)), w, q)
    want, tol = elementwise_reference(pb, X)
    got = out.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - want) <= tol), np.max(np.abs(got - want) / tol)


def test_gradients_match_oracle(fk, setup):
    w, chain, s = setup
    p = _unflat(_flat(_params(4)))
    fk.surrogate_set_params(s, _flat(p))
    n = 512
    q = w.query_configs(n)
    target = np.random.default_rng(5).normal(size=n).astype(np.float32)
    g, loss = fk.surrogate_gradients(s, torch.from_numpy(q).cuda(), torch.from_numpy(target).cuda())
    pb, X = _oracle_with_bf16(p, w, q)
    out, tol_out, want, tol = elementwise_reference(pb, X, target.astype(np.float64))
    got = _unflat(g)
    # the loss: mean of (out - target)^2 with every output within its tolerance
    r = np.abs(out - target)
    assert abs(loss - L.loss(out, target)) <= np.mean(2 * r * tol_out + tol_out ** 2) + 1e-6 * L.loss(out, target)
    for k, _ in ORDER:
        err = np.abs(got[k] - want[k])
        assert np.all(err <= tol[k]), (k, float(np.max(err / tol[k])))
        print(f"{k}: max |err| / tolerance {float(np.max(err / np.maximum(tol[k], 1e-300))):.3f}")


def test_gradients_twelve_point_arm_match_oracle(fk):
    # the 12-point arm's features, an odd number of 128-row tiles (three
    # two-CTA clusters), every gradient entry within its tolerance
    w = synth.workload("arm7m12-n65536")
    chain = fk.chain_from_arm(w.scene.arm)
    s = fk.surrogate_create(chain, seed=3)
    try:
        p = _unflat(_flat(_params(8)))
        fk.surrogate_set_params(s, _flat(p))
        n = 384
        q = w.query_configs(n)
        target = np.random.default_rng(9).normal(size=n).astype(np.float32)
        g, loss = fk.surrogate_gradients(s, torch.from_numpy(q).cuda(), torch.from_numpy(target).cuda())
        pb, X = _oracle_with_bf16(p, w, q)
        out, tol_out, want, tol = elementwise_reference(pb, X, target.astype(np.float64))
        got = _unflat(g)
        r = np.abs(out - target)
        assert abs(loss - L.loss(out, target)) <= np.mean(2 * r * tol_out + tol_out ** 2) + 1e-6 * L.loss(out, target)
        for k, _ in ORDER:
            err = np.abs(got[k] - want[k])
            assert np.all(err <= tol[k]), (k, float(np.max(err / tol[k])))
    finally:
        fk.surrogate_destroy(s)
        fk.fk_chain_destroy(chain)


def test_adam_step_matches_oracle(fk, setup):
    w, chain, s = setup
    s2 = fk.surrogate_create(chain, seed=2)
    try:
        p = _unflat(_flat(_params(6)))
        fk.surrogate_set_params(s2, _flat(p))
        rng = np.random.default_rng(7)
        st = {}
        for it in range(3):
            g = {k: rng.normal(size=shp) for k, shp in ORDER}
            gf = _flat(g)
            fk.surrogate_adam_step(s2, gf, 1e-3)
            L.adam_step(p, _unflat(gf), st, lr=1e-3)
        got = _unflat(fk.surrogate_get_params(s2)[0])
        for k, _ in ORDER:
            np.testing.assert_allclose(got[k], p[k], rtol=1e-4, atol=1e-6)
    finally:
        fk.surrogate_destroy(s2)


def test_train_and_infer_with_fallback(fk, setup):
    w, chain, s = setup
    dev = torch.device("cuda")
    model = fk.fastron_model_create(chain)
    try:
        X = w.train_configs()
        y = torch.empty(w.n_train, dtype=torch.int8, device=dev)
        fk.fk_label(chain, w.scene.boxes, w.scene.radius, torch.from_numpy(X).to(dev), y)
        fk.fastron_train(model, torch.from_numpy(X.astype(np.float64)).to(dev), y, w.gamma, w.beta, w.iter_max,
                         w.s_max)
        qtr = torch.from_numpy(synth.uniform_configs(4242, 1 << 18, 7, w.scene.arm.qlim)).to(dev)
        with pytest.raises(fk.FkError):
            fk.surrogate_train(s, model, qtr, epochs=1, batch=4096, lr=1e-3, holdout=0.125, schedule=7)
        st = fk.surrogate_train(s, model, qtr, epochs=4, batch=4096, lr=1e-3, holdout=0.125)
        assert st["steps"] > 0 and st["loss_last"] < st["loss_first"]
        assert st["tau"] >= 0 and 0 < st["holdout_fallback"] <= 1
        n = 100_000
        q = torch.from_numpy(w.query_configs(n)).to(dev)
        lab = torch.empty(n, dtype=torch.int8, device=dev)
        pred = torch.empty(n, dtype=torch.float32, device=dev)
        nfb = fk.surrogate_infer(s, model, q, lab, pred)
        exact = torch.empty(n, dtype=torch.int8, device=dev)
        fk.fk_score(model, q, exact, rescore=True)
        raw = torch.empty(n, dtype=torch.float32, device=dev)
        fk.surrogate_forward(s, q, raw)
        _, scale, tau = fk.surrogate_get_params(s)
        assert tau == st["tau"]
        p_net = raw.cpu().numpy() * np.float32(scale)
        lab, exact = lab.cpu().numpy(), exact.cpu().numpy()
        assert 0 < nfb < n
        confident = np.abs(p_net) > np.float32(tau)
        # every fallback query carries the exact label
        assert np.array_equal(lab[~confident], exact[~confident])
        assert np.sum(~confident) == nfb
        # the network's answers agree with the exact labels on almost all confident queries
        assert np.mean(lab[confident] == exact[confident]) >= 0.995
    finally:
        fk.fastron_model_destroy(model)


def test_forward_twelve_point_arm_matches_oracle(fk):
    # the 12-point arm's surrogate reads the frame-origin points' features
    w = synth.workload("arm7m12-n65536")
    chain = fk.chain_from_arm(w.scene.arm)
    s = fk.surrogate_create(chain, seed=2)
    try:
        p = _params(4)
        fk.surrogate_set_params(s, _flat(p))
        q = w.query_configs(1000)
        out = torch.empty(1000, dtype=torch.float32, device="cuda")
        fk.surrogate_forward(s, torch.from_numpy(q).cuda(), out)
        pb, X = _oracle_with_bf16(_unflat(_flat(p)), w, q)
        want, tol = elementwise_reference(pb, X)
        assert np.all(np.abs(out.cpu().numpy().astype(np.float64) - want) <= tol)
    finally:
        fk.surrogate_destroy(s)
        fk.fk_chain_destroy(chain)


def test_fused_inference_is_tile_independent(fk, setup):
    # the fused kernel scores 128-query tiles; a query's output must not
    # depend on the tile it falls in or on the padding of the last tile
    w, chain, s = setup
    fk.surrogate_set_params(s, _flat(_params(5)))
    q = torch.from_numpy(w.query_configs(1500)).cuda()
    a = torch.empty(1500, dtype=torch.float32, device="cuda")
    b = torch.empty(1000, dtype=torch.float32, device="cuda")
    fk.surrogate_forward(s, q, a)
    fk.surrogate_forward(s, q[437:1437].contiguous(), b)
    assert torch.equal(a[437:1437], b)
    one = torch.empty(1, dtype=torch.float32, device="cuda")
    fk.surrogate_forward(s, q[999:1000].contiguous(), one)
    assert torch.equal(one, a[999:1000])


def _median_ms(fn, reps=5):
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def test_trained_network_gains_over_the_exact_path(fk):
    """What the learned part adds on the 7-DOF workload (5000 training points,
    4,194,304 queries): trained on 2M of the model's own scores (96 epochs,
    cosine schedule from 3e-3), the network answers most queries by itself
    and the rest take the exact path.  Every fallback label is exact, the
    confident answers differ from the exact labels on at most 1e-4 of the
    queries, and the whole surrogate path takes less time than the exact path
    on the same batch (measured 3.6 ms against 5.4 ms)."""
    dev = torch.device("cuda")
    w = synth.workload("arm7-n5000")
    chain = fk.chain_from_arm(w.scene.arm)
    model = fk.fastron_model_create(chain)
    s = fk.surrogate_create(chain, seed=1)
    try:
        X = w.train_configs()
        y = torch.empty(w.n_train, dtype=torch.int8, device=dev)
        fk.fk_label(chain, w.scene.boxes, w.scene.radius, torch.from_numpy(X).to(dev), y)
        fk.fastron_train(model, torch.from_numpy(X.astype(np.float64)).to(dev), y, w.gamma, w.beta, w.iter_max,
                         w.s_max)
        qtr = torch.from_numpy(synth.uniform_configs(w.seed + 7, 1 << 21, 7, w.scene.arm.qlim)).to(dev)
        st = fk.surrogate_train(s, model, qtr, epochs=96, batch=8192, lr=3e-3, holdout=0.0625,
                                schedule=fk.FK_LR_COSINE)
        del qtr
        n = 1 << 22
        q = torch.from_numpy(w.query_configs(n)).to(dev)
        exact = torch.empty(n, dtype=torch.int8, device=dev)
        lab = torch.empty(n, dtype=torch.int8, device=dev)
        pred = torch.empty(n, dtype=torch.float32, device=dev)
        fk.fk_score(model, q, exact, rescore=True)
        nfb = fk.surrogate_infer(s, model, q, lab, pred)
        raw = torch.empty(n, dtype=torch.float32, device=dev)
        fk.surrogate_forward(s, q, raw)
        _, scale, tau = fk.surrogate_get_params(s)
        confident = (raw.abs() * np.float32(scale) > np.float32(tau)).cpu().numpy()
        labn, exn = lab.cpu().numpy(), exact.cpu().numpy()
        assert int(np.sum(~confident)) == nfb
        assert np.array_equal(labn[~confident], exn[~confident])
        assert nfb / n < 0.5, f"fallback {nfb / n:.3f}"
        assert np.sum(labn != exn) <= 1e-4 * n
        assert st["holdout_fallback"] < 0.5
        t_exact = _median_ms(lambda: fk.fk_score(model, q, exact, rescore=True))
        t_sur = _median_ms(lambda: fk.surrogate_infer(s, model, q, lab))
        assert t_sur < t_exact / 1.1, f"surrogate {t_sur:.2f} ms vs exact {t_exact:.2f} ms"
    finally:
        fk.surrogate_destroy(s)
        fk.fastron_model_destroy(model)
        fk.fk_chain_destroy(chain)


def test_fused_inference_wait_limit_reports_timeout(fk, setup):
    # every bounded wait of the fused kernel gives up at once: the call
    # returns FK_ERR_TIMEOUT without a hang, and the next call with the
    # normal limit succeeds with the same outputs as before
    w, chain, s = setup
    fk.surrogate_set_params(s, _flat(_params(7)))
    q = torch.from_numpy(w.query_configs(4096)).cuda()
    ref = torch.empty(4096, dtype=torch.float32, device="cuda")
    fk.surrogate_forward(s, q, ref)
    out = torch.empty(4096, dtype=torch.float32, device="cuda")
    fk.fk_set_wait_limit(0)
    try:
        with pytest.raises(fk.FkError) as e:
            fk.surrogate_forward(s, q, out)
        assert e.value.code == fk.FK_ERR_TIMEOUT
    finally:
        fk.fk_set_wait_limit(1 << 22)
    fk.surrogate_forward(s, q, out)
    assert torch.equal(out, ref)


def test_training_step_wait_limit_reports_timeout(fk, setup):
    # the training step's kernels (the two-CTA tile kernel, the weight-gradient
    # products, the reduction) with every bounded wait giving up at once: the
    # call returns FK_ERR_TIMEOUT without a hang; with the normal limit the
    # next call gives the same gradient as before, bit for bit
    w, chain, s = setup
    p = _flat(_params(11))
    fk.surrogate_set_params(s, p)
    n = 384
    q = torch.from_numpy(w.query_configs(n)).cuda()
    target = torch.from_numpy(np.random.default_rng(12).normal(size=n).astype(np.float32)).cuda()
    g0, l0 = fk.surrogate_gradients(s, q, target)
    fk.fk_set_wait_limit(0)
    try:
        with pytest.raises(fk.FkError) as e:
            fk.surrogate_gradients(s, q, target)
        assert e.value.code == fk.FK_ERR_TIMEOUT
    finally:
        fk.fk_set_wait_limit(1 << 22)
    fk.surrogate_set_params(s, p)
    g1, l1 = fk.surrogate_gradients(s, q, target)
    assert np.array_equal(g0, g1) and l0 == l1
