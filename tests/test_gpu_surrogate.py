"""GPU surrogate MLP against the FP64 reference (oracle/mlp.py), through the C ABI.

The GPU holds bfloat16 weights and accumulates in FP32; the reference runs in
float64 on the same bfloat16-rounded weights and the same inputs, so the
bars are FP32 accumulation bars: forward probabilities within 1e-5, each
gradient tensor within 1e-3 relative (max-abs over max-abs), the loss within
1e-6. Then: one Adam step against the reference step, and the trained
network recovering a known pass-probability law.
"""
import numpy as np
import pytest

from oracle import mlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

IN, H = 33, 256
SLICES = {"W1": (0, IN * H, (IN, H)), "b1": (IN * H, H, (H,)), "W2": (IN * H + H, H * H, (H, H)),
          "b2": (IN * H + H + H * H, H, (H,)), "W3": (IN * H + 2 * H + H * H, H, (H, 1)),
          "b3": (IN * H + 3 * H + H * H, 1, (1,))}


def unpack(flat):
    return {k: np.asarray(flat[o:o + n], dtype=np.float64).reshape(s) for k, (o, n, s) in SLICES.items()}


def pack(p):
    out = np.zeros(sum(n for _, n, _ in SLICES.values()), dtype=np.float32)
    for k, (o, n, s) in SLICES.items():
        out[o:o + n] = p[k].reshape(-1)
    return out


@pytest.fixture(scope="module")
def arso():
    from paper_2301_07264_gb300 import arso as mod
    return mod


def _setup(arso, seed=0, n=96):
    rng = np.random.default_rng(seed)
    p = mlp.init_params(rng)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.05
    s = arso.surrogate_create(seed)
    arso.surrogate_set_params(s, pack(p))
    arso.surrogate_set_norm(s, np.zeros(IN), np.ones(IN))
    pb = {k: mlp.bf16_round(v) for k, v in p.items()}      # what the GPU computes with
    x = rng.standard_normal((n, IN)).astype(np.float32)
    y = (rng.random(n) < 0.4).astype(np.float32)
    keep = _away_from_kinks(pb, x)
    return s, p, pb, x[keep], y[keep]


def _away_from_kinks(pb, x, margin=3e-5):
    """Rows whose hidden pre-activations all lie more than `margin` (relative to the
    sum of the absolute values of their terms) from zero. ReLU's derivative jumps
    at zero, so for a pre-activation within the FP32 accumulation error of zero the
    gradient mask is decided by rounding order, not by the inputs; the gradient
    comparisons use only rows where both sides must take the same decisions."""
    x = x.astype(np.float64)
    pre1 = x @ pb["W1"] + pb["b1"]
    h1 = np.maximum(pre1, 0.0)
    pre2 = h1 @ pb["W2"] + pb["b2"]
    r1 = np.abs(pre1) / (np.abs(x) @ np.abs(pb["W1"]) + np.abs(pb["b1"]))
    r2 = np.abs(pre2) / (h1 @ np.abs(pb["W2"]) + np.abs(pb["b2"]))
    return (r1.min(axis=1) > margin) & (r2.min(axis=1) > margin)


def test_forward_matches_reference(arso):
    s, p, pb, x, y = _setup(arso)
    dx = torch.from_numpy(x).cuda()
    out = torch.empty(x.shape[0], dtype=torch.float32, device="cuda")
    arso.surrogate_predict(s, dx, out)
    z, _ = mlp.forward(pb, x.astype(np.float64))
    assert np.max(np.abs(out.cpu().numpy() - mlp.sigmoid(z))) < 1e-5


def test_gradients_match_reference(arso):
    s, p, pb, x, y = _setup(arso, seed=1)
    g, loss = arso.surrogate_grads(s, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    z, cache = mlp.forward(pb, x.astype(np.float64))
    ref = mlp.backward(pb, cache, z, y.astype(np.float64))
    assert abs(loss - mlp.bce(z, y.astype(np.float64))) < 1e-6
    got = unpack(g)
    for k in ref:
        scale = np.max(np.abs(ref[k]))
        assert np.max(np.abs(got[k] - ref[k])) <= 1e-3 * scale + 1e-9, k


@pytest.mark.parametrize("n", [1000, 3000])
def test_large_batches_match_reference(arso, n):
    """Several 128-row output tiles with a ragged last one, and weight gradients
    whose batch dimension is split into 256-row chunks (the last one ragged) and
    summed in a fixed order."""
    s, p, pb, x, y = _setup(arso, seed=10 + n, n=n)
    assert x.shape[0] > 0.9 * n
    dx = torch.from_numpy(x).cuda()
    out = torch.empty(x.shape[0], dtype=torch.float32, device="cuda")
    arso.surrogate_predict(s, dx, out)
    z, cache = mlp.forward(pb, x.astype(np.float64))
    assert np.max(np.abs(out.cpu().numpy() - mlp.sigmoid(z))) < 1e-5
    g, loss = arso.surrogate_grads(s, dx, torch.from_numpy(y).cuda())
    ref = mlp.backward(pb, cache, z, y.astype(np.float64))
    assert abs(loss - mlp.bce(z, y.astype(np.float64))) < 1e-6
    got = unpack(g)
    for k in ref:
        scale = np.max(np.abs(ref[k]))
        assert np.max(np.abs(got[k] - ref[k])) <= 1e-3 * scale + 1e-9, k


def test_predict_across_its_row_chunks(arso):
    # predictions run in chunks of 65536 rows; 70,001 rows cross a chunk boundary and
    # end in a ragged 128-row tile
    s, p, pb, x, y = _setup(arso, seed=12, n=96)
    rng = np.random.default_rng(12)
    x = rng.standard_normal((70_001, IN)).astype(np.float32)
    out = torch.empty(x.shape[0], dtype=torch.float32, device="cuda")
    arso.surrogate_predict(s, torch.from_numpy(x).cuda(), out)
    z, _ = mlp.forward(pb, x.astype(np.float64))
    assert np.max(np.abs(out.cpu().numpy() - mlp.sigmoid(z))) < 1e-5


def test_gradients_are_deterministic(arso):
    s, p, pb, x, y = _setup(arso, seed=4, n=2500)
    dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    g1, l1 = arso.surrogate_grads(s, dx, dy)
    g2, l2 = arso.surrogate_grads(s, dx, dy)
    assert np.array_equal(np.asarray(g1), np.asarray(g2))


def test_one_adam_step_matches_reference(arso):
    s, p, pb, x, y = _setup(arso, seed=2, n=64)
    dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    arso.surrogate_train(s, dx, dy, epochs=1, batch=64, lr=1e-3, seed=0)
    z, cache = mlp.forward(pb, x.astype(np.float64))
    g = mlp.backward(pb, cache, z, y.astype(np.float64))
    master = {k: np.asarray(v, dtype=np.float64).copy() for k, v in unpack(pack(p)).items()}
    mlp.adam(master, g, {}, lr=1e-3)
    got = unpack(arso.surrogate_get_params(s))
    for k in master:
        # first Adam step moves each weight by lr * sign(g) (or less where g ~ 0)
        assert np.max(np.abs(got[k] - master[k])) < 2e-5, k


def test_training_learns_a_known_law(arso):
    """Labels drawn from P(pass) = sigmoid(3 - 2 x0 + x1); the trained network's
    prediction approaches that law (binary cross-entropy near its entropy floor)."""
    rng = np.random.default_rng(5)
    n = 200_000
    x = rng.standard_normal((n, IN)).astype(np.float32)
    pr = 1 / (1 + np.exp(-(3 - 2 * x[:, 0] + x[:, 1])))
    y = (rng.random(n) < pr).astype(np.float32)
    s = arso.surrogate_create(3)
    dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    loss = arso.surrogate_train(s, dx, dy, epochs=4, batch=2048, lr=2e-3, seed=1)
    floor = float(np.mean(-(pr * np.log(pr) + (1 - pr) * np.log(1 - pr))))
    assert loss < floor + 0.01
    xt = rng.standard_normal((4096, IN)).astype(np.float32)
    out = torch.empty(4096, dtype=torch.float32, device="cuda")
    arso.surrogate_predict(s, torch.from_numpy(xt).cuda(), out)
    truth = 1 / (1 + np.exp(-(3 - 2 * xt[:, 0] + xt[:, 1])))
    # 200k noisy 0/1 labels over 33 inputs, 31 of them irrelevant: a few percent of
    # estimation noise remains after 4 epochs
    assert np.mean(np.abs(out.cpu().numpy() - truth)) < 0.05


def test_surrogate_search_agrees_with_plain_search(arso):
    """Train on simulator rows from QAOA / brickwork circuits, then bracket the
    tolerable rate (pass fraction >= 2/3) of unseen circuits: the verified
    answer lies within 5% of the plain Monte Carlo search on the same random
    numbers, with fewer plain probes."""
    from paper_2301_07264_gb300 import surrogate_data
    from workloads import circuits as W
    train = [W.qaoa_maxcut(n, 100 + n + 20 * d) for n in (8, 10, 12) for d in range(3)]
    train += [W.brickwork(n, depth, 200 + n + depth) for n in (8, 10, 12) for depth in (4, 8, 12, 16)]
    for c in train:
        c.criterion = W.Criterion("fidelity", threshold=0.9, aggregate="pass")
    x, y = surrogate_data.generate(train, 300_000, seed=1, lp_lo=-4.5, lp_hi=-1.0, p_points=40)
    s = arso.surrogate_create(7)
    arso.surrogate_train(s, x, y, epochs=6, batch=4096, lr=2e-3, seed=2)
    test = [W.brickwork(10, 10, 901), W.qaoa_maxcut(12, 902)]
    for circ in test:
        crit = W.Criterion("fidelity", threshold=0.9, aggregate="pass")
        cc = arso.compile_circuit(circ.n, circ.gates)
        plain = arso.tolerable_rate(cc, crit, 2 / 3, n_traj=4000, seed=3, mode="mc", rel_tol=0.01,
                                    p_lo=1e-5, p_hi=1e-1)
        sur = arso.tolerable_rate_surrogate(cc, crit, 2 / 3, s, n_traj=4000, seed=3, margin=0.1,
                                            p_lo=1e-5, p_hi=1e-1)
        assert sur.used_surrogate == 1
        assert abs(sur.p - plain.p) / plain.p < 0.05, (circ.family, sur.p, plain.p)
        if sur.verified:
            assert sur.probes < plain.probes


def test_gemm_wait_that_runs_out_reports_timeout(arso):
    """The failure path of the tensor-core GEMM's bounded waits: a launch made to
    expect more TMA bytes than arrive gives up (no hang, no fault), the call
    returns ETIMEOUT, and the next call on the same context is correct again."""
    import time
    s, p, pb, x, y = _setup(arso, seed=3, n=300)
    dx = torch.from_numpy(x).cuda()
    out = torch.empty(x.shape[0], dtype=torch.float32, device="cuda")
    arso.debug_stall_next_gemm()
    t0 = time.perf_counter()
    with pytest.raises(arso.ArsoError) as e:
        arso.surrogate_predict(s, dx, out)
    assert e.value.status == arso.ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    arso.surrogate_predict(s, dx, out)
    z, _ = mlp.forward(pb, x.astype(np.float64))
    assert np.max(np.abs(out.cpu().numpy() - mlp.sigmoid(z))) < 1e-5
