"""Surrogate (sur_*) on the GPU against the FP64 MLP oracle.

Gradients of one member on a ragged batch (150 rows = two full 64-row tiles
and a 22-row tail) must match the oracle's BF16-rounded back-propagation;
prediction (ensemble mean and spread, de-standardised) must match the oracle's
forward pass of each member; training must fit a smooth map; the member
spread must grow off the training range, which is what routes a query to the
simulation.
"""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu

RNG_X = dict(phi=(0.1, 0.6), gamma=(1.0, 10.0), zeta=(0.01, 1.0), fp=(0.0, 3.0))


def _rows(n, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    cols = []
    for lo, hi in RNG_X.values():
        mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo) * scale
        cols.append(rng.uniform(mid - half, mid + half, n))
    X = np.stack(cols, axis=1)
    X[:, 1:3] = np.abs(X[:, 1:3]) + 1e-3
    return X.astype(np.float32)


def _smooth_targets(X):
    x = X.astype(np.float64)
    lg, lz = np.log(x[:, 1]), np.log(x[:, 2])
    c = np.arange(40)[None, :]
    return (np.sin(0.3 * c + 2.0 * x[:, :1]) * (1.0 + 0.2 * lg[:, None]) + 0.1 * c * lz[:, None] * 0.1
            + 0.5 * np.cos(0.1 * c * x[:, 3:4])).astype(np.float32)


def _std_inputs(X, mu, sd):
    """The device's input transform in FP32: log of gamma and zeta, then
    (x - mu) / sd; returns the padded [n][16] FP64 matrix fed to the oracle."""
    x = X.astype(np.float32).copy()
    x[:, 1:3] = np.log(np.maximum(x[:, 1:3], np.float32(1e-30)))
    z = (x - mu.astype(np.float32)) / sd.astype(np.float32)
    out = np.zeros((X.shape[0], 16))
    out[:, :4] = z
    return out


def _params32(seed):
    return [np.asarray(a, np.float32) for a in mlp.init_params(seed)]


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


@pytest.fixture
def sur():
    from paper_1310_0998_gb300.surrogate import Surrogate
    s = Surrogate(members=2, max_rows=512, seed=7)
    yield s
    s.close()


def _scaling(seed):
    rng = np.random.default_rng(seed)
    mu_x = np.array([0.35, 1.1, -2.3, 1.5], np.float32)
    sd_x = np.array([0.15, 0.6, 1.2, 0.9], np.float32)
    mu_y = rng.standard_normal(40).astype(np.float32)
    sd_y = (0.5 + rng.uniform(0, 2, 40)).astype(np.float32)
    return mu_x, sd_x, mu_y, sd_y


def test_gradients_match_oracle(sur):
    p = _params32(11)
    sur.set_weights(1, p)
    mu_x, sd_x, mu_y, sd_y = _scaling(12)
    sur.set_scaling(mu_x, sd_x, mu_y, sd_y)
    n = 150
    X = _rows(n, 13)
    Y = np.random.default_rng(14).standard_normal((n, 40)).astype(np.float32)
    loss, g = sur.gradients(1, X, Y)
    x = _std_inputs(X, mu_x, sd_x)
    t = np.zeros((n, 48))
    t[:, :40] = (Y - mu_y) / sd_y
    lo, go = mlp.loss_and_grads([a.astype(np.float64) for a in p], x, t)
    assert abs(loss - lo) <= 1e-3 * lo
    for name, a, b in zip(("W1", "b1", "W2", "b2", "W3", "b3"), g, go):
        assert a.shape == b.shape
        assert _rel(a, b) <= 2e-3, (name, _rel(a, b))
    # padded input columns and output rows get exactly zero gradient
    assert np.all(g[0][:, 4:] == 0) and np.all(g[4][40:] == 0) and np.all(g[5][40:] == 0)


@pytest.mark.parametrize("n", [150, 1, 512])
def test_gradients_tcgen05_equal_mma_sync(sur, n):
    """The training products run on tcgen05 (default) or on warp-level
    mma.sync; both accumulate in FP32 from the same BF16 operands, so the loss
    and every gradient agree to FP32 accumulation-order rounding."""
    p = _params32(31)
    sur.set_weights(0, p)
    sur.set_scaling(*_scaling(32))
    X = _rows(n, 33)
    Y = np.random.default_rng(34).standard_normal((n, 40)).astype(np.float32)
    sur.set_backend(True)
    lt, gt = sur.gradients(0, X, Y)
    sur.set_backend(False)
    lm, gm = sur.gradients(0, X, Y)
    sur.set_backend(True)
    assert abs(lt - lm) <= 1e-5 * abs(lm)
    for name, a, b in zip(("W1", "b1", "W2", "b2", "W3", "b3"), gt, gm):
        assert _rel(a, b) <= 2e-3, (name, _rel(a, b))


def test_single_row_and_full_capacity(sur):
    p = _params32(21)
    sur.set_weights(0, p)
    mu_x, sd_x, mu_y, sd_y = _scaling(22)
    sur.set_scaling(mu_x, sd_x, mu_y, sd_y)
    pd = [a.astype(np.float64) for a in p]
    for n in (1, 512):
        X = _rows(n, 23 + n)
        Y = np.random.default_rng(n).standard_normal((n, 40)).astype(np.float32)
        loss, g = sur.gradients(0, X, Y)
        t = np.zeros((n, 48))
        t[:, :40] = (Y - mu_y) / sd_y
        lo, go = mlp.loss_and_grads(pd, _std_inputs(X, mu_x, sd_x), t)
        assert abs(loss - lo) <= 1e-3 * lo
        for a, b in zip(g, go):
            assert _rel(a, b) <= 2e-3


def test_rejects_oversize_and_bad_member(sur):
    from paper_1310_0998_gb300._lib import DpdError
    with pytest.raises(DpdError):
        sur.gradients(0, _rows(513, 1), np.zeros((513, 40), np.float32))
    with pytest.raises(DpdError):
        sur.gradients(2, _rows(4, 1), np.zeros((4, 40), np.float32))


def test_predict_matches_oracle_members(sur):
    ps = [_params32(31), _params32(32)]
    for k, p in enumerate(ps):
        sur.set_weights(k, p)
    mu_x, sd_x, mu_y, sd_y = _scaling(33)
    sur.set_scaling(mu_x, sd_x, mu_y, sd_y)
    n = 100
    X = _rows(n, 34)
    Y, S = sur.predict(X)
    x = _std_inputs(X, mu_x, sd_x)
    ys = np.stack([mlp.forward([a.astype(np.float64) for a in p], x)["y"][:, :40] * sd_y + mu_y for p in ps])
    mean, spread = ys.mean(axis=0), ys.std(axis=0)
    scale = np.abs(ys).max() + 1.0
    assert np.max(np.abs(Y - mean)) <= 2e-3 * scale
    assert np.max(np.abs(S - spread)) <= 2e-3 * scale


@pytest.mark.parametrize("n", [128, 300, 4096])
def test_tensor_core_prediction(n):
    """Prediction with the tcgen05 forward products (n >= 128 rows, ragged
    tails included) against the mma.sync products and the FP64 oracle."""
    from paper_1310_0998_gb300.surrogate import Surrogate
    s = Surrogate(members=2, max_rows=4096, seed=9)
    try:
        ps = [_params32(61), _params32(62)]
        for k, p in enumerate(ps):
            s.set_weights(k, p)
        mu_x, sd_x, mu_y, sd_y = _scaling(63)
        s.set_scaling(mu_x, sd_x, mu_y, sd_y)
        X = _rows(n, 64)
        s.set_backend(True)
        Yt, St = s.predict(X)
        s.set_backend(False)
        Ym, Sm = s.predict(X)
    finally:
        s.close()
    scale = np.abs(Ym).max() + 1.0
    assert np.max(np.abs(Yt - Ym)) <= 2e-3 * scale
    assert np.max(np.abs(St - Sm)) <= 2e-3 * scale
    x = _std_inputs(X, mu_x, sd_x)
    ys = np.stack([mlp.forward([a.astype(np.float64) for a in p], x)["y"][:, :40] * sd_y + mu_y for p in ps])
    assert np.max(np.abs(Yt - ys.mean(axis=0))) <= 2e-3 * scale


def test_training_fits_and_spread_grows_off_range():
    from paper_1310_0998_gb300.surrogate import Surrogate
    s = Surrogate(members=4, max_rows=1024, seed=3)
    try:
        X = _rows(512, 41)
        Y = _smooth_targets(X)
        first = s.fit(X, Y, epochs=1, batch=64, lr=2e-3)
        last = s.fit(X, Y, epochs=300, batch=64, lr=2e-3)
        assert last < 0.5 * first and last < 0.02, (first, last)
        Xt = _rows(128, 42)
        P, S_in = s.predict(Xt)
        Yt = _smooth_targets(Xt)
        err = np.sqrt(np.mean((P - Yt) ** 2)) / np.std(Yt)
        assert err < 0.15, err
        Xo = _rows(128, 43, scale=4.0)
        _, S_out = s.predict(Xo)
        assert np.median(S_out) > 2.0 * np.median(S_in)
    finally:
        s.close()


def test_query_falls_back_to_simulation():
    """Off the training range the members disagree; such a row is answered by
    a plain simulation of that point, the others by the network."""
    from paper_1310_0998_gb300.surrogate import Surrogate, simulate
    s = Surrogate(members=4, max_rows=1024, seed=5)
    try:
        X = _rows(256, 51)
        s.fit(X, _smooth_targets(X), epochs=100, batch=64, lr=2e-3)
        P, S = s.predict(X)
        threshold = 2.0 * float(np.max(S / (np.abs(P) + 1.0)))
        # stable physics (gamma dt, zeta dt < 1) but 4-6 standard deviations
        # outside the training inputs in ln gamma and ln zeta
        far = np.array([[0.3, 0.05, 20.0, 0.5]], np.float32)
        kw = dict(L=16.0, burn=20, n_snap=2, every=10)
        rows = np.concatenate([X[:1], far])
        Yq, fb = s.query(rows, threshold=threshold, simulate_kw=kw)
        assert not fb[0] and fb[1]
        np.testing.assert_allclose(Yq[0], P[0], rtol=1e-6)
        # the fallback runs row i with seed + i and replica i, as simulate does
        ref = simulate(rows, batched=False, **kw)
        _close_stats(Yq[1], ref[1])
    finally:
        s.close()


def _close_stats(a, b):
    """Two runs of the same point follow the same trajectory bit for bit (the
    step is deterministic), so their statistics differ only by the summation
    order of the FP64 reductions inside the observables, and by the FP32
    rounding of the query's output."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-6)


def test_statistics_batched_equals_sequential():
    """The ensemble path and one simulation at a time give the same
    statistics (same seeds and replica keys)."""
    from paper_1310_0998_gb300.surrogate import simulate
    X = np.array([[0.3, 4.5, 0.1, 1.0], [0.45, 2.0, 0.5, 2.0]], np.float32)
    kw = dict(L=16.0, burn=30, n_snap=2, every=10)
    a = simulate(X, batched=True, **kw)
    b = simulate(X, batched=False, **kw)
    assert np.all(np.isfinite(a))
    _close_stats(a, b)


def test_network_beats_baselines_on_simulator_statistics():
    """Trained on statistics this simulator generates (batched ensemble, short
    runs at L = 32), the network predicts held-out points (plain simulations)
    better than the two predictors that use no model: the training mean, and
    the statistics of the nearest training point in standardised inputs."""
    from paper_1310_0998_gb300 import synth
    from paper_1310_0998_gb300.surrogate import Surrogate, simulate
    kw = dict(L=32.0, burn=600, n_snap=4, every=100)
    X = synth.surrogate_points(320, seed=61).astype(np.float32)
    Xtr, Xte = X[:256], X[256:]
    Ytr = simulate(Xtr, batched=True, seed=0, **kw)
    Yte = simulate(Xte, batched=False, seed=1000, **kw)
    s = Surrogate(members=4, max_rows=1024, seed=9)
    try:
        s.fit(Xtr, Ytr, epochs=300, batch=32, lr=2e-3)
        P, _ = s.predict(Xte)
    finally:
        s.close()
    sd = Ytr.std(axis=0) + 1e-12
    cols = [c for c in range(40) if c != 37]          # the argmax k is integer-valued
    rms = lambda A: float(np.sqrt(np.mean(((A - Yte) / sd)[:, cols] ** 2)))
    z = lambda A: (np.stack([A[:, 0], np.log(A[:, 1]), np.log(A[:, 2]), A[:, 3]], 1))
    ztr, zte = z(Xtr.astype(np.float64)), z(Xte.astype(np.float64))
    mu, sz = ztr.mean(0), ztr.std(0)
    nn = np.argmin((((zte[:, None, :] - ztr[None, :, :]) / sz) ** 2).sum(-1), axis=1)
    e_net, e_mean, e_nn = rms(P), rms(np.broadcast_to(Ytr.mean(0), Yte.shape)), rms(Ytr[nn])
    assert e_net < 0.7 * e_mean and e_net < e_nn, (e_net, e_mean, e_nn)
