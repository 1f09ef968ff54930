"""Pins of the surrogate MLP oracle: BF16 rounding against torch's own
conversion; back-propagation against central finite differences (FP64, no
rounding); padded columns stay inert."""
import numpy as np
import pytest

from oracle import mlp


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10 ** rng.uniform(-8, 8, 20000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 65504.0, 3.0e38, -1e-40]])
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), ref)


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = mlp.init_params(2)
    n = 7
    x = np.zeros((n, 16)); x[:, :4] = rng.standard_normal((n, 4))
    t = np.zeros((n, 48)); t[:, :40] = rng.standard_normal((n, 40))
    loss, g = mlp.loss_and_grads(p, x, t, rounding=False)
    h = 1e-6
    for li, (pi, gi) in enumerate(zip(p, g)):
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in pi.shape)
            if li == 0 and idx[1] >= 4:
                continue
            if li in (4, 5) and idx[0] >= 40:
                continue
            q = [a.copy() for a in p]
            q[li][idx] += h
            lp, _ = mlp.loss_and_grads(q, x, t, rounding=False)
            q[li][idx] -= 2 * h
            lm, _ = mlp.loss_and_grads(q, x, t, rounding=False)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gi[idx]) <= 1e-6 * (1 + abs(fd)), (li, idx, fd, gi[idx])


def test_padding_is_inert():
    rng = np.random.default_rng(3)
    p = mlp.init_params(4)
    x = np.zeros((5, 16)); x[:, :4] = rng.standard_normal((5, 4))
    t = np.zeros((5, 48)); t[:, :40] = rng.standard_normal((5, 40))
    _, g = mlp.loss_and_grads(p, x, t)
    assert np.all(g[0][:, 4:] == 0) and np.all(g[4][40:] == 0) and np.all(g[5][40:] == 0)
