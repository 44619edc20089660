"""Pins for the learned-entry MLP oracle: torch's own BF16 conversion, central
finite differences, torch autograd in FP64, torch.optim.AdamW, torch.topk."""
import numpy as np
import pytest
import torch

from oracle import mlp as M


def tiny(seed=0, d=8, h1=16, h2=16, out=32):
    rng = np.random.default_rng(seed)
    f = lambda *s: (rng.standard_normal(s) * 0.5).astype(np.float32)  # noqa: E731
    return M.MLP(f(h1, d), f(h1), f(h2, h1), f(h2), f(out, h2), f(out))


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(50_000).astype(np.float32) * 1e3,
                        (rng.integers(0, 2**32, 50_000, dtype=np.uint64).astype(np.uint32)
                         .view(np.float32))])
    x = x[np.isfinite(x) & (np.abs(x) < 3e38)]
    # exact ties: low half 0x8000 with both parities of the kept bit
    ties = (np.arange(1000, dtype=np.uint32) << 17 | 0x3F800000 | 0x8000).view(np.float32)
    x = np.concatenate([x, ties, -ties])
    want = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    assert np.array_equal(M.bf16_round(x), want)


def test_gradients_match_finite_differences():
    m = tiny()
    rng = np.random.default_rng(2)
    X = rng.standard_normal((5, 8)).astype(np.float32)
    y = rng.integers(0, 32, 5)
    g = M.gradients(m, X, y, bf16=False)
    h = 1e-3
    for k in M.LAYERS:
        w = getattr(m, k)
        flat = w.reshape(-1)
        for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            orig = float(flat[idx])
            mp = m.copy(); getattr(mp, k).reshape(-1)[idx] = orig + h
            mm = m.copy(); getattr(mm, k).reshape(-1)[idx] = orig - h
            # parameters are FP32: use the values actually stored
            hp = float(getattr(mp, k).reshape(-1)[idx]) - orig
            hm = orig - float(getattr(mm, k).reshape(-1)[idx])
            fd = (M.loss(mp, X, y, bf16=False) - M.loss(mm, X, y, bf16=False)) / (hp + hm)
            assert abs(fd - g[k].reshape(-1)[idx]) <= 1e-5 + 1e-4 * abs(fd), (k, idx)


def test_gradients_match_torch_autograd():
    m = tiny(3, d=12, h1=20, h2=24, out=40)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((7, 12)).astype(np.float32)
    y = rng.integers(0, 40, 7)
    g = M.gradients(m, X, y, bf16=False)
    P = {k: torch.tensor(v.astype(np.float64), requires_grad=True) for k, v in m.params().items()}
    x = torch.tensor(X.astype(np.float64))
    h1 = torch.relu(x @ P["W1"].T + P["b1"])
    h2 = torch.relu(h1 @ P["W2"].T + P["b2"])
    z = h2 @ P["W3"].T + P["b3"]
    L = torch.nn.functional.cross_entropy(z, torch.tensor(y))
    L.backward()
    assert abs(L.item() - M.loss(m, X, y, bf16=False)) < 1e-12
    for k in M.LAYERS:
        np.testing.assert_allclose(g[k], P[k].grad.numpy(), rtol=1e-10, atol=1e-13)


def test_adamw_matches_torch():
    m = tiny(5)
    rng = np.random.default_rng(6)
    X = rng.standard_normal((9, 8)).astype(np.float32)
    y = rng.integers(0, 32, 9)
    opt = M.AdamW(lr=1e-2, wd=0.01)
    P = {k: torch.tensor(v.astype(np.float64), requires_grad=True) for k, v in m.params().items()}
    topt = torch.optim.AdamW(list(P.values()), lr=1e-2, betas=(0.9, 0.999), eps=1e-8, weight_decay=0.01)
    for _ in range(3):
        g = M.gradients(m, X, y, bf16=False)
        for k in M.LAYERS:
            P[k].grad = torch.tensor(g[k])
        topt.step()
        opt.step(m, g)
        for k in M.LAYERS:   # keep both on the same (FP32-rounded) weights
            with torch.no_grad():
                np.testing.assert_allclose(getattr(m, k), P[k].numpy().astype(np.float32), rtol=2e-6, atol=1e-7)
                P[k].copy_(torch.tensor(getattr(m, k).astype(np.float64)))


def test_top_p_and_fallback_probability():
    rng = np.random.default_rng(7)
    z = rng.standard_normal((20, 100))
    z[0, 5] = z[0, 9] = 10.0                       # a tie: smaller index first
    ids, pmax = M.top_p(z, 4)
    vals, tidx = torch.topk(torch.tensor(z), 4, dim=1)
    assert np.array_equal(np.take_along_axis(z, ids.astype(np.int64), 1), vals.numpy())
    assert ids[0, 0] == 5 and ids[0, 1] == 9
    np.testing.assert_allclose(pmax, torch.softmax(torch.tensor(z), 1).max(1).values.numpy(), rtol=1e-12)


def test_standardisation_folds_into_the_first_layer():
    """(x - mean) * inv_std followed by layer 1 is the affine map with
    columns of W1 scaled by inv_std and b1 shifted by -W1' mean: the two
    forms agree up to FP32 rounding of the standardised inputs."""
    rng = np.random.default_rng(11)
    d, h1, h2, out = 12, 16, 16, 20
    m = M.MLP(rng.standard_normal((h1, d)).astype(np.float32), rng.standard_normal(h1).astype(np.float32),
              rng.standard_normal((h2, h1)).astype(np.float32), rng.standard_normal(h2).astype(np.float32),
              rng.standard_normal((out, h2)).astype(np.float32), rng.standard_normal(out).astype(np.float32))
    mean = rng.uniform(20, 80, d).astype(np.float32)
    inv_std = (1.0 / rng.uniform(2, 10, d)).astype(np.float32)
    X = (mean + rng.standard_normal((30, d)) / inv_std).astype(np.float32)
    mn = m.copy()
    mn.mean, mn.inv_std = mean, inv_std
    W1f = (m.W1.astype(np.float64) * inv_std.astype(np.float64)[None, :])
    mf = m.copy()
    mf.W1 = W1f
    mf.b1 = m.b1.astype(np.float64) - W1f @ mean.astype(np.float64)
    z_norm = M.forward(mn, X, bf16=False)["z"]
    Xd = X.astype(np.float64)
    a1 = Xd @ mf.W1.T + mf.b1
    h = np.maximum(a1, 0) @ m.W2.astype(np.float64).T + m.b2
    z_fold = np.maximum(h, 0) @ m.W3.astype(np.float64).T + m.b3
    np.testing.assert_allclose(z_norm, z_fold, rtol=1e-4, atol=1e-4 * np.abs(z_fold).max())
    # identity standardisation changes nothing, bit for bit
    mi = m.copy()
    mi.mean, mi.inv_std = np.zeros(d, np.float32), np.ones(d, np.float32)
    assert np.array_equal(M.forward(mi, X)["z"], M.forward(m, X)["z"])


def test_input_norm_stats_closed_forms():
    """Column 0 is 0..n-1 (mean (n-1)/2, population variance (n^2-1)/12),
    column 1 is constant (std 0: floored at 1e-6 of the largest std),
    column 2 alternates -a, +a (mean 0, std a), column 3 is 2x column 0 + 5."""
    n = 1001
    i = np.arange(n, dtype=np.float64)
    X = np.stack([i, np.full(n, 7.25), np.where(i % 2 == 0, -3.0, 3.0)[:n], 2 * i + 5], axis=1)
    X[-1, 2] = 0.0   # n odd: make the +-a column balance exactly (mean 0)
    mean, inv_std = M.input_norm_stats(X.astype(np.float32))
    sd0 = np.sqrt((n * n - 1) / 12.0)
    sd2 = np.sqrt(2 * 500 * 9.0 / n)
    assert mean[0] == np.float32((n - 1) / 2) and mean[1] == np.float32(7.25) and mean[2] == 0.0
    assert mean[3] == np.float32(n - 1 + 5)
    np.testing.assert_allclose(inv_std[[0, 2, 3]], np.float32([1 / sd0, 1 / sd2, 1 / (2 * sd0)]), rtol=1e-7)
    assert inv_std[1] == np.float32(1.0 / (1e-6 * 2 * sd0))


def test_input_norm_stats_matches_numpy_and_a_planted_mistake_fails():
    rng = np.random.default_rng(5)
    X = (rng.standard_normal((3000, 40)) * rng.uniform(0.1, 50, 40) + rng.uniform(-100, 100, 40)).astype(np.float32)
    mean, inv_std = M.input_norm_stats(X)
    x = X.astype(np.float64)
    assert np.array_equal(mean, x.mean(axis=0).astype(np.float32))
    np.testing.assert_allclose(inv_std, (1.0 / x.std(axis=0)).astype(np.float32), rtol=2.5e-7)
    # sample (n - 1) variance instead of the population one is detected
    wrong = (1.0 / x.std(axis=0, ddof=1)).astype(np.float32)
    assert not np.allclose(inv_std, wrong, rtol=1e-5)


def test_lower_quantile_matches_numpy():
    rng = np.random.default_rng(6)
    for n in (1, 2, 7, 100, 5000):
        v = rng.uniform(0, 1, n).astype(np.float32)
        v[: n // 3] = v[n // 2]    # ties
        for q in (0.0001, 0.05, 0.25, 0.5, 0.999, 1.0):
            assert M.lower_quantile(v, q) == np.quantile(v, q, method="lower")
    v = np.float32([0.9, 0.1, 0.5, 0.3, 0.7])
    assert M.lower_quantile(v, 0.25) == np.float32(0.3)     # position floor(0.25 * 4) = 1
    assert M.lower_quantile(v, 0.2) == np.float32(0.1)      # position floor(0.8) = 0
    assert M.lower_quantile(v, 0.0) == 0.0 and M.lower_quantile(np.float32([]), 0.5) == 0.0
    assert M.lower_quantile(v, 3.0) == np.float32(0.9)
