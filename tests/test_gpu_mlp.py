"""Learned-entry MLP on the GPU (tcgen05 GEMMs) against the FP64 oracle.

Tolerances. The GPU and the oracle feed identical BF16 operands to every
contraction; the GPU accumulates in FP32 (error <= K * 2^-24 relative to the
sum of |products|) and the oracle in FP64. Hidden activations are rounded to
BF16 on both sides, so where the two sums straddle a BF16 rounding boundary
an activation differs by one BF16 ulp (2^-8 relative). Logits are therefore
checked elementwise against 2^-7 times the sum of |products| of the last
layer, and gradients (which pass through two such roundings) by relative
Frobenius norm 1e-2.
"""
import numpy as np
import pytest

from oracle import mlp as M

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2507_17094_gb300 as A
    assert torch.cuda.is_available()
    A.build()


def make_model(d, h1, h2, out, seed):
    rng = np.random.default_rng(seed)
    he = lambda fan: np.sqrt(2.0 / fan)  # noqa: E731
    return M.MLP((rng.standard_normal((h1, d)) * he(d)).astype(np.float32),
                 (rng.standard_normal(h1) * 0.1).astype(np.float32),
                 (rng.standard_normal((h2, h1)) * he(h1)).astype(np.float32),
                 (rng.standard_normal(h2) * 0.1).astype(np.float32),
                 (rng.standard_normal((out, h2)) * he(h2)).astype(np.float32),
                 (rng.standard_normal(out) * 0.1).astype(np.float32))


def gpu_mlp(m, max_batch):
    import paper_2507_17094_gb300 as A
    d, h1, h2, out = m.W1.shape[1], m.W1.shape[0], m.W2.shape[0], m.W3.shape[0]
    g = A.MLP(d, h1, h2, out, max_batch)
    g.set_params(m.W1, m.b1, m.W2, m.b2, m.W3, m.b3)
    return g


@pytest.mark.parametrize("dims", [(96, 256, 128, 1000, 300), (256, 512, 512, 2048, 1024), (64, 128, 128, 128, 8)])
def test_forward_logits_vs_oracle(dims):
    d, h1, h2, out, n = dims
    m = make_model(d, h1, h2, out, seed=1)
    X = np.random.default_rng(2).standard_normal((n, d)).astype(np.float32)
    g = gpu_mlp(m, max(8, (n + 7) // 8 * 8))
    z = g.forward(torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    g.sync()
    f = M.forward(m, X)
    scale = np.abs(f["h2q"]) @ np.abs(M.bf16_round(m.W3).astype(np.float64)).T + np.abs(m.b3)
    err = np.abs(z.cpu().numpy().astype(np.float64) - f["z"])
    assert (err <= 2.0 ** -7 * scale + 1e-5).all(), float((err / (scale + 1e-12)).max())
    g.close()


def test_gradients_vs_oracle():
    d, h1, h2, out, n = 96, 256, 128, 1000, 64
    m = make_model(d, h1, h2, out, seed=3)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((n, d)).astype(np.float32)
    y = rng.integers(0, out, n).astype(np.uint32)
    g = gpu_mlp(m, n)
    loss = torch.zeros(1, device="cuda")
    g.train_step(torch.from_numpy(X).cuda(), torch.from_numpy(y.view(np.int32)).cuda(), lr=0.0, loss=loss)
    torch.cuda.synchronize()
    g.sync()
    want = M.gradients(m, X, y.astype(np.int64))
    got = dict(zip(M.LAYERS, g.get(1)))
    for k in M.LAYERS:
        rel = np.linalg.norm(got[k] - want[k]) / (np.linalg.norm(want[k]) + 1e-30)
        assert rel < 1e-2, (k, rel)
    assert abs(loss.item() - M.loss(m, X, y.astype(np.int64))) < 1e-3 * max(1.0, M.loss(m, X, y.astype(np.int64)))
    # lr = 0 leaves the parameters unchanged
    p = g.get(0)
    assert all(np.array_equal(a, b) for a, b in zip(p, m.params().values()))
    g.close()


def test_adamw_step_vs_oracle():
    # One AdamW step from seeded weights. The oracle steps with its own FP64
    # gradients. A first Adam step moves every weight by lr * g/(|g| + eps),
    # i.e. by +-lr (plus decay), so the two agree to FP32 rounding wherever
    # the gradients agree in sign; they may differ by 2 lr only where a
    # gradient is so small that the GPU's BF16 rounding can flip its sign.
    d, h1, h2, out, n = 64, 128, 128, 256, 32
    lr, wd = 1e-2, 0.01
    m = make_model(d, h1, h2, out, seed=5)
    rng = np.random.default_rng(6)
    X = rng.standard_normal((n, d)).astype(np.float32)
    y = rng.integers(0, out, n).astype(np.uint32)
    g = gpu_mlp(m, n)
    g.train_step(torch.from_numpy(X).cuda(), torch.from_numpy(y.view(np.int32)).cuda(), lr=lr, weight_decay=wd)
    torch.cuda.synchronize()
    g.sync()
    grads = M.gradients(m, X, y.astype(np.int64))
    ref = m.copy()
    M.AdamW(lr=lr, wd=wd).step(ref, grads)
    got = dict(zip(M.LAYERS, g.get(0)))
    for k in M.LAYERS:
        diff = np.abs(got[k].astype(np.float64) - getattr(ref, k))
        small = np.abs(grads[k]) <= 2e-2 * np.sqrt(np.mean(grads[k] ** 2)) + 1e-12
        assert (diff[~small] <= 1e-6 + 1e-6 * np.abs(getattr(ref, k))[~small]).all(), k
        assert (diff <= 2 * lr + 1e-5).all(), k
        assert small.mean() < 0.5, k   # most entries are checked tightly
    g.close()


@pytest.mark.parametrize("P", [1, 8])
def test_fused_top_p(P):
    d, h1, h2, out, n = 96, 256, 256, 3000, 500
    m = make_model(d, h1, h2, out, seed=7)
    X = np.random.default_rng(8).standard_normal((n, d)).astype(np.float32)
    g = gpu_mlp(m, 512)
    Xt = torch.from_numpy(X).cuda()
    z = g.forward(Xt).cpu().numpy().astype(np.float64)
    seeds, pmax = g.predict(Xt, P=P, tau=0.0)
    torch.cuda.synchronize()
    g.sync()
    s = seeds.cpu().numpy().view(np.uint32)
    # 1. self-consistency: the fused epilogue picks the top P of the very
    #    logits the unfused GEMM writes (same FP32 values), ties to the
    #    smaller index, and its softmax maximum matches
    own = np.lexsort((np.broadcast_to(np.arange(out), z.shape), -z), axis=1)[:, :P]
    assert np.array_equal(s, own)
    e = np.exp(z - z.max(axis=1, keepdims=True))
    np.testing.assert_allclose(pmax.cpu().numpy(), 1.0 / e.sum(axis=1), rtol=1e-4)
    # 2. against the oracle's FP64 forward: equal sets except where the P-th
    #    and (P+1)-th oracle logits are closer than twice the row's largest
    #    GPU-oracle logit deviation (a near-tie the two precisions may order
    #    differently)
    f = M.forward(m, X)
    want, _ = M.top_p(f["z"], P)
    zs = np.sort(f["z"], axis=1)[:, ::-1]
    dev = np.abs(z - f["z"]).max(axis=1)
    gap_ok = (zs[:, P - 1] - zs[:, P]) > 2.0 * dev
    same = np.array([set(a) == set(b) for a, b in zip(s, want)])
    assert same[gap_ok].all() and gap_ok.mean() > 0.5, gap_ok.mean()
    # 3. fallback: rows below tau start with ANN_INVALID_ID
    tau = float(np.median(pmax.cpu().numpy()))
    s2, p2 = g.predict(Xt, P=P, tau=tau)
    s2 = s2.cpu().numpy().view(np.uint32)
    low = p2.cpu().numpy() < tau
    assert low.any() and (~low).any()
    assert (s2[low, 0] == 0xFFFFFFFF).all() and np.array_equal(s2[~low], s[~low])
    g.close()


def test_training_reduces_loss():
    # labels = the nearest of 64 random prototypes: learnable
    d, out, n = 96, 64, 1024
    rng = np.random.default_rng(9)
    protos = rng.standard_normal((out, d)).astype(np.float32)
    X = (protos[rng.integers(0, out, 4096)] + 0.3 * rng.standard_normal((4096, d))).astype(np.float32)
    y = np.argmin(((X[:, None, :] - protos[None]) ** 2).sum(-1), axis=1).astype(np.uint32)
    m = make_model(d, 256, 256, out, seed=10)
    g = gpu_mlp(m, n)
    Xt, yt = torch.from_numpy(X).cuda(), torch.from_numpy(y.view(np.int32)).cuda()
    loss = torch.zeros(1, device="cuda")
    losses = []
    for ep in range(15):
        for b in range(0, 4096, n):
            g.train_step(Xt[b:b + n], yt[b:b + n], lr=2e-3, loss=loss)
        losses.append(loss.item())
    g.sync()
    assert losses[-1] < 0.2 * losses[0], losses
    seeds, _ = g.predict(Xt, P=1)
    acc = (seeds.cpu().numpy()[:, 0].view(np.uint32) == y).mean()
    assert acc > 0.9, acc
    g.close()


def test_save_load_round_trip(tmp_path):
    """A saved and reloaded network has bit-identical parameters and logits."""
    import paper_2507_17094_gb300 as A
    m = make_model(64, 128, 128, 256, seed=5)
    g = gpu_mlp(m, 64)
    rng = np.random.default_rng(7)
    g.set_input_norm(rng.uniform(-1, 1, 64), rng.uniform(0.5, 2, 64))
    path = str(tmp_path / "mlp.bin")
    g.save(path)
    h = A.MLP.load(path, max_batch=64)
    assert h.dims == (64, 128, 128, 256)
    for a, b in zip(g.get(0) + list(g.get_input_norm()), h.get(0) + list(h.get_input_norm())):
        assert np.array_equal(a, b)
    X = torch.from_numpy(np.random.default_rng(6).standard_normal((40, 64)).astype(np.float32)).cuda()
    za, zb = g.forward(X), h.forward(X)
    torch.cuda.synchronize()
    assert torch.equal(za, zb)
    g.close()
    h.close()


def test_forward_with_input_standardisation():
    """Queries of magnitude ~50 standardised on the device match the oracle's
    FP32 standardisation followed by the same BF16 network."""
    d, h1, h2, out, n = 256, 512, 512, 1024, 200
    m = make_model(d, h1, h2, out, seed=8)
    rng = np.random.default_rng(9)
    m.mean = rng.uniform(20, 80, d).astype(np.float32)
    m.inv_std = (1.0 / rng.uniform(4, 12, d)).astype(np.float32)
    X = (m.mean + rng.standard_normal((n, d)) / m.inv_std).astype(np.float32)
    g = gpu_mlp(m, 256)
    g.set_input_norm(m.mean, m.inv_std)
    z = g.forward(torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    g.sync()
    f = M.forward(m, X)
    scale = np.abs(f["h2q"]) @ np.abs(M.bf16_round(m.W3).astype(np.float64)).T + np.abs(m.b3)
    err = np.abs(z.cpu().numpy().astype(np.float64) - f["z"])
    assert (err <= 2.0 ** -7 * scale + 1e-5).all(), float((err / (scale + 1e-12)).max())
    g.close()


def ulp_diff(a, b):
    """Distance in FP32 units in the last place (same-sign finite values)."""
    ia = np.asarray(a, np.float32).view(np.int32).astype(np.int64)
    ib = np.asarray(b, np.float32).view(np.int32).astype(np.int64)
    return np.abs(ia - ib)


@pytest.mark.parametrize("n,d", [(20_000, 96), (777, 256), (1, 64)])
def test_fit_input_norm_vs_oracle(n, d):
    """The device statistics (FP64 sums in chunk order) against the oracle's
    FP64 definition: both round one FP64 value to FP32, and the two FP64
    values differ only by summation order (relative 1e-15 at these sizes),
    so the FP32 results agree within one unit in the last place. A constant
    dimension takes the floored inverse."""
    rng = np.random.default_rng(n)
    X = (rng.standard_normal((n, d)) * rng.uniform(0.1, 60, d) + rng.uniform(-90, 90, d)).astype(np.float32)
    X[:, 3] = 12.5
    m = make_model(d, 128, 128, 64, seed=3)
    g = gpu_mlp(m, 64)
    g.fit_input_norm(torch.from_numpy(X).cuda())
    mu, isd = g.get_input_norm()
    want_mu, want_isd = M.input_norm_stats(X)
    assert (ulp_diff(mu, want_mu) <= 1).all() and (ulp_diff(isd, want_isd) <= 1).all()
    g.close()


@pytest.mark.parametrize("n", [1, 2, 5000, 100_003])
def test_confidence_threshold_vs_oracle(n):
    """tau is a rank selection, so it is bit-exact: random top
    probabilities with ties, at fallback fractions 0 .. 1 and beyond."""
    rng = np.random.default_rng(n + 1)
    v = rng.uniform(0.0, 1.0, n).astype(np.float32)
    if n > 4:
        v[: n // 4] = v[n // 2]
        v[-1] = 1.0
    m = make_model(64, 128, 128, 64, seed=3)
    g = gpu_mlp(m, 64)
    vt = torch.from_numpy(v).cuda()
    for q in (0.0, 1e-4, 0.05, 0.5, 0.95, 1.0, 2.0):
        assert g.confidence_threshold(vt, q) == M.lower_quantile(v, q), q
    g.close()


def test_checkpoint_resumes_training(tmp_path):
    """Saving after a few AdamW steps and loading restores the step count
    and the moments: the next step from the loaded copy gives the same
    parameters, bit for bit, as the next step of the original."""
    import paper_2507_17094_gb300 as A
    d, out, n = 64, 128, 64
    m = make_model(d, 128, 128, out, seed=11)
    g = gpu_mlp(m, n)
    rng = np.random.default_rng(12)
    X = torch.from_numpy(rng.standard_normal((n, d)).astype(np.float32)).cuda()
    y = torch.from_numpy(rng.integers(0, out, n).astype(np.int32)).cuda()
    for _ in range(3):
        g.train_step(X, y, lr=1e-3)
    g.sync()
    path = str(tmp_path / "mlp2.bin")
    g.save(path)
    h = A.MLP.load(path, max_batch=n)
    for a, b in zip(g.get(0), h.get(0)):
        assert np.array_equal(a, b)
    g.train_step(X, y, lr=1e-3)
    h.train_step(X, y, lr=1e-3)
    g.sync()
    h.sync()
    for a, b in zip(g.get(0), h.get(0)):
        assert np.array_equal(a, b)
    # a version-1 file (parameters only) still loads, with a fresh optimizer
    raw = open(path, "rb").read()
    dims = np.frombuffer(raw[8:24], np.uint32)
    body = 4 * (dims[1] * dims[0] + dims[1] + dims[2] * dims[1] + dims[2] + dims[3] * dims[2] + dims[3] + 2 * d)
    p1 = str(tmp_path / "mlp1.bin")
    open(p1, "wb").write(b"ANNMLP01" + raw[8:24 + int(body)])
    k = A.MLP.load(p1, max_batch=n)
    for a, b in zip(A.MLP.load(path, max_batch=n).get(0), k.get(0)):
        assert np.array_equal(a, b)
    g.close()
    h.close()
    k.close()


@pytest.mark.parametrize("h2,out,n", [(512, 20_000, 1000), (200, 9_000, 777)])
def test_fused_top_p_many_tiles_per_cta(h2, out, n):
    """Shapes where each persistent CTA computes dozens of tiles across
    several row blocks (the resident-A logits kernel reloads A at each row
    block switch), K = 512 and a ragged K = 200, a ragged last row block: the
    fused top-8 equals the top-8 of the logits the unfused kernel writes."""
    m = make_model(64, 128, h2, out, seed=17)
    X = np.random.default_rng(18).standard_normal((n, 64)).astype(np.float32)
    g = gpu_mlp(m, 1024)
    Xt = torch.from_numpy(X).cuda()
    z = g.forward(Xt).cpu().numpy().astype(np.float64)
    seeds, pmax = g.predict(Xt, P=8, tau=0.0)
    torch.cuda.synchronize()
    g.sync()
    own = np.lexsort((np.broadcast_to(np.arange(out), z.shape), -z), axis=1)[:, :8]
    assert np.array_equal(seeds.cpu().numpy().view(np.uint32), own)
    e = np.exp(z - z.max(axis=1, keepdims=True))
    np.testing.assert_allclose(pmax.cpu().numpy(), 1.0 / e.sum(axis=1), rtol=1e-4)
    g.close()
