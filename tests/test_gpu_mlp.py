"""MLP kernels (BF16 tensor cores, FP32 accumulation) against the FP64 oracle,
and the learned initial guess end to end."""

import numpy as np
import pytest
import torch

from oracle import mlp as OM
from paper_2308_08417_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N = 144
HID = 256


@pytest.fixture(scope="module")
def bbs():
    from paper_2308_08417_gb300 import _build, bbs as mod

    _build.build()
    return mod


@pytest.fixture(scope="module", params=["mma", "tcgen05"])
def net(bbs, request):
    h = bbs.Handle(0)
    m = bbs.MLP(h, N, hidden=HID, seed=7, max_batch=1024)
    m.set_gemm(request.param)
    return m


def sizes():
    return [3 * N, HID, HID, HID, N]


def random_setup(net, seed, M=256):
    rng = np.random.default_rng(seed)
    params = OM.init_params(sizes(), rng)
    net.set_params(torch.as_tensor(OM.flatten(params), dtype=torch.float32))
    # the GPU keeps FP32 masters; the oracle sees the same FP32-rounded values
    params = OM.unflatten(OM.flatten(params).astype(np.float32).astype(np.float64), sizes())
    X = rng.normal(size=(M, 3 * N))
    Xb = OM.to_bf16(X)
    feats = torch.zeros(M, net.in_pad, dtype=torch.bfloat16)
    feats[:, :3 * N] = torch.as_tensor(Xb, dtype=torch.float32).to(torch.bfloat16)
    Y = rng.normal(size=(M, N)).astype(np.float32)
    return params, Xb, feats.cuda(), Y


def test_forward_matches_oracle(net):
    params, Xb, feats, _ = random_setup(net, 1, M=300)
    out = net.forward(feats).cpu().numpy().astype(np.float64)
    ref, _ = OM.forward(params, Xb, round_bf16=True)
    rel = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert rel < 5e-3, rel
    net.check()


def test_gradients_match_oracle(net):
    params, Xb, feats, Y = random_setup(net, 2, M=256)
    targets = torch.as_tensor(Y, device="cuda")
    rows = torch.arange(256, dtype=torch.int32, device="cuda")
    loss = net.gradients(feats, targets, rows)
    g = net.get_grads().cpu().numpy().astype(np.float64)
    ref_loss, ref_grads = OM.loss_and_grads(params, Xb, Y.astype(np.float64), round_bf16=True)
    assert abs(float(loss) - ref_loss) / ref_loss < 1e-3
    ref = OM.flatten(ref_grads)
    o = 0
    for (W_, b_) in ref_grads:
        for part in (W_.ravel(), b_.ravel()):
            seg = g[o:o + part.size]
            rel = np.linalg.norm(seg - part) / np.linalg.norm(part)
            assert rel < 2e-2, (o, rel)
            o += part.size
    assert o == ref.size == net.param_count


def test_training_fits_a_smooth_map(net):
    """Adam on a learnable target (a fixed random linear map of the inputs)
    lowers the loss by a large factor."""
    rng = np.random.default_rng(3)
    params = OM.init_params(sizes(), rng)
    net.set_params(torch.as_tensor(OM.flatten(params), dtype=torch.float32))
    M = 4096
    X = rng.normal(size=(M, 3 * N))
    Wt = rng.normal(size=(3 * N, N)) / np.sqrt(3 * N)
    Y = np.tanh(X @ Wt).astype(np.float32)
    feats = torch.zeros(M, net.in_pad, dtype=torch.bfloat16)
    feats[:, :3 * N] = torch.as_tensor(X, dtype=torch.float32).to(torch.bfloat16)
    feats = feats.cuda()
    targets = torch.as_tensor(Y, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)
    losses = []
    for ep in range(40):
        perm = torch.randperm(M, device="cuda", generator=gen).to(torch.int32)
        for s in range(M // 1024):
            loss = net.train_step(feats, targets, perm[s * 1024:(s + 1) * 1024], 1e-3)
        losses.append(float(loss))
    assert losses[-1] < 0.25 * losses[0], losses


def test_standardisation_and_predict(bbs):
    """Targets are standardised per component with the observed mean and
    standard deviation; predict returns x_prev + out * std + mean."""
    net = bbs.MLP(bbs.Handle(0), N, hidden=HID, seed=11, max_batch=1024)
    net.set_gemm("mma")  # predict through the same layered GEMMs as forward()
    ts = W.time_stepped(num_batch=512, steps=4)
    dev = "cuda"
    A = bbs.DeviceBatch.from_batch(W.make_batch(ts.pattern, ts.values_at(1), "csr"), dev)
    b = torch.as_tensor(ts.rhs_at(1), device=dev)
    rng = np.random.default_rng(4)
    xp = torch.as_tensor(rng.normal(size=(512, N)), device=dev)
    delta = rng.normal(loc=0.2, scale=0.5, size=(512, N))
    xn = xp + torch.as_tensor(delta, device=dev)
    net.observe(A, b, xp, xn)
    net.finalize_stats()
    feats, targets = net.make_samples(A, b, xp, xn)
    d = (xn - xp).cpu().numpy()
    mu, sd = d.mean(axis=0), d.std(axis=0)
    t = targets.cpu().numpy()
    assert np.allclose(t, (d - mu) / sd, rtol=1e-4, atol=1e-4)
    # the diag / b / x_prev columns are standardised too: mean 0, std 1
    f = feats.float().cpu().numpy()[:, :3 * N]
    assert np.abs(f.mean(axis=0)).max() < 2e-2 and np.abs(f.std(axis=0) - 1).max() < 2e-2
    out = net.forward(feats).double().cpu().numpy()
    x0 = net.predict(A, b, xp)
    got = (x0 - xp).cpu().numpy()
    assert np.allclose(got, out * sd + mu, rtol=1e-4, atol=1e-5)


def test_learned_guess_pipeline(bbs):
    """The learned guess end to end on a small time-stepped batch: every solve
    still reaches the tolerance; the report shows what the network gains
    (initial residual and iterations against x0 = x(t-1))."""
    from paper_2308_08417_gb300.learned import TimeStepped

    ts = W.time_stepped(num_batch=2048, steps=40)
    run = TimeStepped(ts, hidden=HID, seed=0, max_batch=2048)
    rep = run.run(train_steps=32, eval_steps=6, epochs=4, batch=2048)
    s = rep.summary()
    print("learned-guess summary:", s)
    assert all(r.converged == 2048 for r in rep.records)
    assert s["final_loss"] < s["first_loss"]
    assert np.isfinite(s["init_residual_learned"]) and np.isfinite(s["iters_learned"])
    # on the held-out training steps the gated guess is no worse than x(t-1)
    assert 0.0 <= s["gate"] <= 1.0 and s["gate_steps"] == 8
    assert s["gate_steps_error_ratio"] <= 1.0 + 1e-9


def test_gate_is_the_least_squares_scale(bbs):
    """The gate gamma is sum c.d / sum c.c over the observed steps (c the
    predicted change, d the true one), limited to [0, 1]; with it the guess's
    squared error over those steps is at most that of x0 = x(t-1)."""
    net = bbs.MLP(bbs.Handle(0), N, hidden=HID, seed=5, max_batch=1024)
    ts = W.time_stepped(num_batch=512, steps=4)
    dev = "cuda"
    rng = np.random.default_rng(9)
    steps = []
    for t in (1, 2, 3):
        A = bbs.DeviceBatch.from_batch(W.make_batch(ts.pattern, ts.values_at(t), "csr"), dev)
        b = torch.as_tensor(ts.rhs_at(t), device=dev)
        xp = torch.as_tensor(rng.normal(size=(512, N)), device=dev)
        xn = xp + torch.as_tensor(rng.normal(scale=0.1, size=(512, N)), device=dev)
        steps.append((A, b, xp, xn))
    for A, b, xp, xn in steps:  # statistics so that the network's change is not tiny
        net.observe(A, b, xp, xn)
    net.finalize_stats()
    assert net.gate() == 1.0  # ungated before a fit
    cs = [(net.predict(A, b, xp) - xp) for A, b, xp, _ in steps]
    for A, b, xp, xn in steps:
        net.gate_observe(A, b, xp, xn)
    net.gate_finalize()
    g = net.gate()
    num = sum(float((c * (xn - xp)).sum()) for c, (_, _, xp, xn) in zip(cs, steps))
    den = sum(float((c * c).sum()) for c in cs)
    want = min(max(num / den, 0.0), 1.0)
    assert 0.0 <= g <= 1.0 and abs(g - want) <= 1e-9 * max(1.0, abs(want))
    err_gated = err_prev = 0.0
    for A, b, xp, xn in steps:
        x0 = net.predict(A, b, xp)
        err_gated += float(((xn - x0) ** 2).sum())
        err_prev += float(((xn - xp) ** 2).sum())
    assert err_gated <= err_prev * (1 + 1e-12)


def _fused_inputs(bbs, B, seed):
    ts = W.time_stepped(num_batch=B, steps=3)
    A = bbs.DeviceBatch.from_batch(W.make_batch(ts.pattern, ts.values_at(2), "csr"), "cuda")
    b = torch.as_tensor(ts.rhs_at(2), device="cuda")
    xp = torch.as_tensor(np.random.default_rng(seed).uniform(-1, 1, (B, N)), device="cuda")
    return ts, A, b, xp


def test_fused_predict_matches_oracle(bbs):
    """The fused tcgen05 network (one kernel for all four layers, 128 systems
    per block, a ragged last tile) against the FP64 oracle's forward pass with
    BF16 rounding where the GPU stores BF16. Standardisation is the identity
    before statistics are set, so x0 - x_prev is the network's output."""
    net = bbs.MLP(bbs.Handle(0), N, hidden=HID, seed=3, max_batch=1024)
    rng = np.random.default_rng(21)
    params = OM.init_params(sizes(), rng)
    net.set_params(torch.as_tensor(OM.flatten(params), dtype=torch.float32))
    params = OM.unflatten(OM.flatten(params).astype(np.float32).astype(np.float64), sizes())
    B = 300
    ts, A, b, xp = _fused_inputs(bbs, B, 5)
    x0 = net.predict(A, b, xp)
    net.check()
    got = (x0 - xp).cpu().numpy()
    vals = ts.values_at(2)
    rows = np.repeat(np.arange(N), np.diff(ts.pattern.row_ptrs))
    diag = vals[:, np.nonzero(rows == ts.pattern.col_idxs)[0]]
    X = np.concatenate([diag, ts.rhs_at(2), xp.cpu().numpy()], axis=1)
    ref, _ = OM.forward(params, OM.to_bf16(X), round_bf16=True)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel < 1e-2, rel


def test_fused_and_layered_paths_agree(bbs):
    """The same network through the fused kernel (tcgen05) and through the
    layered mma.sync GEMMs: predictions and gate statistics agree to BF16
    accuracy."""
    net = bbs.MLP(bbs.Handle(0), N, hidden=HID, seed=8, max_batch=2048)
    B = 1000
    ts, A, b, xp = _fused_inputs(bbs, B, 6)
    noise = torch.as_tensor(np.random.default_rng(2).normal(scale=0.05, size=(B, N)), device="cuda")
    net.observe(A, b, xp, xp + noise)
    net.finalize_stats()
    c = {}
    for kind in ("tcgen05", "mma"):  # gamma = 1 until a gate is fitted
        net.set_gemm(kind)
        c[kind] = net.predict(A, b, xp) - xp
    assert float(torch.linalg.norm(c["tcgen05"] - c["mma"]) / torch.linalg.norm(c["mma"])) < 1e-2
    # a true change that is half the predicted one plus noise: gamma near 0.5
    xn = xp + 0.5 * c["mma"] + 0.1 * torch.linalg.norm(c["mma"]) / np.sqrt(B * N) * noise / 0.05
    g = {}
    for kind in ("tcgen05", "mma"):
        net.set_gemm(kind)
        net.gate_observe(A, b, xp, xn)
        net.gate_finalize()
        g[kind] = net.gate()
        net.check()
    assert 0.3 < g["mma"] < 0.7 and abs(g["tcgen05"] - g["mma"]) < 2e-2 * g["mma"]
