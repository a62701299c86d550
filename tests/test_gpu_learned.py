"""GPU parity of the learned split proposer against the CPU oracle.

The model's FP32 forward pass, loss gradient and Adam steps are compared with the
oracle's FP64 ones within the tolerances FP32 arithmetic allows (forward 1e-5,
gradient 1e-4 relative to the gradient's norm); the splits it leads to, and every
merge made with them, must equal the oracle's exactly.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import NAME, first_diff, from_dev, to_dev

pytestmark = pytest.mark.gpu

H = 32


def _rand_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    p = np.concatenate([rng.normal(0, 4 * scale, H), rng.normal(0, 2 * scale, H),
                        rng.normal(0, 0.3 * scale, H), [rng.normal(0, 0.5)]])
    return p.astype(np.float32)


def _f32_dev(x, dev):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(dev)


def _u64_dev(x, dev):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x).astype(np.uint64).view(np.int64)).to(dev)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_forward_matches_oracle(ipm, dev, orc, seed):
    import torch

    p = _rand_params(seed)
    x = np.linspace(-0.25, 1.25, 3001).astype(np.float32)
    m = ipm.split_model_to_device(p, dev)
    y = torch.empty(x.size, dtype=torch.float32, device=dev)
    ipm.ipm_split_model_forward(m, _f32_dev(x, dev), x.size, y)
    torch.cuda.synchronize()
    want = orc.mlp_forward(p.astype(np.float64), H, x.astype(np.float64))
    got = y.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - want) / (1.0 + np.abs(want))) < 1e-5


@pytest.mark.parametrize("seed", [4, 5, 6])
@pytest.mark.parametrize("n", [1, 31, 4096, 10007])
def test_loss_grad_matches_oracle(ipm, dev, orc, seed, n):
    import torch

    p = _rand_params(seed)
    rng = np.random.default_rng(seed + 100)
    x = rng.random(n).astype(np.float32)
    t = np.clip(x + rng.normal(0, 0.05, n), 0, 1).astype(np.float32)
    m = ipm.split_model_to_device(p, dev)
    g = torch.empty(3 * H + 2, dtype=torch.float32, device=dev)
    ipm.ipm_split_model_loss_grad(m, _f32_dev(x, dev), _f32_dev(t, dev), n, g)
    torch.cuda.synchronize()
    got = g.cpu().numpy().astype(np.float64)
    loss, want = orc.mlp_loss_grad(p.astype(np.float64), H, x.astype(np.float64),
                                   t.astype(np.float64))
    assert abs(got[-1] - loss) <= 1e-5 * (1.0 + loss)
    assert np.linalg.norm(got[:-1] - want) <= 1e-4 * np.linalg.norm(want)


def _train_dev(ipm, dev, buf, la, lb, dt, diags, params, steps, lr):
    import torch

    m = ipm.split_model_to_device(params, dev)
    d = _u64_dev(diags, dev)
    ws = ipm.workspace(ipm.ipm_split_model_train_workspace_bytes(diags.size), dev)
    ipm.ipm_split_model_train(buf, la, lb, NAME[np.dtype(dt)], d, diags.size, m, ws,
                              steps=steps, lr=lr)
    torch.cuda.synchronize()
    assert ipm.ipm_read_device_status(ws) == 0
    return ipm.split_model_from_device(m)


def _oracle_train(orc, a, b, diags, params, steps, lr):
    """The same training on the CPU in FP64: exact targets by replay, then Adam."""
    n = a.size + b.size
    i = orc.splits_replay(a, b, diags.astype(np.uint64))
    x = (diags.astype(np.float64) / n).astype(np.float32).astype(np.float64)
    t = (i.astype(np.float64) / a.size).astype(np.float32).astype(np.float64)
    p = params.astype(np.float64).copy()
    mom, vel = np.zeros_like(p), np.zeros_like(p)
    for step in range(1, steps + 1):
        _, g = orc.mlp_loss_grad(p, H, x, t)
        orc.adam_step(p, mom, vel, g, lr, 0.9, 0.999, 1e-8, step)
    loss, _ = orc.mlp_loss_grad(p, H, x, t)
    return p, loss


@pytest.mark.parametrize("steps", [1, 10])
def test_adam_training_matches_oracle(ipm, dev, orc, steps):
    dt = np.float32
    a, b = W.make_pair("gmm", dt, 30_011, 20_021, seed=7)
    buf = to_dev(np.concatenate([a, b]), dev)
    diags = W.split_training_diagonals(a.size + b.size, 512, seed=3)
    p0 = ipm.split_model_initial_params()
    lr = 1e-3
    got, gloss, gsteps = _train_dev(ipm, dev, buf, a.size, b.size, dt, diags, p0, steps, lr)
    want, wloss = _oracle_train(orc, a, b, diags, p0, steps, lr)
    assert gsteps == steps
    # each Adam step moves a parameter by at most ~lr; FP32 and FP64 agree far closer
    assert np.max(np.abs(got - want)) <= 1e-3 * lr * steps + 1e-6
    assert abs(gloss - wloss) <= 1e-4 * (wloss + 1e-6)


def _gmm_buf(dev, la, lb, seed):
    import torch

    return W.make_buffer_torch(torch, "gmm", np.float32, la, lb, seed, dev)


@pytest.mark.parametrize("P", [1000, 1 << 12])
@pytest.mark.parametrize("dist,dt,ratio", [("gmm", np.float32, 0.75),
                                           ("uniform", np.int32, 0.75),
                                           ("uniform", np.uint64, 0.75),
                                           ("zipf", np.uint32, 1.0)])
def test_learned_splits_exact_and_cheaper(ipm, dev, orc, dist, dt, ratio, P):
    """Trained on the runs, the proposals cut the dependent probe rounds and the
    corrected splits equal the oracle's on every diagonal.  Smooth key distributions
    give a smooth split curve the model fits closely (rounds cut by a quarter or more);
    Zipf keys, where one key is ~18% of each run, put long straight stretches and sharp
    bends into the curve: the proposals are further off and only have to do no worse."""
    import torch

    la, lb = 1_000_003, 900_001
    a, b = W.make_pair(dist, dt, la, lb, seed=11)
    buf = to_dev(np.concatenate([a, b]), dev)
    diags = W.split_training_diagonals(la + lb, 4096, seed=5)
    model = ipm.train_split_model(buf, la, lb, NAME[np.dtype(dt)], _u64_dev(diags, dev),
                                  steps=300, lr=1e-2)
    p, loss, steps = ipm.split_model_from_device(model)
    assert steps == 300 and np.isfinite(loss)
    want = orc.splits_replay(a, b, orc.diagonals(la + lb, P))
    runs = {}
    for name, m in [("learned", model), ("plain", None)]:
        out = torch.empty(P + 1, dtype=torch.int64, device=dev)
        st = torch.zeros(5, dtype=torch.int64, device=dev)
        ipm.ipm_merge_splits_learned(buf, la, lb, NAME[np.dtype(dt)], P, m, out, st)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().astype(np.uint64), want), name
        runs[name] = st.cpu().numpy()
    assert runs["learned"][0] == runs["plain"][0] == P + 1
    # gain: fewer dependent probe rounds per diagonal
    assert runs["learned"][1] < ratio * runs["plain"][1], (P, runs["learned"][1] / runs["plain"][1])


def test_learned_splits_with_a_useless_model(ipm, dev, orc):
    """A model that proposes garbage (NaN, huge, negative) still yields the exact splits."""
    import torch

    dt = np.int32
    la, lb, P = 70_001, 130_003, 999
    a, b = W.make_pair("dup16", dt, la, lb, seed=2)
    buf = to_dev(np.concatenate([a, b]), dev)
    want = orc.splits_replay(a, b, orc.diagonals(la + lb, P))
    bad = [np.full(3 * H + 1, np.nan, np.float32), np.full(3 * H + 1, 1e30, np.float32),
           -_rand_params(9, 10.0)]
    for p in bad:
        m = ipm.split_model_to_device(p, dev)
        out = torch.empty(P + 1, dtype=torch.int64, device=dev)
        ipm.ipm_merge_splits_learned(buf, la, lb, "int32", P, m, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().astype(np.uint64), want)


@pytest.mark.parametrize("dist,dt", [("gmm", np.float32), ("uniform", np.int32),
                                     ("dup16", np.uint32), ("alternation", np.uint64),
                                     ("revdisjoint", np.int32), ("disjoint", np.int64),
                                     ("uniform", np.int64)])
@pytest.mark.parametrize("la,lb", [(1, 1), (5000, 0), (300_007, 299_993), (1_234_567, 77_777)])
def test_merge_inplace_learned_matches_oracle(ipm, dev, orc, dist, dt, la, lb):
    import torch

    a, b = W.make_pair(dist, dt, la, lb, seed=la ^ lb)
    host = np.concatenate([a, b])
    buf = to_dev(host, dev)
    n = la + lb
    if la >= 1:
        diags = W.split_training_diagonals(n, 1024, seed=1)
        model = ipm.train_split_model(buf, la, lb, NAME[np.dtype(dt)], _u64_dev(diags, dev),
                                      steps=100, lr=1e-2)
    else:
        model = ipm.split_model_to_device(ipm.split_model_initial_params(), dev)
    ws = ipm.workspace(ipm.ipm_merge_workspace_bytes(la, lb, NAME[np.dtype(dt)]), dev)
    ipm.ipm_merge_inplace_learned(buf, la, lb, NAME[np.dtype(dt)], model, ws)
    torch.cuda.synchronize()
    assert ipm.ipm_read_device_status(ws) == 0
    assert first_diff(from_dev(buf, dt), orc.merge(a, b)) is None


@pytest.mark.slow
def test_learned_fullsize_gmm_2p28x2(ipm, dev, orc):
    """float32 Gaussian-mixture runs of 2^28 each, P = 2^16: splits sampled against the
    oracle's bisection, the whole merged buffer against the oracle's merge."""
    import torch

    la = lb = 1 << 28
    P = 1 << 16
    buf = _gmm_buf(dev, la, lb, seed=0)
    host = W.as_numpy_keys(buf, np.float32)
    diags = W.split_training_diagonals(la + lb, 4096, seed=0)
    model = ipm.train_split_model(buf, la, lb, "float32", _u64_dev(diags, dev), steps=300,
                                  lr=1e-2)
    out = torch.empty(P + 1, dtype=torch.int64, device=dev)
    st = torch.zeros(5, dtype=torch.int64, device=dev)
    ipm.ipm_merge_splits_learned(buf, la, lb, "float32", P, model, out, st)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.uint64)
    dg = orc.diagonals(la + lb, P)
    for k in np.linspace(0, P, 65).astype(np.int64):
        assert got[k] == orc.split_bsearch(host[:la], host[la:], int(dg[k])), k
    stats = st.cpu().numpy()
    assert stats[1] / stats[0] < 5.0  # well below the ~6 rounds of the plain search
    ws = ipm.workspace(ipm.ipm_merge_workspace_bytes(la, lb, "float32"), dev)
    ipm.ipm_merge_inplace_learned(buf, la, lb, "float32", model, ws)
    torch.cuda.synchronize()
    assert ipm.ipm_read_device_status(ws) == 0
    want = orc.merge(host[:la], host[la:])
    assert first_diff(W.as_numpy_keys(buf, np.float32), want) is None
