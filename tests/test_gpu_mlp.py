"""GPU parity of the surrogate network's kernels against the FP64 reference
(oracle/mlp.py): features, forward, gradient of the MSE loss (BF16 operands,
FP32 accumulation: cosine > 0.999 and relative L2 < 1e-2), the Adam update
(exact up to FP32 rounding given the same gradient), the ensemble statistics,
and convergence of training on a smooth target."""
import math

import numpy as np
import pytest
import torch

from gpu_util import ensure_built
from oracle import mlp as ref
from paper_0903_3852_gb300 import inputs, sde

pytestmark = pytest.mark.gpu


def _flat(params):
    return np.concatenate([p.reshape(-1) for p in params])


def _unflat(vec, layers=ref.LAYERS):
    out, o = [], 0
    for fin, fout in zip(layers[:-1], layers[1:]):
        out.append(vec[o:o + fin * fout].reshape(fout, fin))
        o += fin * fout
        out.append(vec[o:o + fout])
        o += fout
    return out


def _mlp(members=1, max_batch=1024, **kw):
    ensure_built()
    return sde.Mlp(members=members, max_batch=max_batch, **kw)


def test_param_layout_and_count():
    m = _mlp()
    assert m.n_params == ref.n_params() == 133_377
    p = m.get_params(0).cpu().numpy().astype(np.float64)
    layers = _unflat(p)
    for l, (fin, W) in enumerate(zip(ref.LAYERS[:-1], layers[0::2])):
        bound = 1.0 / math.sqrt(fin)
        assert np.all(np.abs(W) <= bound) and W.std() > 0.4 * bound  # U(-b, b) init
    assert m.get_params(0).cpu().numpy().tolist() == m.get_params(0).cpu().numpy().tolist()


def test_features_match_reference_scaling():
    m = _mlp()
    pts = inputs.surrogate_points(777, seed=3)
    X = m.features(sde.points_to_device(pts)).cpu().numpy().astype(np.float64)
    Xr = ref.scale_inputs(*[np.array([p[k] for p in pts]) for k in ("a", "omega", "f", "gamma", "D")])
    assert np.max(np.abs(X - Xr)) <= 2e-6


def _setup(B, seed):
    rng = np.random.default_rng(seed)
    params = ref.init_params(rng)
    X = rng.uniform(-1, 1, (B, 5))
    y = np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2]
    return params, X, y


def test_forward_and_gradient_against_fp64():
    B = 300  # ragged against the 64-row tiles
    params, X, y = _setup(B, 0)
    m = _mlp()
    m.set_params(0, torch.from_numpy(_flat(params).astype(np.float32)).cuda())
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    yd = torch.from_numpy(y.astype(np.float32)).cuda()
    mean, spread = m.forward(Xd)
    out_ref, _ = ref.forward(params, X.astype(np.float32).astype(np.float64))
    got = mean.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(got - out_ref) / np.linalg.norm(out_ref)
    assert rel < 1e-2, rel
    assert np.all(spread.cpu().numpy() == 0.0)
    g, loss = m.grad(0, Xd, yd)
    gref = _flat(ref.backward(params, X.astype(np.float32).astype(np.float64), y.astype(np.float32)))
    gg = g.cpu().numpy().astype(np.float64)
    cos = gg @ gref / (np.linalg.norm(gg) * np.linalg.norm(gref))
    rel = np.linalg.norm(gg - gref) / np.linalg.norm(gref)
    print("grad cosine %.6f rel L2 %.3e" % (cos, rel))
    assert cos > 0.999 and rel < 1e-2
    lref = ref.loss(params, X.astype(np.float32).astype(np.float64), y.astype(np.float32))
    assert abs(loss.item() - lref) <= 1e-2 * lref
    # each layer separately (the small output layer too)
    o = 0
    for fin, fout in zip(ref.LAYERS[:-1], ref.LAYERS[1:]):
        for size in (fin * fout, fout):
            a, b = gg[o:o + size], gref[o:o + size]
            assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b) + 1e-7
            o += size


def test_adam_update_matches_fp64_formula():
    B = 256
    params, X, y = _setup(B, 1)
    m = _mlp(lr=3e-3)
    p0 = _flat(params).astype(np.float32)
    m.set_params(0, torch.from_numpy(p0).cuda())
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    yd = torch.from_numpy(y.astype(np.float32)).cuda()
    g1, _ = m.grad(0, Xd, yd)
    m.train_step(Xd, yd)
    p1 = m.get_params(0).cpu().numpy().astype(np.float64)
    g1 = g1.cpu().numpy().astype(np.float64)
    new, mo, vo = ref.adam_step([p0.astype(np.float64)], [g1], [np.zeros_like(g1)], [np.zeros_like(g1)], 1,
                                lr=3e-3)
    assert np.max(np.abs(p1 - new[0])) <= 1e-6
    g2, _ = m.grad(0, Xd, yd)
    m.train_step(Xd, yd)
    p2 = m.get_params(0).cpu().numpy().astype(np.float64)
    new2, _, _ = ref.adam_step(new, [g2.cpu().numpy().astype(np.float64)], mo, vo, 2, lr=3e-3)
    assert np.max(np.abs(p2 - new2[0])) <= 2e-6


def test_ensemble_mean_and_spread():
    B = 200
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, (B, 5))
    m = _mlp(members=4, seed=7)
    mean, spread = m.forward(torch.from_numpy(X.astype(np.float32)).cuda())
    outs = []
    for q in range(4):
        p = _unflat(m.get_params(q).cpu().numpy().astype(np.float64))
        outs.append(ref.forward(p, X.astype(np.float32).astype(np.float64))[0])
    outs = np.array(outs)
    assert np.max(np.abs(mean.cpu().numpy() - outs.mean(0))) <= 2e-2 * np.abs(outs).max()
    sp = spread.cpu().numpy()
    assert np.all(sp > 0)
    assert np.corrcoef(sp, outs.std(0, ddof=1))[0, 1] > 0.95


def test_training_converges_on_smooth_target():
    rng = np.random.default_rng(4)
    n = 4096
    X = rng.uniform(-1, 1, (n, 5)).astype(np.float32)
    y = (0.5 * np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2] - 0.3 * X[:, 3] ** 2 + 0.1 * X[:, 4]).astype(np.float32)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    m = _mlp(members=2, max_batch=n, lr=2e-3, seed=1)
    loss = torch.zeros(2, device="cuda")
    perm_rng = np.random.default_rng(0)
    for step in range(600):
        idx = torch.from_numpy(perm_rng.integers(0, n, 256)).cuda()
        m.train_step(Xd[idx].contiguous(), yd[idx].contiguous(), loss)
    mean, _ = m.forward(Xd)
    mse = float(((mean - yd) ** 2).mean())
    print("train mse %.3e (target variance %.3e)" % (mse, float(yd.var())))
    assert mse < 0.02 * float(yd.var())


@pytest.mark.parametrize("B", [1, 127, 300, 1029])
def test_tensor_core_forward_against_cuda_core_and_fp64(B):
    """The fused tcgen05 forward (square layers on the tensor cores, 128-point
    tiles, ragged last tile) against the CUDA-core forward of the same
    parameters and against the FP64 reference network, for 4 members with
    different weights.  Both GPU forms round the same operands to BF16; they
    differ in summation order and in the SiLU evaluation, so an activation can
    round to the neighbouring BF16 value: the outputs agree to ~1e-3 of the
    output scale, and each is within the BF16 error of the FP64 network."""
    rng = np.random.default_rng(B)
    X = rng.uniform(-1, 1, (B, 5))
    m = _mlp(members=4, max_batch=2048, seed=11)
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    mean_tc, spread_tc = m.forward(Xd)
    m.check()
    m.use_tensor_cores(False)
    mean_cc, spread_cc = m.forward(Xd)
    m.use_tensor_cores(True)
    outs = []
    for q in range(4):
        p = _unflat(m.get_params(q).cpu().numpy().astype(np.float64))
        outs.append(ref.forward(p, X.astype(np.float32).astype(np.float64))[0])
    outs = np.array(outs)
    scale = max(1.0, np.abs(outs).max())
    a, b = mean_tc.cpu().numpy().astype(np.float64), mean_cc.cpu().numpy().astype(np.float64)
    print("B=%d: |tc - cuda-core| max %.2e, |tc - fp64| max %.2e, |cc - fp64| max %.2e (scale %.2f)"
          % (B, np.abs(a - b).max(), np.abs(a - outs.mean(0)).max(), np.abs(b - outs.mean(0)).max(), scale))
    assert np.all(np.isfinite(a))
    assert np.abs(a - b).max() <= 2e-3 * scale
    assert np.abs(a - outs.mean(0)).max() <= 1e-2 * scale
    sp_tc, sp_cc = spread_tc.cpu().numpy(), spread_cc.cpu().numpy()
    assert np.abs(sp_tc - sp_cc).max() <= 2e-3 * scale


def test_tensor_core_forward_after_training_and_selection():
    """After a few hundred Adam steps (trained weights, not just the initial
    ones) the tensor-core forward still matches the CUDA-core forward; a shape
    without the tensor-core path refuses it."""
    rng = np.random.default_rng(5)
    n = 2048
    X = rng.uniform(-1, 1, (n, 5)).astype(np.float32)
    y = (np.sin(3 * X[:, 0]) * X[:, 1] + X[:, 2] ** 2).astype(np.float32)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    m = _mlp(members=2, max_batch=n, lr=2e-3, seed=2)
    for step in range(300):
        idx = torch.from_numpy(rng.integers(0, n, 256)).cuda()
        m.train_step(Xd[idx].contiguous(), yd[idx].contiguous())
    a, _ = m.forward(Xd)
    m.use_tensor_cores(False)
    b, _ = m.forward(Xd)
    m.check()
    d = (a - b).abs().max().item()
    print("trained: |tc - cuda-core| max %.2e, target scale %.2f" % (d, float(yd.abs().max())))
    assert d <= 2e-3 * max(1.0, float(yd.abs().max()))
    small = _mlp(members=1, max_batch=64, hidden=128)
    with pytest.raises(sde.SDEError) as e:
        small.use_tensor_cores(True)
    assert e.value.status == sde.SDE_ERR_UNSUPPORTED
