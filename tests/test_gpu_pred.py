"""GPU-vs-oracle parity of the offline performance predictor (Sec.
"Performance Prediction Model": seven profiling inputs -> SELU MLP -> the
run's normalised performance), run by the NCF training kernel in its
dense-feature mode.  Tolerances as for NCF: BF16-operand gradients within
2e-2 (relative Frobenius, per group) of the FP64 oracle; predictions within
2e-2 of the magnitude of the terms the output sums."""
import numpy as np
import pytest
import torch

import synth

from gpu_util import DEV, dev, host

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU hosts deselect these
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2508_07605_b300 as ocf  # noqa: E402

NF = 7
SELU_L, SELU_A = 1.0507009873554804934193349852946, 1.6732632423543772848170429916717


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _params(seed):
    rng = np.random.default_rng(seed)
    return _f32(synth.pred_init(rng, NF, out_scale=1.0) + 0.05 * rng.standard_normal(9345))


def _rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("batch,B", [(512, 512), (512, 300), (64, 5)])
def test_pred_gradient_matches_oracle(orc, batch, B):
    runs = synth.make_counters(seed=2, n_apps=8, n_cpu=8, n_gpu=16)
    sel = np.random.default_rng(3).choice(len(runs.y), B, replace=False)
    X, y = _f32(runs.X[sel]), _f32(runs.y[sel])
    params = _params(1)
    h = ocf.Predictor(NF, batch=batch)
    h.set_params(dev(params, torch.float32))
    loss, g = h.grad(dev(X, torch.float32), dev(y, torch.float32))
    torch.cuda.synchronize()
    L, gr = orc.pred_loss_grad(X, y, params, NF)
    assert abs(host(loss)[0] - L) <= 1e-2 * L
    g = host(g)
    w1, b1, w2 = NF * 128, NF * 128 + 128, NF * 128 + 128 + 128 * 64
    for a0, a1 in [(0, w1), (w1, b1), (b1, w2), (w2, len(g))]:
        assert _rel(g[a0:a1], gr[a0:a1]) <= 2e-2, (a0, _rel(g[a0:a1], gr[a0:a1]))
    h.close()


@pytest.mark.parametrize("N", [1, 63, 64, 10007])
def test_pred_inference_matches_oracle(orc, N):
    runs = synth.make_counters(seed=4, n_apps=16, n_cpu=16, n_gpu=64)
    X = _f32(runs.X[:N])
    params = _params(5)
    h = ocf.Predictor(NF, batch=64)
    h.set_params(dev(params, torch.float32))
    y = host(h.infer(dev(X, torch.float32))).astype(np.float64)
    torch.cuda.synchronize()
    layers = orc.pred_unpack(params, NF)
    _, Z2, Y = orc.mlp_forward(X, layers)
    h2 = np.where(Z2 > 0, SELU_L * Z2, SELU_L * SELU_A * np.expm1(np.minimum(Z2, 0)))
    scale = np.abs(h2 * layers[4][:, 0]).sum(1) + abs(layers[5][0])
    err = np.abs(y - Y[:, 0]) / scale
    assert err.max() <= 2e-2, err.max()
    h.close()


def test_pred_adam_step_and_training_track_the_oracle(orc):
    runs = synth.make_counters(seed=6, n_apps=24, n_cpu=8, n_gpu=16)
    train = runs.app < 16
    X, y = _f32(runs.X[train]), _f32(runs.y[train])
    Xh, yh = _f32(runs.X[~train]), _f32(runs.y[~train])
    rng = np.random.default_rng(0)
    params = _f32(synth.pred_init(rng, NF))
    epochs, batch, lr = 15, 256, 3e-3
    perms = synth.ncf_perms(rng, len(y), epochs)
    h = ocf.Predictor(NF, batch=batch)
    h.set_params(dev(params, torch.float32))
    Xd, yd = dev(X, torch.float32), dev(y, torch.float32)
    # the GPU's own gradient of the first batch (for the Adam check below)
    first = perms[0][:batch]
    _, g = h.grad(dev(X[first], torch.float32), dev(y[first], torch.float32))
    L = h.train(Xd, yd, dev(np.stack(perms), torch.int32), lr, losses=True)
    p_g = host(h.get_params()).astype(np.float64)
    torch.cuda.synchronize()
    p_o, L_o = orc.pred_train(X, y, params, NF, perms, batch, lr)
    Lg = host(L)
    assert len(Lg) == len(L_o)
    assert np.abs(Lg[:5] - L_o[:5]).max() <= 2e-2 * L_o[:5].max()
    assert Lg[-10:].mean() <= 1.2 * L_o[-10:].mean() + 1e-5
    rg = np.sqrt(np.mean((orc.pred_forward(Xh, p_g, NF) - yh) ** 2))
    ro = np.sqrt(np.mean((orc.pred_forward(Xh, p_o, NF) - yh) ** 2))
    assert rg <= 1.15 * ro + 2e-3, (rg, ro)
    # the first step's update is Adam on the GPU gradient (checked on a fresh handle)
    h.set_params(dev(params, torch.float32))
    ident = dev(np.arange(len(first), dtype=np.int32)[None, :], torch.int32)
    h.train(dev(X[first], torch.float32), dev(y[first], torch.float32), ident, lr)
    p1 = host(h.get_params()).astype(np.float64)
    ref = params.copy()
    orc.adam(ref, host(g).astype(np.float64), np.zeros_like(ref), np.zeros_like(ref), 1, lr=lr)
    assert np.abs(p1 - ref).max() <= 1e-6 + 1e-3 * lr
    h.close()


def test_pred_argument_errors():
    with pytest.raises(ocf.OpenCFError) as e:
        ocf.Predictor(0)
    assert e.value.code == ocf.INVALID_ARG
    h = ocf.Predictor(NF, batch=64)
    x = torch.zeros(7, device=DEV)
    with pytest.raises(ocf.OpenCFError) as e:
        h.infer(x)                                # parameters not set
    assert e.value.code == ocf.NOT_FITTED
    h.close()


def test_pred_empty_inference():
    h = ocf.Predictor(NF, batch=64)
    h.set_params(dev(_params(2), torch.float32))
    y = h.infer(torch.zeros((0, NF), dtype=torch.float32, device=DEV))
    torch.cuda.synchronize()
    assert y.shape == (0,)
    h.close()


def test_online_full_size_sampled(orc):
    """The online workload at full size, as the benchmark runs it: the
    predictor trained on 1024 apps' runs (20 epochs), V fitted on their dense
    matrix, then 65,536 new apps x 16 profiled runs through predictor ->
    fold-in -> reconstruction + Algorithm 2.  Sampled: predictions against
    the oracle's forward pass with the GPU's trained parameters; fold-in rows
    against the oracle's solves on the GPU's predictions; decisions against
    the oracle's Algorithm 2 on the GPU's own T, bit for bit."""
    from gpu_util import TOL_FP32, solve_err
    n_cpu, n_gpu, k, lam = 16, 64, 16, 0.05
    cpu, gpu = synth.cap_grid(n_cpu, n_gpu)
    n = n_cpu * n_gpu
    f32 = torch.float32
    off = synth.make_counters(seed=0, n_apps=1024, n_cpu=n_cpu, n_gpu=n_gpu)
    rng = np.random.default_rng(0)
    pred = ocf.Predictor(NF, batch=1024)
    pred.set_params(dev(synth.pred_init(rng, NF), f32))
    perms = dev(np.stack(synth.ncf_perms(rng, len(off.y), 20)), torch.int32)
    pred.train(dev(off.X, f32), dev(off.y, f32), perms, 2e-3)
    h = ocf.OpenCF(k=k, lam=lam, sweeps=15, cpu_caps=cpu, gpu_caps=gpu)
    h.set_V(dev(synth.init_factor(rng, n, k), f32))
    h.fit_offline(dev(off.y.reshape(1024, n), f32))
    m_new, runs = 65536, 16
    new = synth.make_counters(seed=1, n_apps=m_new, n_cpu=n_cpu, n_gpu=n_gpu, runs=runs)
    ptr = np.arange(0, m_new * runs + 1, runs, dtype=np.int64)
    y = pred.infer(dev(new.X, f32))
    U, st = h.complete_rows(dev(ptr, torch.int64), dev(new.setting, torch.int32), y)
    _, best, sav = h.predict(U, gamma=0.05, want_T=False)
    y, Ug = host(y).astype(np.float64), host(U).astype(np.float64)
    best, V = host(best), host(h.get_V()).astype(np.float64)
    params = host(pred.get_params()).astype(np.float64)
    apps = np.sort(rng.choice(m_new, 512, replace=False))
    runs_s = (apps[:, None] * runs + np.arange(runs)).ravel()
    # predictions: the test's derived scale, as in the parity test above
    layers = orc.pred_unpack(params, NF)
    _, Z2, Y = orc.mlp_forward(_f32(new.X[runs_s]), layers)
    h2 = np.where(Z2 > 0, SELU_L * Z2, SELU_L * SELU_A * np.expm1(np.minimum(Z2, 0)))
    scale = np.abs(h2 * layers[4][:, 0]).sum(1) + abs(layers[5][0])
    assert (np.abs(y[runs_s] - Y[:, 0]) / scale).max() <= 2e-2
    # fold-in of the sampled apps on the GPU's predictions
    sp = np.arange(0, len(apps) * runs + 1, runs, dtype=np.int64)
    sc = new.setting[runs_s]
    sv = _f32(y[runs_s])
    Uref, sref = orc.half_step(sp, sc, sv, V, lam)
    assert np.array_equal(host(st)[apps], sref)
    assert solve_err(Ug[apps], Uref, V, sp, sc, sv, lam).max() <= TOL_FP32
    # Algorithm 2 on the GPU's T for the sampled apps
    T, b2, _ = h.predict(U[torch.as_tensor(apps, device=DEV)].contiguous(), gamma=0.05)
    assert np.array_equal(host(b2), best[apps])
    bo, _ = orc.select_f32(host(T), cpu, gpu, 0.05)
    assert np.array_equal(host(b2), bo)
