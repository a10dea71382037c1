"""Pins of the oracle's neural collaborative filtering (the paper's CF model,
Sec. "Collaborative Filtering Model": embeddings of the application and of the
power-cap pair, concatenated, through a SELU MLP to one predicted entry).

The oracle is checked against PyTorch's CPU autograd in FP64 (an independent
implementation of embedding lookup, linear layers, SELU, the mean squared
error and back-propagation), against central finite differences, against
torch.optim.Adam for the training loop, and against invariants of the model.
"""
import numpy as np
import pytest
import torch

import synth

D, H1, H2 = 3, 6, 5


def _unpack_t(net, d, h1, h2):
    o = 0
    out = []
    for shape in [(2 * d, h1), (h1,), (h1, h2), (h2,), (h2,), (1,)]:
        size = int(np.prod(shape))
        out.append(net[o:o + size].reshape(shape))
        o += size
    return out


def _torch_loss(ai, sj, r, Ea, Es, net, d, h1, h2):
    W1, b1, W2, b2, w3, b3 = _unpack_t(net, d, h1, h2)
    x = torch.cat([Ea[torch.as_tensor(ai, dtype=torch.long)],
                   Es[torch.as_tensor(sj, dtype=torch.long)]], dim=1)
    h = torch.nn.functional.selu(x @ W1 + b1)
    h = torch.nn.functional.selu(h @ W2 + b2)
    y = h @ w3 + b3
    return y, torch.nn.functional.mse_loss(y, torch.as_tensor(r))


def _case(seed, m=7, n=9, B=40):
    rng = np.random.default_rng(seed)
    net, Ea, Es = synth.ncf_init(rng, m, n, D, H1, H2, emb_scale=0.7, out_scale=1.0)
    net = net + 0.2 * rng.standard_normal(net.shape)   # non-zero biases as well
    ai = rng.integers(0, m, B).astype(np.int32)
    sj = rng.integers(0, n, B).astype(np.int32)
    ai[0], sj[0] = m - 1, n - 1                        # last rows are reached
    r = rng.standard_normal(B)
    return net, Ea, Es, ai, sj, r


@pytest.mark.parametrize("seed", range(3))
def test_ncf_matches_torch_autograd(orc, seed):
    net, Ea, Es, ai, sj, r = _case(seed)
    y = orc.ncf_forward(ai, sj, Ea, Es, net, H1, H2)
    L, gn, ga, gs = orc.ncf_loss_grad(ai, sj, r, Ea, Es, net, H1, H2)
    tn = torch.tensor(net, dtype=torch.float64, requires_grad=True)
    ta = torch.tensor(Ea, dtype=torch.float64, requires_grad=True)
    ts = torch.tensor(Es, dtype=torch.float64, requires_grad=True)
    ty, tL = _torch_loss(ai, sj, r, ta, ts, tn, D, H1, H2)
    tL.backward()
    assert np.abs(y - ty.detach().numpy()).max() <= 1e-13
    assert abs(L - tL.item()) <= 1e-13 * abs(L)
    assert np.abs(gn - tn.grad.numpy()).max() <= 1e-13
    assert np.abs(ga - ta.grad.numpy()).max() <= 1e-13
    assert np.abs(gs - ts.grad.numpy()).max() <= 1e-13
    # rows of indices absent from the batch get no gradient
    absent = np.setdiff1d(np.arange(Ea.shape[0]), ai)
    assert np.all(ga[absent] == 0)


def test_ncf_gradients_finite_differences(orc):
    net, Ea, Es, ai, sj, r = _case(7, B=12)
    _, gn, ga, gs = orc.ncf_loss_grad(ai, sj, r, Ea, Es, net, H1, H2)
    rng = np.random.default_rng(0)
    h = 1e-6
    for arr, g in ((net, gn), (Ea, ga), (Es, gs)):
        flat, gflat = arr.reshape(-1), g.reshape(-1)
        for q in rng.choice(flat.size, min(flat.size, 25), replace=False):
            old = flat[q]
            flat[q] = old + h; Lp = orc.ncf_loss_grad(ai, sj, r, Ea, Es, net, H1, H2)[0]
            flat[q] = old - h; Lm = orc.ncf_loss_grad(ai, sj, r, Ea, Es, net, H1, H2)[0]
            flat[q] = old
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - gflat[q]) <= 1e-6 * max(1.0, abs(fd)), (q, fd, gflat[q])


def test_ncf_predict_is_forward_on_every_pair(orc):
    net, Ea, Es, _, _, _ = _case(3)
    T = orc.ncf_predict(Ea, Es, net, H1, H2)
    m, n = T.shape
    ai, sj = np.divmod(np.arange(m * n), n)
    tn, ta, ts = (torch.tensor(a, dtype=torch.float64) for a in (net, Ea, Es))
    ty, _ = _torch_loss(ai, sj, np.zeros(m * n), ta, ts, tn, D, H1, H2)
    assert np.abs(T.ravel() - ty.numpy()).max() <= 1e-13


def test_ncf_first_layer_splits_over_the_concatenation(orc):
    # x W1 = Ea_i W1[:d] + Es_j W1[d:]: the prediction depends on (i, j) only
    # through the two half-products, so swapping the order of the embedding
    # tables together with the two halves of W1 leaves every prediction equal
    net, Ea, Es, ai, sj, _ = _case(4)
    y = orc.ncf_forward(ai, sj, Ea, Es, net, H1, H2)
    W1 = net[:2 * D * H1].reshape(2 * D, H1)
    net2 = net.copy()
    net2[:2 * D * H1] = np.concatenate([W1[D:], W1[:D]]).ravel()
    y2 = orc.ncf_forward(sj, ai, Es, Ea, net2, H1, H2)
    assert np.abs(y - y2).max() <= 1e-13
    # and permuting the rows of a table together with the indices is invisible
    p = np.random.default_rng(1).permutation(Ea.shape[0])
    inv = np.argsort(p)
    y3 = orc.ncf_forward(inv[ai].astype(np.int32), sj, Ea[p], Es, net, H1, H2)
    assert np.abs(y - y3).max() <= 1e-13


def test_ncf_training_loop_matches_torch_adam(orc):
    rng = np.random.default_rng(5)
    m, n, nnz = 6, 8, 30
    net, Ea, Es = synth.ncf_init(rng, m, n, D, H1, H2, emb_scale=0.5, out_scale=1.0)
    ai = rng.integers(0, m, nnz).astype(np.int32)
    sj = rng.integers(0, n, nnz).astype(np.int32)
    r = rng.random(nnz)
    perms = synth.ncf_perms(rng, nnz, 3)
    batch, lr = 8, 3e-3   # 30 = 8 + 8 + 8 + 6: a shorter last batch every epoch
    net_o, Ea_o, Es_o, losses = orc.ncf_train(ai, sj, r, Ea, Es, net, H1, H2, perms, batch, lr)
    tn = torch.tensor(net, dtype=torch.float64, requires_grad=True)
    ta = torch.tensor(Ea, dtype=torch.float64, requires_grad=True)
    ts = torch.tensor(Es, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tn, ta, ts], lr=lr, betas=(0.9, 0.999), eps=1e-8)
    tl = []
    for perm in perms:
        for b0 in range(0, nnz, batch):
            sel = perm[b0:b0 + batch]
            opt.zero_grad()
            _, L = _torch_loss(ai[sel], sj[sel], r[sel], ta, ts, tn, D, H1, H2)
            L.backward()
            opt.step()
            tl.append(L.item())
    assert len(losses) == 12
    assert np.abs(losses - np.array(tl)).max() <= 1e-12
    assert np.abs(net_o - tn.detach().numpy()).max() <= 1e-12
    assert np.abs(Ea_o - ta.detach().numpy()).max() <= 1e-12
    assert np.abs(Es_o - ts.detach().numpy()).max() <= 1e-12


def test_ncf_learns_a_low_rank_matrix(orc):
    # a small completion task: held-out error well below the column-mean guess
    prob = synth.make_sparse_problem(seed=3, m=80, n_cpu=2, n_gpu=16, rank=2, density=0.4, k=2,
                                     lam=0.05, n_heldout=400)
    ai, sj = synth.coo_from_csr(prob.row_ptr, prob.col)
    rng = np.random.default_rng(0)
    net, Ea, Es = synth.ncf_init(rng, prob.m, prob.n, 8, 32, 16)
    perms = synth.ncf_perms(rng, len(ai), 60)
    net, Ea, Es, losses = orc.ncf_train(ai, sj, prob.val, Ea, Es, net, 32, 16, perms, 64, 3e-3)
    assert losses[-20:].mean() < 0.2 * losses[:5].mean()
    y = orc.ncf_forward(prob.heldout_rows, prob.heldout_cols, Ea, Es, net, 32, 16)
    rmse = np.sqrt(np.mean((y - prob.heldout_truth) ** 2))
    colmean = np.array([prob.val[sj == j].mean() if np.any(sj == j) else prob.val.mean()
                        for j in range(prob.n)])
    base = np.sqrt(np.mean((colmean[prob.heldout_cols] - prob.heldout_truth) ** 2))
    assert rmse < 0.6 * base, (rmse, base)


def test_predictor_training_matches_torch_adam(orc):
    """The offline performance predictor: 7 inputs -> 128 -> 64 SELU -> 1."""
    rng = np.random.default_rng(9)
    runs = synth.make_counters(seed=1, n_apps=6, n_cpu=2, n_gpu=4)
    X, y = runs.X, runs.y
    params = synth.pred_init(rng, 7, out_scale=1.0) + 0.05 * rng.standard_normal(9345)
    perms = synth.ncf_perms(rng, len(y), 2)
    theta, losses = orc.pred_train(X, y, params, 7, perms, 16, 3e-3)
    W = [torch.tensor(p, dtype=torch.float64, requires_grad=True)
         for p in orc.pred_unpack(params, 7)]
    opt = torch.optim.Adam(W, lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    tl = []
    Xt, yt = torch.tensor(X), torch.tensor(y)
    for perm in perms:
        for b0 in range(0, len(y), 16):
            sel = torch.as_tensor(perm[b0:b0 + 16], dtype=torch.long)
            opt.zero_grad()
            h = torch.nn.functional.selu(Xt[sel] @ W[0] + W[1])
            h = torch.nn.functional.selu(h @ W[2] + W[3])
            L = torch.nn.functional.mse_loss((h @ W[4] + W[5])[:, 0], yt[sel])
            L.backward()
            opt.step()
            tl.append(L.item())
    assert np.abs(losses - np.array(tl)).max() <= 1e-12
    ref = np.concatenate([w.detach().numpy().ravel() for w in W])
    assert np.abs(theta - ref).max() <= 1e-12
