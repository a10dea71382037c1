"""GPU-vs-oracle parity of the streaming refit of V: the per-setting sums of
the V-half-step's normal equations, seeded with an offline block and grown by
batches of new applications (fold-in against the current V, then every
setting re-solved).  Checked stepwise: the oracle's state is fed the GPU's own
factors of each batch, so both sides hold the same sums up to rounding."""
import numpy as np
import pytest
import torch

import synth

from gpu_util import TOL_FP32, TOL_FP64, csr_dev, dev, host, rounded, row_rel_err, solve_err

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU hosts deselect these
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2508_07605_b300 as ocf  # noqa: E402

DT = {"fp32": torch.float32, "fp64": torch.float64}
# FP32: the sums are accumulated in FP32 over every ingested observation
# (up to ~500 per setting here), so a setting's solve carries that rounding
# on top of the per-solve gate.
TOL = {"fp32": 20 * TOL_FP32, "fp64": 100 * TOL_FP64}


def _block(rng, m, n, density, dt):
    rows, cols = [], []
    for i in range(m):
        c = np.nonzero(rng.random(n) < density)[0]
        if len(c) == 0:
            c = np.array([rng.integers(n)])
        rows.append(np.full(len(c), i)); cols.append(c)
    cols = np.concatenate(cols).astype(np.int32)
    ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum([len(r) for r in rows], out=ptr[1:])
    return ptr, cols, rounded(0.2 + rng.random(len(cols)), dt)


@pytest.mark.parametrize("precision,k,weighted", [("fp32", 16, False), ("fp32", 32, False),
                                                  ("fp32", 8, False), ("fp32", 16, True),
                                                  ("fp64", 8, False), ("fp64", 32, True)])
def test_stream_stepwise_parity(orc, precision, k, weighted):
    rng = np.random.default_rng(40 + k)
    dt = DT[precision]
    n, lam = 128, 0.05
    off = _block(rng, 600, n, 0.3, dt)
    U_off = rounded(rng.standard_normal((600, k)) / np.sqrt(k), dt)
    h = ocf.OpenCF(k=k, lam=lam, precision=precision, weighted_lambda=weighted)
    h.set_V(dev(np.zeros((n, k)), dt))
    h.stream_begin(*csr_dev(*off, dt), dev(U_off, dt))
    V0 = host(h.get_V()).astype(np.float64)
    torch.cuda.synchronize()
    ref = orc.StreamState(n, k, lam, weighted)
    ref.add(*off, U_off)
    assert row_rel_err(V0, ref.V).max() <= TOL[precision]
    Vprev = V0
    for b, (mb, dens) in enumerate([(200, 0.05), (1, 0.5), (350, 0.1)]):
        batch = _block(rng, mb, n, dens, dt)
        U, st = h.stream_ingest(*csr_dev(*batch, dt))
        V = host(h.get_V()).astype(np.float64)
        torch.cuda.synchronize()
        fold = orc.half_step_wr if weighted else orc.half_step
        Uref, sref = fold(*batch, Vprev, lam)
        assert np.array_equal(host(st), sref)
        assert row_rel_err(host(U), Uref).max() <= TOL[precision], b
        ref.add(*batch, host(U).astype(np.float64))
        assert row_rel_err(V, ref.V).max() <= TOL[precision], (b, row_rel_err(V, ref.V).max())
        Vprev = V


def test_stream_untouched_settings_and_errors(orc):
    rng = np.random.default_rng(5)
    n, k, lam = 64, 16, 0.05
    off = _block(rng, 300, n - 4, 0.3, torch.float32)        # settings 60..63 never observed
    U_off = rounded(rng.standard_normal((300, k)) / 4, torch.float32)
    h = ocf.OpenCF(k=k, lam=lam)
    h.set_V(dev(np.ones((n, k)), torch.float32))
    with pytest.raises(ocf.OpenCFError) as e:
        h.stream_ingest(*csr_dev(*off, torch.float32))
    assert e.value.code == ocf.NOT_FITTED
    h.stream_begin(*csr_dev(*off, torch.float32), dev(U_off, torch.float32))
    V = host(h.get_V())
    torch.cuda.synchronize()
    assert np.all(V[n - 4:] == 0)
    h.set_V(dev(np.ones((n, k)), torch.float32))                # a new V ends the stream
    with pytest.raises(ocf.OpenCFError) as e:
        h.stream_ingest(*csr_dev(*off, torch.float32))
    assert e.value.code == ocf.NOT_FITTED
    hb = ocf.OpenCF(k=32, lam=lam, precision="bf16_gram")
    hb.set_V(dev(np.ones((n, 32)), torch.float32))
    with pytest.raises(ocf.OpenCFError) as e:
        hb.stream_begin(*csr_dev(*off, torch.float32), dev(np.zeros((300, 32)), torch.float32))
    assert e.value.code == ocf.UNSUPPORTED


def test_stream_empty_batch_keeps_V(orc):
    rng = np.random.default_rng(9)
    n, k, lam = 96, 16, 0.05
    off = _block(rng, 400, n, 0.3, torch.float32)
    U_off = rounded(rng.standard_normal((400, k)) / 4, torch.float32)
    h = ocf.OpenCF(k=k, lam=lam)
    h.set_V(dev(np.zeros((n, k)), torch.float32))
    h.stream_begin(*csr_dev(*off, torch.float32), dev(U_off, torch.float32))
    V0 = host(h.get_V()).copy()
    empty = (np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    U, st = h.stream_ingest(*csr_dev(*empty, torch.float32))
    V1 = host(h.get_V())
    torch.cuda.synchronize()
    assert U.shape == (0, k) and st.shape == (0,)
    assert row_rel_err(V1, V0).max() <= 1e-6     # re-solved from the same sums


def test_stream_sums_exchange_emulated_on_one_gpu(orc):
    """Two handles stand for two ranks: each adds its shard's terms, the
    increments are summed (what the all-reduce of paper_2508_07605_b300.shard
    does across processes) and installed in both; V then equals that of one
    handle that ingested every row."""
    rng = np.random.default_rng(13)
    n, k, lam = 96, 16, 0.05
    dt = torch.float32
    off = _block(rng, 500, n, 0.3, dt)
    U_off = rounded(rng.standard_normal((500, k)) / 4, dt)
    new = _block(rng, 300, n, 0.08, dt)

    def rows(blk, r0, r1):
        p, c, v = blk
        return p[r0:r1 + 1] - p[r0], c[p[r0]:p[r1]], v[p[r0]:p[r1]]

    one = ocf.OpenCF(k=k, lam=lam)
    one.set_V(dev(np.zeros((n, k)), dt))
    one.stream_begin(*csr_dev(*off, dt), dev(U_off, dt))
    U_one, _ = one.stream_ingest(*csr_dev(*new, dt))
    ranks = [ocf.OpenCF(k=k, lam=lam) for _ in range(2)]
    cuts = [(0, 250), (250, 500)]
    for h, (r0, r1) in zip(ranks, cuts):
        h.set_V(dev(np.zeros((n, k)), dt))
        h.stream_begin(*csr_dev(*rows(off, r0, r1), dt), dev(U_off[r0:r1], dt))
    tot = [sum(x) for x in zip(*[h.stream_sums() for h in ranks])]
    for h in ranks:
        h.stream_set_sums(*tot)
    base = [t.clone() for t in tot]
    Us = []
    for h, (r0, r1) in zip(ranks, [(0, 120), (120, 300)]):
        U, _ = h.stream_ingest(*csr_dev(*rows(new, r0, r1), dt))
        Us.append(U)
    incs = [[c - b for c, b in zip(h.stream_sums(), base)] for h in ranks]
    tot = [b + i0 + i1 for b, i0, i1 in zip(base, *incs)]
    for h in ranks:
        h.stream_set_sums(*tot)
    torch.cuda.synchronize()
    Vone = host(one.get_V()).astype(np.float64)
    for h in ranks:
        assert row_rel_err(host(h.get_V()), Vone).max() <= 1e-4
    assert row_rel_err(host(torch.cat(Us)), host(U_one)).max() <= 1e-5
    # the counts are exact
    assert torch.equal(tot[2], one.stream_sums()[2])


def test_stream_full_size_stepwise_sampled(orc):
    """The streaming workload at full size (offline fit of the 2048-app block,
    then 16 batches of 8192 new apps, one graph launch each, as the benchmark
    runs it), step by step: sampled new apps' factors against the oracle's
    fold-in from the GPU's previous V, and every setting of V against the
    oracle's sums re-solved over the same factors."""
    w = synth.make_stream(seed=0)
    off = w.offline
    cpu, gpu = off.caps()
    f32 = torch.float32
    h = ocf.OpenCF(k=off.k, lam=off.lam, sweeps=off.sweeps, cpu_caps=cpu, gpu_caps=gpu)
    o_csr = csr_dev(off.row_ptr, off.col, off.val, f32)
    h.set_V(dev(off.V0, f32))
    U_off = h.fit_csr(*o_csr, off.n)
    h.stream_begin(*o_csr, U_off)
    ref = orc.StreamState(off.n, off.k, off.lam)
    ref.add(off.row_ptr, off.col, rounded(off.val, f32), host(U_off).astype(np.float64))
    V = host(h.get_V()).astype(np.float64)
    assert row_rel_err(V, ref.V).max() <= TOL_FP32
    rng = np.random.default_rng(0)
    for b, (p, c, v) in enumerate(w.batches):
        U, st = h.stream_ingest(*csr_dev(p, c, v, f32))
        Ug = host(U).astype(np.float64)
        rows = np.sort(rng.choice(len(p) - 1, 256, replace=False))
        sp = [0]; sc = []; sv = []
        for i in rows:
            sc.append(c[p[i]:p[i + 1]]); sv.append(rounded(v[p[i]:p[i + 1]], f32))
            sp.append(sp[-1] + p[i + 1] - p[i])
        sp = np.array(sp); sc = np.concatenate(sc); sv = np.concatenate(sv)
        Uref, sref = orc.half_step(sp, sc, sv, V, off.lam)
        assert np.array_equal(host(st)[rows], sref)
        assert solve_err(Ug[rows], Uref, V, sp, sc, sv, off.lam).max() <= TOL_FP32, b
        ref.add(p, c, rounded(v, f32), Ug)
        V = host(h.get_V()).astype(np.float64)
        assert row_rel_err(V, ref.V).max() <= TOL_FP32, (b, row_rel_err(V, ref.V).max())
