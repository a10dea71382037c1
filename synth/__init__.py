"""Seeded synthetic inputs for the OPEN online-phase completion path.

This module only *generates inputs*: performance matrices, observation masks,
initial factors, held-out samples and cap grids.  It holds none of the
method's arithmetic (no Gram, no solve, no selection), so both the CUDA path
and the FP64 oracle can be fed from it without sharing any method code.

The paper's matrices come from profiling real applications under CPU/GPU
power caps (Sec. "Putting it all together", Eq. 1; Sec. "Online Performance
Prediction"); none of that data exists here.  The recipes below stand in for
it, with the shapes of the paper's problem: rows are applications, columns are
(CPU cap, GPU cap) settings in CPU-major order ``j = c_idx * n_gpu + g_idx``,
the offline block is dense, and each new application contributes a handful of
online-profiled entries.

Readings of details the paper leaves unstated:
  * noise ``N(0, 0.01)`` is a standard deviation of 0.01, added after
    normalisation, never clipped;
  * the exp-transformed matrix is normalised by its global min and max;
  * a "rank-r ground truth" is ``U V^T / max|U V^T|`` so it stays exactly
    rank r;
  * CPU caps are ``linspace(120, 270, n_cpu)`` W and GPU caps
    ``linspace(100, 250, n_gpu)`` W (the paper enumerates no grid);
  * random draws of the method itself (the initial V of ALS, the initial MLP
    weights) are generated here and passed in as inputs.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

NOISE_STD = 0.01


def cap_grid(n_cpu: int, n_gpu: int):
    """CPU and GPU cap values in watts (ascending)."""
    return (np.linspace(120.0, 270.0, n_cpu), np.linspace(100.0, 250.0, n_gpu))


@dataclasses.dataclass
class CompletionProblem:
    """One sparse completion problem in CSR form plus what scores it."""
    m: int
    n: int
    k: int
    lam: float
    sweeps: int
    row_ptr: np.ndarray          # int64[m+1]
    col: np.ndarray              # int32[nnz], strictly increasing per row
    val: np.ndarray              # float64[nnz] observed (noisy) values
    V0: np.ndarray               # float64[n, k] initial V of ALS
    n_cpu: int = 1
    n_gpu: int = 1
    heldout_rows: Optional[np.ndarray] = None   # int64
    heldout_cols: Optional[np.ndarray] = None   # int64
    heldout_truth: Optional[np.ndarray] = None  # float64, noiseless
    truth: Optional[np.ndarray] = None          # dense noiseless truth when small

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def caps(self):
        return cap_grid(self.n_cpu, self.n_gpu)


def csr_from_positions(pos: np.ndarray, m: int, n: int):
    """CSR (row_ptr, col) of sorted flattened positions ``i * n + j``."""
    rows = pos // n
    cols = (pos - rows * n).astype(np.int32)
    counts = np.bincount(rows, minlength=m).astype(np.int64)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, cols, rows


def bernoulli_positions(rng: np.random.Generator, total: int, p: float) -> np.ndarray:
    """Sorted positions of an i.i.d. Bernoulli(p) mask over ``total`` cells.

    Successive gaps of a Bernoulli process are Geometric(p), so drawing gaps
    gives the same distribution as drawing every cell, at O(p * total) cost.
    """
    if p >= 1.0:
        return np.arange(total, dtype=np.int64)
    est = int(p * total + 8.0 * math.sqrt(p * total + 1.0) + 64)
    chunks = []
    last = -1
    while True:
        gaps = rng.geometric(p, size=est).astype(np.int64)
        pos = last + np.cumsum(gaps)
        chunks.append(pos)
        last = int(pos[-1])
        if last >= total:
            break
    pos = np.concatenate(chunks)
    return pos[pos < total]


def sample_unobserved(rng, m, n, observed_pos, count):
    """Seeded sample of ``count`` distinct unobserved cells (rows, cols)."""
    count = int(min(count, m * n - len(observed_pos)))
    picked = np.empty(0, dtype=np.int64)
    while len(picked) < count:
        cand = rng.integers(0, m * n, size=2 * (count - len(picked)) + 16)
        cand = np.unique(cand)
        cand = cand[~np.isin(cand, observed_pos, assume_unique=False)]
        cand = cand[~np.isin(cand, picked)]
        picked = np.concatenate([picked, cand])
    picked = np.sort(picked[:count])
    rows = picked // n
    return rows, picked - rows * n


def init_factor(rng, n, k, scale=0.1):
    """Initial V of ALS: ``scale * N(0, 1)`` entries (n x k)."""
    return scale * rng.standard_normal((n, k))


# ---------------------------------------------------------------------------
# Workload 1: 64 apps x 120 settings (8 CPU x 15 GPU caps), exp-transformed
# rank-4 truth, 48 fully observed offline rows + 16 new rows with 6 entries.
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class OfflineOnlineProblem:
    offline: np.ndarray          # dense [m_off, n] noisy offline block
    new: CompletionProblem       # CSR of the new rows (row indices local)
    joint: CompletionProblem     # CSR of all rows (offline + new)
    truth: np.ndarray            # dense noiseless truth [m, n]
    m_off: int


def make_small_offline_online(seed: int = 0, m: int = 64, m_off: int = 48,
                              n_cpu: int = 8, n_gpu: int = 15, rank: int = 4,
                              k: int = 8, lam: float = 0.1, sweeps: int = 20,
                              obs_per_new_row: int = 6) -> OfflineOnlineProblem:
    rng = np.random.default_rng(seed)
    n = n_cpu * n_gpu
    Ut = rng.standard_normal((m, rank)) / 2.0
    Vt = rng.standard_normal((n, rank)) / 2.0
    T0 = np.exp(Ut @ Vt.T)
    truth = (T0 - T0.min()) / (T0.max() - T0.min())
    noisy = truth + rng.normal(0.0, NOISE_STD, size=(m, n))
    offline = noisy[:m_off].copy()
    new_cols = [np.sort(rng.choice(n, size=obs_per_new_row, replace=False))
                for _ in range(m - m_off)]
    V0 = init_factor(rng, n, k)

    def build(rows_cols):
        ptr = [0]
        cols, vals = [], []
        for i, cs in rows_cols:
            cols.append(np.asarray(cs, dtype=np.int32))
            vals.append(noisy[i, cs])
            ptr.append(ptr[-1] + len(cs))
        return (np.asarray(ptr, dtype=np.int64), np.concatenate(cols).astype(np.int32),
                np.concatenate(vals).astype(np.float64))

    new_rc = [(m_off + t, c) for t, c in enumerate(new_cols)]
    p_new, c_new, v_new = build(new_rc)
    all_rc = [(i, np.arange(n)) for i in range(m_off)] + new_rc
    p_all, c_all, v_all = build(all_rc)
    # held-out: every unobserved entry of the new rows
    hr, hc = [], []
    for t, cs in enumerate(new_cols):
        un = np.setdiff1d(np.arange(n), cs)
        hr.append(np.full(len(un), t, dtype=np.int64))
        hc.append(un.astype(np.int64))
    hr = np.concatenate(hr)
    hc = np.concatenate(hc)
    new = CompletionProblem(m - m_off, n, k, lam, sweeps, p_new, c_new, v_new, V0.copy(),
                            n_cpu, n_gpu, hr, hc, truth[m_off + hr, hc], truth[m_off:].copy())
    joint = CompletionProblem(m, n, k, lam, sweeps, p_all, c_all, v_all, V0.copy(),
                              n_cpu, n_gpu, hr + m_off, hc, truth[m_off + hr, hc], truth.copy())
    return OfflineOnlineProblem(offline, new, joint, truth, m_off)


# ---------------------------------------------------------------------------
# Workload 2 (and the generic sparse recipe): rank-r truth U V^T / max|U V^T|,
# U, V ~ N(0,1)/2, Bernoulli(density) mask, N(0, 0.01) noise.
# ---------------------------------------------------------------------------
def make_sparse_problem(seed: int = 0, m: int = 4096, n_cpu: int = 16, n_gpu: int = 64,
                        rank: int = 16, density: float = 0.05, k: int = 16,
                        lam: float = 0.05, sweeps: int = 15, n_heldout: int = 1 << 17,
                        keep_truth: bool = False, rng=None) -> CompletionProblem:
    rng = np.random.default_rng(seed) if rng is None else rng
    n = n_cpu * n_gpu
    Ut = rng.standard_normal((m, rank)) / 2.0
    Vt = rng.standard_normal((n, rank)) / 2.0
    M = Ut @ Vt.T
    scale = float(np.abs(M).max())
    truth = M / scale
    pos = bernoulli_positions(rng, m * n, density)
    row_ptr, col, rows = csr_from_positions(pos, m, n)
    val = truth.ravel()[pos] + rng.normal(0.0, NOISE_STD, size=len(pos))
    V0 = init_factor(rng, n, k)
    hr, hc = sample_unobserved(rng, m, n, pos, n_heldout)
    return CompletionProblem(m, n, k, lam, sweeps, row_ptr, col, val.astype(np.float64), V0,
                             n_cpu, n_gpu, hr, hc, truth[hr, hc],
                             truth if keep_truth else None)


def make_c2(seed: int = 0, **kw) -> CompletionProblem:
    """4096 apps x 1024 settings (16 x 64 caps), rank 16, 5 % observed, k=16,
    lambda=0.05, 15 sweeps."""
    return make_sparse_problem(seed=seed, **kw)


# ---------------------------------------------------------------------------
# Workload 3: many independent problems of uneven size.
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class BatchedProblems:
    problems: List[CompletionProblem]

    def __len__(self):
        return len(self.problems)

    def concat(self):
        """Concatenated CSR/V0 arrays with per-problem offsets (int64)."""
        P = len(self.problems)
        m = np.array([p.m for p in self.problems], dtype=np.int64)
        n = np.array([p.n for p in self.problems], dtype=np.int64)
        k = np.array([p.k for p in self.problems], dtype=np.int32)
        nnz = np.array([p.nnz for p in self.problems], dtype=np.int64)
        row_off = np.zeros(P + 1, dtype=np.int64); np.cumsum(m, out=row_off[1:])
        col_off = np.zeros(P + 1, dtype=np.int64); np.cumsum(n, out=col_off[1:])
        nnz_off = np.zeros(P + 1, dtype=np.int64); np.cumsum(nnz, out=nnz_off[1:])
        uf = np.zeros(P + 1, dtype=np.int64); np.cumsum(m * k, out=uf[1:])
        vf = np.zeros(P + 1, dtype=np.int64); np.cumsum(n * k, out=vf[1:])
        # row_ptr of each problem is local (starts at 0); concatenated row_ptr
        # holds global nnz offsets and has sum(m) + 1 entries.
        row_ptr = np.zeros(int(row_off[-1]) + 1, dtype=np.int64)
        for t, p in enumerate(self.problems):
            row_ptr[row_off[t]:row_off[t + 1] + 1] = p.row_ptr + nnz_off[t]
        col = np.concatenate([p.col for p in self.problems]).astype(np.int32)
        val = np.concatenate([p.val for p in self.problems])
        V0 = np.concatenate([p.V0.ravel() for p in self.problems])
        return dict(m=m, n=n, k=k, row_off=row_off, col_off=col_off, nnz_off=nnz_off,
                    u_off=uf, v_off=vf, row_ptr=row_ptr, col=col, val=val, V0=V0)


def make_batched(seed: int = 0, n_problems: int = 10000, m_range=(32, 512),
                 n_range=(64, 1024), density_range=(0.02, 0.20), rank_range=(8, 32),
                 lam: float = 0.05, sweeps: int = 15, n_heldout: int = 64) -> BatchedProblems:
    """Apps, settings and density log-uniform over their ranges, rank uniform
    over the integers, solver k equal to the rank.  Settings counts are
    factored into a CPU x GPU grid only nominally (n_cpu=1)."""
    rng = np.random.default_rng(seed)
    probs = []
    lm = np.log(m_range); ln = np.log(n_range); ld = np.log(density_range)
    for _ in range(n_problems):
        m = int(round(math.exp(rng.uniform(lm[0], lm[1]))))
        n = int(round(math.exp(rng.uniform(ln[0], ln[1]))))
        d = float(math.exp(rng.uniform(ld[0], ld[1])))
        r = int(rng.integers(rank_range[0], rank_range[1] + 1))
        probs.append(make_sparse_problem(m=m, n_cpu=1, n_gpu=n, rank=r, density=d, k=r,
                                         lam=lam, sweeps=sweeps, n_heldout=n_heldout,
                                         rng=rng))
    return BatchedProblems(probs)


# ---------------------------------------------------------------------------
# Workloads 4 and 5 are too large for numpy on the host; they are drawn with
# torch (CPU or CUDA device) from a seeded generator.  Only inputs are made.
# ---------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def torch_bernoulli_csr(gen, m: int, n: int, p: float, device):
    """CSR of an i.i.d. Bernoulli(p) mask over m x n via geometric gaps
    (inverse-CDF draws), entirely on ``device``."""
    torch = _torch()
    total = m * n
    est = int(p * total + 8.0 * math.sqrt(p * total + 1.0) + 64)
    logq = math.log1p(-p)
    chunks = []
    last = -1
    while True:
        u = torch.rand(est, generator=gen, device=device, dtype=torch.float64)
        gaps = torch.floor(torch.log1p(-u) / logq).to(torch.int64) + 1
        pos = last + torch.cumsum(gaps, 0)
        chunks.append(pos)
        last = int(pos[-1].item())
        if last >= total:
            break
    pos = torch.cat(chunks)
    pos = pos[pos < total]
    rows = torch.div(pos, n, rounding_mode="floor")
    cols = (pos - rows * n).to(torch.int32)
    counts = torch.bincount(rows, minlength=m)
    row_ptr = torch.zeros(m + 1, dtype=torch.int64, device=device)
    row_ptr[1:] = torch.cumsum(counts, 0)
    return row_ptr, cols, rows


@dataclasses.dataclass
class LargeSparseProblem:
    m: int
    n: int
    k: int
    lam: float
    n_cpu: int
    n_gpu: int
    row_ptr: object   # torch int64 [m+1]
    col: object       # torch int32 [nnz]
    val: object       # torch float32 [nnz]
    Ut: object        # torch float32 [m, rank]  (ground-truth factors)
    Vt: object        # torch float32 [n, rank]
    scale: float
    V: object         # torch float32 [n, k]  fixed V for the fold-in


def make_large_foldin(seed: int = 0, m: int = 1 << 20, n_cpu: int = 64, n_gpu: int = 64,
                      rank: int = 32, k: int = 32, density: float = 0.01, lam: float = 0.05,
                      device="cuda") -> LargeSparseProblem:
    """1M apps x 4096 settings (64 x 64 caps), 1 % observed, k=32.  The fixed
    V of the fold-in is the ground-truth V plus 1 % noise (a stand-in for an
    offline fit), so the fold-in works on a realistic, well-posed V."""
    torch = _torch()
    n = n_cpu * n_gpu
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    Ut = torch.randn(m, rank, generator=gen, device=device) / 2.0
    Vt = torch.randn(n, rank, generator=gen, device=device) / 2.0
    scale = 0.0
    step = max(1, (1 << 26) // n)
    for s in range(0, m, step):
        scale = max(scale, float((Ut[s:s + step] @ Vt.T).abs().max().item()))
    row_ptr, col, rows = torch_bernoulli_csr(gen, m, n, density, device)
    nnz = col.numel()
    val = torch.empty(nnz, dtype=torch.float32, device=device)
    step = 1 << 24
    for s in range(0, nnz, step):
        r = rows[s:s + step]
        c = col[s:s + step].to(torch.int64)
        val[s:s + step] = (Ut[r] * Vt[c]).sum(1) / scale
    val += NOISE_STD * torch.randn(nnz, generator=gen, device=device)
    V = (Vt[:, :k] if rank >= k else torch.nn.functional.pad(Vt, (0, k - rank)))
    V = (V + 0.01 * torch.randn(V.shape, generator=gen, device=device)).contiguous()
    del rows
    return LargeSparseProblem(m, n, k, lam, n_cpu, n_gpu, row_ptr, col, val, Ut, Vt, scale, V)


@dataclasses.dataclass
class LearnedWorkload:
    n: int
    n_cpu: int
    n_gpu: int
    k: int
    lam: float
    s_obs: int
    scale: float
    Vt: object        # ground-truth setting factors [n, rank] (torch), smooth in the caps
    A: object         # trait loadings [traits, rank]
    gen: object       # torch generator for app draws
    device: object
    rank: int
    traits: int
    spread: float

    def V_fixed(self):
        """The fixed setting factors of the handle, V = Vt / sqrt(scale), so
        that a row of normalised runtimes is (u / sqrt(scale)) V^T."""
        return (self.Vt / math.sqrt(self.scale)).contiguous()

    def draw_apps(self, count: int):
        """``count`` new apps: noisy rows [count, n], noiseless rows, and
        ``s_obs`` distinct observed settings per app (sorted, int32)."""
        torch = _torch()
        z = torch.randn(count, self.traits, generator=self.gen, device=self.device)
        Ua = z @ self.A + self.spread * torch.randn(count, self.rank, generator=self.gen,
                                                    device=self.device)
        clean = (Ua @ self.Vt.T) / self.scale
        noisy = clean + NOISE_STD * torch.randn(clean.shape, generator=self.gen,
                                                device=self.device)
        keys = torch.rand(count, self.n, generator=self.gen, device=self.device)
        obs = torch.topk(keys, self.s_obs, dim=1).indices.sort(dim=1).values.to(torch.int32)
        return noisy, clean, obs


def dense_rows_csr(rows):
    """CSR of fully observed rows [m, n] (every setting, in index order)."""
    torch = _torch()
    m, n = rows.shape
    dev = rows.device
    row_ptr = torch.arange(0, (m + 1) * n, n, dtype=torch.int64, device=dev)
    col = torch.arange(n, dtype=torch.int32, device=dev).repeat(m)
    return row_ptr, col, rows.reshape(-1).contiguous()


def learned_pool(wl: "LearnedWorkload", handle, count: int, chunk: int = 65536):
    """Training pool of the learned warm start: ``count`` apps, each with its
    ``s_obs`` observed entries (features) and, as target, the factor the
    plain fold-in computes from the app's full noisy profile.  Returns
    (col [count, s_obs] int32, val [count, s_obs] float32, U_target [count, k])."""
    torch = _torch()
    cols, vals, tgts = [], [], []
    for s in range(0, count, chunk):
        c = min(chunk, count - s)
        noisy, _, obs = wl.draw_apps(c)
        U, _ = handle.complete_rows(*dense_rows_csr(noisy))
        cols.append(obs)
        vals.append(torch.gather(noisy, 1, obs.to(torch.int64)))
        tgts.append(U)
        del noisy
    return torch.cat(cols), torch.cat(vals), torch.cat(tgts)


def observed_csr(rows, obs):
    """CSR of the entries ``obs`` [m, s] (sorted per row) of ``rows`` [m, n]."""
    torch = _torch()
    m, s = obs.shape
    row_ptr = torch.arange(0, (m + 1) * s, s, dtype=torch.int64, device=rows.device)
    val = torch.gather(rows, 1, obs.to(torch.int64)).reshape(-1).contiguous()
    return row_ptr, obs.reshape(-1).contiguous(), val


def make_learned(seed: int = 0, n_cpu: int = 64, n_gpu: int = 64, rank: int = 32, k: int = 32,
                 lam: float = 0.05, s_obs: int = 16, traits: int = 4, spread: float = 0.05,
                 smooth_terms: int = 6, device="cuda") -> LearnedWorkload:
    """Workload of the learned warm start (4096 settings, k = 32, 16 observed
    settings per new app).

    Runtime varies smoothly with the caps, so each true setting factor is a
    random combination of low-frequency cosines of the normalised caps:
    Vt[j] = sum_{a,b < smooth_terms} cos(pi a c_j) cos(pi b g_j) w_ab with
    w_ab ~ N(0, I) * 0.6^(a+b).  Applications share a few traits (compute vs
    memory intensity and the like): u = z A + spread * e, z ~ N(0, I_traits),
    A ~ N(0, 1/traits), e ~ N(0, I).  Rows are u Vt^T / scale plus N(0, 0.01)
    noise, scale = max |u Vt^T| over a 4096-app draw."""
    torch = _torch()
    n = n_cpu * n_gpu
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    c = torch.linspace(0.0, 1.0, n_cpu, device=device, dtype=torch.float64)
    g = torch.linspace(0.0, 1.0, n_gpu, device=device, dtype=torch.float64)
    cc = c.repeat_interleave(n_gpu)
    gg = g.repeat(n_cpu)
    basis = []
    for a in range(smooth_terms):
        for b in range(smooth_terms):
            basis.append(torch.cos(math.pi * a * cc) * torch.cos(math.pi * b * gg) * 0.6 ** (a + b))
    Phi = torch.stack(basis, 1).float()
    W = torch.randn(Phi.shape[1], rank, generator=gen, device=device)
    Vt = (Phi @ W).contiguous()
    A = torch.randn(traits, rank, generator=gen, device=device) / math.sqrt(traits)
    z = torch.randn(4096, traits, generator=gen, device=device)
    Uo = z @ A + spread * torch.randn(4096, rank, generator=gen, device=device)
    scale = float((Uo @ Vt.T).abs().max().item())
    return LearnedWorkload(n, n_cpu, n_gpu, k, lam, s_obs, scale, Vt, A, gen, device, rank,
                           traits, spread)


def mlp_init(rng: np.random.Generator, sizes=(48, 256, 256, 32), out_scale: float = 1.0):
    """LeCun-normal initial weights (the SELU recommendation of Klambauer et
    al. 2017) and zero biases; W_l is stored [in, out] row-major.  The last
    layer's weights are multiplied by ``out_scale`` (targets far smaller than
    one train faster from a small initial output)."""
    params = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        params.append(rng.standard_normal((a, b)) / math.sqrt(a))
        params.append(np.zeros(b))
    params[-2] = params[-2] * out_scale
    return params


# ---------------------------------------------------------------------------
# GPU power traces for Algorithm 1: a CPU phase (data preparation) near idle
# power, then, for most jobs, a GPU phase well above the threshold with brief
# dips (kernel gaps, synchronisation), as in the paper's GROMACS and BERT
# traces (Fig. "power_pattern").  Readings every 0.2 s.
# ---------------------------------------------------------------------------
def make_power_traces(seed: int = 0, n_traces: int = 1024, length: int = 3000,
                      p_cpu: float = 45.0, p_gpu: float = 200.0, dip_rate: float = 0.02,
                      never: float = 0.2) -> np.ndarray:
    """float32 [n_traces, length]: CPU phase N(p_cpu, 5) W for a uniform random
    number of readings, then GPU phase N(p_gpu, 30) W with a reading below
    60 W at rate dip_rate; a fraction `never` of jobs stays in the CPU phase."""
    rng = np.random.default_rng(seed)
    P = rng.normal(p_cpu, 5.0, (n_traces, length)).astype(np.float32)
    start = rng.integers(0, max(length, 1), n_traces)
    gpu_jobs = rng.random(n_traces) >= never
    pos = np.arange(length)[None, :]
    in_gpu = (pos >= start[:, None]) & gpu_jobs[:, None]
    G = rng.normal(p_gpu, 30.0, (n_traces, length)).astype(np.float32)
    dips = rng.random((n_traces, length)) < dip_rate
    G[dips] = rng.uniform(20.0, 59.0, int(dips.sum())).astype(np.float32)
    P[in_gpu] = G[in_gpu]
    return P


# ---------------------------------------------------------------------------
# Neural collaborative filtering (the paper's CF model): initial parameters and
# the per-epoch visiting orders of the observed entries (both are random draws
# of the method, so they are inputs to the GPU path and the oracle alike).
NCF_D, NCF_H1, NCF_H2 = 32, 128, 64


def ncf_init(rng: np.random.Generator, m: int, n: int, d: int = NCF_D, h1: int = NCF_H1,
             h2: int = NCF_H2, emb_scale: float = 0.1, out_scale: float = 0.1):
    """(net, Ea, Es): embeddings N(0, emb_scale^2); LeCun-normal MLP weights
    [in, out] row-major, zero biases, the output weights scaled by out_scale;
    net packed as [W1 (2d x h1), b1, W2 (h1 x h2), b2, w3 (h2), b3]."""
    W1 = rng.standard_normal((2 * d, h1)) / math.sqrt(2 * d)
    W2 = rng.standard_normal((h1, h2)) / math.sqrt(h1)
    w3 = rng.standard_normal(h2) / math.sqrt(h2) * out_scale
    net = np.concatenate([W1.ravel(), np.zeros(h1), W2.ravel(), np.zeros(h2), w3, np.zeros(1)])
    Ea = rng.standard_normal((m, d)) * emb_scale
    Es = rng.standard_normal((n, d)) * emb_scale
    return net, Ea, Es


def ncf_perms(rng: np.random.Generator, nnz: int, epochs: int):
    """One random visiting order of the observed entries per epoch."""
    return [rng.permutation(nnz).astype(np.int32) for _ in range(epochs)]


def coo_from_csr(row_ptr, col):
    """(app index, setting index) of every observed entry, in CSR order."""
    ai = np.repeat(np.arange(len(row_ptr) - 1, dtype=np.int32), np.diff(row_ptr))
    return ai, np.asarray(col, dtype=np.int32)


# ---------------------------------------------------------------------------
# Streaming refit: an offline block (workload 2's matrix) and a stream of new
# applications from the same rank-16 model, each profiled online under a few
# settings (Sec. "Online Performance Prediction").
@dataclasses.dataclass
class StreamWorkload:
    offline: CompletionProblem
    batches: list          # [(row_ptr, col, val)] per batch of new applications
    truth_new: np.ndarray  # [m_new, n] noiseless rows of the new applications
    batch: int


def make_stream(seed: int = 0, n_batches: int = 16, batch: int = 8192, obs: int = 16,
                truth_rows: int = 2048) -> StreamWorkload:
    rng = np.random.default_rng(seed)
    off = make_sparse_problem(seed=seed, keep_truth=False)
    n, rank = off.n, 16
    # the offline matrix's generator, re-drawn with the same seed, gives its V;
    # new applications draw fresh U rows from the same distribution
    g = np.random.default_rng(seed)
    Ut = g.standard_normal((off.m, rank)) / 2.0
    Vt = g.standard_normal((n, rank)) / 2.0
    scale = float(np.abs(Ut @ Vt.T).max())
    batches, truth = [], []
    for _ in range(n_batches):
        Un = rng.standard_normal((batch, rank)) / 2.0
        cols = np.sort(np.argsort(rng.random((batch, n)), axis=1)[:, :obs], axis=1)
        rows = np.repeat(np.arange(batch), obs)
        tv = np.einsum("bk,bok->bo", Un, Vt[cols]) / scale
        val = (tv + rng.normal(0.0, NOISE_STD, size=tv.shape)).ravel()
        ptr = np.arange(0, batch * obs + 1, obs, dtype=np.int64)
        batches.append((ptr, cols.ravel().astype(np.int32), val))
        if len(truth) * batch < truth_rows:
            truth.append(Un @ Vt.T / scale)
    return StreamWorkload(off, batches, np.concatenate(truth)[:truth_rows], batch)


# ---------------------------------------------------------------------------
# Offline performance predictor: synthetic profiling runs.  Each application
# has a CPU share of its baseline runtime and how memory-bound its CPU and GPU
# parts are; a run under caps (c, g) yields the paper's seven inputs (CPU cap,
# GPU cap, memory throughput, IPS, SM clock, DRAM active, FP active) and the
# normalised performance in the matrix's unit: runtime / baseline runtime
# (1 at the largest caps, larger under tighter caps).
@dataclasses.dataclass
class CounterRuns:
    X: np.ndarray      # [N, 7] inputs, each scaled to about [0, 1]
    y: np.ndarray      # [N] normalised runtime (runtime / runtime at the largest caps)
    app: np.ndarray    # [N] application index
    setting: np.ndarray  # [N] setting index (CPU-major)


@dataclasses.dataclass
class AppTraits:
    cpu_share: np.ndarray
    mem_c: np.ndarray
    mem_g: np.ndarray
    flop: np.ndarray
    ips0: np.ndarray


def counter_runs(traits: AppTraits, app: np.ndarray, setting: np.ndarray, n_cpu: int,
                 n_gpu: int, rng: Optional[np.random.Generator] = None,
                 noise: float = 0.02) -> CounterRuns:
    """Runs (app[r], setting[r]) of the synthetic applications: the seven inputs
    (with multiplicative noise when rng is given) and the normalised runtime."""
    cpu, gpu = cap_grid(n_cpu, n_gpu)
    c = cpu[setting // n_gpu] / cpu[-1]
    g = gpu[setting % n_gpu] / gpu[-1]
    a = app
    s_cpu = c ** (0.3 + 0.5 * (1.0 - traits.mem_c[a]))           # CPU speed under its cap
    clk = np.minimum(1.0, 1.1 * g ** 0.6)                         # SM clock / max clock
    s_gpu = traits.mem_g[a] * (1.0 - 0.2 * (1.0 - g)) + (1.0 - traits.mem_g[a]) * clk
    y = traits.cpu_share[a] / s_cpu + (1.0 - traits.cpu_share[a]) / s_gpu
    mult = (lambda: np.exp(rng.normal(0.0, noise, len(a)))) if rng is not None else (lambda: 1.0)
    X = np.stack([
        (cpu[setting // n_gpu] - cpu[0]) / (cpu[-1] - cpu[0]),
        (gpu[setting % n_gpu] - gpu[0]) / (gpu[-1] - gpu[0]),
        traits.mem_c[a] * s_cpu ** 0.5 * mult(),                   # memory throughput
        traits.ips0[a] * s_cpu * (1.0 - 0.5 * traits.mem_c[a]) * mult(),   # IPS
        clk * mult(),                                              # SM clock
        traits.mem_g[a] * (1.0 - 0.2 * (1.0 - g)) / (s_gpu + 1e-9) * 0.8 * mult(),   # DRAM active
        traits.flop[a] * clk * (1.0 - 0.5 * traits.mem_g[a]) * mult(),   # FP active
    ], axis=1)
    return CounterRuns(X.astype(np.float64), y.astype(np.float64), app.astype(np.int32),
                       setting.astype(np.int32))


def make_traits(rng: np.random.Generator, n_apps: int) -> AppTraits:
    return AppTraits(rng.uniform(0.05, 0.6, n_apps), rng.uniform(0.0, 1.0, n_apps),
                     rng.uniform(0.0, 1.0, n_apps), rng.uniform(0.2, 1.0, n_apps),
                     rng.uniform(0.5, 1.0, n_apps))


def make_counters(seed: int = 0, n_apps: int = 512, n_cpu: int = 16, n_gpu: int = 64,
                  runs: Optional[int] = None, noise: float = 0.02) -> CounterRuns:
    """All settings of every application (runs None) or `runs` random settings
    each (in increasing setting order per application)."""
    rng = np.random.default_rng(seed)
    n = n_cpu * n_gpu
    traits = make_traits(rng, n_apps)
    if runs is None:
        app = np.repeat(np.arange(n_apps), n)
        setting = np.tile(np.arange(n), n_apps)
    else:
        app = np.repeat(np.arange(n_apps), runs)
        keys = rng.random((n_apps, n))
        setting = np.sort(np.argpartition(keys, runs - 1, axis=1)[:, :runs], axis=1).ravel()
    return counter_runs(traits, app, setting, n_cpu, n_gpu, rng, noise)


def pred_init(rng: np.random.Generator, n_features: int = 7, out_scale: float = 0.1):
    """Predictor parameters [W1 (n_features x 128), b1, W2 (128 x 64), b2, w3, b3]
    (LeCun-normal weights, zero biases, output weights scaled), packed."""
    W1 = rng.standard_normal((n_features, NCF_H1)) / math.sqrt(n_features)
    W2 = rng.standard_normal((NCF_H1, NCF_H2)) / math.sqrt(NCF_H1)
    w3 = rng.standard_normal(NCF_H2) / math.sqrt(NCF_H2) * out_scale
    return np.concatenate([W1.ravel(), np.zeros(NCF_H1), W2.ravel(), np.zeros(NCF_H2), w3,
                           np.zeros(1)])
