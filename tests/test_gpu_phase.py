"""Algorithm 1 (phase-transition detection) on the GPU over many traces,
against the oracle's step-by-step circular-buffer version: detection indices
bit for bit."""
import numpy as np
import pytest
import torch

import synth

from gpu_util import DEV, host

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2508_07605_b300 as ocf  # noqa: E402


@pytest.mark.parametrize("n,L", [(1, 24), (1, 25), (7, 31), (300, 1000), (2049, 257), (4, 256),
                                 (5, 512), (64, 3000)])
def test_phase_detect_matches_oracle(orc, n, L):
    P = synth.make_power_traces(seed=n + L, n_traces=n, length=L)
    got = host(ocf.phase_detect(torch.as_tensor(P, device=DEV)))
    assert np.array_equal(got, orc.phase_detect(P))


def test_phase_detect_edges(orc):
    L = 200
    P = np.full((6, L), 40.0, np.float32)
    P[1] = 60.0                          # equal to the threshold: not below
    P[2, 50:75] = 90.0                   # exactly one window
    P[3, 50:74] = 90.0                   # one reading short
    P[4, :] = 100.0
    P[4, 100] = np.nan                   # not a number is not below the threshold
    P[4, 10] = 59.99                     # a dip restarts the window
    P[5, 170:] = 150.0                   # runs into the end of the trace
    got = host(ocf.phase_detect(torch.as_tensor(P, device=DEV)))
    want = orc.phase_detect(P)
    assert np.array_equal(got, want)
    assert list(want) == [-1, 24, 74, -1, 35, 194]


def test_phase_detect_runs_across_chunk_boundaries(orc):
    # the kernel streams 256 readings at a time: runs that start before a
    # multiple of 256 and end after it, and dips right at the boundary
    L = 1100
    P = np.full((6, L), 40.0, np.float32)
    P[0, 250:300] = 90.0                 # report at 274, in the second chunk
    P[1, 232:1100] = 90.0                # report at 256, the boundary reading
    P[2, 231:1100] = 90.0                # report at 255, the last of the first chunk
    P[3, 240:1100] = 90.0
    P[3, 256] = 10.0                     # dip at the boundary: report at 281
    P[4, 500:1100] = 90.0
    P[4, 511:513] = 10.0                 # dips either side of 512: report at 537
    P[5, 1075:] = 90.0                   # the last reading completes the window
    got = host(ocf.phase_detect(torch.as_tensor(P, device=DEV)))
    want = orc.phase_detect(P)
    assert np.array_equal(got, want)
    assert list(want) == [274, 256, 255, 281, 537, 1099]


@pytest.mark.parametrize("window,p_th", [(1, 60.0), (5, 120.0), (100, 60.0)])
def test_phase_detect_other_windows_and_strided_rows(orc, window, p_th):
    P = synth.make_power_traces(seed=window, n_traces=500, length=600)
    big = torch.zeros(500, 640, device=DEV)
    big[:, :600] = torch.as_tensor(P, device=DEV)
    got = host(ocf.phase_detect(big[:, :600], p_th=p_th, window=window))
    assert np.array_equal(got, orc.phase_detect(P, p_th=p_th, window=window, intervals=1))


def test_phase_detect_rejects_bad_window():
    with pytest.raises(ocf.OpenCFError):
        ocf.phase_detect(torch.zeros(2, 10, device=DEV), window=0)


@pytest.mark.parametrize("window", [1, 2, 7, 8, 9, 31, 257])
@pytest.mark.parametrize("L,ld", [(700, 700), (700, 701), (1024, 1024)])
def test_phase_detect_dense_dips(orc, window, L, ld):
    # frequent dips and not-a-number readings: short runs everywhere, both the
    # walk used below an 8-reading window and the one-step test used above it,
    # on rows that start on and off the 16-byte grid
    rng = np.random.default_rng(window * 7 + L + ld)
    P = np.where(rng.random((300, L)) < 0.05, 10.0, 90.0).astype(np.float32)
    P[rng.random(P.shape) < 0.01] = np.nan
    big = torch.zeros(300, ld, device=DEV)
    big[:, :L] = torch.as_tensor(P, device=DEV)
    got = host(ocf.phase_detect(big[:, :L], window=window))
    assert np.array_equal(got, orc.phase_detect(P, window=window, intervals=1))


def test_phase_detect_full_size_sampled(orc):
    """The Algorithm 1 workload at full size (2^17 traces x 3000 readings, one
    launch as the benchmark times it): every 32nd trace and the last 64
    against the oracle, bit for bit."""
    n, L = 1 << 17, 3000
    P = synth.make_power_traces(seed=0, n_traces=n, length=L)
    got = host(ocf.phase_detect(torch.as_tensor(P, device=DEV)))
    samp = np.concatenate([np.arange(0, n, 32), np.arange(n - 64, n)])
    assert np.array_equal(got[samp], orc.phase_detect(P[samp]))
    assert 0.5 < np.mean(got >= 0) < 0.95   # both outcomes occur at scale
