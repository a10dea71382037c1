"""Pins of the oracle's streaming refit of V (incremental per-setting normal
equations) against the batch half-step over the union of ingested rows, against
numpy's least squares, and against its own invariants (batch splitting,
untouched settings)."""
import numpy as np
import pytest

import synth


def _csr(rng, m, n, density):
    rows, cols = [], []
    for i in range(m):
        c = np.nonzero(rng.random(n) < density)[0]
        rows.append(np.full(len(c), i)); cols.append(c)
    rows = np.concatenate(rows); cols = np.concatenate(cols).astype(np.int32)
    ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=ptr[1:])
    return ptr, cols, rng.random(len(cols))


def _stack(parts):
    """Concatenate CSR blocks (rows in order)."""
    ptrs, cols, vals, off = [np.zeros(1, np.int64)], [], [], 0
    for p, c, v in parts:
        ptrs.append(p[1:] + off); off += p[-1]; cols.append(c); vals.append(v)
    return np.concatenate(ptrs), np.concatenate(cols), np.concatenate(vals)


@pytest.mark.parametrize("weighted", [False, True])
def test_stream_equals_batch_half_step_over_the_union(orc, weighted):
    rng = np.random.default_rng(0)
    n, k, lam = 40, 5, 0.1
    off = _csr(rng, 60, n, 0.5)
    U_off = rng.standard_normal((60, k))
    st = orc.StreamState(n, k, lam, weighted)
    st.add(*off, U_off)
    b1 = _csr(rng, 25, n, 0.2)
    b2 = _csr(rng, 30, n, 0.1)
    U1, _ = st.ingest(*b1)
    U2, _ = st.ingest(*b2)
    ptr, col, val = _stack([off, b1, b2])
    U = np.vstack([U_off, U1, U2])
    cptr, cidx, cval = orc.transpose(ptr, col, val, n)
    solve = orc.half_step_wr if weighted else orc.half_step
    Vref, sref = solve(cptr, cidx, cval, U, lam)
    assert np.abs(st.V - Vref).max() <= 1e-11 * max(1.0, np.abs(Vref).max())
    assert np.array_equal(st.status, sref)
    # the new rows' factors are the fold-in against the V current at their arrival
    fold = orc.half_step_wr if weighted else orc.half_step
    V_after_off = orc.StreamState(n, k, lam, weighted)
    V_after_off.add(*off, U_off)
    U1_ref, _ = fold(*b1, V_after_off.V, lam)
    assert np.abs(U1 - U1_ref).max() <= 1e-12 * max(1.0, np.abs(U1_ref).max())


def test_stream_column_is_ridge_least_squares(orc):
    rng = np.random.default_rng(1)
    n, k, lam = 12, 4, 0.3
    p, c, v = _csr(rng, 50, n, 0.4)
    U = rng.standard_normal((50, k))
    st = orc.StreamState(n, k, lam)
    st.add(p, c, v, U)
    rows = np.repeat(np.arange(50), np.diff(p))
    for j in range(n):
        sel = c == j
        A = np.vstack([U[rows[sel]], np.sqrt(lam) * np.eye(k)])
        y = np.concatenate([v[sel], np.zeros(k)])
        ref = np.linalg.lstsq(A, y, rcond=None)[0] if sel.any() else np.zeros(k)
        assert np.abs(st.V[j] - ref).max() <= 1e-10


def test_stream_batch_split_invariance_and_untouched_settings(orc):
    rng = np.random.default_rng(2)
    n, k, lam = 30, 6, 0.05
    p, c, v = _csr(rng, 90, n - 3, 0.3)          # the last three settings are never observed
    U = rng.standard_normal((90, k))
    one = orc.StreamState(n, k, lam)
    one.add(p, c, v, U)
    three = orc.StreamState(n, k, lam)
    for a, b in [(0, 20), (20, 61), (61, 90)]:
        sp = p[a:b + 1] - p[a]
        three.add(sp, c[p[a]:p[b]], v[p[a]:p[b]], U[a:b])
    assert np.abs(one.G - three.G).max() <= 1e-12 * np.abs(one.G).max()
    assert np.abs(one.V - three.V).max() <= 1e-11
    assert np.all(one.V[-3:] == 0) and np.all(one.status[-3:] == orc.EMPTY_ROW)
    assert np.array_equal(one.cnt[:n - 3], np.bincount(c, minlength=n - 3))
