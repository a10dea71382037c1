"""Helpers shared by the GPU parity tests: device copies of synthetic inputs
and the error measures the tolerances are stated in."""
import numpy as np
import torch

DEV = torch.device("cuda", 0)

# Tolerances (per-row relative 2-norm error against the FP64 oracle fed the
# identical inputs).  FP32: the gate the method's FP32 path is held to;
# FP64: rounding of a k x k Cholesky with modest condition numbers.
TOL_FP32 = 1e-5
TOL_FP64 = 1e-12


def dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device=DEV, dtype=dtype)


def csr_dev(row_ptr, col, val, dtype):
    return dev(row_ptr, torch.int64), dev(col, torch.int32), dev(val, dtype)


def host(t):
    return t.detach().cpu().numpy()


def row_rel_err(gpu, ref, floor=1e-30):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    num = np.linalg.norm(gpu - ref, axis=1)
    den = np.maximum(np.linalg.norm(ref, axis=1), floor)
    return num / den


def rounded(a, dtype):
    """The values a kernel of the given precision actually sees, as FP64."""
    return np.asarray(a, dtype=np.float32 if dtype == torch.float32 else np.float64).astype(
        np.float64)


def solve_err(gpu, ref, F, ptr, col, val, lam, weighted=False):
    """Per-row error of ridge solves, scaled by what FP32 rounding can reach.

    Dividing by |u_ref| alone overstates the error when the right-hand side
    sum b = sum_t r_t f_t cancels (u tiny next to its terms): its rounding
    error is ~eps * sum_t |r_t| |f_t|, carried through A^{-1}.  The scale is
    max(|u_ref|, |A^{-1}|_2 * |sum_t |r_t| |f_t||).  weighted: row i carries
    lambda * s_i (s_i its observation count) instead of lambda."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    out = np.zeros(len(ref))
    k = F.shape[1]
    for i in range(len(ref)):
        c = col[ptr[i]:ptr[i + 1]]
        r = val[ptr[i]:ptr[i + 1]]
        if len(c) == 0:
            out[i] = np.linalg.norm(gpu[i])
            continue
        A = F[c].T @ F[c] + lam * (len(c) if weighted else 1) * np.eye(k)
        babs = (np.abs(r)[:, None] * np.abs(F[c])).sum(0)
        scale = max(np.linalg.norm(ref[i]), np.linalg.norm(np.linalg.inv(A), 2) *
                    np.linalg.norm(babs))
        out[i] = np.linalg.norm(gpu[i] - ref[i]) / max(scale, 1e-300)
    return out
