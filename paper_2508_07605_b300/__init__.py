"""Python binding of ``libopen_cf.so`` (see include/open_cf.h).

Argument marshalling only: tensors are checked for device, dtype and layout,
their ``data_ptr()`` and the current CUDA stream are passed to the C ABI, and
outputs are allocated with torch.  Every computation runs in the library's
CUDA kernels; if the library cannot be loaded the import fails loudly -- there
is no CPU path.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import buildlib as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = _build.LIB

OK, INVALID_ARG, NOT_FITTED, CUDA_ERROR, OUT_OF_MEMORY, UNSUPPORTED, TIMEOUT = 0, -1, -2, -3, -4, -5, -6
ROW_OK, ROW_NOT_SPD, ROW_EMPTY, ROW_FALLBACK_USED, ROW_BAD_INPUT = 0, 1, 2, 3, 4
FP64, FP32, BF16_GRAM = 0, 1, 2
_PRECISION = {"fp64": FP64, "fp32": FP32, "bf16_gram": BF16_GRAM}
MAX_K = 32


class OpenCFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"open_cf error {code}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("lambda_", ctypes.c_double), ("sweeps", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("precision", ctypes.c_int),
                ("cholesky_fp64", ctypes.c_int32), ("n_cpu_caps", ctypes.c_int32),
                ("n_gpu_caps", ctypes.c_int32),
                ("cpu_caps_w_host", ctypes.POINTER(ctypes.c_double)),
                ("gpu_caps_w_host", ctypes.POINTER(ctypes.c_double)),
                ("device", ctypes.c_int32), ("mlp_fallback_threshold", ctypes.c_float),
                ("weighted_lambda", ctypes.c_int32)]


_V, _I64, _I32, _F, _D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_double

_SIGNATURES = {
    "open_cf_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(_V)]),
    "open_cf_destroy": (None, [_V]),
    "open_cf_last_error": (ctypes.c_char_p, [_V]),
    "open_cf_set_wait_limit": (ctypes.c_int, [_V, _I32]),
    "open_cf_check": (ctypes.c_int, [_V]),
    "open_cf_set_V": (ctypes.c_int, [_V, _V, _I64, _V]),
    "open_cf_get_V": (ctypes.c_int, [_V, _V, _V]),
    "open_cf_fit_offline": (ctypes.c_int, [_V, _V, _I64, _I64, _I64, _V, _V, _V]),
    "open_cf_fit_csr": (ctypes.c_int, [_V, _I64, _I64, _I64, _V, _V, _V, _V, _V, _V, _V, _V]),
    "open_cf_complete_rows": (ctypes.c_int, [_V, _I64, _I64, _V, _V, _V, _V, _V, _I32, _V]),
    "open_cf_complete_rows_checked": (ctypes.c_int,
                                      [_V, _I64, _I64, _V, _V, _V, _V, _V, _V, _I32, _V]),
    "open_cf_normal_residual": (ctypes.c_int, [_V, _I64, _I64, _V, _V, _V, _V, _V, _V]),
    "open_cf_predict": (ctypes.c_int, [_V, _V, _I64, _V, _V, _V, _F, _I32, _V]),
    "open_cf_save": (ctypes.c_int, [_V, _V, _I64, ctypes.POINTER(_I64)]),
    "open_cf_load": (ctypes.c_int, [_V, _V, _I64]),
    "open_cf_complete_select_host": (ctypes.c_int, [_V, _I64, _I64, _V, _V, _I32, _V, _I32, _F,
                                                    _I32, _V, _V, _V, _V, _I64, _V]),
    "open_cf_select": (ctypes.c_int, [_V, _V, _I64, _I64, _V, _V, _F, _I32, _V]),
    "open_cf_objective": (ctypes.c_int, [_V, _I64, _I64, _V, _V, _V, _V, _V, _V, _V]),
    "open_cf_csr_to_csc": (ctypes.c_int, [_V, _I64, _I64, _I64, _V, _V, _V, _V, _V, _V, _V]),
    "open_cf_validate_csr": (ctypes.c_int, [_V, _I64, _I64, _I64, _V, _V, _V,
                                            ctypes.POINTER(_I32), _V]),
    "open_cf_csr_to_csc_noalloc": (ctypes.c_int, [_I64, _I64, _I64, _V, _V, _V, _V, _V, _V, _V]),
    "open_cf_batched_fit": (ctypes.c_int, [_V, _I64, _V, _V, _V, _V, _I64, _V, _V, _V, _V, _V,
                                           _V]),
    "open_cf_batched_tune": (ctypes.c_int, [_V, _I64, _V, _V, _V, _V, _I64, _V, _V, _V, _V, _V,
                                            _V]),
    "open_cf_mlp_set_params": (ctypes.c_int, [_V, _V, _V]),
    "open_cf_mlp_get_params": (ctypes.c_int, [_V, _V, _V]),
    "open_cf_mlp_train_step": (ctypes.c_int, [_V, _I64, _I64, _V, _V, _V, _V, _F, _V, _V, _V]),
    "open_cf_mlp_infer": (ctypes.c_int, [_V, _I64, _I64, _V, _V, _V, _V, _V, _V, _V]),
    "open_cf_phase_detect": (ctypes.c_int, [_V, _I64, _I64, _I64, _F, _I32, _V, _V]),
    "open_cf_fma_peak": (ctypes.c_int, [_I32, _I32, ctypes.POINTER(_D)]),
    "open_cf_stream_begin": (ctypes.c_int, [_V, _I64, _I64, _V, _V, _V, _V, _V]),
    "open_cf_stream_ingest": (ctypes.c_int, [_V, _I64, _I64, _V, _V, _V, _V, _V, _V]),
    "open_cf_stream_sums": (ctypes.c_int, [_V, _V, _V, _V, _V]),
    "open_cf_stream_set_sums": (ctypes.c_int, [_V, _V, _V, _V, _V]),
    "open_cf_ncf_create": (ctypes.c_int, [_I64, _I32, _V, _I32, _V, _I32, ctypes.c_int,
                                          ctypes.POINTER(_V)]),
    "open_cf_ncf_destroy": (None, [_V]),
    "open_cf_ncf_last_error": (ctypes.c_char_p, [_V]),
    "open_cf_ncf_set_params": (ctypes.c_int, [_V, _V, _V, _V, _V]),
    "open_cf_ncf_get_params": (ctypes.c_int, [_V, _V, _V, _V, _V]),
    "open_cf_ncf_train": (ctypes.c_int, [_V, _I64, _V, _V, _V, _I32, _V, _F, _V, _V]),
    "open_cf_ncf_grad": (ctypes.c_int, [_V, _I64, _V, _V, _V, _V, _V, _V, _V, _V]),
    "open_cf_ncf_predict": (ctypes.c_int, [_V, _V, _F, _I32, _V, _V, _V]),
    "open_cf_ncf_skipped": (ctypes.c_int, [_V, ctypes.POINTER(_I64)]),
    "open_cf_ncf_check": (ctypes.c_int, [_V]),
    "open_cf_ncf_set_wait_limit": (ctypes.c_int, [_V, _I32]),
    "open_cf_pred_create": (ctypes.c_int, [_I32, _I32, ctypes.c_int, ctypes.POINTER(_V)]),
    "open_cf_pred_destroy": (None, [_V]),
    "open_cf_pred_last_error": (ctypes.c_char_p, [_V]),
    "open_cf_pred_set_params": (ctypes.c_int, [_V, _V, _V]),
    "open_cf_pred_get_params": (ctypes.c_int, [_V, _V, _V]),
    "open_cf_pred_train": (ctypes.c_int, [_V, _I64, _V, _V, _I32, _V, _F, _V, _V]),
    "open_cf_pred_grad": (ctypes.c_int, [_V, _I64, _V, _V, _V, _V, _V]),
    "open_cf_pred_infer": (ctypes.c_int, [_V, _I64, _V, _V, _V]),
}

MLP_PARAMS = 86560   # OPEN_CF_MLP_PARAMS
NCF_D, NCF_H1, NCF_H2, NCF_NET = 32, 128, 64, 16641   # OPEN_CF_NCF_*

_lib = None


def build(force: bool = False) -> str:
    """Compile the CUDA library in-tree (nvcc, sm_103a)."""
    return _build.build(force=force)


def lib():
    """Load libopen_cf.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        if not _build.up_to_date():
            _build.build()
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return sorted(_SIGNATURES)


def phase_detect(power, p_th: float = 60.0, window: int = 25):
    """Algorithm 1 on every row of `power` (float32 CUDA tensor [traces, len],
    unit column stride): index of the reading that reports a transition, or -1."""
    if power.dtype != torch.float32 or not power.is_cuda or power.dim() != 2 or \
            power.stride(1) != 1:
        raise ValueError("power must be a 2-D float32 CUDA tensor with unit column stride")
    n, L = power.shape
    out = torch.empty(n, dtype=torch.int64, device=power.device)
    stream = ctypes.c_void_p(torch.cuda.current_stream(power.device).cuda_stream)
    with torch.cuda.device(power.device):
        rc = lib().open_cf_phase_detect(_ptr(power), n, L, power.stride(0), float(p_th),
                                        int(window), _ptr(out), stream)
    if rc != OK:
        raise OpenCFError(rc, "open_cf_phase_detect failed")
    return out


def fma_peak(fp64: bool = False, device: int = 0) -> float:
    """Measured FP32 (or FP64) FMA throughput of the device, TFLOP/s."""
    out = _D(0.0)
    rc = lib().open_cf_fma_peak(int(fp64), int(device), ctypes.byref(out))
    if rc != OK:
        raise OpenCFError(rc, "open_cf_fma_peak failed")
    return float(out.value)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


class OpenCF:
    """Handle of the completion engine (open_cf_create / open_cf_destroy)."""

    def __init__(self, k: int, lam: float, sweeps: int = 15, precision: str = "fp32",
                 cholesky_fp64: bool = False, cpu_caps=None, gpu_caps=None, device: int = 0,
                 mlp_fallback_threshold: float = 0.02, weighted_lambda: bool = False):
        self._h = ctypes.c_void_p(0)
        self.k, self.lam, self.sweeps = int(k), float(lam), int(sweeps)
        self.precision = precision
        self.device = torch.device("cuda", device)
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        cpu = [] if cpu_caps is None else [float(c) for c in cpu_caps]
        gpu = [] if gpu_caps is None else [float(g) for g in gpu_caps]
        self._cpu = (ctypes.c_double * max(1, len(cpu)))(*cpu)
        self._gpu = (ctypes.c_double * max(1, len(gpu)))(*gpu)
        self.n_cpu, self.n_gpu = len(cpu), len(gpu)
        cfg = Config(self.k, self.lam, self.sweeps, 0, _PRECISION[precision], int(cholesky_fp64),
                     len(cpu), len(gpu), ctypes.cast(self._cpu, ctypes.POINTER(ctypes.c_double)),
                     ctypes.cast(self._gpu, ctypes.POINTER(ctypes.c_double)), device,
                     float(mlp_fallback_threshold), int(bool(weighted_lambda)))
        rc = lib().open_cf_create(ctypes.byref(cfg), ctypes.byref(self._h))
        if rc != OK:
            raise OpenCFError(rc, "open_cf_create failed")
        self.n = None

    def close(self):
        if self._h and self._h.value:
            lib().open_cf_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers ---------------------------------------------------------
    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _check(self, rc):
        if rc != OK:
            raise OpenCFError(rc, lib().open_cf_last_error(self._h).decode())

    def _real(self, t, name):
        if t.device != self.device or t.dtype != self.dtype or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {self.dtype} tensor on {self.device}")
        return t

    def _csr(self, row_ptr, col, val):
        if row_ptr.dtype != torch.int64 or col.dtype != torch.int32:
            raise ValueError("row_ptr must be int64 and col int32")
        for t, nm in ((row_ptr, "row_ptr"), (col, "col")):
            if t.device != self.device or not t.is_contiguous():
                raise ValueError(f"{nm} must be contiguous on {self.device}")
        self._real(val, "val")
        return row_ptr.numel() - 1, col.numel()

    def _empty(self, *shape, dtype=None):
        return torch.empty(*shape, dtype=dtype or self.dtype, device=self.device)

    # -- API ---------------------------------------------------------------
    def last_error(self) -> str:
        return lib().open_cf_last_error(self._h).decode()

    def set_wait_limit(self, polls: int = -1):
        """Bound of the tensor-core pipelines' waits in polls (0: give up at once,
        -1: the default)."""
        self._check(lib().open_cf_set_wait_limit(self._h, int(polls)))

    def check(self):
        """Raise OpenCFError(TIMEOUT) if a tensor-core pipeline wait gave up since
        the last check (synchronises the device; clears the flags)."""
        with torch.cuda.device(self.device):
            self._check(lib().open_cf_check(self._h))

    def set_V(self, V):
        self._real(V, "V")
        if V.dim() != 2 or V.shape[1] != self.k:
            raise ValueError("V must be [n, k]")
        self._check(lib().open_cf_set_V(self._h, _ptr(V), V.shape[0], self._stream()))
        self.n = V.shape[0]

    def get_V(self):
        out = self._empty(self.n, self.k)
        self._check(lib().open_cf_get_V(self._h, _ptr(out), self._stream()))
        return out

    def fit_offline(self, P, J_hist: bool = False):
        self._real(P, "P")
        m, n = P.shape
        U = self._empty(m, self.k)
        J = self._empty(2 * self.sweeps, dtype=torch.float64) if J_hist else None
        self._check(lib().open_cf_fit_offline(self._h, _ptr(P), m, n, P.stride(0), _ptr(U),
                                              _ptr(J), self._stream()))
        return (U, J) if J_hist else U

    def fit_csr(self, row_ptr, col, val, n: int, J_hist: bool = False, status: bool = False):
        m, nnz = self._csr(row_ptr, col, val)
        U = self._empty(m, self.k)
        J = self._empty(2 * self.sweeps, dtype=torch.float64) if J_hist else None
        rs = self._empty(m, dtype=torch.int32) if status else None
        cs = self._empty(n, dtype=torch.int32) if status else None
        self._check(lib().open_cf_fit_csr(self._h, m, n, nnz, _ptr(row_ptr), _ptr(col), _ptr(val),
                                          _ptr(U), _ptr(rs), _ptr(cs), _ptr(J), self._stream()))
        out = [U]
        if J_hist:
            out.append(J)
        if status:
            out += [rs, cs]
        return out[0] if len(out) == 1 else tuple(out)

    def complete_rows(self, row_ptr, col, val, joint: bool = False):
        m, nnz = self._csr(row_ptr, col, val)
        U = self._empty(m, self.k)
        st = self._empty(m, dtype=torch.int32)
        self._check(lib().open_cf_complete_rows(self._h, m, nnz, _ptr(row_ptr), _ptr(col),
                                                _ptr(val), _ptr(U), _ptr(st), int(joint),
                                                self._stream()))
        return U, st

    def complete_rows_checked(self, row_ptr, col, val, refine: bool = False, U=None, st=None,
                              resid=None):
        """Fold-in with the per-row normal-equation residual (and optionally one
        refinement step); returns (U, status, resid).  Output tensors may be
        passed in to be reused."""
        m, nnz = self._csr(row_ptr, col, val)
        U = self._empty(m, self.k) if U is None else U
        st = self._empty(m, dtype=torch.int32) if st is None else st
        resid = self._empty(m, dtype=torch.float32) if resid is None else resid
        self._check(lib().open_cf_complete_rows_checked(
            self._h, m, nnz, _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(U), _ptr(st),
            _ptr(resid), int(bool(refine)), self._stream()))
        return U, st, resid

    def complete_select_host(self, row_ptr, col, val, check: int = 2, gamma: float = 0.05,
                             baseline: int = -1, best=None, saving=None, status=None,
                             resid=None, chunk_rows: int = 0):
        """Fold-in (check 0: plain, 1: residual check, 2: check + one refinement
        step) and Algorithm 2 for a CSR in host memory (col int32, or uint16 to
        send a quarter fewer bytes), decisions back in host memory; the copies of one chunk of rows overlap the solves of the one
        before (pin the host tensors for that).  Returns (best, saving, status,
        resid) host tensors (status / resid None unless passed in); the work is
        queued on the current stream: synchronise it before reading them."""
        if row_ptr.dtype != torch.int64 or val.dtype != torch.float32:
            raise ValueError("row_ptr int64, val float32")
        if col.dtype not in (torch.int32, torch.uint16):
            raise ValueError("col int32, or uint16 for up to 65,535 settings")
        for t, nm in ((row_ptr, "row_ptr"), (col, "col"), (val, "val")):
            if t.device.type != "cpu" or not t.is_contiguous():
                raise ValueError(f"{nm} must be a contiguous host tensor")
        m, nnz = row_ptr.numel() - 1, col.numel()
        best = torch.empty(m, dtype=torch.int32, pin_memory=True) if best is None else best
        saving = torch.empty(m, dtype=torch.float32, pin_memory=True) if saving is None else saving
        for t in (best, saving, status, resid):
            if t is not None and (t.device.type != "cpu" or not t.is_contiguous() or
                                  t.numel() != m):
                raise ValueError("outputs must be contiguous host tensors of m elements")
        self._check(lib().open_cf_complete_select_host(
            self._h, m, nnz, _ptr(row_ptr), _ptr(col), 2 if col.dtype == torch.uint16 else 4,
            _ptr(val), int(check), float(gamma),
            int(baseline), _ptr(best), _ptr(saving), _ptr(status), _ptr(resid), int(chunk_rows),
            self._stream()))
        return best, saving, status, resid

    def save(self) -> bytes:
        """Checkpoint of the handle's state (V, learned warm start with its Adam
        state, streaming sums) as bytes; waits for the device."""
        size = _I64(0)
        self._check(lib().open_cf_save(self._h, None, 0, ctypes.byref(size)))
        buf = ctypes.create_string_buffer(size.value)
        self._check(lib().open_cf_save(self._h, buf, size.value, ctypes.byref(size)))
        return buf.raw[:size.value]

    def load(self, data: bytes):
        """Restore a checkpoint made by save() on a handle of the same configuration."""
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        self._check(lib().open_cf_load(self._h, buf, len(data)))
        n = int.from_bytes(bytes(data[48:56]), "little", signed=True)   # the header's settings
        if n > 0:
            self.n = n

    def normal_residual(self, row_ptr, col, val, U):
        """Per-row relative normal-equation residual of the given factors."""
        m, nnz = self._csr(row_ptr, col, val)
        self._real(U, "U")
        resid = self._empty(m, dtype=torch.float32)
        self._check(lib().open_cf_normal_residual(self._h, m, nnz, _ptr(row_ptr), _ptr(col),
                                                  _ptr(val), _ptr(U), _ptr(resid),
                                                  self._stream()))
        return resid

    def predict(self, U, gamma: float = 0.05, baseline: int = -1, want_T: bool = True,
                want_select: bool = True):
        self._real(U, "U")
        m = U.shape[0]
        T = self._empty(m, self.n) if want_T else None
        best = self._empty(m, dtype=torch.int32) if want_select else None
        sav = self._empty(m, dtype=torch.float32) if want_select else None
        self._check(lib().open_cf_predict(self._h, _ptr(U), m, _ptr(T), _ptr(best), _ptr(sav),
                                          float(gamma), int(baseline), self._stream()))
        return T, best, sav

    def select(self, T, gamma: float = 0.05, baseline: int = -1):
        if T.dtype != torch.float32 or T.device != self.device or T.stride(1) != 1:
            raise ValueError("T must be float32 on the device with unit column stride")
        m = T.shape[0]
        best = self._empty(m, dtype=torch.int32)
        sav = self._empty(m, dtype=torch.float32)
        self._check(lib().open_cf_select(self._h, _ptr(T), m, T.stride(0), _ptr(best), _ptr(sav),
                                         float(gamma), int(baseline), self._stream()))
        return best, sav

    def stream_begin(self, row_ptr, col, val, U):
        """Seed the streaming refit with rows and their factors U (m x k); V is
        re-solved over them."""
        m, nnz = self._csr(row_ptr, col, val)
        self._real(U, "U")
        self._check(lib().open_cf_stream_begin(self._h, m, nnz, _ptr(row_ptr), _ptr(col),
                                               _ptr(val), _ptr(U), self._stream()))

    def stream_ingest(self, row_ptr, col, val, out=None, status=None):
        """A batch of new applications: (U_new, status); V is refitted in place.
        `out` (m x k) and `status` (int32 m) may be given to reuse buffers."""
        m, nnz = self._csr(row_ptr, col, val)
        U = out if out is not None else self._empty(m, self.k)
        st = status if status is not None else self._empty(m, dtype=torch.int32)
        self._real(U, "out")
        if U.shape != (m, self.k) or st.shape != (m,) or st.dtype != torch.int32:
            raise ValueError("out must be m x k and status int32 of length m")
        self._check(lib().open_cf_stream_ingest(self._h, m, nnz, _ptr(row_ptr), _ptr(col),
                                                _ptr(val), _ptr(U), _ptr(st), self._stream()))
        return U, st

    def stream_sums(self):
        """(G [n, KP, KP], b [n, KP], counts [n]) of the streaming refit."""
        n = self.get_V().shape[0]
        kp = 8 if self.k <= 8 else (16 if self.k <= 16 else 32)
        G = self._empty(n, kp, kp)
        b = self._empty(n, kp)
        cnt = torch.empty(n, dtype=torch.int64, device=self.device)
        self._check(lib().open_cf_stream_sums(self._h, _ptr(G), _ptr(b), _ptr(cnt),
                                              self._stream()))
        return G, b, cnt

    def stream_set_sums(self, G, b, cnt):
        """Install sums (e.g. totals over several processes) and re-solve V."""
        for t, nm in ((G, "G"), (b, "b")):
            self._real(t, nm)
        if cnt.dtype != torch.int64 or cnt.device != self.device or not cnt.is_contiguous():
            raise ValueError("counts must be a contiguous int64 tensor on the device")
        self._check(lib().open_cf_stream_set_sums(self._h, _ptr(G), _ptr(b), _ptr(cnt),
                                                  self._stream()))

    def objective(self, row_ptr, col, val, U, row_rmse: bool = False):
        m, nnz = self._csr(row_ptr, col, val)
        self._real(U, "U")
        J = self._empty(1, dtype=torch.float64)
        rr = self._empty(m, dtype=torch.float32) if row_rmse else None
        self._check(lib().open_cf_objective(self._h, m, nnz, _ptr(row_ptr), _ptr(col), _ptr(val),
                                            _ptr(U), _ptr(J), _ptr(rr), self._stream()))
        return (J, rr) if row_rmse else J

    def csr_to_csc(self, row_ptr, col, val, n: int):
        m, nnz = self._csr(row_ptr, col, val)
        cptr = self._empty(n + 1, dtype=torch.int64)
        ridx = self._empty(max(nnz, 1), dtype=torch.int32)
        cval = self._empty(max(nnz, 1))
        self._check(lib().open_cf_csr_to_csc(self._h, m, n, nnz, _ptr(row_ptr), _ptr(col),
                                             _ptr(val), _ptr(cptr), _ptr(ridx), _ptr(cval),
                                             self._stream()))
        return cptr, ridx[:nnz], cval[:nnz]

    def batched_fit(self, m, n, k, nnz_p, row_ptr, col, val, V, want_U: bool = True):
        """Batched completion: m, n, k, nnz_p are host int sequences (one entry
        per problem); row_ptr/col/val the stacked CSR on the device; V the
        stacked initial V (float32, overwritten in place with the fitted V)."""
        import numpy as np
        m = np.ascontiguousarray(m, dtype=np.int64); n = np.ascontiguousarray(n, dtype=np.int64)
        k = np.ascontiguousarray(k, dtype=np.int32)
        nz = np.ascontiguousarray(nnz_p, dtype=np.int64)
        self._csr(row_ptr, col, val)
        self._real(V, "V")
        U = self._empty(int((m * k).sum())) if want_U else None
        self._check(lib().open_cf_batched_fit(
            self._h, len(m), m.ctypes.data, n.ctypes.data, k.ctypes.data, nz.ctypes.data,
            col.numel(), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(V), _ptr(U), self._stream()))
        return U

    def batched_tune(self, m, n, k, nnz_p, row_ptr, col, val, V_scratch):
        import numpy as np
        m = np.ascontiguousarray(m, dtype=np.int64); n = np.ascontiguousarray(n, dtype=np.int64)
        k = np.ascontiguousarray(k, dtype=np.int32)
        nz = np.ascontiguousarray(nnz_p, dtype=np.int64)
        W = (ctypes.c_int32 * 4)()
        self._check(lib().open_cf_batched_tune(
            self._h, len(m), m.ctypes.data, n.ctypes.data, k.ctypes.data, nz.ctypes.data,
            col.numel(), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(V_scratch), W,
            self._stream()))
        return tuple(int(w) for w in W)   # warps large, warps small, cut %, CTAs per SM

    # -- learned warm start ------------------------------------------------
    def _f32(self, t, name, numel=None):
        if t.device != self.device or t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float32 tensor on {self.device}")
        if numel is not None and t.numel() != numel:
            raise ValueError(f"{name} must have {numel} entries")
        return t

    def mlp_set_params(self, params):
        self._f32(params, "params", MLP_PARAMS)
        self._check(lib().open_cf_mlp_set_params(self._h, _ptr(params), self._stream()))

    def mlp_get_params(self):
        out = self._empty(MLP_PARAMS, dtype=torch.float32)
        self._check(lib().open_cf_mlp_get_params(self._h, _ptr(out), self._stream()))
        return out

    def mlp_train_step(self, row_ptr, col, val, U_target, lr: float = 1e-3, loss=None,
                       grads: bool = False):
        """One Adam step (grads False) or the gradient alone (grads True,
        parameters unchanged).  ``loss``: optional float64 device tensor of
        one element that receives the loss before the update."""
        B, nnz = self._csr(row_ptr, col, val)
        self._f32(U_target, "U_target", B * self.k)
        if loss is not None and (loss.dtype != torch.float64 or loss.device != self.device):
            raise ValueError("loss must be a float64 tensor on the device")
        g = self._empty(MLP_PARAMS, dtype=torch.float32) if grads else None
        self._check(lib().open_cf_mlp_train_step(self._h, B, nnz, _ptr(row_ptr), _ptr(col),
                                                 _ptr(val), _ptr(U_target), float(lr),
                                                 _ptr(loss), _ptr(g), self._stream()))
        return g

    def mlp_infer(self, row_ptr, col, val, row_rmse: bool = False):
        m, nnz = self._csr(row_ptr, col, val)
        U = self._empty(m, self.k, dtype=torch.float32)
        st = self._empty(m, dtype=torch.int32)
        rr = self._empty(m, dtype=torch.float32) if row_rmse else None
        self._check(lib().open_cf_mlp_infer(self._h, m, nnz, _ptr(row_ptr), _ptr(col), _ptr(val),
                                            _ptr(U), _ptr(st), _ptr(rr), self._stream()))
        return (U, st, rr) if row_rmse else (U, st)

    def validate_csr(self, row_ptr, col, val, n: int) -> int:
        m, nnz = self._csr(row_ptr, col, val)
        res = ctypes.c_int32(-1)
        self._check(lib().open_cf_validate_csr(self._h, m, n, nnz, _ptr(row_ptr), _ptr(col),
                                               _ptr(val), ctypes.byref(res), self._stream()))
        return int(res.value)


class NCF:
    """Handle of neural collaborative filtering (open_cf_ncf_create / destroy):
    m applications, the CPU-major cap grid's n settings, mini-batch capacity
    `batch` (a multiple of 64)."""

    def __init__(self, m: int, cpu_caps, gpu_caps, batch: int = 1024, device: int = 0):
        self._h = ctypes.c_void_p(0)
        self.m = int(m)
        self.n = len(cpu_caps) * len(gpu_caps)
        self.batch = int(batch)
        self.device = torch.device("cuda", device)
        cpu = (ctypes.c_double * len(cpu_caps))(*[float(c) for c in cpu_caps])
        gpu = (ctypes.c_double * len(gpu_caps))(*[float(g) for g in gpu_caps])
        h = ctypes.c_void_p(0)
        rc = lib().open_cf_ncf_create(self.m, len(cpu_caps), cpu, len(gpu_caps), gpu, self.batch,
                                      device, ctypes.byref(h))
        if rc != OK:
            raise OpenCFError(rc, "open_cf_ncf_create failed")
        self._h = h

    def close(self):
        if self._h:
            lib().open_cf_ncf_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != OK:
            msg = lib().open_cf_ncf_last_error(self._h)
            raise OpenCFError(rc, msg.decode() if msg else "")

    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _t(self, t, dtype, numel, name):
        if t.dtype != dtype or t.device != self.device or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {dtype} tensor on {self.device}")
        if numel is not None and t.numel() != numel:
            raise ValueError(f"{name} must have {numel} elements")
        return t

    def set_params(self, net, Ea, Es):
        self._t(net, torch.float32, NCF_NET, "net")
        self._t(Ea, torch.float32, self.m * NCF_D, "Ea")
        self._t(Es, torch.float32, self.n * NCF_D, "Es")
        with torch.cuda.device(self.device):
            self._check(lib().open_cf_ncf_set_params(self._h, _ptr(net), _ptr(Ea), _ptr(Es),
                                                     self._stream()))

    def get_params(self):
        net = torch.empty(NCF_NET, dtype=torch.float32, device=self.device)
        Ea = torch.empty(self.m, NCF_D, dtype=torch.float32, device=self.device)
        Es = torch.empty(self.n, NCF_D, dtype=torch.float32, device=self.device)
        with torch.cuda.device(self.device):
            self._check(lib().open_cf_ncf_get_params(self._h, _ptr(net), _ptr(Ea), _ptr(Es),
                                                     self._stream()))
        return net, Ea, Es

    def _coo(self, app, setting, val):
        nnz = app.numel()
        self._t(app, torch.int32, nnz, "app")
        self._t(setting, torch.int32, nnz, "setting")
        self._t(val, torch.float32, nnz, "val")
        return nnz

    def steps(self, nnz: int, epochs: int) -> int:
        return epochs * ((nnz + self.batch - 1) // self.batch)

    def train(self, app, setting, val, perms, lr: float, losses: bool = False):
        """perms: int32 [epochs, nnz] visiting orders.  Returns the per-step
        losses (float64 tensor) when asked, else None."""
        nnz = self._coo(app, setting, val)
        epochs = perms.shape[0] if perms.dim() == 2 else 0
        self._t(perms, torch.int32, epochs * nnz, "perms")
        L = torch.empty(self.steps(nnz, epochs), dtype=torch.float64,
                        device=self.device) if losses else None
        with torch.cuda.device(self.device):
            self._check(lib().open_cf_ncf_train(self._h, nnz, _ptr(app), _ptr(setting), _ptr(val),
                                                epochs, _ptr(perms), float(lr), _ptr(L),
                                                self._stream()))
        return L

    def grad(self, app, setting, val):
        """(loss, g_net, g_Ea, g_Es) of one batch, no update."""
        B = self._coo(app, setting, val)
        loss = torch.empty(1, dtype=torch.float64, device=self.device)
        gn = torch.empty(NCF_NET, dtype=torch.float32, device=self.device)
        ga = torch.empty(self.m, NCF_D, dtype=torch.float32, device=self.device)
        gs = torch.empty(self.n, NCF_D, dtype=torch.float32, device=self.device)
        with torch.cuda.device(self.device):
            self._check(lib().open_cf_ncf_grad(self._h, B, _ptr(app), _ptr(setting), _ptr(val),
                                               _ptr(loss), _ptr(gn), _ptr(ga), _ptr(gs),
                                               self._stream()))
        return loss, gn, ga, gs

    def predict(self, gamma: float = 0.05, T: bool = True, select: bool = True,
                baseline: int = -1):
        """(T [m, n] or None, best [m] or None, saving [m] or None)."""
        Tt = torch.empty(self.m, self.n, dtype=torch.float32, device=self.device) if T else None
        best = torch.empty(self.m, dtype=torch.int32, device=self.device) if select else None
        sav = torch.empty(self.m, dtype=torch.float32, device=self.device) if select else None
        with torch.cuda.device(self.device):
            self._check(lib().open_cf_ncf_predict(self._h, _ptr(Tt), float(gamma), int(baseline),
                                                  _ptr(best), _ptr(sav), self._stream()))
        return Tt, best, sav

    def skipped(self) -> int:
        c = _I64(0)
        with torch.cuda.device(self.device):
            self._check(lib().open_cf_ncf_skipped(self._h, ctypes.byref(c)))
        return int(c.value)

    def check(self):
        with torch.cuda.device(self.device):
            self._check(lib().open_cf_ncf_check(self._h))

    def set_wait_limit(self, polls: int = -1):
        self._check(lib().open_cf_ncf_set_wait_limit(self._h, int(polls)))


class Predictor:
    """Offline performance predictor (open_cf_pred_*): n_features dense inputs
    -> 128 -> 64 SELU units -> one output, trained on the mean squared error."""

    def __init__(self, n_features: int = 7, batch: int = 1024, device: int = 0):
        self._h = ctypes.c_void_p(0)
        self.nf, self.batch = int(n_features), int(batch)
        self.device = torch.device("cuda", device)
        self.n_params = self.nf * NCF_H1 + (NCF_NET - 2 * NCF_D * NCF_H1)
        h = ctypes.c_void_p(0)
        rc = lib().open_cf_pred_create(self.nf, self.batch, device, ctypes.byref(h))
        if rc != OK:
            raise OpenCFError(rc, "open_cf_pred_create failed")
        self._h = h

    def close(self):
        if self._h:
            lib().open_cf_pred_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != OK:
            msg = lib().open_cf_pred_last_error(self._h)
            raise OpenCFError(rc, msg.decode() if msg else "")

    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _t(self, t, dtype, numel, name):
        if t.dtype != dtype or t.device != self.device or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {dtype} tensor on {self.device}")
        if numel is not None and t.numel() != numel:
            raise ValueError(f"{name} must have {numel} elements")
        return t

    def set_params(self, params):
        self._t(params, torch.float32, self.n_params, "params")
        with torch.cuda.device(self.device):
            self._check(lib().open_cf_pred_set_params(self._h, _ptr(params), self._stream()))

    def get_params(self):
        p = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        with torch.cuda.device(self.device):
            self._check(lib().open_cf_pred_get_params(self._h, _ptr(p), self._stream()))
        return p

    def _xy(self, X, y):
        N = y.numel()
        self._t(X, torch.float32, N * self.nf, "X")
        self._t(y, torch.float32, N, "y")
        return N

    def train(self, X, y, perms, lr: float, losses: bool = False):
        N = self._xy(X, y)
        epochs = perms.shape[0] if perms.dim() == 2 else 0
        self._t(perms, torch.int32, epochs * N, "perms")
        L = torch.empty(epochs * ((N + self.batch - 1) // self.batch), dtype=torch.float64,
                        device=self.device) if losses else None
        with torch.cuda.device(self.device):
            self._check(lib().open_cf_pred_train(self._h, N, _ptr(X), _ptr(y), epochs,
                                                 _ptr(perms), float(lr), _ptr(L), self._stream()))
        return L

    def grad(self, X, y):
        B = self._xy(X, y)
        loss = torch.empty(1, dtype=torch.float64, device=self.device)
        g = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        with torch.cuda.device(self.device):
            self._check(lib().open_cf_pred_grad(self._h, B, _ptr(X), _ptr(y), _ptr(loss), _ptr(g),
                                                self._stream()))
        return loss, g

    def infer(self, X):
        N = X.numel() // self.nf
        self._t(X, torch.float32, N * self.nf, "X")
        y = torch.empty(N, dtype=torch.float32, device=self.device)
        with torch.cuda.device(self.device):
            self._check(lib().open_cf_pred_infer(self._h, N, _ptr(X), _ptr(y), self._stream()))
        return y
