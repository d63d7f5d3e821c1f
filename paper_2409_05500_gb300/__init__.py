"""GB300 (sm_103a) approximate-ordering VarLiNGAM.

Thin Python binding over the C ABI declared in include/varlingam_gb300.h.
The functions below carry the C names and only marshal arguments: every step
of the method runs in the library's CUDA kernels.  PyTorch supplies device
memory and streams.  There is no CPU fallback: if the shared library is
missing or cannot be loaded, importing this package raises.

Quick use::

    import torch, paper_2409_05500_gb300 as vl
    h = vl.Handle()                              # current CUDA device/stream
    out = vl.fit(h, X_cuda_float64, p=1)         # dict of device tensors
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvarlingam_gb300.so")

VL_OK = 0
STATUS_NAMES = {
    0: "VL_OK", 1: "VL_ERR_ARG", 2: "VL_ERR_SHAPE", 3: "VL_ERR_RANK",
    4: "VL_ERR_DEGENERATE", 5: "VL_ERR_NONFINITE", 6: "VL_ERR_CUDA", 7: "VL_ERR_NOMEM",
    8: "VL_ERR_TIMEOUT", 9: "VL_ERR_UNSUPPORTED",
}
VL_PREC_FP64 = 0
VL_PREC_MIXED = 1
VL_PREC_MIXED_CERTIFIED = 2
PRECISIONS = {"fp64": VL_PREC_FP64, "mixed": VL_PREC_MIXED,
              "mixed_certified": VL_PREC_MIXED_CERTIFIED}

EXPORTED = ("vl_create", "vl_destroy", "vl_set_stream", "vl_reserve", "vl_sync",
            "vl_last_error", "vl_profile_events", "vl_kernel_launches", "vl_fit", "vl_var_fit",
            "vl_pairwise_measure", "vl_causal_order", "vl_causal_order_noalloc",
            "vl_causal_order_certified", "vl_causal_order_standard", "vl_fit_b",
            "vl_fit_batched", "vl_fit_batched_async", "vl_sfu_rate", "vl_var_select",
            "vl_bootstrap_resample", "vl_bootstrap")
CRITERIA = {"aic": 0, "bic": 1, "hq": 2}


class VLError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class vl_instance(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("ldx", ctypes.c_int64), ("m", ctypes.c_int),
                ("n", ctypes.c_int), ("p", ctypes.c_int), ("order", ctypes.c_void_p),
                ("B0", ctypes.c_void_p), ("Btau", ctypes.c_void_p), ("M", ctypes.c_void_p),
                ("D", ctypes.c_void_p)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; "
            "g.build()'` (nvcc for sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, I64, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    sig = {
        "vl_create": [ctypes.POINTER(P), I, P, S],
        "vl_destroy": [P],
        "vl_set_stream": [P, P],
        "vl_reserve": [P, I, I, I],
        "vl_sync": [P],
        "vl_var_fit": [P, P, I64, I, I, I, I, P, P],
        "vl_var_select": [P, P, I64, I, I, I, I, I, P, P],
        "vl_bootstrap_resample": [P, P, I64, I, I, I, ctypes.c_uint64, I64, I, P],
        "vl_bootstrap": [P, P, I64, I, I, I, I, I, ctypes.c_uint64, ctypes.c_double, I, P, P],
        "vl_pairwise_measure": [P, P, I64, I, I, I, P, P, P],
        "vl_causal_order": [P, P, I, P, P],
        "vl_causal_order_noalloc": [P, P, I, P, P],
        "vl_causal_order_certified": [P, P, P, I64, I, I, P, P, P],
        "vl_causal_order_standard": [P, P, I64, I, I, I, P, P],
        "vl_fit_b": [P, P, I64, I, I, P, P, I, I, P, P],
        "vl_fit_batched": [P, ctypes.POINTER(vl_instance), I, I, ctypes.POINTER(I)],
        "vl_fit_batched_async": [P, ctypes.POINTER(vl_instance), I, I, P],
        "vl_fit": [P, P, I64, I, I, I, I, P, P, P, P, P],
        "vl_profile_events": [P, P, P],
        "vl_sfu_rate": [I, P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = I
    lib.vl_last_error.argtypes = [P]
    lib.vl_last_error.restype = ctypes.c_char_p
    lib.vl_kernel_launches.argtypes = []
    lib.vl_kernel_launches.restype = ctypes.c_ulonglong
    return lib


_lib = _load()


def lib() -> ctypes.CDLL:
    return _lib


def sfu_rate(device: int = 0):
    """Measured (ex2, lg2) results per clock per SM of the special-function
    unit (diagnostic)."""
    e, l = ctypes.c_double(), ctypes.c_double()
    code = _lib.vl_sfu_rate(device, ctypes.byref(e), ctypes.byref(l))
    if code != VL_OK:
        raise VLError(code, "vl_sfu_rate failed")
    return e.value, l.value


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(_lib.vl_kernel_launches())


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("library arguments must be CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("library arguments must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _rows_ptr(t: torch.Tensor):
    """A matrix whose rows may be strided (a column slice of a wider one):
    unit stride within a row, the row stride passed beside the pointer."""
    if not t.is_cuda:
        raise ValueError("library arguments must be CUDA tensors")
    if t.dim() != 2 or t.stride(1) != 1 or t.stride(0) < t.shape[1]:
        raise ValueError("matrix arguments need unit stride within a row")
    return ctypes.c_void_p(t.data_ptr())


class Handle:
    """Owns a vl_handle bound to a CUDA device and stream (default: the
    current torch device and stream)."""

    def __init__(self, device: Optional[int] = None, stream: Optional[torch.cuda.Stream] = None,
                 workspace_bytes: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA is not available: this library has no CPU path")
        self.device = torch.cuda.current_device() if device is None else device
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        code = _lib.vl_create(ctypes.byref(h), self.device, ctypes.c_void_p(self.stream.cuda_stream),
                              workspace_bytes)
        if code != VL_OK:
            raise VLError(code, "vl_create failed")
        self.h = h

    def check(self, code: int, what: str):
        if code != VL_OK:
            raise VLError(code, f"{what}: {_lib.vl_last_error(self.h).decode()}")

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        self.check(_lib.vl_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)), "vl_set_stream")

    def profile_events(self, start: Optional[torch.cuda.Event], stop: Optional[torch.cuda.Event]):
        """Record start/stop around the pairwise-moment kernel of later calls."""
        a = ctypes.c_void_p(start.cuda_event) if start is not None else None
        b = ctypes.c_void_p(stop.cuda_event) if stop is not None else None
        self.check(_lib.vl_profile_events(self.h, a, b), "vl_profile_events")

    def sync(self):
        self.check(_lib.vl_sync(self.h), "vl_sync")

    def close(self):
        if getattr(self, "h", None):
            _lib.vl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- C names
def vl_var_fit(h: Handle, X: torch.Tensor, p: int, prec: str, M: torch.Tensor,
               E: Optional[torch.Tensor]) -> None:
    m, n = X.shape
    h.check(_lib.vl_var_fit(h.h, _ptr(X), X.stride(0), m, n, p, PRECISIONS[prec], _ptr(M),
                            _ptr(E)), "vl_var_fit")


def vl_var_select(h: Handle, X: torch.Tensor, p_max: int, criterion: str, prec: str,
                  values: torch.Tensor, p_best: torch.Tensor) -> None:
    """Lag order by AIC, BIC or HQ over p = 1..p_max (see the header):
    values (p_max FP64) and p_best (one int32) are device outputs."""
    m, n = X.shape
    h.check(_lib.vl_var_select(h.h, _ptr(X), X.stride(0), m, n, p_max, CRITERIA[criterion],
                               PRECISIONS[prec], _ptr(values), _ptr(p_best)), "vl_var_select")


def vl_bootstrap_resample(h: Handle, X: torch.Tensor, block_len: int, seed: int, b0: int,
                          Xb: torch.Tensor) -> None:
    """Moving-block resamples b0 .. b0 + nb - 1 of X into Xb (nb x m x n,
    contiguous; see the header for the block starts)."""
    m, n = X.shape
    nb = Xb.shape[0]
    h.check(_lib.vl_bootstrap_resample(h.h, _rows_ptr(X), X.stride(0), m, n, block_len, seed, b0, nb,
                                       _ptr(Xb)), "vl_bootstrap_resample")


def vl_bootstrap(h: Handle, X: torch.Tensor, p: int, n_resamples: int, block_len: int,
                 seed: int, threshold: float, prec: str, edge_prob: torch.Tensor,
                 order_prob: torch.Tensor) -> None:
    """The whole method on n_resamples moving-block resamples: edge_prob and
    order_prob (m x m FP64, device) receive the fraction of resamples with
    |B0[i, j]| > threshold and with i before j in the causal order."""
    m, n = X.shape
    h.check(_lib.vl_bootstrap(h.h, _rows_ptr(X), X.stride(0), m, n, p, n_resamples, block_len, seed,
                              threshold, PRECISIONS[prec], _ptr(edge_prob), _ptr(order_prob)),
            "vl_bootstrap")


def vl_pairwise_measure(h: Handle, E: torch.Tensor, prec: str, Hx: Optional[torch.Tensor],
                        Hr: Optional[torch.Tensor], D: Optional[torch.Tensor]) -> None:
    m, n_eff = E.shape
    h.check(_lib.vl_pairwise_measure(h.h, _ptr(E), E.stride(0), m, n_eff, PRECISIONS[prec],
                                     _ptr(Hx), _ptr(Hr), _ptr(D)), "vl_pairwise_measure")


def vl_causal_order(h: Handle, D: torch.Tensor, order: torch.Tensor,
                    gap: Optional[torch.Tensor] = None) -> None:
    m = D.shape[0]
    h.check(_lib.vl_causal_order(h.h, _ptr(D), m, _ptr(order), _ptr(gap)), "vl_causal_order")


def vl_causal_order_certified(h: Handle, D: torch.Tensor, E: torch.Tensor, order: torch.Tensor,
                              gap: Optional[torch.Tensor] = None,
                              stats: Optional[torch.Tensor] = None) -> None:
    """Algorithm 1 on a mixed-precision D with near ties decided on FP64
    entries recomputed from E (the data D was measured from).  stats: 4 int32
    on the device (steps re-decided, pairs re-evaluated, picks changed, steps
    left unverified) or None."""
    m, n_eff = E.shape
    h.check(_lib.vl_causal_order_certified(h.h, _ptr(D), _ptr(E), E.stride(0), m, n_eff,
                                           _ptr(order), _ptr(gap), _ptr(stats)),
            "vl_causal_order_certified")


def vl_causal_order_noalloc(D: torch.Tensor, order: torch.Tensor,
                            gap: Optional[torch.Tensor] = None,
                            stream: Optional[torch.cuda.Stream] = None) -> None:
    """Allocation-free ordering on `stream` (default: the current stream);
    m <= 512.  See include/varlingam_gb300.h for its rules."""
    st = stream if stream is not None else torch.cuda.current_stream()
    code = _lib.vl_causal_order_noalloc(ctypes.c_void_p(st.cuda_stream), _ptr(D), D.shape[0],
                                        _ptr(order), _ptr(gap))
    if code != VL_OK:
        raise VLError(code, "vl_causal_order_noalloc")


def vl_causal_order_standard(h: Handle, E: torch.Tensor, prec: str, order: torch.Tensor,
                             gap: Optional[torch.Tensor] = None) -> None:
    """The iterative search of Section 3 (Eq. 4 refinement every iteration)."""
    m, n_eff = E.shape
    h.check(_lib.vl_causal_order_standard(h.h, _ptr(E), E.stride(0), m, n_eff,
                                          PRECISIONS[prec], _ptr(order), _ptr(gap)),
            "vl_causal_order_standard")


def vl_fit_b(h: Handle, E: torch.Tensor, order: torch.Tensor, M: Optional[torch.Tensor],
             prec: str, B0: torch.Tensor, Btau: Optional[torch.Tensor]) -> None:
    m, n_eff = E.shape
    p = 0 if M is None else M.shape[0]
    h.check(_lib.vl_fit_b(h.h, _ptr(E), E.stride(0), m, n_eff, _ptr(order), _ptr(M), p,
                          PRECISIONS[prec], _ptr(B0), _ptr(Btau)), "vl_fit_b")


def vl_fit(h: Handle, X: torch.Tensor, p: int, prec: str, M: torch.Tensor, order: torch.Tensor,
           B0: torch.Tensor, Btau: torch.Tensor, D: Optional[torch.Tensor] = None) -> None:
    """Whole method on one series, asynchronous on the handle's stream."""
    m, n = X.shape
    h.check(_lib.vl_fit(h.h, _ptr(X), X.stride(0), m, n, p, PRECISIONS[prec], _ptr(M),
                        _ptr(order), _ptr(B0), _ptr(Btau), _ptr(D)), "vl_fit")


def _instances(instances):
    arr = (vl_instance * len(instances))()
    for k, d in enumerate(instances):
        X = d["X"]
        arr[k] = vl_instance(X.data_ptr(), X.stride(0), X.shape[0], X.shape[1], int(d["p"]),
                             d["order"].data_ptr(), d["B0"].data_ptr(), d["Btau"].data_ptr(),
                             d["M"].data_ptr(), d["D"].data_ptr() if d.get("D") is not None else None)
    return arr


def vl_fit_batched(h: Handle, instances: Sequence[Dict[str, torch.Tensor]], prec: str):
    """instances: dicts with X (m x n float64 CUDA), p, and output tensors
    order, B0, Btau, M and optionally D.  Returns the per-instance status
    codes (0 = ok)."""
    arr = _instances(instances)
    status = (ctypes.c_int * len(instances))()
    code = _lib.vl_fit_batched(h.h, arr, len(instances), PRECISIONS[prec], status)
    out = [int(s) for s in status]
    if code != VL_OK and all(s == VL_OK for s in out):  # a failure of the call itself
        h.check(code, "vl_fit_batched")
    return out


def vl_fit_batched_async(h: Handle, instances: Sequence[Dict[str, torch.Tensor]], prec: str,
                         dev_status: torch.Tensor) -> None:
    """The batch enqueued without host synchronisation (mixed precisions);
    dev_status: int32 CUDA tensor of len(instances), filled on the device.
    The instance array is kept on the handle object until the next call, so
    a captured graph of this call stays valid."""
    arr = _instances(instances)
    h._batch_keepalive = arr
    h.check(_lib.vl_fit_batched_async(h.h, arr, len(instances), PRECISIONS[prec],
                                      _ptr(dev_status)), "vl_fit_batched_async")


# ------------------------------------------------------------ conveniences
def alloc_outputs(m: int, p: int, device=None) -> Dict[str, torch.Tensor]:
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    f64 = dict(dtype=torch.float64, device=dev)
    return {
        "M": torch.empty((p, m, m), **f64), "B0": torch.empty((m, m), **f64),
        "Btau": torch.empty((p, m, m), **f64), "D": torch.empty((m, m), **f64),
        "order": torch.empty((m,), dtype=torch.int32, device=dev),
    }


def fit(h: Handle, X: torch.Tensor, p: int, prec: str = "mixed", steps: bool = False):
    """Whole method on one series (device tensor X, m x n float64).  With
    steps=True the four calls run separately and E, Hx, Hr, D and the gaps
    are returned too; otherwise the single fused call vl_fit."""
    m, n = X.shape
    out = alloc_outputs(m, p, X.device.index)
    if not steps:
        vl_fit(h, X, p, prec, out["M"], out["order"], out["B0"], out["Btau"], out["D"])
        h.sync()
        return out
    f64 = dict(dtype=torch.float64, device=X.device)
    E = torch.empty((m, n - p), **f64)
    out.update(E=E, Hx=torch.empty((m,), **f64), Hr=torch.empty((m, m), **f64),
               gap=torch.empty((m,), **f64))
    vl_var_fit(h, X, p, prec, out["M"], E)
    vl_pairwise_measure(h, E, prec, out["Hx"], out["Hr"], out["D"])
    if prec == "mixed_certified":
        out["cert_stats"] = torch.zeros(4, dtype=torch.int32, device=X.device)
        vl_causal_order_certified(h, out["D"], E, out["order"], out["gap"], out["cert_stats"])
    else:
        vl_causal_order(h, out["D"], out["order"], out["gap"])
    vl_fit_b(h, E, out["order"], out["M"], prec, out["B0"], out["Btau"])
    h.sync()
    return out
