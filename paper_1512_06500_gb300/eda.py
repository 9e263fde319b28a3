"""Python binding of the C ABI in include/eda.h (argument marshalling only).

Every step of the method runs in the CUDA library ``_lib/libeda_gb300.so``; this module only
passes device pointers, sizes and the current CUDA stream. PyTorch supplies device memory
and streams. There is no CPU fallback: if the library is missing or no GPU is present the
calls raise.

Layouts: a d x n column-major sample block is a C-contiguous tensor of shape (n, d) (one
sample per row of the tensor), so ``X.data_ptr()`` with leading dimension d is exactly the
paper's X = [chi_1 .. chi_n].
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libeda_gb300.so")

EDA_F64, EDA_F32, EDA_BF16, EDA_BF16X2, EDA_F64_TC = 0, 1, 2, 3, 4
OP_SW, OP_SB, OP_M, OP_N = 0, 1, 2, 3

STATUS = {
    0: "EDA_OK", -1: "EDA_ERR_INVALID_ARG", -2: "EDA_ERR_BAD_LABELS", -3: "EDA_ERR_NONFINITE",
    -4: "EDA_ERR_OOM", -5: "EDA_ERR_CUDA", -6: "EDA_ERR_TIMEOUT", -7: "EDA_ERR_BREAKDOWN",
    -8: "EDA_ERR_NOT_CONVERGED",
}

# every symbol include/eda.h declares
EXPORTS = [
    "eda_config_default", "eda_build", "eda_build_from_factors", "eda_apply_exp", "eda_solve",
    "eda_project", "eda_get_factors", "eda_get_dims", "eda_destroy", "eda_strerror",
    "eda_last_cuda_error", "eda_last_cuda_error_string", "eda_kernel_launches",
    "eda_profile_enable", "eda_profile_reset", "eda_profile_read", "eda_profile_work",
    "eda_lowrank_exp_apply_noalloc", "eda_solve_batched", "eda_solve_arnoldi", "eda_solve_direct",
]


class EdaError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = f"{where}: {STATUS.get(code, code)}"
        if code == -5 and _lib is not None:
            msg += f" ({_lib.eda_last_cuda_error_string().decode()})"
        super().__init__(msg)


class Config(ctypes.Structure):
    _fields_ = [
        ("prec", ctypes.c_int32), ("block_b", ctypes.c_int32), ("m_max", ctypes.c_int32),
        ("check_every", ctypes.c_int32), ("tau", ctypes.c_double), ("c2", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("true_residuals", ctypes.c_int32), ("m_form", ctypes.c_int32),
        ("wait_limit", ctypes.c_int32), ("tc_min_mi", ctypes.c_int32), ("tc_fused", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 3),
    ]


class SolveInfo(ctypes.Structure):
    _fields_ = [
        ("converged", ctypes.c_int32), ("iters", ctypes.c_int32), ("mapplies", ctypes.c_int32),
        ("basis_cols", ctypes.c_int32), ("refills", ctypes.c_int32), ("checks", ctypes.c_int32),
        ("refine_iters", ctypes.c_int32), ("reserved0", ctypes.c_int32), ("c2", ctypes.c_double), ("lmax_w", ctypes.c_double), ("lmax_b", ctypes.c_double),
        ("max_relres_est", ctypes.c_double), ("max_relres_true", ctypes.c_double),
        ("ms_solve", ctypes.c_double), ("relres", ctypes.POINTER(ctypes.c_double)),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "relres"}


class Problem(ctypes.Structure):
    _fields_ = [
        ("X", ctypes.c_void_p), ("x_dtype", ctypes.c_int32), ("k", ctypes.c_int32),
        ("d", ctypes.c_int64), ("n", ctypes.c_int64), ("ldx", ctypes.c_int64),
        ("labels", ctypes.c_void_p), ("t", ctypes.c_int32), ("block_b", ctypes.c_int32),
        ("tol", ctypes.c_double), ("V", ctypes.c_void_p), ("lam", ctypes.c_void_p),
        ("status", ctypes.c_int32), ("reserved", ctypes.c_int32), ("info", SolveInfo),
    ]


_lib = None


def load(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "eda_config_default": ([P(Config)], ctypes.c_int),
        "eda_build": ([vp, i32, i64, i64, i64, vp, i32, P(Config), vp, P(vp)], ctypes.c_int),
        "eda_build_from_factors": ([vp, i64, vp, i64, i64, P(Config), vp, P(vp)], ctypes.c_int),
        "eda_apply_exp": ([vp, i32, f64, vp, vp, i64, i32, i32, vp], ctypes.c_int),
        "eda_solve": ([vp, i32, f64, vp, i32, vp, vp, vp, P(SolveInfo), vp], ctypes.c_int),
        "eda_project": ([vp, vp, i32, vp, i32, i64, i64, vp, vp], ctypes.c_int),
        "eda_get_factors": ([vp] + [vp] * 10 + [vp], ctypes.c_int),
        "eda_get_dims": ([vp, P(i64), P(i64), P(i32), P(f64), P(f64), P(f64)], ctypes.c_int),
        "eda_destroy": ([vp], None),
        "eda_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "eda_last_cuda_error": ([], ctypes.c_int),
        "eda_last_cuda_error_string": ([], ctypes.c_char_p),
        "eda_kernel_launches": ([], ctypes.c_uint64),
        "eda_profile_enable": ([ctypes.c_int], ctypes.c_int),
        "eda_profile_reset": ([], ctypes.c_int),
        "eda_profile_read": ([ctypes.c_char_p, P(f64), P(i64)], ctypes.c_int),
        "eda_profile_work": ([ctypes.c_char_p, P(f64), P(f64)], ctypes.c_int),
        "eda_lowrank_exp_apply_noalloc": ([vp, i64, i32, vp, vp, vp, i64, i32, vp], ctypes.c_int),
        "eda_solve_batched": ([P(Problem), i32, P(Config), i32, vp], ctypes.c_int),
        "eda_solve_arnoldi": ([vp, i32, f64, vp, vp, P(SolveInfo), vp], ctypes.c_int),
        "eda_solve_direct": ([vp, i32, vp, vp, P(SolveInfo), vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(code, where):
    if code != 0:
        raise EdaError(code, where)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _need_cuda(t, name, dtype=None):
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}")


def _dtype_code(t):
    if t.dtype == torch.float64:
        return EDA_F64
    if t.dtype == torch.float32:
        return EDA_F32
    raise ValueError("sample blocks must be float64 or float32")


def config(**kw) -> Config:
    """eda_config with the library defaults, then the given fields overridden."""
    c = Config()
    _check(load().eda_config_default(ctypes.byref(c)), "eda_config_default")
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def kernel_launches() -> int:
    return int(load().eda_kernel_launches())


def profile_enable(on=True):
    _check(load().eda_profile_enable(1 if on else 0), "eda_profile_enable")


def profile_reset():
    _check(load().eda_profile_reset(), "eda_profile_reset")


def profile_read(region: str):
    """(total device ms, calls) of a library region since the last reset."""
    ms, calls = ctypes.c_double(), ctypes.c_int64()
    _check(load().eda_profile_read(region.encode(), ctypes.byref(ms), ctypes.byref(calls)), "eda_profile_read")
    return ms.value, calls.value


def solve_batched(problems, cfg=None, workers=0, stream=None):
    """Solve independent problems side by side (eda_solve_batched).

    problems: sequence of dicts with X ((n, d) CUDA tensor, float64 or float32), labels ((n,) int32
    CUDA tensor), k, t, tol and optionally block_b. Returns (results, code): one dict per problem
    with V ((t, d) float64), lam ((t,) float64), status and info, and the batch status.
    """
    arr = (Problem * len(problems))()
    keep = []
    for i, pr in enumerate(problems):
        X, lab = pr["X"], pr["labels"]
        _need_cuda(X, "X")
        _need_cuda(lab, "labels", torch.int32)
        n, d = X.shape
        t = int(pr["t"])
        V = torch.empty((t, d), dtype=torch.float64, device=X.device)
        lam = torch.empty(t, dtype=torch.float64, device=X.device)
        keep.append((V, lam))
        arr[i] = Problem(X=X.data_ptr(), x_dtype=_dtype_code(X), k=int(pr["k"]), d=d, n=n, ldx=d,
                         labels=lab.data_ptr(), t=t, block_b=int(pr.get("block_b", 0)), tol=float(pr["tol"]),
                         V=V.data_ptr(), lam=lam.data_ptr(), status=0)
    c = cfg if cfg is not None else config(block_b=0)
    code = load().eda_solve_batched(arr, len(problems), ctypes.byref(c), int(workers), _stream(stream))
    if code not in (0, -8):
        raise EdaError(code, "eda_solve_batched")
    out = []
    for i, (V, lam) in enumerate(keep):
        out.append(dict(V=V, lam=lam, status=arr[i].status, info=arr[i].info.as_dict()))
    return out, code


def profile_work(region: str):
    """(algorithmic FLOPs, algorithmic bytes) the library counted for a region since the last reset."""
    fl, by = ctypes.c_double(), ctypes.c_double()
    _check(load().eda_profile_work(region.encode(), ctypes.byref(fl), ctypes.byref(by)), "eda_profile_work")
    return fl.value, by.value


class Handle:
    """A built EDA problem (owns the library handle)."""

    def __init__(self, ptr, device):
        self._h = ptr
        self.device = device
        d, n, k = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        c2, lw, lb = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(load().eda_get_dims(self._h, ctypes.byref(d), ctypes.byref(n), ctypes.byref(k), ctypes.byref(c2),
                                   ctypes.byref(lw), ctypes.byref(lb)), "eda_get_dims")
        self.d, self.n, self.k = d.value, n.value, k.value
        self.c2, self.lmax_w, self.lmax_b = c2.value, lw.value, lb.value

    def close(self):
        if self._h:
            load().eda_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def apply_exp(self, op, X, alpha=0.0, out=None, stream=None):
        """Y = exp(alpha H H^T) X (op SW/SB) or Y = M X (op M); X: (b, d) CUDA tensor.

        float64 X uses the FP64 factors; float32 X uses the handle's working precision
        (single-precision sweeps, or bf16 H on the tensor cores).
        """
        _need_cuda(X, "X")
        b, d = X.shape
        if d != self.d:
            raise ValueError("X has the wrong dimension")
        Y = out if out is not None else torch.empty_like(X)
        _check(load().eda_apply_exp(self._h, op, float(alpha), _ptr(X), _ptr(Y), d, b, _dtype_code(X),
                                    _stream(stream)), "eda_apply_exp")
        return Y

    def solve(self, t, tol, V0=None, want_y=False, relres=False, stream=None, check=True):
        """t dominant pairs: returns (V (t, d), lam (t,), Y or None, info dict, status)."""
        dev = self.device
        V = torch.empty((t, self.d), dtype=torch.float64, device=dev)
        lam = torch.empty(t, dtype=torch.float64, device=dev)
        Y = torch.empty((t, self.d), dtype=torch.float64, device=dev) if want_y else None
        info = SolveInfo()
        rr = (ctypes.c_double * t)() if relres else None
        if rr is not None:
            info.relres = ctypes.cast(rr, ctypes.POINTER(ctypes.c_double))
        b0 = 0
        if V0 is not None:
            _need_cuda(V0, "V0", torch.float64)
            b0 = V0.shape[0]
        code = load().eda_solve(self._h, t, float(tol), _ptr(V0), b0, _ptr(V), _ptr(lam), _ptr(Y), ctypes.byref(info),
                                _stream(stream))
        if check and code not in (0, -8):
            raise EdaError(code, "eda_solve")
        out = info.as_dict()
        if rr is not None:
            out["relres"] = list(rr)
        return V, lam, Y, out, code

    def solve_arnoldi(self, t, tol, relres=False, stream=None, check=True):
        """t dominant pairs of the nonsymmetric form (block Arnoldi): returns (V (t, d), lam (t,), info, status)."""
        dev = self.device
        V = torch.empty((t, self.d), dtype=torch.float64, device=dev)
        lam = torch.empty(t, dtype=torch.float64, device=dev)
        info = SolveInfo()
        rr = (ctypes.c_double * t)() if relres else None
        if rr is not None:
            info.relres = ctypes.cast(rr, ctypes.POINTER(ctypes.c_double))
        code = load().eda_solve_arnoldi(self._h, t, float(tol), _ptr(V), _ptr(lam), ctypes.byref(info),
                                        _stream(stream))
        if check and code not in (0, -8):
            raise EdaError(code, "eda_solve_arnoldi")
        out = info.as_dict()
        if rr is not None:
            out["relres"] = list(rr)
        return V, lam, out, code

    def solve_direct(self, t, stream=None, check=True):
        """t dominant pairs solved exactly in span([H_W H_B]): returns (V (t, d), lam (t,), info, status)."""
        dev = self.device
        V = torch.empty((t, self.d), dtype=torch.float64, device=dev)
        lam = torch.empty(t, dtype=torch.float64, device=dev)
        info = SolveInfo()
        code = load().eda_solve_direct(self._h, t, _ptr(V), _ptr(lam), ctypes.byref(info), _stream(stream))
        if check and code != 0:
            raise EdaError(code, "eda_solve_direct")
        return V, lam, info.as_dict(), code

    def project(self, V, Xq, stream=None):
        """P = V^T Xq; V: (t, d) float64, Xq: (m, d) float64 -> P (m, t)."""
        _need_cuda(V, "V", torch.float64)
        _need_cuda(Xq, "Xq", torch.float64)
        t = V.shape[0]
        m = Xq.shape[0]
        P = torch.empty((m, t), dtype=torch.float64, device=V.device)
        _check(load().eda_project(self._h, _ptr(V), t, _ptr(Xq), EDA_F64, m, self.d, _ptr(P), _stream(stream)),
               "eda_project")
        return P

    def factors(self, stream=None):
        """Device copies of the build results (H_W, H_B as (cols, d) tensors, Grams, K, eigenvalues)."""
        dev = self.device
        f64 = dict(dtype=torch.float64, device=dev)
        n, k, d = self.n, self.k, self.d
        out = dict(
            HW=torch.empty((n, d), **f64), HB=torch.empty((k, d), **f64),
            counts=torch.empty(k, dtype=torch.int32, device=dev), perm=torch.empty(n, dtype=torch.int32, device=dev),
            GW=torch.empty((n, n), **f64), GB=torch.empty((k, k), **f64), KW=torch.empty((n, n), **f64),
            KB=torch.empty((k, k), **f64), evals_w=torch.empty(n, **f64), evals_b=torch.empty(k, **f64),
        )
        has_labels = True
        code = load().eda_get_factors(self._h, *[_ptr(out[x]) for x in
                                                 ("HW", "HB", "counts", "perm", "GW", "GB", "KW", "KB", "evals_w",
                                                  "evals_b")], _stream(stream))
        if code == -1:   # built from factors: no labels
            has_labels = False
            code = load().eda_get_factors(self._h, _ptr(out["HW"]), _ptr(out["HB"]), None, None, _ptr(out["GW"]),
                                          _ptr(out["GB"]), _ptr(out["KW"]), _ptr(out["KB"]), _ptr(out["evals_w"]),
                                          _ptr(out["evals_b"]), _stream(stream))
            out.pop("counts")
            out.pop("perm")
        _check(code, "eda_get_factors")
        out["has_labels"] = has_labels
        return out


def build(X, labels, k, cfg: Config | None = None, stream=None) -> Handle:
    """eda_build on samples X ((n, d) float64/float32 CUDA tensor) and int32 labels."""
    _need_cuda(X, "X")
    _need_cuda(labels, "labels", torch.int32)
    n, d = X.shape
    h = ctypes.c_void_p()
    c = cfg if cfg is not None else config()
    _check(load().eda_build(_ptr(X), _dtype_code(X), d, n, d, _ptr(labels), int(k), ctypes.byref(c), _stream(stream),
                            ctypes.byref(h)), "eda_build")
    return Handle(h, X.device)


def build_from_factors(HW, HB, cfg: Config | None = None, stream=None) -> Handle:
    """eda_build_from_factors; HW: (n, d), HB: (kb, d) float64 CUDA tensors (column-major d x n, d x kb)."""
    _need_cuda(HW, "HW", torch.float64)
    _need_cuda(HB, "HB", torch.float64)
    n, d = HW.shape
    kb = HB.shape[0]
    h = ctypes.c_void_p()
    c = cfg if cfg is not None else config()
    _check(load().eda_build_from_factors(_ptr(HW), n, _ptr(HB), kb, d, ctypes.byref(c), _stream(stream),
                                         ctypes.byref(h)), "eda_build_from_factors")
    return Handle(h, HW.device)


def lowrank_exp_apply_noalloc(H, K, X, out=None, stream=None):
    """Y = X + H K (H^T X) without any device allocation (fixed library scratch).

    H: (m, d) float64 CUDA tensor (column-major d x m), K: (m, m), X: (b, d). The library
    rejects m * b above 174762 with EDA_ERR_INVALID_ARG.
    """
    for t, nm in ((H, "H"), (K, "K"), (X, "X")):
        _need_cuda(t, nm, torch.float64)
    m, d = H.shape
    b = X.shape[0]
    Y = out if out is not None else torch.empty_like(X)
    _check(load().eda_lowrank_exp_apply_noalloc(_ptr(H), d, m, _ptr(K), _ptr(X), _ptr(Y), d, b, _stream(stream)),
           "eda_lowrank_exp_apply_noalloc")
    return Y
