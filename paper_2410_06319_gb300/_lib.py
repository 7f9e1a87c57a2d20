"""ctypes marshalling for liblsq.so (see include/lsq.h for every contract)."""
import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
HEADER = os.path.join(ROOT, "include", "lsq.h")


def library_path():
    return os.path.join(HERE, "_lib", "liblsq.so")


if not os.path.exists(library_path()):
    raise ImportError(
        "liblsq.so is not built: run `python paper_2410_06319_gb300/build.py` "
        "(or __graft_entry__.build()); the solver has no non-CUDA fallback")

lib = ctypes.CDLL(library_path())

PREC = {"auto": -1, "f64": 0, "f32": 1, "f16": 2, "bf16": 3, "e4m3": 4, "bf16x3": 5, "f64x2": 6}
STATUS = {0: "LSQ_OK", 1: "LSQ_NOT_CONVERGED", -1: "LSQ_E_INVAL", -2: "LSQ_E_RANK",
          -3: "LSQ_E_BREAKDOWN", -4: "LSQ_E_NONFINITE", -5: "LSQ_E_CUDA", -6: "LSQ_E_TIMEOUT",
          -7: "LSQ_E_NOMEM", -8: "LSQ_E_UNSUPPORTED", -9: "LSQ_E_SIZE"}


#: kernels timed with opts.timing (order of lsq_info.kern_ms)
KERNELS = ["sketch_gemm", "lsqr_pass", "fgmres_pass", "residual_pass", "arnoldi_step", "fgmres_trsv",
           "sketch_fix", "spare7"]


class Opts(ctypes.Structure):
    _fields_ = [("lda", ctypes.c_int64), ("lsqr_maxit", ctypes.c_int32),
                ("ir_maxit", ctypes.c_int32), ("gmres_maxit", ctypes.c_int32),
                ("no_escalate", ctypes.c_int32), ("no_colscale", ctypes.c_int32),
                ("ir_stop", ctypes.c_int32), ("timing", ctypes.c_int32),
                ("no_graph", ctypes.c_int32), ("sketch_exact", ctypes.c_int32),
                ("gmres_tol", ctypes.c_double), ("kappa_hint", ctypes.c_double),
                ("Y_in", ctypes.c_void_p), ("R_in", ctypes.c_void_p), ("x0_in", ctypes.c_void_p),
                ("sketch_kchunk", ctypes.c_int64), ("wait_limit_us", ctypes.c_int32),
                ("expire_sync", ctypes.c_int32), ("sketch_kind", ctypes.c_int32),
                ("sparse_zeta", ctypes.c_int32), ("ops_escalated", ctypes.c_int32),
                ("aug_alpha", ctypes.c_double), ("h_in_ur", ctypes.c_int32),
                ("batch_mode", ctypes.c_int32), ("batch_grid", ctypes.c_int32),
                ("arnoldi", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("lsqr_its", ctypes.c_int32), ("lsqr_flag", ctypes.c_int32),
                ("ir_its", ctypes.c_int32), ("gmres_its_total", ctypes.c_int32),
                ("escalated", ctypes.c_int32), ("ir_converged", ctypes.c_int32),
                ("gmres_its", ctypes.c_int32 * 32),
                ("lsqr_normr", ctypes.c_double), ("lsqr_normar", ctypes.c_double),
                ("lsqr_normA", ctypes.c_double), ("kappa_R_est", ctypes.c_double),
                ("ir_dx_rel", ctypes.c_double), ("ir_dr_rel", ctypes.c_double),
                ("stage_ms", ctypes.c_double * 8), ("gpu_launches", ctypes.c_int64),
                ("ir_dx_hist", ctypes.c_double * 32), ("ir_dr_hist", ctypes.c_double * 32),
                ("gmres_relres", ctypes.c_double * 32),
                ("kern_ms", ctypes.c_double * 8), ("kern_launches", ctypes.c_int64 * 8),
                ("arnoldi_second_passes", ctypes.c_int64), ("us_used", ctypes.c_int32),
                ("sketches", ctypes.c_int32), ("aug_alpha", ctypes.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["gmres_its"] = list(self.gmres_its)[: max(0, self.ir_its)]
        for k in ("ir_dx_hist", "ir_dr_hist", "gmres_relres"):
            d[k] = list(getattr(self, k))[: max(0, self.ir_its)]
        d["stage_ms"] = dict(zip(["cast", "sketch", "qr", "lsqr", "residual", "fgmres", "update",
                                  "total"], list(self.stage_ms)))
        d["kern_ms"] = dict(zip(KERNELS, list(self.kern_ms)))
        d["kern_launches"] = dict(zip(KERNELS, list(self.kern_launches)))
        return d


class Problem(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("b", ctypes.c_void_p), ("m", ctypes.c_int64),
                ("n", ctypes.c_int64), ("s", ctypes.c_int64), ("lda", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("x", ctypes.c_void_p), ("r", ctypes.c_void_p)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_TUPLE = [_P, _P, _P, _I64, _I64, _I64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
          ctypes.c_double, ctypes.c_uint64, ctypes.POINTER(Opts)]
lib.lsq_create.argtypes = [ctypes.POINTER(_P), _P]
lib.lsq_destroy.argtypes = [_P]
lib.lsq_status_string.argtypes = [ctypes.c_int]
lib.lsq_status_string.restype = ctypes.c_char_p
lib.lsq_last_cuda_error.argtypes = [_P]
lib.lsq_last_cuda_error.restype = ctypes.c_char_p
lib.lsq_opts_default.argtypes = [ctypes.POINTER(Opts)]
lib.lsq_sizeof.argtypes = [ctypes.c_int]
lib.lsq_sizeof.restype = ctypes.c_size_t
lib.lsq_sketch.argtypes = _TUPLE + [_P]
lib.lsq_qr_r.argtypes = _TUPLE + [_P, _P]
lib.lsq_lsqr.argtypes = _TUPLE + [_P, ctypes.POINTER(Info)]
lib.lsq_lsir.argtypes = _TUPLE + [_P, _P, ctypes.POINTER(Info)]
lib.lsq_lsir_host.argtypes = _TUPLE + [_P, _P, ctypes.POINTER(Info)]
lib.lsq_ir_step.argtypes = _TUPLE + [_P, _P, _P, ctypes.POINTER(Info)]
lib.lsq_omega.argtypes = [_P, _I64, _I64, _I64, ctypes.c_int, ctypes.c_uint64, _P]
lib.lsq_lsir_batched.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(Problem), ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.POINTER(Opts),
                                 ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(Info)]
lib.lsq_qr_r_noalloc.argtypes = [_P, _I64, _I64, ctypes.c_int, _P, _P, _P]
lib.lsq_probe_fma_rate.argtypes = [ctypes.c_int, _P, ctypes.POINTER(ctypes.c_double)]
lib.lsq_residual.argtypes = [_P, _P, _P, _I64, _I64, ctypes.c_int, ctypes.POINTER(Opts), _P, _P, _P, _P]
for _f in ("lsq_create", "lsq_destroy", "lsq_sketch", "lsq_qr_r", "lsq_lsqr", "lsq_lsir", "lsq_lsir_host", "lsq_ir_step",
           "lsq_omega", "lsq_lsir_batched", "lsq_qr_r_noalloc", "lsq_probe_fma_rate", "lsq_residual"):
    getattr(lib, _f).restype = ctypes.c_int


def declared_functions():
    """Names of the functions declared in include/lsq.h."""
    with open(HEADER) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lsq_[a-z_0-9]+)\s*\(", text)))


class LsqError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} {detail}".strip())


def _ptr(x):
    """Device pointer of a torch tensor (checked: CUDA, contiguous) or a raw int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not x.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return x.data_ptr()


def _prec(p):
    return PREC[p] if isinstance(p, str) else int(p)


class Handle:
    """Owns an lsq_handle bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, stream=None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self._h = _P()
        st = lib.lsq_create(ctypes.byref(self._h), _P(stream))
        if st != 0:
            raise LsqError(st, "lsq_create")

    @property
    def ptr(self):
        return self._h

    def last_cuda_error(self):
        return lib.lsq_last_cuda_error(self._h).decode()

    def close(self):
        if self._h:
            lib.lsq_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _opts(opts):
    if opts is None:
        return Opts()
    if isinstance(opts, Opts):
        return opts
    o = Opts()
    for k, v in opts.items():
        if k in ("Y_in", "R_in", "x0_in"):
            v = _ptr(v)
        setattr(o, k, v)
    return o


def _check(h, st, where, allow=(0, 1)):
    if st not in allow:
        raise LsqError(st, where, h.last_cuda_error() if st == -5 else "")
    return st


def _tuple(h, A, b, m, n, s, u_s, u_p, u_w, u_r, tol, seed, opts):
    o = _opts(opts)
    return [h.ptr, _ptr(A), _ptr(b), m, n, s, _prec(u_s), _prec(u_p), _prec(u_w), _prec(u_r),
            float(tol), int(seed), ctypes.byref(o)], o


def lsq_sketch(h, A, b, m, n, s, u_s, u_p, u_w, u_r, tol, seed, opts, Y):
    args, _o = _tuple(h, A, b, m, n, s, u_s, u_p, u_w, u_r, tol, seed, opts)
    return _check(h, lib.lsq_sketch(*args, _ptr(Y)), "lsq_sketch")


def lsq_qr_r(h, A, b, m, n, s, u_s, u_p, u_w, u_r, tol, seed, opts, R, xs):
    args, _o = _tuple(h, A, b, m, n, s, u_s, u_p, u_w, u_r, tol, seed, opts)
    return _check(h, lib.lsq_qr_r(*args, _ptr(R), _ptr(xs)), "lsq_qr_r")


def lsq_lsqr(h, A, b, m, n, s, u_s, u_p, u_w, u_r, tol, seed, opts, x, info=None):
    args, _o = _tuple(h, A, b, m, n, s, u_s, u_p, u_w, u_r, tol, seed, opts)
    info = info if info is not None else Info()
    st = _check(h, lib.lsq_lsqr(*args, _ptr(x), ctypes.byref(info)), "lsq_lsqr")
    return st, info


def lsq_lsir(h, A, b, m, n, s, u_s, u_p, u_w, u_r, tol, seed, opts, x, r, info=None):
    args, _o = _tuple(h, A, b, m, n, s, u_s, u_p, u_w, u_r, tol, seed, opts)
    info = info if info is not None else Info()
    st = _check(h, lib.lsq_lsir(*args, _ptr(x), _ptr(r), ctypes.byref(info)), "lsq_lsir")
    return st, info


def lsq_ir_step(h, A, b, m, n, s, u_s, u_p, u_w, u_r, tol, seed, opts, R, x, r, info=None):
    """One refinement step of Algorithm 2 from (x, r), both overwritten (device tensors)."""
    args, _o = _tuple(h, A, b, m, n, s, u_s, u_p, u_w, u_r, tol, seed, opts)
    info = info if info is not None else Info()
    st = _check(h, lib.lsq_ir_step(*args, _ptr(R), _ptr(x), _ptr(r), ctypes.byref(info)), "lsq_ir_step")
    return st, info


def lsq_residual(h, A, b, m, n, u_r, opts, x, r, f, g):
    """[f; g] = [b - r - A x; -A^T r] in u_r (Alg. 2 refinement residual), device tensors."""
    o = _opts(opts)
    return _check(h, lib.lsq_residual(h.ptr, _ptr(A), _ptr(b), m, n, _prec(u_r), ctypes.byref(o), _ptr(x),
                                      _ptr(r), _ptr(f), _ptr(g)), "lsq_residual")


def _host_ptr(x):
    """Host pointer of a contiguous FP64 numpy array or CPU torch tensor (or a raw int)."""
    if x is None or isinstance(x, int):
        return x
    if hasattr(x, "is_cuda"):
        if x.is_cuda or not x.is_contiguous() or x.element_size() != 8:
            raise ValueError("expected a contiguous FP64 CPU tensor")
        return x.data_ptr()
    if x.dtype.itemsize != 8 or not x.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a contiguous FP64 array")
    return x.ctypes.data


def lsq_lsir_host(h, A, b, m, n, s, u_s, u_p, u_w, u_r, tol, seed, opts, x, r, info=None):
    """lsq_lsir on host arrays (numpy or CPU tensors; page-locked tensors copy fastest)."""
    o = _opts(opts)
    info = info if info is not None else Info()
    st = lib.lsq_lsir_host(h.ptr, _host_ptr(A), _host_ptr(b), m, n, s, _prec(u_s), _prec(u_p), _prec(u_w),
                           _prec(u_r), float(tol), int(seed), ctypes.byref(o), _host_ptr(x), _host_ptr(r),
                           ctypes.byref(info))
    return _check(h, st, "lsq_lsir_host"), info


def lsq_lsir_batched(h, problems, u_s, u_p, u_w, u_r, tol, opts=None):
    """problems: list of dicts with A, b, m, n, s, seed, x, r (tensors or pointers), optional lda.

    Returns (aggregate status, per-problem statuses, per-problem Info)."""
    k = len(problems)
    arr = (Problem * max(1, k))()
    for i, pr in enumerate(problems):
        arr[i] = Problem(_ptr(pr["A"]), _ptr(pr["b"]), pr["m"], pr["n"], pr["s"], pr.get("lda", 0),
                         int(pr.get("seed", 0)), _ptr(pr["x"]), _ptr(pr.get("r")))
    sts = (ctypes.c_int32 * max(1, k))()
    infos = (Info * max(1, k))()
    o = _opts(opts)
    st = lib.lsq_lsir_batched(h.ptr, k, arr, _prec(u_s), _prec(u_p), _prec(u_w), _prec(u_r),
                              float(tol), ctypes.byref(o), sts, infos)
    _check(h, st, "lsq_lsir_batched")
    return st, list(sts)[:k], list(infos)[:k]


def lsq_omega(h, s, j0, cols, u_s, seed, out):
    return _check(h, lib.lsq_omega(h.ptr, s, j0, cols, _prec(u_s), int(seed), _ptr(out)),
                  "lsq_omega", allow=(0,))


def lsq_qr_r_noalloc(Y, s, n, u_p, R, c=None, stream=None):
    """QR of a sketch in the library's fixed device scratch (no allocation, no handle).

    Returns the status; raises LsqError on errors other than LSQ_E_SIZE, which is
    returned so callers can fall back to lsq_qr_r.
    """
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    st = lib.lsq_qr_r_noalloc(_ptr(Y), s, n, _prec(u_p), _ptr(R), _ptr(c), _P(stream))
    if st not in (0, -9):
        raise LsqError(st, "lsq_qr_r_noalloc")
    return st


def lsq_probe_fma_rate(which="f64", stream=None):
    """FMAs per second of the current device (which = "f64" or "f32")."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    out = ctypes.c_double(0.0)
    st = lib.lsq_probe_fma_rate({"f64": 0, "f32": 1}[which], _P(stream), ctypes.byref(out))
    if st != 0:
        raise LsqError(st, "lsq_probe_fma_rate")
    return out.value
