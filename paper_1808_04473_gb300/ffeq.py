"""Thin ctypes binding over the C ABI of ``libffeq.so`` (``include/ffeq.h``).

Every function here marshals arguments and calls the library entry point of the
same name; all arithmetic runs in the CUDA kernels.  There is no fallback: if
the library has not been built, or a call fails, an exception is raised.

Tensors are ``torch`` tensors (device memory and streams come from PyTorch);
complex arrays are ``torch.complex64``.  ``equalize`` is a convenience wrapper
that allocates the outputs and calls ``ffeq_plan_create`` + ``ffeq_equalize``.
"""
from __future__ import annotations

import ctypes
import os
import re

PD, FD = 0, 1
FP32, TF32X3, BF16X3, FP16X3 = 0, 1, 2, 3
UNBIASED, LITERAL = 0, 1
LMMSE, ZF, MRC, LAMA = 0, 1, 2, 3

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libffeq.so")
INCLUDE_DIR = os.path.join(os.path.dirname(_HERE), "include")
HEADER_PATH = os.path.join(INCLUDE_DIR, "ffeq.h")
HEADER_PATHS = [HEADER_PATH, os.path.join(INCLUDE_DIR, "ffeq_batch.h")]

_STATUS = {0: "FFEQ_OK", 1: "FFEQ_ERR_INVALID_ARG", 2: "FFEQ_ERR_UNSUPPORTED", 3: "FFEQ_ERR_CUDA",
           4: "FFEQ_ERR_TIMEOUT"}


class FfeqError(RuntimeError):
    """A non-OK status returned by the library."""

    def __init__(self, func: str, status: int, detail: str = ""):
        self.status = status
        super().__init__(f"{func} -> {_STATUS.get(status, status)}{': ' + detail if detail else ''}")


class ffeq_problem(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int), ("U", ctypes.c_int), ("C", ctypes.c_int), ("n_sc", ctypes.c_int),
                ("n_sym", ctypes.c_int), ("arch", ctypes.c_int), ("precision", ctypes.c_int),
                ("estimate", ctypes.c_int), ("llr_bits", ctypes.c_int), ("refine", ctypes.c_int),
                ("refine_fp64", ctypes.c_int), ("equalizer", ctypes.c_int), ("lama_iters", ctypes.c_int)]


class ffeq_instance(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int), ("U", ctypes.c_int), ("C", ctypes.c_int), ("n_sc", ctypes.c_int),
                ("n_sym", ctypes.c_int), ("N0", ctypes.c_float), ("Es", ctypes.c_float),
                ("h_off", ctypes.c_longlong), ("y_off", ctypes.c_longlong), ("z_off", ctypes.c_longlong),
                ("sigma2_off", ctypes.c_longlong), ("llr_off", ctypes.c_longlong), ("info_off", ctypes.c_longlong)]


class ffeq_batch_config(ctypes.Structure):
    _fields_ = [("arch", ctypes.c_int), ("precision", ctypes.c_int), ("estimate", ctypes.c_int),
                ("llr_bits", ctypes.c_int), ("h_elems", ctypes.c_longlong), ("y_elems", ctypes.c_longlong),
                ("z_elems", ctypes.c_longlong), ("sigma2_elems", ctypes.c_longlong),
                ("llr_elems", ctypes.c_longlong), ("info_elems", ctypes.c_longlong), ("equalizer", ctypes.c_int),
                ("lama_iters", ctypes.c_int)]


_lib = None
_vp, _sz, _f, _i = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_float, ctypes.c_int
_SIGS = {
    "ffeq_version": ([], _i),
    "ffeq_status_string": ([_i], ctypes.c_char_p),
    "ffeq_last_cuda_error": ([], ctypes.c_char_p),
    "ffeq_plan_create": ([ctypes.POINTER(_vp), ctypes.POINTER(ffeq_problem)], _i),
    "ffeq_plan_create_clusters": ([ctypes.POINTER(_vp), ctypes.POINTER(ffeq_problem), ctypes.POINTER(_i)], _i),
    "ffeq_plan_destroy": ([_vp], None),
    "ffeq_workspace_size": ([_vp, ctypes.POINTER(_sz)], _i),
    "ffeq_equalize": ([_vp, _vp, _vp, _f, _f, _vp, _vp, _vp, _vp, _vp, _sz, _vp], _i),
    "ffeq_local_preprocess": ([_vp, _vp, _vp, _vp, _sz, _vp], _i),
    "ffeq_fuse_equalize": ([_vp, _vp, _sz, _f, _f, _vp, _vp, _vp, _vp, _vp], _i),
    "ffeq_host_staging_size": ([_vp, ctypes.POINTER(_sz)], _i),
    "ffeq_equalize_host": ([_vp, _vp, _vp, _f, _f, _vp, _vp, _vp, _vp, _vp, _sz, _vp], _i),
    "ffeq_fd_train_workspace_size": ([_vp, ctypes.POINTER(_sz)], _i),
    "ffeq_fd_train_forward": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp], _i),
    "ffeq_fd_train_backward": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp], _i),
    "ffeq_fd_optimal_workspace_size": ([_vp, ctypes.POINTER(_sz)], _i),
    "ffeq_fd_optimal_backward": ([_vp, _vp, _vp, _f, _f, _vp, _vp, _vp, _vp, _sz, _vp], _i),
    "ffeq_equalize_noalloc": ([_vp, _vp, _vp, _f, _f, _vp, _vp, _vp, _vp, _vp], _i),
    "ffeq_device_status": ([ctypes.POINTER(_i), _i], _i),
    "ffeq_plan_set_tuning": ([_vp, ctypes.POINTER(_i), _i], _i),
    "ffeq_plan_get_tuning": ([_vp, ctypes.POINTER(_i), _i], _i),
    "ffeq_plan_autotune": ([_vp, _vp, _vp, _f, _f, _vp, _vp, _vp, _vp, _vp, _sz, _vp, _i], _i),
    "ffeq_plan_autotune_sets": ([_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i, _f, _f, _vp, _vp, _vp, _vp, _vp,
                                 _sz, _vp, _i], _i),
    "ffeq_batch_create": ([ctypes.POINTER(_vp), ctypes.POINTER(ffeq_batch_config), ctypes.POINTER(ffeq_instance),
                           _i], _i),
    "ffeq_batch_destroy": ([_vp], None),
    "ffeq_batch_workspace_size": ([_vp, ctypes.POINTER(_sz)], _i),
    "ffeq_batch_upload": ([_vp, _vp, _sz, _vp], _i),
    "ffeq_batch_equalize": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp], _i),
    "ffeq_batch_autotune": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp, _i], _i),
    "ffeq_batch_groups": ([_vp], _i),
    "ffeq_batch_get_tuning": ([_vp, ctypes.POINTER(_i), _i], _i),
    "ffeq_batch_set_tuning": ([_vp, ctypes.POINTER(_i), _i], _i),
}


def lib():
    """Load ``libffeq.so`` once (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def header_symbols() -> list[str]:
    """Names of the functions declared in ``include/ffeq.h`` and ``include/ffeq_batch.h``."""
    text = "".join(open(h).read() for h in HEADER_PATHS)
    return sorted(set(re.findall(r"\b(ffeq_[a-z_]+)\s*\(", text)))


def _check(func: str, status: int):
    if status != 0:
        detail = lib().ffeq_last_cuda_error().decode() if status == 3 else ""
        raise FfeqError(func, status, detail)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensors passed to libffeq must be contiguous")
        return t.data_ptr()
    if hasattr(t, "ctypes"):                       # numpy array (host buffers)
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to libffeq must be C-contiguous")
        return t.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(t)!r}")


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class Plan:
    """Owner of an ``ffeq_plan*`` (destroyed with the object)."""

    def __init__(self, handle: int, problem: ffeq_problem):
        self.handle = handle
        self.problem = problem

    def __del__(self):
        if self.handle and _lib is not None:
            _lib.ffeq_plan_destroy(self.handle)
            self.handle = None


def ffeq_version() -> int:
    return lib().ffeq_version()


def ffeq_plan_create(B: int, U: int, C: int, n_sc: int, n_sym: int, arch: int = PD, precision: int = FP32,
                     estimate: int = UNBIASED, llr_bits: int = 0, refine: int = 0, refine_fp64: int = 0,
                     cluster_sizes=None, equalizer: int = LMMSE, lama_iters: int = 0) -> Plan:
    """Create a plan; ``cluster_sizes`` (C antenna counts summing to B) for clusters of unequal size."""
    p = ffeq_problem(B, U, C, n_sc, n_sym, arch, precision, estimate, llr_bits, refine, refine_fp64, equalizer,
                     lama_iters)
    h = _vp()
    if cluster_sizes is None:
        _check("ffeq_plan_create", lib().ffeq_plan_create(ctypes.byref(h), ctypes.byref(p)))
    else:
        if len(cluster_sizes) != C:
            raise ValueError("cluster_sizes must have C entries")
        sizes = (_i * len(cluster_sizes))(*[int(v) for v in cluster_sizes])
        _check("ffeq_plan_create_clusters", lib().ffeq_plan_create_clusters(ctypes.byref(h), ctypes.byref(p), sizes))
    return Plan(h.value, p)


def ffeq_workspace_size(plan: Plan) -> int:
    n = _sz()
    _check("ffeq_workspace_size", lib().ffeq_workspace_size(plan.handle, ctypes.byref(n)))
    return n.value


def ffeq_host_staging_size(plan: Plan) -> int:
    n = _sz()
    _check("ffeq_host_staging_size", lib().ffeq_host_staging_size(plan.handle, ctypes.byref(n)))
    return n.value


def ffeq_equalize(plan: Plan, H, y, N0: float, Es: float, z, sigma2, llr=None, info=None, workspace=None,
                  workspace_bytes: int = 0, stream=None) -> None:
    _check("ffeq_equalize", lib().ffeq_equalize(
        plan.handle, _ptr(H), _ptr(y), float(N0), float(Es), _ptr(z), _ptr(sigma2), _ptr(llr), _ptr(info),
        _ptr(workspace), workspace_bytes, _stream(stream)))


def ffeq_local_preprocess(plan: Plan, H, y, workspace, workspace_bytes: int, stream=None) -> None:
    _check("ffeq_local_preprocess", lib().ffeq_local_preprocess(
        plan.handle, _ptr(H), _ptr(y), _ptr(workspace), workspace_bytes, _stream(stream)))


def ffeq_fuse_equalize(plan: Plan, workspace, workspace_bytes: int, N0: float, Es: float, z, sigma2, llr=None,
                       info=None, stream=None) -> None:
    _check("ffeq_fuse_equalize", lib().ffeq_fuse_equalize(
        plan.handle, _ptr(workspace), workspace_bytes, float(N0), float(Es), _ptr(z), _ptr(sigma2), _ptr(llr),
        _ptr(info), _stream(stream)))


def ffeq_equalize_host(plan: Plan, H, y, N0: float, Es: float, z, sigma2, llr=None, info=None, staging=None,
                       staging_bytes: int = 0, stream=None) -> None:
    _check("ffeq_equalize_host", lib().ffeq_equalize_host(
        plan.handle, _ptr(H), _ptr(y), float(N0), float(Es), _ptr(z), _ptr(sigma2), _ptr(llr), _ptr(info),
        _ptr(staging), staging_bytes, _stream(stream)))


def ffeq_fd_train_workspace_size(plan: Plan) -> int:
    n = _sz()
    _check("ffeq_fd_train_workspace_size", lib().ffeq_fd_train_workspace_size(plan.handle, ctypes.byref(n)))
    return n.value


def ffeq_fd_train_forward(plan: Plan, H, y, rho_c, nu, z, workspace, workspace_bytes: int, stream=None) -> None:
    _check("ffeq_fd_train_forward", lib().ffeq_fd_train_forward(
        plan.handle, _ptr(H), _ptr(y), _ptr(rho_c), _ptr(nu), _ptr(z), _ptr(workspace), workspace_bytes,
        _stream(stream)))


def ffeq_fd_train_backward(plan: Plan, H, y, rho_c, nu, gz, gH, gy, grho, gnu, workspace, workspace_bytes: int,
                           stream=None) -> None:
    _check("ffeq_fd_train_backward", lib().ffeq_fd_train_backward(
        plan.handle, _ptr(H), _ptr(y), _ptr(rho_c), _ptr(nu), _ptr(gz), _ptr(gH), _ptr(gy), _ptr(grho), _ptr(gnu),
        _ptr(workspace), workspace_bytes, _stream(stream)))


def ffeq_fd_optimal_workspace_size(plan: Plan) -> int:
    n = _sz()
    _check("ffeq_fd_optimal_workspace_size", lib().ffeq_fd_optimal_workspace_size(plan.handle, ctypes.byref(n)))
    return n.value


def ffeq_fd_optimal_backward(plan: Plan, H, y, N0: float, Es: float, gz, gH, gy, workspace, workspace_bytes: int,
                             stream=None) -> None:
    _check("ffeq_fd_optimal_backward", lib().ffeq_fd_optimal_backward(
        plan.handle, _ptr(H), _ptr(y), float(N0), float(Es), _ptr(gz), _ptr(gH), _ptr(gy), _ptr(workspace),
        workspace_bytes, _stream(stream)))


def ffeq_equalize_noalloc(plan: Plan, H, y, N0: float, Es: float, z, sigma2, llr=None, info=None,
                          stream=None) -> None:
    """``ffeq_equalize`` for callers that cannot allocate device memory: no workspace
    argument, the library's fixed 64 MiB per-device array is used instead (calls
    must not overlap on the GPU; the first call on a device must precede any
    stream capture)."""
    _check("ffeq_equalize_noalloc", lib().ffeq_equalize_noalloc(
        plan.handle, _ptr(H), _ptr(y), float(N0), float(Es), _ptr(z), _ptr(sigma2), _ptr(llr), _ptr(info),
        _stream(stream)))


def ffeq_plan_set_tuning(plan: Plan, tuning) -> None:
    """``tuning`` = (contraction shape, staged subcarriers); see include/ffeq.h."""
    buf = (_i * 2)(*[int(v) for v in tuning])
    _check("ffeq_plan_set_tuning", lib().ffeq_plan_set_tuning(plan.handle, buf, 2))


def ffeq_plan_get_tuning(plan: Plan) -> tuple[int, int]:
    buf = (_i * 2)()
    _check("ffeq_plan_get_tuning", lib().ffeq_plan_get_tuning(plan.handle, buf, 2))
    return (buf[0], buf[1])


def ffeq_plan_autotune(plan: Plan, H, y, N0: float, Es: float, z, sigma2, llr=None, info=None, workspace=None,
                       workspace_bytes: int = 0, stream=None, reps: int = 10) -> tuple[int, int]:
    _check("ffeq_plan_autotune", lib().ffeq_plan_autotune(
        plan.handle, _ptr(H), _ptr(y), float(N0), float(Es), _ptr(z), _ptr(sigma2), _ptr(llr), _ptr(info),
        _ptr(workspace), workspace_bytes, _stream(stream), int(reps)))
    return ffeq_plan_get_tuning(plan)


def ffeq_plan_autotune_sets(plan: Plan, Hs, ys, N0: float, Es: float, z, sigma2, llr=None, info=None, workspace=None,
                            workspace_bytes: int = 0, stream=None, reps: int = 10) -> tuple[int, int]:
    """Autotune over several input sets (lists of device buffers), read in rotation."""
    if len(Hs) != len(ys) or not Hs:
        raise ValueError("Hs and ys must be non-empty lists of the same length")
    harr = (_vp * len(Hs))(*[_ptr(h) for h in Hs])
    yarr = (_vp * len(ys))(*[_ptr(v) for v in ys])
    _check("ffeq_plan_autotune_sets", lib().ffeq_plan_autotune_sets(
        plan.handle, harr, yarr, len(Hs), float(N0), float(Es), _ptr(z), _ptr(sigma2), _ptr(llr), _ptr(info),
        _ptr(workspace), workspace_bytes, _stream(stream), int(reps)))
    return ffeq_plan_get_tuning(plan)


def ffeq_device_status(clear: bool = True) -> int:
    code = _i()
    _check("ffeq_device_status", lib().ffeq_device_status(ctypes.byref(code), int(clear)))
    return code.value


def ffeq_status_string(status: int) -> str:
    return lib().ffeq_status_string(status).decode()


# --------------------------------------------------------------------- uneven batches

class Batch:
    """Owner of an ``ffeq_batch*`` (destroyed with the object)."""

    def __init__(self, handle: int, config: ffeq_batch_config, instances):
        self.handle = handle
        self.config = config
        self.instances = instances

    def __del__(self):
        if self.handle and _lib is not None:
            _lib.ffeq_batch_destroy(self.handle)
            self.handle = None


def ffeq_batch_create(config: ffeq_batch_config, instances) -> Batch:
    """``instances``: a sequence of ``ffeq_instance`` (copied into a C array)."""
    arr = (ffeq_instance * max(1, len(instances)))(*instances)
    h = _vp()
    _check("ffeq_batch_create", lib().ffeq_batch_create(ctypes.byref(h), ctypes.byref(config), arr,
                                                        len(instances)))
    return Batch(h.value, config, list(instances))


def ffeq_batch_workspace_size(batch: Batch) -> int:
    n = _sz()
    _check("ffeq_batch_workspace_size", lib().ffeq_batch_workspace_size(batch.handle, ctypes.byref(n)))
    return n.value


def ffeq_batch_upload(batch: Batch, workspace, workspace_bytes: int, stream=None) -> None:
    _check("ffeq_batch_upload", lib().ffeq_batch_upload(batch.handle, _ptr(workspace), workspace_bytes,
                                                        _stream(stream)))


def ffeq_batch_equalize(batch: Batch, H, y, z, sigma2, llr=None, info=None, workspace=None, workspace_bytes: int = 0,
                        stream=None) -> None:
    _check("ffeq_batch_equalize", lib().ffeq_batch_equalize(
        batch.handle, _ptr(H), _ptr(y), _ptr(z), _ptr(sigma2), _ptr(llr), _ptr(info), _ptr(workspace),
        workspace_bytes, _stream(stream)))


def ffeq_batch_autotune(batch: Batch, H, y, z, sigma2, llr=None, info=None, workspace=None,
                        workspace_bytes: int = 0, stream=None, reps: int = 10) -> None:
    _check("ffeq_batch_autotune", lib().ffeq_batch_autotune(
        batch.handle, _ptr(H), _ptr(y), _ptr(z), _ptr(sigma2), _ptr(llr), _ptr(info), _ptr(workspace),
        workspace_bytes, _stream(stream), int(reps)))


def ffeq_batch_groups(batch: Batch) -> int:
    return lib().ffeq_batch_groups(batch.handle)


def ffeq_batch_get_tuning(batch: Batch) -> list[tuple[int, int, int, int]]:
    """Per user group: (users padded, contraction stages, solve threads per CTA, lanes per row)."""
    g = ffeq_batch_groups(batch)
    buf = (_i * max(1, 4 * g))()
    _check("ffeq_batch_get_tuning", lib().ffeq_batch_get_tuning(batch.handle, buf, 4 * g))
    return [tuple(buf[4 * k:4 * k + 4]) for k in range(g)]


def ffeq_batch_set_tuning(batch: Batch, tuning) -> None:
    flat = [int(v) for t in tuning for v in t]
    buf = (_i * max(1, len(flat)))(*flat)
    _check("ffeq_batch_set_tuning", lib().ffeq_batch_set_tuning(batch.handle, buf, len(flat)))


def pack_batch(specs, arch: int = PD, precision: int = FP32, estimate: int = UNBIASED, llr_bits: int = 0,
               with_info: bool = True, equalizer: int = LMMSE, lama_iters: int = 0):
    """Lay instances out back to back in flat buffers.

    ``specs``: sequence of ``(B, U, C, n_sc, n_sym, N0, Es)``.  Offsets of the
    complex arrays are kept even (16-byte aligned rows when B is even); sigma^2
    is ``[n_sc][n_sym][U]`` per instance for LAMA, else ``[n_sc][U]``.
    Returns ``(config, instances)``.
    """
    def even(x):
        return x + (x & 1)
    offs = dict(h=0, y=0, z=0, s2=0, llr=0, info=0)
    inst = []
    for (B, U, C, n_sc, n_sym, N0, Es) in specs:
        Ceff = C if arch == FD else 1
        inst.append(ffeq_instance(B, U, C, n_sc, n_sym, float(N0), float(Es), offs["h"], offs["y"], offs["z"],
                                  offs["s2"], offs["llr"], offs["info"]))
        offs["h"] = even(offs["h"] + n_sc * U * B)
        offs["y"] = even(offs["y"] + n_sc * n_sym * B)
        offs["z"] = even(offs["z"] + n_sc * n_sym * U)
        offs["s2"] += n_sc * U * (n_sym if equalizer == LAMA else 1)
        offs["llr"] += n_sc * n_sym * U * llr_bits
        offs["info"] += n_sc * Ceff
    cfg = ffeq_batch_config(arch, precision, estimate, llr_bits, offs["h"], offs["y"], offs["z"], offs["s2"],
                            offs["llr"], offs["info"] if with_info else 0, equalizer, lama_iters)
    return cfg, inst


# --------------------------------------------------------------------- convenience

def equalize(H, y, N0: float, Es: float, C: int, arch: int = PD, estimate: int = UNBIASED, llr_bits: int = 0,
             with_info: bool = False, stream=None, precision: int = FP32, refine: int = 0,
             refine_fp64: int = 0, cluster_sizes=None, equalizer: int = LMMSE, lama_iters: int = 0) -> dict:
    """Allocate outputs on ``H.device`` and run one equalization (returns torch tensors)."""
    import torch
    if H.dtype != torch.complex64 or y.dtype != torch.complex64:
        raise TypeError("H and y must be complex64")
    if not H.is_cuda or not y.is_cuda:
        raise ValueError("H and y must be CUDA tensors (there is no CPU path)")
    n_sc, U, B = H.shape
    n_sym = y.shape[1]
    if tuple(y.shape) != (n_sc, n_sym, B):
        raise ValueError("y must be [n_sc][n_sym][B]")
    plan = ffeq_plan_create(B, U, C, n_sc, n_sym, arch, precision, estimate, llr_bits, refine, refine_fp64,
                            cluster_sizes, equalizer, lama_iters)
    dev = H.device
    s2_shape = (n_sc, n_sym, U) if equalizer == LAMA else (n_sc, U)     # LAMA: per received vector
    out = {"z": torch.empty((n_sc, n_sym, U), dtype=torch.complex64, device=dev),
           "sigma2": torch.empty(s2_shape, dtype=torch.float32, device=dev)}
    if llr_bits:
        out["llr"] = torch.empty((n_sc, n_sym, U, llr_bits), dtype=torch.float32, device=dev)
    if with_info:
        out["info"] = torch.empty((n_sc, C if arch == FD else 1), dtype=torch.int32, device=dev)
    ws_bytes = ffeq_workspace_size(plan)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev) if ws_bytes else None
    ffeq_equalize(plan, H, y, N0, Es, out["z"], out["sigma2"], out.get("llr"), out.get("info"), ws, ws_bytes,
                  stream)
    return out
