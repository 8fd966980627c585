"""Python binding of the HPS leaf-reduction library (C ABI in include/hps.h).

Argument marshalling only: every step of the leaf reduction runs in the CUDA
kernels of ``libhps.so``.  Functions keep the C names.  Buffer arguments take
a torch tensor (its ``data_ptr()`` is passed; dtype, device and contiguity are
checked), a raw integer address, or None for a NULL pointer.  A non-OK status
raises ``HpsError``.  If the library has not been built, importing works but
the first call raises: there is no CPU fallback.

Build it with ``python -m paper_2503_04033_gb300.build`` (or
``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os

__all__ = [
    "HPS_OK", "HPS_EINVAL", "HPS_ENOMEM", "HPS_ESINGULAR", "HPS_ENOCONV", "HPS_ECUDA", "HPS_ETIMEOUT",
    "HPS_FP64", "HPS_FP32_IR", "HPS_BF16_IR", "HPS_OPT_IR_MAX_ITERS", "HPS_OPT_IR_TOL", "HPS_OPT_BLOCK",
    "HPS_OPT_TENSOR_CORES", "HPS_OPT_SYNC", "HPS_OPT_TEST_SINGULAR_BOX", "HPS_OPT_TEST_TC_TIMEOUT", "HpsError", "LeafKind", "load_library", "library_path",
    "hps_create", "hps_destroy", "hps_set_option", "hps_leaf_sizes", "hps_leaf_nodes", "hps_workspace_per_box",
    "hps_leaf_build_dtn", "hps_leaf_particular", "hps_leaf_reconstruct", "hps_assemble_interface_blocks",
    "hps_last_refinement", "hps_profile_enable", "hps_profile_reset", "hps_profile_get", "hps_status_string",
    "EXPORTED_SYMBOLS", "KERNEL_CLASSES", "hps_leaf_build_dtn_noalloc", "hps_leaf_groups", "LeafGroup",
    "HPS_OPT_AUTOTUNE", "HPS_OPT_GRAPHS", "HPS_OPT_TC_EPILOGUE", "HPS_OPT_LU_UNIT", "HPS_OPT_TC_FUSE", "HPS_OPT_RESIDUAL_DF", "HPS_OPT_FP16_OPERANDS", "HPS_OPT_GROUPS_CONCURRENT", "hps_mlp_create", "hps_mlp_destroy", "hps_mlp_num_params",
    "hps_mlp_copy_params", "hps_mlp_forward", "hps_mlp_grad", "hps_mlp_target", "hps_mlp_grad_target",
    "hps_mlp_adam_step", "hps_lowrank_dtn",
    "hps_dtn_gate", "hps_selftest_conversions", "hps_leaf_factor", "hps_leaf_solve_factored",
    "hps_leaf_reconstruct_factored", "hps_leaf_factors_destroy", "hps_leaf_apply",
    "hps_interface_factor", "hps_interface_solve", "hps_interface_info", "hps_interface_destroy",
    "hps_interface_plan", "hps_interface_last_refinement", "hps_leaf2d_solve", "hps_leaf2d_reconstruct",
    "hps_leaf2d_sizes", "hps_interface2d_factor", "hps_interface2d_plan", "hps_leaf_cross_sizes",
    "hps_leaf_cross_nodes", "hps_leaf_cross_solve", "hps_leaf_cross_reconstruct", "hps_leaf_iti",
    "hps_leaf_iti_solve", "hps_leaf_iti_reconstruct", "hps_iti_assemble", "hps_iti_rhs",
    "hps_mixed_layout", "hps_mixed_face_coords", "hps_mixed_assemble", "hps_mixed_reduce", "hps_mixed_traces",
]

HPS_OK, HPS_EINVAL, HPS_ENOMEM, HPS_ESINGULAR, HPS_ENOCONV, HPS_ECUDA, HPS_ETIMEOUT = range(7)
HPS_FP64, HPS_FP32_IR, HPS_BF16_IR = 0, 1, 2
HPS_OPT_IR_MAX_ITERS, HPS_OPT_IR_TOL, HPS_OPT_BLOCK, HPS_OPT_TENSOR_CORES, HPS_OPT_SYNC = 1, 2, 3, 4, 5
HPS_OPT_AUTOTUNE, HPS_OPT_GRAPHS, HPS_OPT_TC_EPILOGUE, HPS_OPT_LU_UNIT, HPS_OPT_TC_FUSE = 6, 7, 8, 10, 11
HPS_OPT_RESIDUAL_DF, HPS_OPT_FP16_OPERANDS = 12, 13
HPS_OPT_GROUPS_CONCURRENT = 14
HPS_OPT_TEST_SINGULAR_BOX = 100
HPS_OPT_TEST_TC_TIMEOUT = 101

EXPORTED_SYMBOLS = (
    "hps_create", "hps_destroy", "hps_set_option", "hps_leaf_sizes", "hps_leaf_nodes", "hps_workspace_per_box",
    "hps_leaf_build_dtn", "hps_leaf_particular", "hps_leaf_reconstruct", "hps_assemble_interface_blocks",
    "hps_last_refinement", "hps_profile_enable", "hps_profile_reset", "hps_profile_get", "hps_status_string",
    "hps_leaf_build_dtn_noalloc", "hps_leaf_groups", "hps_mlp_create", "hps_mlp_destroy", "hps_mlp_num_params",
    "hps_mlp_copy_params", "hps_mlp_forward", "hps_mlp_grad", "hps_mlp_target", "hps_mlp_grad_target",
    "hps_mlp_adam_step", "hps_lowrank_dtn",
    "hps_dtn_gate", "hps_selftest_conversions", "hps_leaf_factor", "hps_leaf_solve_factored",
    "hps_leaf_reconstruct_factored", "hps_leaf_factors_destroy", "hps_leaf_apply",
    "hps_interface_factor", "hps_interface_solve", "hps_interface_info", "hps_interface_destroy",
    "hps_interface_plan", "hps_interface_last_refinement", "hps_leaf2d_solve", "hps_leaf2d_reconstruct",
    "hps_interface2d_factor", "hps_interface2d_plan", "hps_leaf_cross_sizes", "hps_leaf_cross_nodes",
    "hps_leaf_cross_solve", "hps_leaf_cross_reconstruct", "hps_leaf_iti", "hps_leaf_iti_solve",
    "hps_leaf_iti_reconstruct", "hps_iti_assemble", "hps_iti_rhs", "hps_mixed_layout",
    "hps_mixed_face_coords", "hps_mixed_assemble", "hps_mixed_reduce", "hps_mixed_traces",
)

# Kernel classes of hps_profile_get.
KERNEL_CLASSES = ("build", "panel", "update_cudacore", "update_tcgen05", "gather", "residual_fp64",
                  "refine_update", "dn_fp64", "update_tcgen05_refine", "pack", "residual_df",
                  "bookkeeping", "residual_df64")

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


def library_path() -> str:
    return os.path.join(_HERE, "libhps.so")


class HpsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        super().__init__(f"{where}: {hps_status_string(status)} (status {status})")


class LeafKind(ctypes.Structure):
    """hps_leaf_kind: polynomial order p, box sides h[3], wavenumber kappa, and
    optionally the first-order field beta (device [nbox, 3, p^3] float64 tensor
    or address) of -Lap u + div(beta u) - kappa^2 b u."""
    _fields_ = [("p", ctypes.c_int), ("h", ctypes.c_double * 3), ("kappa", ctypes.c_double),
                ("beta", ctypes.c_void_p)]

    def __init__(self, p: int, h, kappa: float, beta=None):
        hh = list(h) if hasattr(h, "__len__") else [h, h, h]
        super().__init__(int(p), (ctypes.c_double * 3)(*[float(x) for x in hh]), float(kappa),
                         _ptr(beta, _f64() if beta is not None and not isinstance(beta, int) else None))
        self._beta_ref = beta   # keeps the tensor alive while the kind is


class LeafGroup(ctypes.Structure):
    """hps_leaf_group: one order p / box size h of a mixed batch, per-box kappa."""
    _fields_ = [("p", ctypes.c_int), ("h", ctypes.c_double * 3), ("nbox", ctypes.c_int),
                ("kappa", ctypes.POINTER(ctypes.c_double)), ("b", ctypes.c_void_p), ("T", ctypes.c_void_p),
                ("S", ctypes.c_void_p), ("nrhs", ctypes.c_int), ("f", ctypes.c_void_p), ("v", ctypes.c_void_p),
                ("hflux", ctypes.c_void_p), ("box_status", ctypes.c_void_p)]


def load_library() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -m paper_2503_04033_gb300.build); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    i64p = ctypes.POINTER(ctypes.c_int64)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    kp = ctypes.POINTER(LeafKind)
    sig = {
        "hps_create": (i, [ctypes.POINTER(vp), i, sz]),
        "hps_destroy": (None, [vp]),
        "hps_set_option": (i, [vp, i, d]),
        "hps_leaf_sizes": (i, [i, ip, ip]),
        "hps_selftest_conversions": (i, [i, ctypes.c_longlong, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_longlong)]),
        "hps_leaf_nodes": (i, [i, dp, dp, dp]),
        "hps_workspace_per_box": (sz, [i, i]),
        "hps_leaf_build_dtn": (i, [vp, kp, i, vp, vp, vp, i, vp, vp]),
        "hps_leaf_particular": (i, [vp, kp, i, i, vp, vp, vp, vp, i, vp, vp]),
        "hps_leaf_reconstruct": (i, [vp, kp, i, i, vp, vp, vp, vp, vp, i, vp, vp]),
        "hps_leaf_factor": (i, [vp, kp, i, vp, i, i, vp, vp, ctypes.POINTER(vp)]),
        "hps_leaf_solve_factored": (i, [vp, i, vp, vp, vp, vp, vp]),
        "hps_leaf_reconstruct_factored": (i, [vp, i, vp, vp, vp, vp, vp]),
        "hps_leaf_factors_destroy": (None, [vp]),
        "hps_leaf_apply": (i, [vp, kp, i, i, vp, vp, vp, vp]),
        "hps_interface_factor": (i, [vp, i, ip, vp, i, i, vp, ctypes.POINTER(vp)]),
        "hps_interface_last_refinement": (i, [vp, ip, dp]),
        "hps_leaf2d_solve": (i, [i, dp, d, i, vp, i, vp, vp, vp, vp, vp, vp, vp]),
        "hps_interface2d_factor": (i, [vp, i, ip, vp, i, i, vp, ctypes.POINTER(vp)]),
        "hps_interface2d_plan": (i, [i, ip, ip, ip, ip, ip]),
        "hps_leaf2d_reconstruct": (i, [i, i, i, vp, vp, vp, vp, vp]),
        "hps_leaf_cross_sizes": (i, [i, ip, ip]),
        "hps_leaf_cross_nodes": (i, [i, dp, dp, dp]),
        "hps_leaf_cross_solve": (i, [i, dp, d, i, vp, vp, vp, i, vp, vp, vp, vp, vp, vp, vp]),
        "hps_leaf_cross_reconstruct": (i, [i, i, i, vp, vp, vp, vp, vp]),
        "hps_leaf_iti": (i, [kp, d, i, vp, vp, vp, vp]),
        "hps_leaf_iti_solve": (i, [kp, d, i, vp, i, vp, vp, vp, vp, vp, vp, vp]),
        "hps_leaf_iti_reconstruct": (i, [i, d, i, i, vp, vp, vp, vp, vp, vp, vp, vp]),
        "hps_iti_assemble": (i, [i, vp, vp, vp, vp, vp, vp]),
        "hps_iti_rhs": (i, [i, vp, d, vp, vp, vp]),
        "hps_mixed_layout": (i, [vp, vp, vp, vp, vp, vp]),
        "hps_mixed_face_coords": (i, [vp, vp, vp, vp, vp]),
        "hps_mixed_assemble": (i, [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "hps_mixed_reduce": (i, [vp, vp, vp, vp]),
        "hps_mixed_traces": (i, [vp, vp, vp, vp]),
        "hps_interface_solve": (i, [vp, i, vp, vp, vp, vp]),
        "hps_interface_info": (i, [vp, ip, ip, ip, ctypes.POINTER(sz)]),
        "hps_interface_destroy": (None, [vp]),
        "hps_interface_plan": (i, [i, ip, ip, ip, ip, ip]),
        "hps_assemble_interface_blocks": (i, [i, ip, dp, i64p, i64p, i64p, dp, i64p, i64p, i64p, dp, i64p, i64p]),
        "hps_last_refinement": (i, [vp, i, ip, dp]),
        "hps_profile_enable": (i, [vp, i]),
        "hps_profile_reset": (i, [vp]),
        "hps_profile_get": (i, [vp, i, ctypes.POINTER(ctypes.c_longlong), dp, dp, dp]),
        "hps_status_string": (ctypes.c_char_p, [i]),
        "hps_leaf_build_dtn_noalloc": (i, [kp, i, vp, vp, vp, vp]),
        "hps_leaf_groups": (i, [vp, i, ctypes.POINTER(LeafGroup), i, vp]),
        "hps_mlp_create": (i, [i, i, i, i, i, i, ctypes.c_ulonglong, ctypes.POINTER(vp)]),
        "hps_mlp_destroy": (None, [vp]),
        "hps_mlp_num_params": (sz, [vp]),
        "hps_mlp_copy_params": (i, [vp, i, ctypes.POINTER(ctypes.c_float), i]),
        "hps_mlp_forward": (i, [vp, i, vp, vp, vp, vp]),
        "hps_mlp_grad": (i, [vp, i, vp, vp, vp, d, dp, vp]),
        "hps_mlp_target": (i, [i, i, vp, vp, d, vp, vp]),
        "hps_mlp_grad_target": (i, [vp, i, vp, vp, dp, vp]),
        "hps_mlp_adam_step": (i, [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, vp]),
        "hps_lowrank_dtn": (i, [i, i, i, vp, d, vp, vp, vp, vp]),
        "hps_dtn_gate": (i, [vp, kp, i, vp, vp, i, ctypes.c_ulonglong, i, d, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, where: str) -> None:
    if status != HPS_OK:
        raise HpsError(status, where)


def _sizes_or_zero(p: int):
    """(n, m) of order p, or (0, 0) when the library rejects p (the call
    itself then reports it)."""
    n, m = ctypes.c_int(), ctypes.c_int()
    if load_library().hps_leaf_sizes(int(p), ctypes.byref(n), ctypes.byref(m)) != HPS_OK:
        return 0, 0
    return n.value, m.value


def _need(x, count: int, what: str) -> None:
    """Refuses (ValueError, before any launch) a tensor with fewer than
    count elements where the library will read or write count; addresses
    passed as ints are the caller's responsibility."""
    import torch
    if isinstance(x, torch.Tensor) and x.numel() < count:
        raise ValueError(f"{what}: {x.numel()} elements, the call needs {count}")


def _ptr(x, dtype=None):
    """Device address of a tensor (checked), an int, or None.  A pinned host
    tensor passes too: its address is device-accessible (mapped)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    import torch
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"expected a torch tensor, int or None, got {type(x)}")
    if not x.is_cuda and not x.is_pinned():
        raise ValueError("expected a CUDA tensor or a pinned host tensor")
    if not x.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and x.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {x.dtype}")
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _f64():
    import torch
    return torch.float64


def _i32():
    import torch
    return torch.int32


def hps_status_string(status: int) -> str:
    try:
        return load_library().hps_status_string(int(status)).decode()
    except RuntimeError:
        return f"status {status}"


def hps_create(device: int = 0, workspace_bytes_max: int = 0) -> int:
    ctx = ctypes.c_void_p()
    _check(load_library().hps_create(ctypes.byref(ctx), int(device), int(workspace_bytes_max)), "hps_create")
    return ctx.value


def hps_destroy(ctx: int) -> None:
    load_library().hps_destroy(ctx)


def hps_set_option(ctx: int, option: int, value: float) -> None:
    _check(load_library().hps_set_option(ctx, int(option), float(value)), "hps_set_option")


def hps_selftest_conversions(device: int = 0, n: int = 1 << 24, seed: int = 1):
    """(double->float, float->double) mismatch counts of the integer-pipe
    conversions against the hardware ones (both 0 when correct)."""
    out = (ctypes.c_longlong * 2)()
    _check(load_library().hps_selftest_conversions(int(device), int(n), int(seed), out), "hps_selftest_conversions")
    return int(out[0]), int(out[1])


def hps_leaf_sizes(p: int):
    n, m = ctypes.c_int(), ctypes.c_int()
    _check(load_library().hps_leaf_sizes(int(p), ctypes.byref(n), ctypes.byref(m)), "hps_leaf_sizes")
    return n.value, m.value


def hps_leaf_nodes(p: int, lo, h):
    import numpy as np
    lo3 = (ctypes.c_double * 3)(*[float(v) for v in lo])
    hh = list(h) if hasattr(h, "__len__") else [h, h, h]
    h3 = (ctypes.c_double * 3)(*[float(v) for v in hh])
    out = np.empty((p ** 3, 3), dtype=np.float64)
    _check(load_library().hps_leaf_nodes(int(p), lo3, h3, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           "hps_leaf_nodes")
    return out


def hps_workspace_per_box(p: int, prec: int = HPS_FP32_IR) -> int:
    return int(load_library().hps_workspace_per_box(int(p), int(prec)))


def hps_leaf_build_dtn(ctx, kind: LeafKind, nbox: int, b, T, S=None, prec: int = HPS_FP32_IR,
                       box_status=None, stream=None) -> None:
    n, m = _sizes_or_zero(kind.p)
    _need(b, nbox * kind.p ** 3, "b")
    _need(T, nbox * m * m, "T")
    _need(S, nbox * n * m, "S")
    _need(box_status, nbox, "box_status")
    f64 = _f64() if not isinstance(b, int) else None
    _check(load_library().hps_leaf_build_dtn(
        ctx, ctypes.byref(kind), int(nbox), _ptr(b, f64), _ptr(T, f64), _ptr(S, f64), int(prec),
        _ptr(box_status, _i32() if box_status is not None and not isinstance(box_status, int) else None),
        _stream(stream)), "hps_leaf_build_dtn")


def hps_leaf_particular(ctx, kind: LeafKind, nbox: int, nrhs: int, b, f, v, h, prec: int = HPS_FP32_IR,
                        box_status=None, stream=None) -> None:
    n, m = _sizes_or_zero(kind.p)
    _need(b, nbox * kind.p ** 3, "b")
    _need(f, nbox * nrhs * kind.p ** 3, "f")
    _need(v, nbox * nrhs * n, "v")
    _need(h, nbox * nrhs * m, "h")
    _need(box_status, nbox, "box_status")
    f64 = _f64() if not isinstance(b, int) else None
    _check(load_library().hps_leaf_particular(
        ctx, ctypes.byref(kind), int(nbox), int(nrhs), _ptr(b, f64), _ptr(f, f64), _ptr(v, f64), _ptr(h, f64),
        int(prec), _ptr(box_status, _i32() if box_status is not None and not isinstance(box_status, int) else None),
        _stream(stream)), "hps_leaf_particular")


def hps_leaf_reconstruct(ctx, kind: LeafKind, nbox: int, nrhs: int, b, S, v, ub, ui, prec: int = HPS_FP32_IR,
                         box_status=None, stream=None) -> None:
    n, m = _sizes_or_zero(kind.p)
    if S is None:
        _need(b, nbox * kind.p ** 3, "b")
    _need(S, nbox * n * m, "S")
    _need(v, nbox * nrhs * n, "v")
    _need(ub, nbox * nrhs * m, "ub")
    _need(ui, nbox * nrhs * n, "ui")
    _need(box_status, nbox, "box_status")
    f64 = _f64() if not isinstance(ub, int) else None
    _check(load_library().hps_leaf_reconstruct(
        ctx, ctypes.byref(kind), int(nbox), int(nrhs), _ptr(b, f64), _ptr(S, f64), _ptr(v, f64), _ptr(ub, f64),
        _ptr(ui, f64), int(prec),
        _ptr(box_status, _i32() if box_status is not None and not isinstance(box_status, int) else None),
        _stream(stream)), "hps_leaf_reconstruct")


def hps_leaf_factor(ctx, kind: LeafKind, nbox: int, b, nrhs_max: int, prec: int = HPS_FP32_IR, box_status=None,
                    stream=None):
    """Factors A_ii of every box once; returns the handle for
    hps_leaf_solve_factored / hps_leaf_reconstruct_factored."""
    out = ctypes.c_void_p()
    _check(load_library().hps_leaf_factor(
        ctx, ctypes.byref(kind), int(nbox), _ptr(b, _f64() if not isinstance(b, int) else None), int(nrhs_max),
        int(prec), _ptr(box_status, _i32() if box_status is not None and not isinstance(box_status, int) else None),
        _stream(stream), ctypes.byref(out)), "hps_leaf_factor")
    return out


def hps_leaf_solve_factored(factors, nrhs: int, f, v, h, box_status=None, stream=None) -> None:
    f64 = _f64() if not isinstance(f, int) else None
    _check(load_library().hps_leaf_solve_factored(
        factors, int(nrhs), _ptr(f, f64), _ptr(v, f64), _ptr(h, f64),
        _ptr(box_status, _i32() if box_status is not None and not isinstance(box_status, int) else None),
        _stream(stream)), "hps_leaf_solve_factored")


def hps_leaf_reconstruct_factored(factors, nrhs: int, v, ub, ui, box_status=None, stream=None) -> None:
    f64 = _f64() if not isinstance(ub, int) else None
    _check(load_library().hps_leaf_reconstruct_factored(
        factors, int(nrhs), _ptr(v, f64), _ptr(ub, f64), _ptr(ui, f64),
        _ptr(box_status, _i32() if box_status is not None and not isinstance(box_status, int) else None),
        _stream(stream)), "hps_leaf_reconstruct_factored")


def hps_leaf_apply(ctx, kind: LeafKind, nbox: int, nfield: int, b, u, out, stream=None) -> None:
    """out = A u at the interior nodes of full nodal fields [nbox, nfield, p^3]."""
    f64 = _f64() if not isinstance(u, int) else None
    _check(load_library().hps_leaf_apply(ctx, ctypes.byref(kind), int(nbox), int(nfield), _ptr(b, f64), _ptr(u, f64),
                                         _ptr(out, f64), _stream(stream)), "hps_leaf_apply")


def hps_leaf_factors_destroy(factors) -> None:
    load_library().hps_leaf_factors_destroy(factors)


def hps_interface_factor(ctx, p: int, nb, T, nrhs_max: int = 1, prec: int = HPS_FP64, stream=None):
    """Factors the interface system of an nb grid of boxes from their DtN maps
    T [nbox, m, m] (device), in FP64 or FP32 with FP64 refinement in each
    solve; returns the handle for hps_interface_solve."""
    out = ctypes.c_void_p()
    nb3 = (ctypes.c_int * 3)(*[int(v) for v in nb])
    _check(load_library().hps_interface_factor(ctx, int(p), nb3, _ptr(T, _f64() if not isinstance(T, int) else None),
                                               int(nrhs_max), int(prec), _stream(stream), ctypes.byref(out)),
           "hps_interface_factor")
    return out


def hps_interface2d_factor(ctx, p: int, nb, T, nrhs_max: int = 1, prec: int = HPS_FP64, stream=None):
    """hps_interface_factor for an nb[0] x nb[1] grid of 2-D boxes (maps T [nbox, m, m], m = 4 (p-2))."""
    out = ctypes.c_void_p()
    nb2 = (ctypes.c_int * 2)(*[int(v) for v in nb])
    _check(load_library().hps_interface2d_factor(ctx, int(p), nb2, _ptr(T, _f64() if not isinstance(T, int) else None),
                                                 int(nrhs_max), int(prec), _stream(stream), ctypes.byref(out)),
           "hps_interface2d_factor")
    return out


def hps_interface2d_plan(p: int, nb):
    """The merge tree of a 2-D grid (host only): (nodes [n_merge, 8], lists)."""
    import numpy as np
    lib = load_library()
    nb2 = (ctypes.c_int * 2)(*[int(v) for v in nb])
    nm, nl = ctypes.c_int(), ctypes.c_int()
    _check(lib.hps_interface2d_plan(int(p), nb2, ctypes.byref(nm), ctypes.byref(nl), None, None),
           "hps_interface2d_plan")
    nodes = np.zeros((max(nm.value, 1), 8), dtype=np.int32)
    lists = np.zeros(max(nl.value, 1), dtype=np.int32)
    ip = ctypes.POINTER(ctypes.c_int)
    _check(lib.hps_interface2d_plan(int(p), nb2, ctypes.byref(nm), ctypes.byref(nl), nodes.ctypes.data_as(ip),
                                    lists.ctypes.data_as(ip)), "hps_interface2d_plan")
    return nodes[:nm.value], lists[:nl.value]


def hps_interface_last_refinement(iface):
    """(corrections, last relative correction) of the last FP32_IR solve."""
    a, b = ctypes.c_int(), ctypes.c_double()
    _check(load_library().hps_interface_last_refinement(iface, ctypes.byref(a), ctypes.byref(b)),
           "hps_interface_last_refinement")
    return a.value, b.value


def hps_interface_solve(iface, nrhs: int, h, g, ub, stream=None) -> None:
    """u_b [nbox, nrhs, m] on every box face from the leaf fluxes h and the
    Dirichlet values g (both [nbox, nrhs, m]; g None for g = 0)."""
    f64 = _f64() if not isinstance(h, int) else None
    _check(load_library().hps_interface_solve(iface, int(nrhs), _ptr(h, f64), _ptr(g, f64), _ptr(ub, f64),
                                              _stream(stream)), "hps_interface_solve")


def hps_interface_info(iface):
    """(merges, levels, largest separator in nodes, device bytes held)."""
    a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
    _check(load_library().hps_interface_info(iface, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                             ctypes.byref(d)), "hps_interface_info")
    return a.value, b.value, c.value, d.value


def hps_interface_destroy(iface) -> None:
    load_library().hps_interface_destroy(iface)


def hps_interface_plan(p: int, nb):
    """The merge tree (host only): (nodes [n_merge, 8] int32, lists int32), see hps.h."""
    import numpy as np
    lib = load_library()
    nb3 = (ctypes.c_int * 3)(*[int(v) for v in nb])
    nm, nl = ctypes.c_int(), ctypes.c_int()
    _check(lib.hps_interface_plan(int(p), nb3, ctypes.byref(nm), ctypes.byref(nl), None, None), "hps_interface_plan")
    nodes = np.zeros((max(nm.value, 1), 8), dtype=np.int32)
    lists = np.zeros(max(nl.value, 1), dtype=np.int32)
    ip = ctypes.POINTER(ctypes.c_int)
    _check(lib.hps_interface_plan(int(p), nb3, ctypes.byref(nm), ctypes.byref(nl), nodes.ctypes.data_as(ip),
                                  lists.ctypes.data_as(ip)), "hps_interface_plan")
    return nodes[:nm.value], lists[:nl.value]


def hps_leaf2d_sizes(p: int):
    """(n, m) = ((p-2)^2, 4 (p-2)) of a 2-D box."""
    if p < 3 or p > 24:
        raise HpsError(HPS_EINVAL, "hps_leaf2d_sizes")
    return (p - 2) ** 2, 4 * (p - 2)


def hps_leaf2d_solve(p: int, h, kappa: float, nbox: int, b, nrhs: int = 0, f=None, T=None, S=None, v=None,
                     hflux=None, box_status=None, stream=None) -> None:
    """2-D boxes: T, S, and for nrhs loads v, h (device tensors, see hps.h)."""
    f64 = _f64() if not isinstance(b, int) else None
    hh = (ctypes.c_double * 2)(*[float(x) for x in (h if hasattr(h, "__len__") else (h, h))])
    _check(load_library().hps_leaf2d_solve(
        int(p), hh, float(kappa), int(nbox), _ptr(b, f64), int(nrhs), _ptr(f, f64), _ptr(T, f64), _ptr(S, f64),
        _ptr(v, f64), _ptr(hflux, f64),
        _ptr(box_status, _i32() if box_status is not None and not isinstance(box_status, int) else None),
        _stream(stream)), "hps_leaf2d_solve")


def hps_leaf2d_reconstruct(p: int, nbox: int, nrhs: int, S, v, ub, ui, stream=None) -> None:
    f64 = _f64() if not isinstance(S, int) else None
    _check(load_library().hps_leaf2d_reconstruct(int(p), int(nbox), int(nrhs), _ptr(S, f64), _ptr(v, f64),
                                                 _ptr(ub, f64), _ptr(ui, f64), _stream(stream)),
           "hps_leaf2d_reconstruct")


def hps_leaf_cross_sizes(p: int):
    """(n, m) = ((p-2)^3, 6 (p-1)^2) of a box with Legendre face grids."""
    n, m = ctypes.c_int(), ctypes.c_int()
    _check(load_library().hps_leaf_cross_sizes(int(p), ctypes.byref(n), ctypes.byref(m)), "hps_leaf_cross_sizes")
    return n.value, m.value


def hps_leaf_cross_nodes(p: int, lo, h) -> np.ndarray:
    """[m, 3] coordinates of the box's Legendre face nodes."""
    import numpy as np
    _, m = hps_leaf_cross_sizes(p)
    lo3 = np.ascontiguousarray(np.broadcast_to(np.asarray(lo, dtype=np.float64), (3,)))
    h3 = np.ascontiguousarray(np.broadcast_to(np.asarray(h, dtype=np.float64), (3,)))
    out = np.empty((m, 3))
    dp = ctypes.POINTER(ctypes.c_double)
    _check(load_library().hps_leaf_cross_nodes(int(p), lo3.ctypes.data_as(dp), h3.ctypes.data_as(dp),
                                               out.ctypes.data_as(dp)), "hps_leaf_cross_nodes")
    return out


def hps_leaf_cross_solve(p: int, h, kappa: float, nbox: int, C, d, b, nrhs: int = 0, f=None, T=None, S=None,
                         v=None, hflux=None, box_status=None, stream=None) -> None:
    """Cross-term leaves: T, S, and for nrhs loads v, h (device tensors, see hps.h)."""
    f64 = _f64() if not isinstance(b, int) else None
    h3 = [float(x) for x in h] if hasattr(h, "__len__") else [float(h)] * 3
    hh = (ctypes.c_double * 3)(*h3)
    _check(load_library().hps_leaf_cross_solve(
        int(p), hh, float(kappa), int(nbox), _ptr(C, f64), _ptr(d, f64), _ptr(b, f64), int(nrhs), _ptr(f, f64),
        _ptr(T, f64), _ptr(S, f64), _ptr(v, f64), _ptr(hflux, f64),
        _ptr(box_status, _i32() if box_status is not None and not isinstance(box_status, int) else None),
        _stream(stream)), "hps_leaf_cross_solve")


def hps_leaf_cross_reconstruct(p: int, nbox: int, nrhs: int, S, v, ub, ui, stream=None) -> None:
    f64 = _f64() if not isinstance(S, int) else None
    _check(load_library().hps_leaf_cross_reconstruct(int(p), int(nbox), int(nrhs), _ptr(S, f64), _ptr(v, f64),
                                                     _ptr(ub, f64), _ptr(ui, f64), _stream(stream)),
           "hps_leaf_cross_reconstruct")


def hps_leaf_iti(kind: LeafKind, eta: float, nbox: int, b, R, box_status=None, stream=None) -> None:
    """Leaf impedance-to-impedance maps R [nbox][m][m] (a complex128 tensor)
    of boxes b [nbox][p^3] (see include/hps.h)."""
    import torch
    if not isinstance(R, int) and R.dtype != torch.complex128:
        raise ValueError("R must be complex128")
    if 4 <= kind.p <= 16:                  # the orders hps_leaf_iti accepts (others: HPS_EINVAL from the call)
        n, m = _sizes_or_zero(kind.p)
        _need(b, nbox * kind.p ** 3, "b")
        _need(R, nbox * m * m, "R")
        _need(box_status, nbox, "box_status")
    f64 = _f64() if not isinstance(b, int) else None
    _check(load_library().hps_leaf_iti(
        ctypes.byref(kind), float(eta), int(nbox), _ptr(b, f64), _ptr(R, None),
        _ptr(box_status, _i32() if box_status is not None and not isinstance(box_status, int) else None),
        _stream(stream)), "hps_leaf_iti")


def _mixed_args(nb, p_box):
    import numpy as np
    nb3 = np.ascontiguousarray(nb, dtype=np.int32).reshape(3)
    pb = np.ascontiguousarray(p_box, dtype=np.int32).reshape(-1)
    if pb.size != int(np.prod(nb3)):
        raise ValueError("p_box needs one order per box")
    return nb3, pb


def _host_ptrs(arrs):
    """A C array of host addresses of float64 numpy arrays (kept alive by the caller)."""
    import numpy as np
    for a in arrs:
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
            raise ValueError("expected contiguous float64 numpy arrays")
    return (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])


def hps_mixed_layout(nb, p_box):
    """(n_iface, n_dir, face_p, face_off) of a mixed-order grid (host)."""
    import numpy as np
    nb3, pb = _mixed_args(nb, p_box)
    nx, ny, nz = (int(v) for v in nb3)
    nfaces = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1) + 2 * (ny * nz + nx * nz + nx * ny)
    nfaces = max(nfaces, 1) if min(nx, ny, nz) >= 1 else 1   # bad sizes: the library answers HPS_EINVAL
    ni, nd = ctypes.c_int64(), ctypes.c_int64()
    fp = np.zeros(nfaces, dtype=np.int32)
    fo = np.zeros(nfaces + 1, dtype=np.int64)
    _check(load_library().hps_mixed_layout(nb3.ctypes.data, pb.ctypes.data, ctypes.byref(ni), ctypes.byref(nd),
                                           fp.ctypes.data, fo.ctypes.data), "hps_mixed_layout")
    return ni.value, nd.value, fp, fo


def hps_mixed_face_coords(nb, p_box, lo, L):
    import numpy as np
    nb3, pb = _mixed_args(nb, p_box)
    ni, nd, _, _ = hps_mixed_layout(nb, p_box)
    lo3 = np.ascontiguousarray(lo, dtype=np.float64).reshape(3)
    L3 = np.ascontiguousarray(L, dtype=np.float64).reshape(3)
    xyz = np.empty((ni + nd, 3))
    _check(load_library().hps_mixed_face_coords(nb3.ctypes.data, pb.ctypes.data, lo3.ctypes.data, L3.ctypes.data,
                                                xyz.ctypes.data), "hps_mixed_face_coords")
    return xyz


def hps_mixed_assemble(nb, p_box, T_boxes):
    """COO triplets (rows, cols, vals, rows_d, cols_d, vals_d) of the
    interface system from host DtN maps T_boxes[tau] [m_tau, m_tau]."""
    import numpy as np
    nb3, pb = _mixed_args(nb, p_box)
    Ts = [np.ascontiguousarray(t, dtype=np.float64) for t in T_boxes]
    ptrs = _host_ptrs(Ts)
    lib = load_library()
    nnz, nnz_d = ctypes.c_int64(), ctypes.c_int64()
    _check(lib.hps_mixed_assemble(nb3.ctypes.data, pb.ctypes.data, ptrs, ctypes.byref(nnz), None, None, None,
                                  ctypes.byref(nnz_d), None, None, None), "hps_mixed_assemble")
    r, c, v = np.empty(nnz.value, np.int64), np.empty(nnz.value, np.int64), np.empty(nnz.value)
    rd, cd, vd = np.empty(nnz_d.value, np.int64), np.empty(nnz_d.value, np.int64), np.empty(nnz_d.value)
    _check(lib.hps_mixed_assemble(nb3.ctypes.data, pb.ctypes.data, ptrs, ctypes.byref(nnz), r.ctypes.data,
                                  c.ctypes.data, v.ctypes.data, ctypes.byref(nnz_d), rd.ctypes.data, cd.ctypes.data,
                                  vd.ctypes.data), "hps_mixed_assemble")
    return r, c, v, rd, cd, vd


def hps_mixed_reduce(nb, p_box, h_boxes):
    """sum_tau Q_tau h_tau [n_iface + n_dir] from host fluxes h_boxes[tau] [m_tau]."""
    import numpy as np
    nb3, pb = _mixed_args(nb, p_box)
    hs = [np.ascontiguousarray(x, dtype=np.float64).reshape(-1) for x in h_boxes]
    ni, nd, _, _ = hps_mixed_layout(nb, p_box)
    r = np.empty(ni + nd)
    _check(load_library().hps_mixed_reduce(nb3.ctypes.data, pb.ctypes.data, _host_ptrs(hs), r.ctypes.data),
           "hps_mixed_reduce")
    return r


def hps_mixed_traces(nb, p_box, u):
    """Per box the face-node values P_tau u (list of host arrays [m_tau])."""
    import numpy as np
    nb3, pb = _mixed_args(nb, p_box)
    uu = np.ascontiguousarray(u, dtype=np.float64)
    out = [np.empty(6 * (int(p) - 2) ** 2) for p in pb]
    _check(load_library().hps_mixed_traces(nb3.ctypes.data, pb.ctypes.data, uu.ctypes.data, _host_ptrs(out)),
           "hps_mixed_traces")
    return out


def hps_leaf_iti_solve(kind: LeafKind, eta: float, nbox: int, b, nrhs: int = 0, f=None, R=None, S=None, v=None,
                       hout=None, box_status=None, stream=None) -> None:
    """ItI maps with the interior operator and loads (complex128 outputs; see include/hps.h)."""
    import torch
    for name, t in (("R", R), ("S", S), ("v", v), ("hout", hout)):
        if t is not None and not isinstance(t, int) and t.dtype != torch.complex128:
            raise ValueError(f"{name} must be complex128")
    if 4 <= kind.p <= 16:
        n, m = _sizes_or_zero(kind.p)
        _need(b, nbox * kind.p ** 3, "b")
        _need(f, nbox * nrhs * kind.p ** 3, "f")
        _need(R, nbox * m * m, "R")
        _need(S, nbox * n * m, "S")
        _need(v, nbox * nrhs * n, "v")
        _need(hout, nbox * nrhs * m, "hout")
        _need(box_status, nbox, "box_status")
    f64 = _f64()
    _check(load_library().hps_leaf_iti_solve(
        ctypes.byref(kind), float(eta), int(nbox), _ptr(b, f64), int(nrhs), _ptr(f, f64), _ptr(R, None),
        _ptr(S, None), _ptr(v, None), _ptr(hout, None),
        _ptr(box_status, _i32() if box_status is not None and not isinstance(box_status, int) else None),
        _stream(stream)), "hps_leaf_iti_solve")


def hps_leaf_iti_reconstruct(p: int, eta: float, nbox: int, nrhs: int, R, S, v, hout, fin, ui=None, ub=None,
                             stream=None) -> None:
    if 4 <= p <= 16:
        n, m = _sizes_or_zero(p)
        _need(fin, nbox * nrhs * m, "fin")
        _need(ui, nbox * nrhs * n, "ui")
        _need(ub, nbox * nrhs * m, "ub")
        _need(R, nbox * m * m, "R")
        _need(S, nbox * n * m, "S")
    _check(load_library().hps_leaf_iti_reconstruct(int(p), float(eta), int(nbox), int(nrhs), _ptr(R, None),
                                                   _ptr(S, None), _ptr(v, None), _ptr(hout, None), _ptr(fin, None),
                                                   _ptr(ui, None), _ptr(ub, None), _stream(stream)),
           "hps_leaf_iti_reconstruct")


def hps_iti_assemble(p: int, nb, R_host):
    """COO (rows, cols, vals complex) of the two-level ItI system from host
    maps R_host [nbox, m, m] (complex128 numpy)."""
    import numpy as np
    nb3 = np.ascontiguousarray(nb, dtype=np.int32).reshape(3)
    Rh = np.ascontiguousarray(R_host, dtype=np.complex128)
    lib = load_library()
    nnz = ctypes.c_int64()
    _check(lib.hps_iti_assemble(int(p), nb3.ctypes.data, Rh.ctypes.data, ctypes.byref(nnz), None, None, None),
           "hps_iti_assemble")
    r, c = np.empty(nnz.value, np.int64), np.empty(nnz.value, np.int64)
    v = np.empty(nnz.value, np.complex128)
    _check(lib.hps_iti_assemble(int(p), nb3.ctypes.data, Rh.ctypes.data, ctypes.byref(nnz), r.ctypes.data,
                                c.ctypes.data, v.ctypes.data), "hps_iti_assemble")
    return r, c, v


def hps_iti_rhs(p: int, nb, eta: float, hout_host=None, g_face=None):
    """rhs [nbox m] (complex128) of the two-level ItI system (host)."""
    import numpy as np
    nb3 = np.ascontiguousarray(nb, dtype=np.int32).reshape(3)
    nbox = int(np.prod(nb3))
    m = 6 * (int(p) - 2) ** 2
    ho = None if hout_host is None else np.ascontiguousarray(hout_host, dtype=np.complex128).reshape(nbox, m)
    gf = None if g_face is None else np.ascontiguousarray(g_face, dtype=np.float64).reshape(nbox, m)
    out = np.empty(nbox * m, np.complex128)
    _check(load_library().hps_iti_rhs(int(p), nb3.ctypes.data, float(eta), None if ho is None else ho.ctypes.data,
                                      None if gf is None else gf.ctypes.data, out.ctypes.data), "hps_iti_rhs")
    return out


def hps_last_refinement(ctx, nbox: int):
    import numpy as np
    it = np.zeros(nbox, dtype=np.int32)
    rel = np.zeros(nbox, dtype=np.float64)
    _check(load_library().hps_last_refinement(ctx, int(nbox), it.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                              rel.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           "hps_last_refinement")
    return it, rel


def hps_assemble_interface_blocks(p: int, nb, T_host=None):
    """Returns (rows, cols, vals, rows_d, cols_d, vals_d, n_iface, n_dir) as numpy
    arrays (COO, unsummed) from host DtN blocks T_host [nbox, m, m]."""
    import numpy as np
    lib = load_library()
    nb3 = (ctypes.c_int * 3)(*[int(v) for v in nb])
    c64 = ctypes.c_int64
    nnz, nnz_d, ni, nd = c64(), c64(), c64(), c64()
    _check(lib.hps_assemble_interface_blocks(int(p), nb3, None, ctypes.byref(nnz), None, None, None,
                                             ctypes.byref(nnz_d), None, None, None, ctypes.byref(ni),
                                             ctypes.byref(nd)), "hps_assemble_interface_blocks")
    if T_host is None:
        return nnz.value, nnz_d.value, ni.value, nd.value
    T_host = np.ascontiguousarray(T_host, dtype=np.float64)
    rows, cols, vals = (np.empty(nnz.value, np.int64), np.empty(nnz.value, np.int64), np.empty(nnz.value))
    rd, cd, vd = (np.empty(nnz_d.value, np.int64), np.empty(nnz_d.value, np.int64), np.empty(nnz_d.value))
    P = ctypes.POINTER
    i64 = lambda a: a.ctypes.data_as(P(c64))
    f64 = lambda a: a.ctypes.data_as(P(ctypes.c_double))
    _check(lib.hps_assemble_interface_blocks(int(p), nb3, f64(T_host), ctypes.byref(nnz), i64(rows), i64(cols),
                                             f64(vals), ctypes.byref(nnz_d), i64(rd), i64(cd), f64(vd),
                                             ctypes.byref(ni), ctypes.byref(nd)), "hps_assemble_interface_blocks")
    return rows, cols, vals, rd, cd, vd, ni.value, nd.value


def hps_profile_enable(ctx, on: bool = True) -> None:
    _check(load_library().hps_profile_enable(ctx, int(bool(on))), "hps_profile_enable")


def hps_profile_reset(ctx) -> None:
    _check(load_library().hps_profile_reset(ctx), "hps_profile_reset")


def hps_profile_get(ctx, cls: int):
    """(launches, ms, flops, bytes) accumulated for kernel class cls."""
    n = ctypes.c_longlong()
    ms, fl, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load_library().hps_profile_get(ctx, int(cls), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl),
                                          ctypes.byref(by)), "hps_profile_get")
    return n.value, ms.value, fl.value, by.value


def hps_leaf_build_dtn_noalloc(kind: LeafKind, nbox: int, b, T, box_status=None, stream=None) -> None:
    """FP64 DtN build that allocates no device memory (see include/hps.h)."""
    f64 = _f64() if not isinstance(b, int) else None
    _check(load_library().hps_leaf_build_dtn_noalloc(
        ctypes.byref(kind), int(nbox), _ptr(b, f64), _ptr(T, f64),
        _ptr(box_status, _i32() if box_status is not None and not isinstance(box_status, int) else None),
        _stream(stream)), "hps_leaf_build_dtn_noalloc")


def hps_leaf_groups(ctx, groups, prec: int = HPS_FP32_IR, stream=None) -> None:
    """groups: list of dicts with keys p, h, kappa (host sequence, one per box),
    b, T (or None), S (or None), f/v/hflux (or None) and box_status (or None);
    nbox is len(kappa) and nrhs is taken from v's shape."""
    import numpy as np
    arr = (LeafGroup * max(1, len(groups)))()
    keep = []
    f64 = _f64()
    for i, g in enumerate(groups):
        kap = np.ascontiguousarray(np.asarray(g["kappa"], dtype=np.float64))
        keep.append(kap)
        hh = g["h"] if hasattr(g["h"], "__len__") else [g["h"]] * 3
        v = g.get("v")
        arr[i].p = int(g["p"])
        arr[i].h = (ctypes.c_double * 3)(*[float(x) for x in hh])
        arr[i].nbox = int(len(kap))
        arr[i].kappa = kap.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        n_g, m_g = _sizes_or_zero(int(g["p"]))
        nb_g, nr_g = int(len(kap)), (int(v.shape[1]) if v is not None else 0)
        _need(g["b"], nb_g * int(g["p"]) ** 3, "b")
        _need(g.get("T"), nb_g * m_g * m_g, "T")
        _need(g.get("S"), nb_g * n_g * m_g, "S")
        _need(g.get("f"), nb_g * nr_g * int(g["p"]) ** 3, "f")
        _need(v, nb_g * nr_g * n_g, "v")
        _need(g.get("hflux"), nb_g * nr_g * m_g, "hflux")
        _need(g.get("box_status"), nb_g, "box_status")
        arr[i].b = _ptr(g["b"], f64)
        arr[i].T = _ptr(g.get("T"), f64)
        arr[i].S = _ptr(g.get("S"), f64)
        arr[i].nrhs = int(v.shape[1]) if v is not None else 0
        arr[i].f = _ptr(g.get("f"), f64)
        arr[i].v = _ptr(v, f64)
        arr[i].hflux = _ptr(g.get("hflux"), f64)
        bs = g.get("box_status")
        arr[i].box_status = _ptr(bs, _i32() if bs is not None and not isinstance(bs, int) else None)
    _check(load_library().hps_leaf_groups(ctx, len(groups), arr, int(prec), _stream(stream)), "hps_leaf_groups")


# ---- learned low-rank correction and its residual gate

def hps_mlp_create(device: int, n_in: int, n_h1: int, n_h2: int, m: int, rank: int, seed: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load_library().hps_mlp_create(int(device), int(n_in), int(n_h1), int(n_h2), int(m), int(rank),
                                         int(seed), ctypes.byref(h)), "hps_mlp_create")
    return h.value


def hps_mlp_destroy(net) -> None:
    load_library().hps_mlp_destroy(net)


def hps_mlp_num_params(net) -> int:
    return int(load_library().hps_mlp_num_params(net))


def hps_mlp_copy_params(net, which: int = 0, host=None, to_device: bool = False):
    """which = 0 parameters, 1 gradients; returns the host FP32 array (or loads
    `host` into the network when to_device)."""
    import numpy as np
    if host is None:
        host = np.empty(hps_mlp_num_params(net), dtype=np.float32)
    host = np.ascontiguousarray(host, dtype=np.float32)
    _check(load_library().hps_mlp_copy_params(net, int(which), host.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                              int(bool(to_device))), "hps_mlp_copy_params")
    return host


def hps_mlp_forward(net, B: int, b, U, V, stream=None) -> None:
    f64 = _f64()
    _check(load_library().hps_mlp_forward(net, int(B), _ptr(b, f64), _ptr(U, f64), _ptr(V, f64), _stream(stream)),
           "hps_mlp_forward")


def hps_mlp_grad(net, B: int, b, T, T0, scale: float, want_loss: bool = True, stream=None):
    f64 = _f64()
    loss = ctypes.c_double()
    _check(load_library().hps_mlp_grad(net, int(B), _ptr(b, f64), _ptr(T, f64), _ptr(T0, f64), float(scale),
                                       ctypes.byref(loss) if want_loss else None, _stream(stream)), "hps_mlp_grad")
    return loss.value if want_loss else None


def hps_mlp_target(nbox: int, m: int, T, T0, scale: float, D, stream=None) -> None:
    """D = float((T - T0) / scale) on the device (D a float32 tensor)."""
    import torch
    _check(load_library().hps_mlp_target(int(nbox), int(m), _ptr(T, _f64()), _ptr(T0, _f64()), float(scale),
                                         _ptr(D, torch.float32), _stream(stream)), "hps_mlp_target")


def hps_mlp_grad_target(net, B: int, b, D, want_loss: bool = True, stream=None):
    import torch
    loss = ctypes.c_double()
    _check(load_library().hps_mlp_grad_target(net, int(B), _ptr(b, _f64()), _ptr(D, torch.float32),
                                              ctypes.byref(loss) if want_loss else None, _stream(stream)),
           "hps_mlp_grad_target")
    return loss.value if want_loss else None


def hps_mlp_adam_step(net, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                      stream=None) -> None:
    _check(load_library().hps_mlp_adam_step(net, float(lr), float(beta1), float(beta2), float(eps), _stream(stream)),
           "hps_mlp_adam_step")


def hps_lowrank_dtn(nbox: int, m: int, rank: int, T0, scale: float, U, V, T, stream=None) -> None:
    f64 = _f64()
    _check(load_library().hps_lowrank_dtn(int(nbox), int(m), int(rank), _ptr(T0, f64), float(scale), _ptr(U, f64),
                                          _ptr(V, f64), _ptr(T, f64), _stream(stream)), "hps_lowrank_dtn")


def hps_dtn_gate(ctx, kind: LeafKind, nbox: int, b, T_hat, nprobe: int, seed: int, iters: int, tol: float,
                 accept, err, stream=None) -> None:
    f64 = _f64()
    _check(load_library().hps_dtn_gate(ctx, ctypes.byref(kind), int(nbox), _ptr(b, f64), _ptr(T_hat, f64),
                                       int(nprobe), int(seed), int(iters), float(tol), _ptr(accept, _i32()),
                                       _ptr(err, f64), _stream(stream)), "hps_dtn_gate")
