"""Plain FP64 CPU oracle for the HPS leaf-box reduction (arXiv:2503.04033).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never imports it and shares no code with it.

The arithmetic lives in ``hps_oracle.c`` (plain loops, FP64); this module
compiles it with gcc on first use and wraps it with ctypes and numpy.  What
each routine computes, with the paper passage it follows:

* ``nodes``, ``diff``: Chebyshev-Lobatto points and the 1-D spectral
  differentiation matrix (Sec. 2.1, Trefethen's collocation).
* ``leaf_matrix``: the local equilibrium matrix A^tau (Algorithm 1): interior
  rows are the Helmholtz operator of Eq. 2, face rows the outward normal
  derivative of Eq. 4, edge and corner nodes dropped (Remark 1).
* ``leaf_dtn``: S = -A_ii^{-1} A_ib and T = A_bb + A_bi S (Sec. 2.2, Eq. 8).
* ``leaf_particular``: v = A_ii^{-1} f_i and h = A_bi v (Sec. 2.2 steps 1-2).
* ``leaf_reconstruct``: u_i = v + S u_b (Sec. 2.2 step 4).
* ``*_2d``: the same for a p x p grid per box (the 2-D form of the method,
  Sec. 1 and Sec. 3.2; four edges of p - 2 nodes, corners dropped).

``oracle.global_solve`` adds the interface system and the dense brute-force
check; ``oracle.pins`` holds the closed forms the tests pin the oracle to.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hps_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``hps_oracle.c`` into ``liboracle.so`` (gcc, OpenMP, FP64, no
    FMA contraction so that x86 and Arm hosts round alike)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-std=c99", "-D_DEFAULT_SOURCE", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            c_int, c_double = ctypes.c_int, ctypes.c_double
            sig = {
                "oc_sizes": (c_int, [c_int, ip, ip]),
                "oc_nodes": (None, [c_int, dp]),
                "oc_diff": (None, [c_int, dp]),
                "oc_node_coords": (None, [c_int, dp, dp, dp]),
                "oc_kept_index": (c_int, [c_int, c_int, c_int, c_int]),
                "oc_leaf_matrix": (None, [c_int, dp, c_double, dp, dp, dp]),
                "oc_split_blocks": (None, [c_int, dp, dp, dp, dp, dp]),
                "oc_lu": (c_int, [c_int, dp, ip]),
                "oc_lu_solve": (None, [c_int, dp, ip, c_int, dp]),
                "oc_leaf_dtn": (c_int, [c_int, dp, c_double, dp, dp, dp, dp]),
                "oc_leaf_particular": (c_int, [c_int, dp, c_double, dp, dp, c_int, dp, dp, dp]),
                "oc_leaf_reconstruct": (c_int, [c_int, dp, c_double, dp, dp, c_int, dp, dp, dp]),
                "oc_batch_dtn": (None, [c_int, dp, c_double, c_int, dp, dp, dp, ip, c_int]),
                "oc_max_threads": (c_int, []),
                "oc2_sizes": (c_int, [c_int, ip, ip]),
                "oc2_node_coords": (None, [c_int, dp, dp, dp]),
                "oc2_kept_index": (c_int, [c_int, c_int, c_int]),
                "oc2_leaf_matrix": (None, [c_int, dp, c_double, dp, dp]),
                "oc2_leaf_dtn": (c_int, [c_int, dp, c_double, dp, dp, dp]),
                "oc2_leaf_particular": (c_int, [c_int, dp, c_double, dp, c_int, dp, dp, dp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _h3(h):
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), (3,))
    return np.ascontiguousarray(h)


def sizes(p: int):
    """(n, m) = ((p-2)^3 interior nodes, 6 (p-2)^2 face nodes)."""
    q = p - 2
    return q ** 3, 6 * q * q


def max_threads() -> int:
    return int(_load().oc_max_threads())


def nodes(p: int) -> np.ndarray:
    t = np.empty(p)
    _load().oc_nodes(p, _dp(t))
    return t


def diff(p: int) -> np.ndarray:
    """Reference-interval ([-1,1]) differentiation matrix, p x p."""
    D = np.empty((p, p))
    _load().oc_diff(p, _dp(D))
    return D


def node_coords(p: int, lo, h) -> np.ndarray:
    """[p^3, 3] coordinates of a box's nodes in grid order (x fastest)."""
    xyz = np.empty((p ** 3, 3))
    _load().oc_node_coords(p, _dp(_h3(lo)), _dp(_h3(h)), _dp(xyz))
    return xyz


def kept_index(p: int, i: int, j: int, k: int) -> int:
    return int(_load().oc_kept_index(p, i, j, k))


def _beta(beta, p: int):
    """None, or the velocity-like field as a contiguous [3, p^3] array."""
    if beta is None:
        return None
    return np.ascontiguousarray(np.asarray(beta, np.float64).reshape(3, p ** 3))


def leaf_matrix(p: int, h, kappa: float, b: np.ndarray, beta=None) -> np.ndarray:
    """Kept-node collocation matrix of -Lap u + div(beta u) - kappa^2 b u
    (beta None: no first-order term)."""
    n, m = sizes(p)
    A = np.empty((n + m, n + m))
    bt = _beta(beta, p)
    _load().oc_leaf_matrix(p, _dp(_h3(h)), float(kappa), _dp(np.ascontiguousarray(b, np.float64)),
                           _dp(bt) if bt is not None else None, _dp(A))
    return A


def apply_interior(p: int, h, kappa: float, b: np.ndarray, u: np.ndarray, beta=None) -> np.ndarray:
    """A u at the interior nodes for a full nodal field u [p^3] (grid order):
    the interior rows of the kept-node collocation matrix (Eq. 2), applied
    to u's interior and face values; 0 at every other node."""
    from .global_solve import face_node_grid_indices, interior_grid_indices
    n, m = sizes(p)
    ii, fi = interior_grid_indices(p), face_node_grid_indices(p)
    A = leaf_matrix(p, h, kappa, b, beta)
    out = np.zeros(p ** 3)
    out[ii] = A[:n, :] @ np.concatenate([u[ii], u[fi]])
    return out


def split_blocks(p: int, A: np.ndarray):
    n, m = sizes(p)
    Aii, Aib, Abi, Abb = (np.empty(s) for s in ((n, n), (n, m), (m, n), (m, m)))
    _load().oc_split_blocks(p, _dp(np.ascontiguousarray(A)), _dp(Aii), _dp(Aib), _dp(Abi), _dp(Abb))
    return Aii, Aib, Abi, Abb


def lu(A: np.ndarray):
    """(LU, piv, info) of the oracle's own partial-pivot LU."""
    n = A.shape[0]
    LU = np.array(A, dtype=np.float64, order="C", copy=True)
    piv = np.empty(n, dtype=np.int32)
    info = _load().oc_lu(n, _dp(LU), _ip(piv))
    return LU, piv, int(info)


def lu_solve(LU: np.ndarray, piv: np.ndarray, B: np.ndarray) -> np.ndarray:
    n = LU.shape[0]
    X = np.array(B, dtype=np.float64, order="C", copy=True)
    if X.ndim == 1:
        X = X.reshape(n, 1)
    _load().oc_lu_solve(n, _dp(LU), _ip(piv), X.shape[1], _dp(X))
    return X.reshape(B.shape)


def leaf_dtn(p: int, h, kappa: float, b: np.ndarray, want_S: bool = True, beta=None):
    """(T [m,m], S [n,m] or None, info) for one box."""
    n, m = sizes(p)
    T = np.empty((m, m))
    S = np.empty((n, m)) if want_S else None
    info = _load().oc_leaf_dtn(p, _dp(_h3(h)), float(kappa),
                               _dp(np.ascontiguousarray(b, np.float64)), _dp(_beta(beta, p)), _dp(T), _dp(S))
    return T, S, int(info)


def leaf_particular(p: int, h, kappa: float, b: np.ndarray, f: np.ndarray, beta=None):
    """(v [nrhs,n], h [nrhs,m], info); f is [nrhs, p^3] (or [p^3])."""
    n, m = sizes(p)
    f2 = np.ascontiguousarray(np.atleast_2d(f), np.float64)
    nrhs = f2.shape[0]
    v = np.empty((nrhs, n))
    hf = np.empty((nrhs, m))
    info = _load().oc_leaf_particular(p, _dp(_h3(h)), float(kappa),
                                      _dp(np.ascontiguousarray(b, np.float64)), _dp(_beta(beta, p)), nrhs,
                                      _dp(f2), _dp(v), _dp(hf))
    return v, hf, int(info)


def leaf_reconstruct(p: int, h, kappa: float, b: np.ndarray, v: np.ndarray, ub: np.ndarray, beta=None):
    """(u_i [nrhs,n], info) with u_i = v + S u_b."""
    n, m = sizes(p)
    v2 = np.ascontiguousarray(np.atleast_2d(v), np.float64)
    ub2 = np.ascontiguousarray(np.atleast_2d(ub), np.float64)
    ui = np.empty_like(v2)
    info = _load().oc_leaf_reconstruct(p, _dp(_h3(h)), float(kappa),
                                       _dp(np.ascontiguousarray(b, np.float64)), _dp(_beta(beta, p)), v2.shape[0],
                                       _dp(v2), _dp(ub2), _dp(ui))
    return ui, int(info)


def batch_dtn(p: int, h, kappa: float, b: np.ndarray, want_S: bool = False, nthreads: int = 0):
    """Algorithm 1's box loop over a batch b [nbox, p^3]: (T, S or None, status)."""
    n, m = sizes(p)
    b = np.ascontiguousarray(b, np.float64)
    nbox = b.shape[0]
    T = np.empty((nbox, m, m))
    S = np.empty((nbox, n, m)) if want_S else None
    status = np.empty(nbox, dtype=np.int32)
    _load().oc_batch_dtn(p, _dp(_h3(h)), float(kappa), nbox, _dp(b), _dp(T), _dp(S), _ip(status), int(nthreads))
    return T, S, status


# ------------------------------------------------------------------ 2-D


def sizes_2d(p: int):
    n, m = ctypes.c_int(), ctypes.c_int()
    if _load().oc2_sizes(int(p), ctypes.byref(n), ctypes.byref(m)) != 0:
        raise ValueError(f"p = {p} too small")
    return n.value, m.value


def node_coords_2d(p: int, lo, h) -> np.ndarray:
    out = np.empty((p * p, 2))
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    h = np.ascontiguousarray(np.broadcast_to(np.asarray(h, dtype=np.float64), (2,)))
    _load().oc2_node_coords(int(p), _dp(lo), _dp(h), _dp(out))
    return out


def kept_index_2d(p: int, i: int, j: int) -> int:
    return _load().oc2_kept_index(int(p), int(i), int(j))


def _h2(h):
    return np.ascontiguousarray(np.broadcast_to(np.asarray(h, dtype=np.float64), (2,)))


def leaf_matrix_2d(p: int, h, kappa: float, b: np.ndarray) -> np.ndarray:
    n, m = sizes_2d(p)
    A = np.empty((n + m, n + m))
    _load().oc2_leaf_matrix(int(p), _dp(_h2(h)), float(kappa), _dp(np.ascontiguousarray(b, dtype=np.float64)), _dp(A))
    return A


def leaf_dtn_2d(p: int, h, kappa: float, b: np.ndarray, want_S: bool = True):
    """(T [m, m], S [n, m] or None, info) of one 2-D box."""
    n, m = sizes_2d(p)
    T = np.empty((m, m))
    S = np.empty((n, m)) if want_S else None
    info = _load().oc2_leaf_dtn(int(p), _dp(_h2(h)), float(kappa), _dp(np.ascontiguousarray(b, dtype=np.float64)),
                                _dp(T), _dp(S) if S is not None else None)
    return T, S, info


def leaf_particular_2d(p: int, h, kappa: float, b: np.ndarray, f: np.ndarray):
    """(v [nrhs, n], h [nrhs, m], info) for loads f [nrhs, p^2]."""
    n, m = sizes_2d(p)
    f = np.ascontiguousarray(np.atleast_2d(f), dtype=np.float64)
    nrhs = f.shape[0]
    v = np.empty((nrhs, n))
    hf = np.empty((nrhs, m))
    info = _load().oc2_leaf_particular(int(p), _dp(_h2(h)), float(kappa),
                                       _dp(np.ascontiguousarray(b, dtype=np.float64)), nrhs, _dp(f), _dp(v), _dp(hf))
    return v, hf, info
