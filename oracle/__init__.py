"""CPU oracle for GP population evaluation -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path:
the arithmetic lives in ``tgp_oracle.c`` (plain C, binary64, recursive tree
walk), this module only marshals numpy arrays through ctypes.

What it follows (TensorGP, arXiv 2103.07512): the tensor phenotype over a
rank-2 grid (Sec. 3.1), the operators of Table 1 with their protections and the
pi-scaled trigonometry of Sec. 3.2, the Pagie polynomial of Eq. 1 and the RMSE
fitness of Sec. 4.1 / Table 2.  The readings taken where the paper is silent are
listed at the top of ``tgp_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tgp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

PREFIX, POSTFIX = 0, 1
TARGET_PAGIE, TARGET_VALUES = 0, 1

# opcode numbering of the token stream (terminals, then Table 1 functions)
X, Y, CONST, ADD, SUB, MUL, DIV, SIN, COS, NEG, ABS, MIN, MAX = range(13)
TAN, EXP, LOG, POW, MDIST, SQRT, SIGN, CLIP, MOD, FRAC, IF = range(13, 24)

_lib = None

# A test may point the wrapper at a deliberately broken copy of the oracle
# (tests/test_oracle_mutants.py) to show that the pins catch the mistake.
_OVERRIDE = os.environ.get("TGP_ORACLE_LIB_OVERRIDE")


def build(force: bool = False) -> str:
    """Compiles liboracle.so next to its source (gcc, no fp contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11",
                               "-ffp-contract=off", "-fno-fast-math",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        if _OVERRIDE:
            lib = ctypes.CDLL(_OVERRIDE)
        else:
            build()
            lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float
        lib.oracle_eval.argtypes = [P, P, i64, P, i32, i32, i32, i32, f32, f32, f32, f32,
                                    i64, P, P, P, P, P, i32]
        lib.oracle_eval.restype = ctypes.c_int
        lib.oracle_fitness.argtypes = [P, P, i64, P, i32, i32, i32, i32, f32, f32, f32, f32,
                                       i32, P, i64, P, P, P, P, P, i32]
        lib.oracle_fitness.restype = ctypes.c_int
        lib.oracle_fitness_parts.argtypes = [P, P, i64, P, i32, i32, i32, i32, f32, f32, f32, f32,
                                             i32, P, i64, P, i32, ctypes.c_double, P, P, P, i64, P]
        lib.oracle_fitness_parts.restype = ctypes.c_int
        lib.oracle_pagie.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.oracle_pagie.restype = ctypes.c_double
        lib.oracle_sinpi.argtypes = [ctypes.c_double]
        lib.oracle_sinpi.restype = ctypes.c_double
        lib.oracle_cospi.argtypes = [ctypes.c_double]
        lib.oracle_cospi.restype = ctypes.c_double
        lib.oracle_grid_point.argtypes = [i32, i32, f32, f32, f32, f32, i64,
                                          ctypes.POINTER(f32), ctypes.POINTER(f32)]
        lib.oracle_grid_point.restype = None
        lib.oracle_arity.argtypes = [i32]
        lib.oracle_arity.restype = ctypes.c_int
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _pop_arrays(ops, imm, tree_off):
    ops = np.ascontiguousarray(ops, dtype=np.int32)
    imm = np.ascontiguousarray(imm, dtype=np.float32)
    tree_off = np.ascontiguousarray(tree_off, dtype=np.int64)
    if ops.size == 0:
        ops = np.zeros(1, np.int32)[:0]
    return ops, imm, tree_off


TRIG_MODES = {"pi": 0, "rad": 1}


def _trig(trig):
    if trig not in TRIG_MODES:
        raise ValueError(f"trig must be one of {sorted(TRIG_MODES)}")
    return TRIG_MODES[trig]


def evaluate(ops, imm, tree_off, order, W, H, xlo, xhi, ylo, yhi, pts=None, with_bound=False, trig="pi"):
    """Phenotypes of every tree.

    trig: "pi" (sin(a) = sin(pi a), Sec. 3.2) or "rad" (radians, the footnote
    of Table 1); it applies to sin, cos and tan.

    Returns (v64 [T, n], v32 [T, n], flags [T, n]) where n = H*W (all points in
    flat order) or len(pts).  v32 is the FP32-faithful evaluation, flags marks
    points where a division saw |denominator| < 1e-6.  With with_bound=True a
    fourth array [T, n] bounds |any binary32 evaluation - exact| per element.
    """
    lib = _load()
    ops, imm, tree_off = _pop_arrays(ops, imm, tree_off)
    T = tree_off.size - 1
    if pts is None:
        n = W * H
        pts_arr = None
    else:
        pts_arr = np.ascontiguousarray(pts, dtype=np.int64)
        n = pts_arr.size
    v64 = np.empty((T, n), np.float64)
    v32 = np.empty((T, n), np.float32)
    fl = np.empty((T, n), np.uint8)
    eb = np.empty((T, n), np.float64) if with_bound else None
    rc = lib.oracle_eval(_ptr(ops), _ptr(imm), imm.size, _ptr(tree_off), T, order,
                         W, H, xlo, xhi, ylo, yhi, n, _ptr(pts_arr), _ptr(v64), _ptr(v32), _ptr(fl),
                         _ptr(eb), _trig(trig))
    if rc != 0:
        raise OracleError(f"oracle_eval failed: {rc}")
    if with_bound:
        return v64, v32, fl.astype(bool), eb
    return v64, v32, fl.astype(bool)


def fitness(ops, imm, tree_off, order, W, H, xlo, xhi, ylo, yhi, target=None, pts=None,
            with_bound=False, trig="pi"):
    """RMSE of every tree against Pagie (target None) or a [H*W] value array
    (trig as for evaluate).

    Returns (rmse64 [T], rmse32 [T], n_flagged [T]); with with_bound=True also
    rmse_err [T], the L2 bound of the per-element binary32 error bounds.
    """
    lib = _load()
    ops, imm, tree_off = _pop_arrays(ops, imm, tree_off)
    T = tree_off.size - 1
    if target is None:
        kind, tv = TARGET_PAGIE, None
    else:
        kind, tv = TARGET_VALUES, np.ascontiguousarray(target, dtype=np.float64).reshape(-1)
        if tv.size != W * H:
            raise ValueError("target must hold H*W values")
    if pts is None:
        n, pts_arr = 0, None
    else:
        pts_arr = np.ascontiguousarray(pts, dtype=np.int64)
        n = pts_arr.size
    r64 = np.empty(T, np.float64)
    r32 = np.empty(T, np.float64)
    nf = np.empty(T, np.int64)
    re = np.empty(T, np.float64) if with_bound else None
    rc = lib.oracle_fitness(_ptr(ops), _ptr(imm), imm.size, _ptr(tree_off), T, order,
                            W, H, xlo, xhi, ylo, yhi, kind, _ptr(tv), n, _ptr(pts_arr),
                            _ptr(r64), _ptr(r32), _ptr(nf), _ptr(re), _trig(trig))
    if rc != 0:
        raise OracleError(f"oracle_fitness failed: {rc}")
    if with_bound:
        return r64, r32, nf, re
    return r64, r32, nf


PART_NAMES = ("s64", "s32", "s64_c", "s32_c", "se_c", "n_c", "n_flagged", "n_excluded")


def fitness_parts(ops, imm, tree_off, order, W, H, xlo, xhi, ylo, yhi, target=None, pts=None, trig="pi",
                  tol=1e-4, ex_cap=None):
    """Sums behind the fitness comparison (see oracle_fitness_parts in
    tgp_oracle.c): a dict of [T] arrays named by PART_NAMES, plus "ex_tree"
    and "ex_pt", the (tree, flat point) pairs of the elements that are not
    comparable (an unbounded error bound, or the FP32-faithful value further
    than tol (1 + |v64|) from the binary64 one)."""
    lib = _load()
    ops, imm, tree_off = _pop_arrays(ops, imm, tree_off)
    T = tree_off.size - 1
    if target is None:
        kind, tv = TARGET_PAGIE, None
    else:
        kind, tv = TARGET_VALUES, np.ascontiguousarray(target, dtype=np.float64).reshape(-1)
        if tv.size != W * H:
            raise ValueError("target must hold H*W values")
    if pts is None:
        n, pts_arr = 0, None
    else:
        pts_arr = np.ascontiguousarray(pts, dtype=np.int64)
        n = pts_arr.size
    sums = np.zeros((max(T, 1), 8), np.float64)
    cap = int(ex_cap) if ex_cap is not None else max(1024, (T * (n if pts is not None else W * H)) // 8)
    while True:
        ex_tree = np.empty(cap, np.int32)
        ex_pt = np.empty(cap, np.int64)
        ex_n = ctypes.c_int64()
        rc = lib.oracle_fitness_parts(_ptr(ops), _ptr(imm), imm.size, _ptr(tree_off), T, order,
                                      W, H, xlo, xhi, ylo, yhi, kind, _ptr(tv), n, _ptr(pts_arr), _trig(trig),
                                      float(tol), _ptr(sums), _ptr(ex_tree), _ptr(ex_pt), cap, ctypes.byref(ex_n))
        if rc != 0:
            raise OracleError(f"oracle_fitness_parts failed: {rc}")
        if ex_n.value <= cap:
            break
        cap = ex_n.value
    out = {k: sums[:T, i].copy() for i, k in enumerate(PART_NAMES)}
    out["ex_tree"] = ex_tree[:ex_n.value].copy()
    out["ex_pt"] = ex_pt[:ex_n.value].copy()
    return out


def pagie(x: float, y: float) -> float:
    """Eq. 1 at one point, binary64."""
    return _load().oracle_pagie(float(x), float(y))


def sinpi(a: float) -> float:
    return _load().oracle_sinpi(float(a))


def cospi(a: float) -> float:
    return _load().oracle_cospi(float(a))


def grid_point(W, H, xlo, xhi, ylo, yhi, p):
    """Binary32 coordinates (x, y) of flat grid index p."""
    x = ctypes.c_float()
    y = ctypes.c_float()
    _load().oracle_grid_point(W, H, xlo, xhi, ylo, yhi, p, ctypes.byref(x), ctypes.byref(y))
    return x.value, y.value


def arity(op: int) -> int:
    return _load().oracle_arity(op)
