"""tgp: GB300-native evaluation of GP expression-tree populations.

Thin ctypes binding of libtgp (C ABI in include/tgp.h): argument marshalling
only -- every step of the evaluation runs in the library's host compiler and
CUDA kernels.  The entry points keep the C names without the ``tgp_`` prefix.
PyTorch is used only for device memory and streams.

Importing this package does not load the library; the first call does, and
raises if libtgp.so is missing or fails to load (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtgp.so")

OK = 0
E_INVALID, E_TOKENS, E_NOMEM, E_BUDGET, E_CUDA, E_TIMEOUT, E_DEVICE_CHECK, E_BUSY = range(-1, -9, -1)
PREFIX, POSTFIX = 0, 1
TARGET_PAGIE, TARGET_TENSOR, TARGET_TOKENS = 0, 1, 2
F_HOST_ONLY, F_NO_DEDUP, F_TIME_KERNELS, F_NO_SIMPLIFY, F_TRIG_RADIANS, F_NO_COLUMNS = 1, 2, 4, 8, 16, 32
N_OPS = 24

EXPORTS = ["tgp_create", "tgp_destroy", "tgp_last_error", "tgp_load_domain", "tgp_release_domain",
           "tgp_compile_population", "tgp_release_population", "tgp_evaluate", "tgp_fitness",
           "tgp_fitness_dev", "tgp_stats_get", "tgp_debug_plan", "tgp_debug_layout",
           "tgp_calibrate_op_costs", "tgp_calibrate_peak", "tgp_plan_work", "tgp_fitness_noalloc", "tgp_fitness_graph", "tgp_autotune",
           "tgp_server_create", "tgp_server_destroy", "tgp_server_submit", "tgp_server_wait",
           "tgp_server_stats_get", "tgp_evolve", "tgp_population_tokens", "tgp_load_domain_rows",
           "tgp_fitness_sse_dev"]


class TgpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tgp error {code}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("cache_budget_bytes", ctypes.c_int64),
                ("points_per_thread", ctypes.c_int32), ("threads_per_block", ctypes.c_int32),
                ("n_groups", ctypes.c_int32), ("cache_min_cost", ctypes.c_int32),
                ("plan_threads", ctypes.c_int32), ("cache_ids_max", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class TargetTokens(ctypes.Structure):
    _fields_ = [("ops", ctypes.c_void_p), ("imm", ctypes.c_void_p), ("n_ops", ctypes.c_int64),
                ("n_imm", ctypes.c_int64), ("order", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("tree_nodes", ctypes.c_int64), ("dag_nodes", ctypes.c_int64),
                ("dag_internal", ctypes.c_int64), ("code_instrs", ctypes.c_int64),
                ("n_groups", ctypes.c_int64), ("n_items", ctypes.c_int64),
                ("points_per_thread", ctypes.c_int32), ("threads_per_block", ctypes.c_int32),
                ("slots", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("cache_entries", ctypes.c_int64), ("cache_bytes", ctypes.c_int64),
                ("cache_hits", ctypes.c_int64), ("cache_inserts", ctypes.c_int64),
                ("cache_evictions", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("eval_ms_sum", ctypes.c_double), ("eval_timed", ctypes.c_int64),
                ("cache_reserved", ctypes.c_int64), ("cache_id_nodes", ctypes.c_int64),
                ("cache_id_rebuilds", ctypes.c_int64), ("reserved", ctypes.c_int64 * 3)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


class ServerConfig(ctypes.Structure):
    _fields_ = [("streams", ctypes.c_int32), ("max_batch_trees", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_int64), ("reserved", ctypes.c_int64 * 6)]


class Job(ctypes.Structure):
    _fields_ = [("ops", ctypes.c_void_p), ("imm", ctypes.c_void_p), ("n_imm", ctypes.c_int64),
                ("tree_off", ctypes.c_void_p), ("n_trees", ctypes.c_int32), ("order", ctypes.c_int32),
                ("W", ctypes.c_int32), ("H", ctypes.c_int32),
                ("xlo", ctypes.c_float), ("xhi", ctypes.c_float), ("ylo", ctypes.c_float), ("yhi", ctypes.c_float),
                ("target_kind", ctypes.c_int32), ("target_tokens", ctypes.c_void_p)]


class JobInfo(ctypes.Structure):
    _fields_ = [("submit_ns", ctypes.c_int64), ("launch_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64),
                ("batch", ctypes.c_int64), ("batch_jobs", ctypes.c_int32), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int64 * 4)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "submitted", "completed", "failed", "batches", "max_batch_jobs", "max_in_flight", "domains_resident",
        "domains_loaded", "domains_released", "bytes_in_use", "max_bytes_in_use", "hbm_budget_bytes", "queued",
        "worker_busy_ns", "domain_load_ns", "max_batch_domains", "adopt_ns", "fitness_ns")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


class EvolveConfig(ctypes.Structure):
    _fields_ = [("tournament", ctypes.c_int32), ("p_crossover", ctypes.c_float), ("p_mutation", ctypes.c_float),
                ("elitism", ctypes.c_int32), ("max_depth", ctypes.c_int32), ("mutation_depth", ctypes.c_int32),
                ("functions", ctypes.c_void_p), ("n_functions", ctypes.c_int32),
                ("const_lo", ctypes.c_float), ("const_hi", ctypes.c_float), ("seed", ctypes.c_uint64),
                ("reserved", ctypes.c_int64 * 4)]


_lib = None


def lib():
    """Loads libtgp.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        from . import build as _build
        if _build.stale():
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libtgp.so not found at {LIB_PATH}")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
        sig = {
            "tgp_create": [P, P],
            "tgp_destroy": [P],
            "tgp_load_domain": [P, i32, i32, f32, f32, f32, f32, i32, P, P],
            "tgp_load_domain_rows": [P, i32, i32, f32, f32, f32, f32, i32, i32, i32, P, P],
            "tgp_fitness_sse_dev": [P, i64, i64, P, P],
            "tgp_release_domain": [P, i64],
            "tgp_compile_population": [P, P, P, i64, P, i32, i32, P],
            "tgp_release_population": [P, i64],
            "tgp_evaluate": [P, i64, i64, P, P],
            "tgp_fitness": [P, i64, i64, P, P, i32],
            "tgp_fitness_dev": [P, i64, i64, P, P],
            "tgp_stats_get": [P, P],
            "tgp_debug_plan": [P, i64, i64, P, i64, P, P, i64, P],
            "tgp_debug_layout": [P, i32],
            "tgp_calibrate_op_costs": [P, P],
            "tgp_calibrate_peak": [P, P, P],
            "tgp_plan_work": [P, i64, i64, P],
            "tgp_fitness_noalloc": [P, i64, i64, P, P],
            "tgp_fitness_graph": [P, i64, i64, P, P],
            "tgp_autotune": [P, i64, i64, P, P, P, P],
            "tgp_server_create": [P, P, P],
            "tgp_server_destroy": [P],
            "tgp_server_submit": [P, P, P],
            "tgp_server_wait": [P, i64, i64, P, P],
            "tgp_server_stats_get": [P, P],
            "tgp_evolve": [P, i64, P, P, P],
            "tgp_population_tokens": [P, i64, P, i64, P, i64, P, i64, P, P, P],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.tgp_last_error.argtypes = [P]
        L.tgp_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    if hasattr(a, "data_ptr"):      # torch tensor
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError(f"cannot pass {type(a)} as a pointer")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return ctypes.c_void_p(s)
    return ctypes.c_void_p(s.cuda_stream)   # torch.cuda.Stream


class Context:
    """A libtgp context on one CUDA device (or host-only for plan inspection)."""

    def __init__(self, device=0, host_only=False, cache_budget_bytes=0, points_per_thread=0,
                 threads_per_block=0, n_groups=0, dedup=True, time_kernels=False, cache_min_cost=0,
                 simplify=True, trig="pi", plan_threads=0, columns=True, cache_ids_max=0):
        """trig: "pi" (sin(a) = sin(pi a), Sec. 3.2) or "rad" (radians, the
        footnote of Table 1), for sin, cos and tan."""
        if trig not in ("pi", "rad"):
            raise ValueError('trig must be "pi" or "rad"')
        self._L = lib()
        cfg = Config()
        cfg.device = device
        cfg.flags = ((F_HOST_ONLY if host_only else 0) | (0 if dedup else F_NO_DEDUP)
                     | (F_TIME_KERNELS if time_kernels else 0) | (0 if simplify else F_NO_SIMPLIFY)
                     | (F_TRIG_RADIANS if trig == "rad" else 0) | (0 if columns else F_NO_COLUMNS))
        cfg.cache_budget_bytes = cache_budget_bytes
        cfg.points_per_thread = points_per_thread
        cfg.threads_per_block = threads_per_block
        cfg.n_groups = n_groups
        cfg.cache_min_cost = cache_min_cost
        cfg.plan_threads = plan_threads
        cfg.cache_ids_max = cache_ids_max
        h = ctypes.c_void_p()
        self._h = None
        self._check(self._L.tgp_create(ctypes.byref(h), ctypes.byref(cfg)))
        self._h = h

    def _check(self, rc):
        if rc != OK:
            msg = self._L.tgp_last_error(None).decode(errors="replace")
            raise TgpError(rc, msg)

    def close(self):
        if self._h is not None:
            self._L.tgp_destroy(self._h)
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

    # ---------------------------------------------------------------- ABI

    def load_domain(self, W, H, xlo=-5.0, xhi=5.0, ylo=-5.0, yhi=5.0, target=None,
                    target_tokens=None, rows=None):
        """tgp_load_domain: Pagie target by default; `target` = float32 [H*W]
        array (numpy or torch, host or device); `target_tokens` = (ops, imm, order).
        rows = (row0, n_rows): tgp_load_domain_rows, the band of rows row0 ..
        row0 + n_rows - 1 of the W x H grid (`target` then holds the band's
        n_rows*W values)."""
        out = ctypes.c_int64()
        keep = None
        if rows is not None:
            row0, n_rows = int(rows[0]), int(rows[1])

            def load(kind, tgt):
                return self._L.tgp_load_domain_rows(self._h, W, H, xlo, xhi, ylo, yhi, row0, n_rows, kind, tgt,
                                                    ctypes.byref(out))
        else:
            n_rows = H

            def load(kind, tgt):
                return self._L.tgp_load_domain(self._h, W, H, xlo, xhi, ylo, yhi, kind, tgt, ctypes.byref(out))
        if target_tokens is not None:
            ops, imm, order = target_tokens
            ops = np.ascontiguousarray(ops, np.int32)
            imm = np.ascontiguousarray(imm, np.float32)
            tt = TargetTokens(ops.ctypes.data, imm.ctypes.data if imm.size else None,
                              ops.size, imm.size, order)
            keep = (ops, imm, tt)
            rc = load(TARGET_TOKENS, ctypes.byref(tt))
        elif target is not None:
            if isinstance(target, np.ndarray):
                target = np.ascontiguousarray(target, np.float32)
                if target.size != W * n_rows:
                    raise ValueError("target must hold one value per point of the domain")
            keep = target
            rc = load(TARGET_TENSOR, _ptr(target))
        else:
            rc = load(TARGET_PAGIE, None)
        del keep
        self._check(rc)
        return out.value

    def release_domain(self, dom):
        self._check(self._L.tgp_release_domain(self._h, dom))

    def compile_population(self, ops, imm, tree_off, order=PREFIX):
        """tgp_compile_population from token arrays (or an inputs.Tokens)."""
        ops = np.ascontiguousarray(ops, np.int32)
        imm = np.ascontiguousarray(imm, np.float32)
        tree_off = np.ascontiguousarray(tree_off, np.int64)
        out = ctypes.c_int64()
        self._check(self._L.tgp_compile_population(
            self._h, _ptr(ops), _ptr(imm) if imm.size else None, imm.size, _ptr(tree_off),
            tree_off.size - 1, order, ctypes.byref(out)))
        return out.value

    def compile_tokens(self, tok):
        return self.compile_population(tok.ops, tok.imm, tok.tree_off, tok.order)

    def release_population(self, pop):
        self._check(self._L.tgp_release_population(self._h, pop))

    def evolve(self, pop, rmse, seed, tournament=0, p_crossover=0.0, p_mutation=0.0, elitism=0, max_depth=0,
               mutation_depth=0, functions=None, const_range=(0.0, 0.0)):
        """tgp_evolve: the next generation of `pop` from its RMSE values, as a
        new population handle (zero arguments take the library's defaults)."""
        rmse = np.ascontiguousarray(rmse, np.float64)
        fn = None if functions is None else np.ascontiguousarray(functions, np.int32)
        cfg = EvolveConfig(tournament=tournament, p_crossover=p_crossover, p_mutation=p_mutation,
                           elitism=elitism, max_depth=max_depth, mutation_depth=mutation_depth,
                           functions=None if fn is None else fn.ctypes.data,
                           n_functions=0 if fn is None else fn.size,
                           const_lo=const_range[0], const_hi=const_range[1], seed=seed)
        out = ctypes.c_int64()
        self._check(self._L.tgp_evolve(self._h, pop, _ptr(rmse), ctypes.byref(cfg), ctypes.byref(out)))
        return out.value

    def population_tokens(self, pop):
        """tgp_population_tokens: the population's trees as prefix tokens (inputs.Tokens)."""
        from .inputs import Tokens
        no, ni, nt = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        sizes = (ctypes.byref(no), ctypes.byref(ni), ctypes.byref(nt))
        self._check(self._L.tgp_population_tokens(self._h, pop, None, 0, None, 0, None, 0, *sizes))
        ops = np.empty(no.value, np.int32)
        imm = np.empty(ni.value, np.float32)
        off = np.empty(nt.value + 1, np.int64)
        self._check(self._L.tgp_population_tokens(self._h, pop, _ptr(ops), ops.size, _ptr(imm), imm.size,
                                                  _ptr(off), off.size, *sizes))
        return Tokens(ops, imm, off, PREFIX)

    def evaluate(self, pop, dom, out, stream=None):
        """tgp_evaluate into a device float32 buffer [n_trees, H*W] (torch tensor)."""
        self._check(self._L.tgp_evaluate(self._h, pop, dom, _stream(stream), _ptr(out)))

    def fitness(self, pop, dom, n_trees, stream=None, blocking=True, out=None):
        """tgp_fitness: returns a float64 numpy array of n_trees RMSE values."""
        if out is None:
            out = np.empty(n_trees, np.float64)
        self._check(self._L.tgp_fitness(self._h, pop, dom, _stream(stream), _ptr(out), int(blocking)))
        return out

    def fitness_dev(self, pop, dom, out, stream=None):
        """tgp_fitness_dev: RMSE into a device float64 buffer (torch tensor)."""
        self._check(self._L.tgp_fitness_dev(self._h, pop, dom, _stream(stream), _ptr(out)))

    def fitness_sse_dev(self, pop, dom, out, stream=None):
        """tgp_fitness_sse_dev: sums of squared residuals (binary64) into a
        device float64 buffer (torch tensor)."""
        self._check(self._L.tgp_fitness_sse_dev(self._h, pop, dom, _stream(stream), _ptr(out)))

    def fitness_graph(self, pop, dom, out, stream=None):
        """tgp_fitness_graph: RMSE into a device float64 buffer through a
        captured CUDA graph (captured on the first call, replayed after)."""
        self._check(self._L.tgp_fitness_graph(self._h, pop, dom, _stream(stream), _ptr(out)))

    def autotune(self, pop, dom, stream=None):
        """tgp_autotune: returns (K, groups, kernel ms) of the fastest shape."""
        k = ctypes.c_int32()
        g = ctypes.c_int32()
        ms = ctypes.c_double()
        self._check(self._L.tgp_autotune(self._h, pop, dom, _stream(stream), ctypes.byref(k), ctypes.byref(g),
                                         ctypes.byref(ms)))
        return k.value, g.value, ms.value

    def fitness_noalloc(self, pop, dom, out, stream=None):
        """tgp_fitness_noalloc: RMSE into a device float64 buffer without any
        device allocation by the library (fixed scratch; see include/tgp.h)."""
        self._check(self._L.tgp_fitness_noalloc(self._h, pop, dom, _stream(stream), _ptr(out)))

    def stats(self):
        s = Stats()
        self._check(self._L.tgp_stats_get(self._h, ctypes.byref(s)))
        return s.as_dict()

    def debug_plan(self, pop, n_points):
        """tgp_debug_plan: decoded bytecode [n, 6] int32 and group offsets."""
        n = ctypes.c_int64()
        g = ctypes.c_int32()
        self._check(self._L.tgp_debug_plan(self._h, pop, n_points, None, 0, ctypes.byref(n), None, 0,
                                           ctypes.byref(g)))
        ins = np.zeros((n.value, 6), np.int32)
        off = np.zeros(g.value + 1, np.int64)
        self._check(self._L.tgp_debug_plan(self._h, pop, n_points, _ptr(ins), n.value, ctypes.byref(n),
                                           _ptr(off), off.size, ctypes.byref(g)))
        return ins, off

    def calibrate_peak(self):
        """tgp_calibrate_peak: measured binary32 lane operations per second
        of straight-line add chains and of fused multiply-add chains."""
        a = ctypes.c_double()
        f = ctypes.c_double()
        self._check(self._L.tgp_calibrate_peak(self._h, ctypes.byref(a), ctypes.byref(f)))
        return a.value, f.value

    def plan_work(self, pop, dom):
        """tgp_plan_work: evaluations per operator the fitness launches plan
        ([N_OPS] float64), and the residuals formed at tree roots."""
        w = np.zeros(N_OPS + 1, np.float64)
        self._check(self._L.tgp_plan_work(self._h, pop, dom, _ptr(w)))
        return w[:N_OPS], float(w[N_OPS])

    def calibrate_op_costs(self):
        c = np.zeros(N_OPS, np.float64)
        self._check(self._L.tgp_calibrate_op_costs(self._h, _ptr(c)))
        return c


class Server:
    """tgp_server: a serving loop on a context (worker thread in the library).

    submit() queues a job (tokens scored on a grid against the Pagie target
    or a target tree) and returns its id; wait() returns its RMSE values and
    timeline.  Jobs on the same domain that wait together are fused into one
    launch; launches on different streams overlap on the device."""

    def __init__(self, ctx, streams=0, max_batch_trees=0, hbm_budget_bytes=0):
        self._L = lib()
        self.ctx = ctx
        cfg = ServerConfig()
        cfg.streams = streams
        cfg.max_batch_trees = max_batch_trees
        cfg.hbm_budget_bytes = hbm_budget_bytes
        h = ctypes.c_void_p()
        self._h = None
        ctx._check(self._L.tgp_server_create(ctx._h, ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._trees = {}

    def close(self):
        if self._h is not None:
            self._L.tgp_server_destroy(self._h)
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

    def submit(self, tok, W, H, xlo=-5.0, xhi=5.0, ylo=-5.0, yhi=5.0, target_tokens=None):
        """Queues a job; `tok` is an inputs.Tokens, `target_tokens` = (ops, imm, order) or None (Pagie)."""
        ops = np.ascontiguousarray(tok.ops, np.int32)
        imm = np.ascontiguousarray(tok.imm, np.float32)
        off = np.ascontiguousarray(tok.tree_off, np.int64)
        j = Job(ops.ctypes.data, imm.ctypes.data if imm.size else None, imm.size, off.ctypes.data,
                off.size - 1, tok.order, W, H, xlo, xhi, ylo, yhi, TARGET_PAGIE, None)
        keep = None
        if target_tokens is not None:
            t_ops, t_imm, t_order = target_tokens
            t_ops = np.ascontiguousarray(t_ops, np.int32)
            t_imm = np.ascontiguousarray(t_imm, np.float32)
            tt = TargetTokens(t_ops.ctypes.data, t_imm.ctypes.data if t_imm.size else None, t_ops.size,
                              t_imm.size, t_order)
            keep = (t_ops, t_imm, tt)
            j.target_kind = TARGET_TOKENS
            j.target_tokens = ctypes.cast(ctypes.pointer(tt), ctypes.c_void_p)
        out = ctypes.c_int64()
        self.ctx._check(self._L.tgp_server_submit(self._h, ctypes.byref(j), ctypes.byref(out)))
        del keep
        self._trees[out.value] = int(off.size - 1)
        return out.value

    def wait(self, job_id, timeout=None):
        """(rmse float64[n_trees], info dict); raises TgpError (E_TIMEOUT when not done in time)."""
        n = self._trees.get(job_id, 0)
        rmse = np.empty(max(n, 1), np.float64)
        info = JobInfo()
        us = -1 if timeout is None else int(timeout * 1e6)
        rc = self._L.tgp_server_wait(self._h, job_id, us, _ptr(rmse), ctypes.byref(info))
        if rc != E_TIMEOUT:
            self._trees.pop(job_id, None)
        self.ctx._check(rc)
        return rmse[:n], info.as_dict()

    def stats(self):
        s = ServerStats()
        self.ctx._check(self._L.tgp_server_stats_get(self._h, ctypes.byref(s)))
        return s.as_dict()


def debug_layout():
    out = np.zeros(2, np.int32)
    rc = lib().tgp_debug_layout(_ptr(out), 2)
    if rc != OK:
        raise TgpError(rc, "debug_layout")
    return {"n_opnd": int(out[0]), "n_forms": int(out[1])}
