"""Element and fitness comparison of the CUDA path against the CPU oracle.

Tolerances (stated for the hot path): an element passes when
|gpu - ref64| <= 1e-4 * (1 + |ref64|); a fitness passes when
|gpu - ref| <= 1e-5 * |ref| (plus an absolute floor of 1e-6 for fits that are
exact in binary64, where only binary32 round-off remains).

Elements are classified first:
  * excluded: some division of the tree saw |denominator| < 1e-6 (oracle flag);
  * ill-conditioned: the oracle's own FP32-faithful value disagrees with its
    binary64 value beyond the element tolerance -- no binary32 program can
    match binary64 there; these are checked against the FP32-faithful value
    instead (same tolerance), and counted.
A tree with excluded or ill-conditioned elements has its fitness checked
against the oracle's FP32-faithful fitness.
"""
from __future__ import annotations

import numpy as np

ELEM_TOL = 1e-4
FIT_RTOL = 1e-5
FIT_ATOL = 1e-6


def close(a, b, tol=ELEM_TOL):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    with np.errstate(all="ignore"):
        same = (a == b) | (np.isnan(a) & np.isnan(b))
        near = np.abs(a - b) <= tol * (1.0 + np.abs(b))
    return same | near


def classify(gpu, v64, v32, flags):
    """Returns a dict of boolean masks and counts (arrays shaped [T, n])."""
    gpu = np.asarray(gpu, np.float32)
    excl = np.asarray(flags, bool)
    ill = ~close(v32, v64) & ~excl
    ok64 = close(gpu, v64)
    ok32 = close(gpu, v32)
    fail_well = ~excl & ~ill & ~ok64
    fail_ill = ill & ~ok32
    return {
        "excluded": excl, "ill": ill, "fail_well": fail_well, "fail_ill": fail_ill,
        "n": int(gpu.size), "n_excluded": int(excl.sum()), "n_ill": int(ill.sum()),
        "n_fail_well": int(fail_well.sum()), "n_fail_ill": int(fail_ill.sum()),
    }


def assert_elements(gpu, v64, v32, flags, max_ill_fail_frac=1e-3, context=""):
    c = classify(gpu, v64, v32, flags)
    if c["n_fail_well"]:
        idx = np.argwhere(c["fail_well"])[:5]
        raise AssertionError(f"{context}: {c['n_fail_well']} well-conditioned elements off "
                             f"(first {idx.tolist()}: gpu {np.asarray(gpu)[tuple(idx.T)]} "
                             f"ref {np.asarray(v64)[tuple(idx.T)]})")
    assert c["n_fail_ill"] <= max_ill_fail_frac * c["n"], \
        f"{context}: {c['n_fail_ill']} ill-conditioned elements off the FP32-faithful value"
    return c


FLT_MAX = float(np.finfo(np.float32).max)


def assert_fitness(gpu, r64, r32, tree_flagged, n_points, context=""):
    """tree_flagged[t]: tree t has excluded or ill-conditioned elements.

    Squared residuals are summed in binary32 per warp before the binary64
    reduction, so a tree whose squared-error sum exceeds FLT_MAX (a squared
    residual above FLT_MAX, or a warp's sum of them) may legitimately give +inf
    where binary64 stays finite; +inf is accepted exactly when the oracle's
    sum of squares N * rmse^2 is at least FLT_MAX / 2."""
    gpu = np.asarray(gpu, np.float64)
    bad = []
    for t in range(gpu.size):
        ref = r32[t] if tree_flagged[t] else r64[t]
        g = gpu[t]
        if np.isinf(ref) or np.isinf(g):
            # binary32 overflow of a squared residual turns a huge finite sum
            # into +inf; accept +inf when the reference sum is beyond FLT_MAX
            if np.isinf(ref) and np.isinf(g):
                continue
            if np.isinf(g) and n_points * float(r64[t]) ** 2 >= FLT_MAX / 2:
                continue
            bad.append((t, g, ref))
            continue
        if abs(g - ref) > FIT_RTOL * abs(ref) + FIT_ATOL:
            # a flagged tree may still match binary64
            if tree_flagged[t] and abs(g - r64[t]) <= FIT_RTOL * abs(r64[t]) + FIT_ATOL:
                continue
            bad.append((t, g, ref))
    assert not bad, f"{context}: fitness off for {len(bad)} trees, first {bad[:5]}"


def oracle_fitness_chunk(args):
    """Worker for a spawn process pool: oracle fitness of one chunk of trees."""
    import oracle
    ops, imm, off, order, g, target = args
    return oracle.fitness(ops, imm, off, order, g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi, target=target)
