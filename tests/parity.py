"""Element and fitness comparison of the CUDA path against the CPU oracle.

Element rule.  An element passes when |gpu - v64| <= 1e-4 * (1 + |v64|) (the
stated tolerance), or when |gpu - v64| <= E, where E is the oracle's forward
error bound for ANY binary32 evaluation of that tree at that point (correctly
rounded + - * / sqrt, sin/cos(pi a), exp, log within 2 ulp, tan within 4, pow
within 8; see oracle/tgp_oracle.c).  The second clause covers ill-conditioned
elements (e.g. a division by a difference of nearly equal values) that no
binary32 program can get within the fixed tolerance.  Excluded from the element
check, and counted: elements where a division saw |denominator| < 1e-6 (the
stated exclusion), elements whose bound is unbounded (undecided zero test of a
denominator or an if condition, a jump of sign/frac/mod within the bound, a
pole, binary32 overflow), and, when the FP32-faithful values are passed,
elements not finite in binary64 but finite in the FP32-faithful walk.
Otherwise, where v64 is not finite, the GPU value must not be finite either.

Fitness rule.  |gpu - r64| <= 1e-5 |r64| + R + 1e-6, where R = sqrt(mean E^2)
bounds the RMSE change caused by the element errors (triangle inequality in
the L2 norm) and 1e-6 absorbs binary32 round-off of exact fits.  Trees with an
unbounded element are not fitness-checked (counted).  Squared residuals are
summed in binary32 per warp, so +inf is accepted when N * r64^2 >= FLT_MAX / 2.
"""
from __future__ import annotations

import warnings

import numpy as np

ELEM_TOL = 1e-4
FIT_RTOL = 1e-5
FIT_ATOL = 1e-6
FLT_MAX = float(np.finfo(np.float32).max)


def close(a, b, tol=ELEM_TOL):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    with np.errstate(all="ignore"):
        same = (a == b) | (np.isnan(a) & np.isnan(b))
        near = np.abs(a - b) <= tol * (1.0 + np.abs(b))
    return same | near


def classify(gpu, v64, flags, bound, v32=None):
    """Masks and counts for arrays shaped [T, n].  With v32 (the oracle's
    FP32-faithful values), an element that is not finite in binary64 but
    finite in the FP32-faithful walk (a binary32 evaluation took another
    branch of an undecided test: an if condition, a sign, a pole) is excluded
    instead of requiring a non-finite device value."""
    g = np.asarray(gpu, np.float64)
    v64 = np.asarray(v64, np.float64)
    fin64 = np.isfinite(v64)
    unbounded = fin64 & ~np.isfinite(bound)
    excluded = np.asarray(flags, bool) | unbounded
    must_be_nonfinite = ~fin64
    if v32 is not None:
        diverged = ~fin64 & np.isfinite(np.asarray(v32, np.float64))
        excluded = excluded | diverged
        must_be_nonfinite = must_be_nonfinite & ~diverged
    with np.errstate(all="ignore"):
        by_tol = close(g, v64)
        by_bound = np.abs(g - v64) <= bound
    fail = (fin64 & ~excluded & ~(by_tol | by_bound)) | (must_be_nonfinite & np.isfinite(g))
    ill = fin64 & ~excluded & ~by_tol & by_bound
    return {
        "excluded": excluded, "ill": ill, "fail": fail,
        "n": int(g.size), "n_excluded": int(excluded.sum()), "n_unbounded": int(unbounded.sum()),
        "n_ill": int(ill.sum()), "n_fail": int(fail.sum()),
    }


def assert_elements(gpu, v64, flags, bound, context="", v32=None):
    c = classify(gpu, v64, flags, bound, v32)
    if c["n_fail"]:
        idx = np.argwhere(c["fail"])[:5]
        sel = tuple(idx.T)
        raise AssertionError(f"{context}: {c['n_fail']} of {c['n']} elements off "
                             f"(first {idx.tolist()}: gpu {np.asarray(gpu)[sel]} ref {np.asarray(v64)[sel]} "
                             f"bound {np.asarray(bound)[sel]})")
    return c


def assert_fitness(gpu, r64, rmse_err, n_points, context=""):
    gpu = np.asarray(gpu, np.float64)
    bad = []
    skipped = 0
    for t in range(gpu.size):
        g, ref, R = gpu[t], float(r64[t]), float(rmse_err[t])
        if not np.isfinite(R):
            skipped += 1
            continue
        if np.isinf(ref) or np.isinf(g):
            if np.isinf(ref) and np.isinf(g):
                continue
            if np.isinf(g) and n_points * ref * ref >= FLT_MAX / 2:
                continue
            bad.append((t, g, ref, R))
            continue
        if abs(g - ref) > FIT_RTOL * abs(ref) + R + FIT_ATOL:
            bad.append((t, g, ref, R))
    assert not bad, f"{context}: fitness off for {len(bad)} trees, first {bad[:5]}"
    if skipped:
        warnings.warn(f"{context}: {skipped} of {gpu.size} trees have an unbounded element; fitness not checked")
    return skipped


def assert_fitness_of_phenotype(gpu_fit, phenotype, target, trees, context="", rtol=1e-4):
    """For trees whose oracle fitness is not comparable (an unbounded element):
    the device RMSE against the binary64 RMSE of the device's own phenotype
    (checks the fused residual-and-reduction step on exactly those trees).
    rtol covers the binary32 target and the binary32 per-warp sums."""
    ref = rmse_of(np.asarray(phenotype)[trees], target)
    got = np.asarray(gpu_fit, np.float64)[trees]
    n = np.asarray(phenotype).shape[1]
    bad = []
    for t, g, r in zip(trees, got, ref):
        if np.isinf(r) or np.isinf(g):
            if not (np.isinf(g) and (np.isinf(r) or n * r * r >= FLT_MAX / 2)):
                bad.append((int(t), g, r))
        elif abs(g - r) > rtol * abs(r) + FIT_ATOL:
            bad.append((int(t), g, r))
    assert not bad, f"{context}: device fitness off its own phenotype for {len(bad)} trees, first {bad[:5]}"


def grid_target(g):
    """Eq. 1 in binary64 at the grid's binary32 points, flat in point order."""
    import oracle
    return np.array([oracle.pagie(*oracle.grid_point(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi, p)) for p in range(g.N)])


def oracle_fitness_chunk(args):
    """Worker for a spawn process pool: oracle fitness of one chunk of trees."""
    import oracle
    ops, imm, off, order, g, target = args
    return oracle.fitness(ops, imm, off, order, g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi, target=target,
                          with_bound=True)


def oracle_eval_chunk(args):
    """Worker for a spawn process pool: oracle phenotypes (with bounds) of one
    chunk of trees at the listed points (all points when pts is None)."""
    import oracle
    ops, imm, off, order, g, pts = args
    return oracle.evaluate(ops, imm, off, order, g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi, pts=pts,
                           with_bound=True)


def rmse_of(phenotype, target):
    """binary64 RMSE of each row of a phenotype against a target (+inf when not finite)."""
    ph = np.asarray(phenotype, np.float64)
    with np.errstate(all="ignore"):
        r = np.sqrt(np.mean((ph - np.asarray(target, np.float64)) ** 2, axis=1))
    return np.where(np.isfinite(r), r, np.inf)
