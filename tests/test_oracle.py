"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value is a closed
form, an exact rational derived from Eq. 1, an independent numpy restatement of
a single operator, or brute force written separately in this file.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2103_07512_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def toks(*exprs, order=I.PREFIX):
    return I.to_tokens([I.parse_string(e) for e in exprs], order)


def ev(exprs, W, H, lo=-5.0, hi=5.0, order=I.PREFIX):
    t = toks(*exprs, order=order)
    return oracle.evaluate(t.ops, t.imm, t.tree_off, order, W, H, lo, hi, lo, hi)


def np_grid(W, H, lo=-5.0, hi=5.0):
    """Independent restatement of the binary32 grid reading: inclusive
    linspace, x along columns, y along rows, flat index row*W + col."""
    f = np.float32
    sx = (f(hi) - f(lo)) / f(W - 1) if W > 1 else f(0)
    sy = (f(hi) - f(lo)) / f(H - 1) if H > 1 else f(0)
    cols = np.arange(W, dtype=np.float32)
    rows = np.arange(H, dtype=np.float32)
    xs = f(lo) + cols * sx
    ys = f(lo) + rows * sy
    X = np.tile(xs, H).astype(np.float64)
    Y = np.repeat(ys, W).astype(np.float64)
    return X, Y


# ---------------------------------------------------------------- Eq. 1

def test_pagie_golden_points():
    rows = [l.split() for l in open(os.path.join(GOLD, "pagie_points.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) >= 8
    for x, y, num, den in rows:
        exp = float(Fraction(int(num), int(den)))
        got = oracle.pagie(float(x), float(y))
        assert got == pytest.approx(exp, rel=1e-15, abs=1e-15), (x, y)


def test_pagie_symmetry_and_limit():
    for x, y in [(0.3, -2.0), (4.0, 1.5)]:
        assert oracle.pagie(x, y) == oracle.pagie(-x, y) == oracle.pagie(y, x)
    assert oracle.pagie(1e6, 1e6) == pytest.approx(2.0, rel=1e-12)


# ---------------------------------------------------------------- grid

@pytest.mark.parametrize("W,H", [(1, 1), (2, 3), (7, 5), (64, 64), (33, 17)])
def test_grid_matches_binary32_linspace(W, H):
    X, Y = np_grid(W, H)
    for p in range(W * H):
        x, y = oracle.grid_point(W, H, -5.0, 5.0, -5.0, 5.0, p)
        assert (x, y) == (X[p], Y[p])
    # endpoints: first column / row is exactly lo
    assert oracle.grid_point(W, H, -5.0, 5.0, -5.0, 5.0, 0) == (-5.0, -5.0)


def test_grid_endpoints_close_to_hi():
    x, y = oracle.grid_point(64, 64, -5.0, 5.0, -5.0, 5.0, 64 * 64 - 1)
    assert abs(x - 5.0) < 1e-5 and abs(y - 5.0) < 1e-5


# ---------------------------------------------------------------- closed forms

def test_x_plus_y_and_x_times_x():
    W, H = 7, 5
    X, Y = np_grid(W, H)
    v64, v32, fl = ev(["add(x, y)", "mult(x, x)", "x", "y", "sub(x, y)"], W, H)
    assert np.array_equal(v64[0], X + Y)
    assert np.array_equal(v64[1], X * X)
    assert np.array_equal(v64[2], X)
    assert np.array_equal(v64[3], Y)
    assert np.array_equal(v64[4], X - Y)
    assert not fl.any()
    # FP32-faithful values are the binary32 roundings of single IEEE ops
    f = np.float32
    assert np.array_equal(v32[0], (X.astype(f) + Y.astype(f)))
    assert np.array_equal(v32[1], (X.astype(f) * X.astype(f)))


PAGIE_TREE = ("add(div(mult(mult(x, x), mult(x, x)), add(1.0, mult(mult(x, x), mult(x, x)))),"
              " div(mult(mult(y, y), mult(y, y)), add(1.0, mult(mult(y, y), mult(y, y)))))")


def test_pagie_as_tree_has_zero_rmse():
    t = toks(PAGIE_TREE)
    r64, r32, nf = oracle.fitness(t.ops, t.imm, t.tree_off, 0, 64, 64, -5, 5, -5, 5)
    assert r64[0] < 1e-15
    assert r32[0] < 1e-6  # binary32 roundoff only
    assert nf[0] == 0


def test_rmse_of_zero_tree_is_rms_of_target():
    W, H = 33, 17
    t = toks("sub(x, x)")
    r64, _, _ = oracle.fitness(t.ops, t.imm, t.tree_off, 0, W, H, -5, 5, -5, 5)
    X, Y = np_grid(W, H)
    P = X ** 4 / (1 + X ** 4) + Y ** 4 / (1 + Y ** 4)
    assert r64[0] == pytest.approx(math.sqrt(np.mean(P ** 2)), rel=1e-14)


def test_rmse_by_hand_on_2x2_grid():
    # grid 2x2 over [-5,5]: points (+-5, +-5); P = 2*625/626 at all four
    a = Fraction(625, 313)
    t = toks("x", "add(x, y)", "0.5")
    r64, _, _ = oracle.fitness(t.ops, t.imm, t.tree_off, 0, 2, 2, -5, 5, -5, 5)
    ex = math.sqrt(float(((Fraction(-5) - a) ** 2 + (Fraction(5) - a) ** 2) / 2))
    exy = math.sqrt(float(((Fraction(-10) - a) ** 2 + 2 * a ** 2 + (Fraction(10) - a) ** 2) / 4))
    ec = math.sqrt(float((Fraction(1, 2) - a) ** 2))
    assert r64[0] == pytest.approx(ex, rel=1e-15)
    assert r64[1] == pytest.approx(exy, rel=1e-15)
    assert r64[2] == pytest.approx(ec, rel=1e-15)


def test_rmse_against_given_values_divides_by_n():
    W, H = 3, 2
    target = np.arange(6, dtype=np.float64)
    t = toks("0.0")
    r64, _, _ = oracle.fitness(t.ops, t.imm, t.tree_off, 0, W, H, -5, 5, -5, 5, target=target)
    assert r64[0] == pytest.approx(math.sqrt(sum(v * v for v in range(6)) / 6), rel=1e-15)


def test_nonfinite_fitness_is_inf():
    # x^1024 by repeated squaring: 5^1024 overflows binary64 (and binary32)
    e = "0.9"
    big = "mult(mult(x, x), mult(x, x))"
    for _ in range(8):
        big = f"mult({big}, {big})"
    t = toks(big, e, f"sin({big})")
    r64, r32, _ = oracle.fitness(t.ops, t.imm, t.tree_off, 0, 4, 4, -5, 5, -5, 5)
    assert math.isinf(r64[0]) and math.isinf(r32[0])
    assert math.isfinite(r64[1])
    # sin(pi * inf) is NaN; a NaN phenotype also gives fitness +inf
    assert r64[2] == math.inf and r32[2] == math.inf


# ---------------------------------------------------------------- operators

def test_trig_is_pi_scaled_special_values():
    # Sec. 3.2: argument multiplied by pi
    assert oracle.sinpi(0.5) == 1.0
    assert oracle.cospi(1.0) == -1.0
    assert oracle.sinpi(1.0) == 0.0
    assert oracle.cospi(0.5) == 0.0
    assert oracle.sinpi(-0.5) == -1.0
    assert oracle.sinpi(2.5) == 1.0
    assert oracle.cospi(-3.0) == -1.0
    assert oracle.sinpi(1e7 + 0.5) == 1.0


def test_trig_against_numpy_for_moderate_arguments():
    a = np.linspace(-7.3, 7.3, 1001)
    s = np.array([oracle.sinpi(v) for v in a])
    c = np.array([oracle.cospi(v) for v in a])
    assert np.allclose(s, np.sin(np.pi * a), rtol=0, atol=1e-14)
    assert np.allclose(c, np.cos(np.pi * a), rtol=0, atol=1e-14)
    # not the unscaled (radian) functions, and not swapped (Table 1 typo)
    assert not np.allclose(s, np.sin(a), atol=1e-3)
    assert not np.allclose(s, np.cos(np.pi * a), atol=1e-3)


def test_trig_periodicity_and_parity():
    for a in [0.1, 0.37, 1.9, 3.25]:
        assert oracle.sinpi(a + 2) == pytest.approx(oracle.sinpi(a), abs=1e-14)
        assert oracle.sinpi(-a) == -oracle.sinpi(a)
        assert oracle.cospi(-a) == oracle.cospi(a)
        assert oracle.sinpi(a) ** 2 + oracle.cospi(a) ** 2 == pytest.approx(1.0, abs=1e-15)


def test_special_trees():
    W, H = 7, 5
    X, Y = np_grid(W, H)
    v64, _, fl = ev(["sin(0.5)", "cos(1.0)", "div(x, sub(y, y))", "neg(neg(x))", "abs(neg(x))",
                     "min(x, y)", "max(x, y)", "div(x, y)", "neg(x)", "cos(x)"], W, H)
    assert np.all(v64[0] == 1.0)
    assert np.all(v64[1] == -1.0)
    assert np.all(v64[2] == 0.0)        # protected division
    assert fl[2].all()                   # denominator 0 is flagged near-singular
    assert np.array_equal(v64[3], X)
    assert np.array_equal(v64[4], np.abs(X))
    assert np.array_equal(v64[5], np.minimum(X, Y))
    assert np.array_equal(v64[6], np.maximum(X, Y))
    with np.errstate(divide="ignore", invalid="ignore"):
        q = np.where(Y == 0, 0.0, X / Y)
    assert np.array_equal(v64[7], q)
    assert np.array_equal(v64[8], -X)
    assert np.allclose(v64[9], np.cos(np.pi * X), atol=2e-15, rtol=0)


def test_protected_division_negative_zero():
    # sub(x, x) is +0; neg of it is -0: both are zero denominators
    v64, v32, _ = ev(["div(1.0, neg(sub(x, x)))", "div(0.25, mult(x, 0.0))"], 3, 3)
    assert np.all(v64 == 0.0) and np.all(v32 == 0.0)


def test_near_singular_flag():
    # denominator x - c where c is 1e-7 away from a grid coordinate
    W, H = 3, 1   # x in {-5, 0, 5}
    v64, _, fl = ev(["div(1.0, sub(x, 1e-7))", "div(1.0, sub(x, 1e-3))", "add(x, 1e-9)"], W, H)
    assert fl[0].tolist() == [False, True, False]
    assert not fl[1].any() and not fl[2].any()


# ---------------------------------------------------------------- FP32-faithful

def test_fp32_faithful_single_ops_equal_numpy_binary32():
    rng = np.random.default_rng(5)
    W, H = 16, 8
    X, Y = np_grid(W, H)
    f = np.float32
    x32, y32 = X.astype(f), Y.astype(f)
    c = f(rng.uniform(-1, 1))
    cs = repr(float(c))
    v64, v32, _ = ev([f"add(x, {cs})", f"sub({cs}, y)", f"mult(x, y)", f"div(x, {cs})",
                      "min(x, y)", "max(x, neg(y))", "abs(sub(x, y))"], W, H)
    with np.errstate(all="ignore"):
        exp = [x32 + c, c - y32, x32 * y32, x32 / c, np.minimum(x32, y32),
               np.maximum(x32, -y32), np.abs(x32 - y32)]
    for i, e in enumerate(exp):
        assert np.array_equal(v32[i], e), i


def test_fp32_faithful_rounds_every_node():
    # (x*c1)*c2 in binary32 differs from x*(c1*c2) rounded once for some x
    W, H = 64, 1
    v64, v32, _ = ev(["mult(mult(x, 0.1), 0.3)"], W, H)
    X, _ = np_grid(W, H)
    f = np.float32
    assert np.array_equal(v32[0], (X.astype(f) * f(0.1)) * f(0.3))


# ---------------------------------------------------------------- encodings

def test_prefix_equals_postfix_on_random_population():
    tok, g = I.small_population(seed=0)
    post = I.convert_order(tok, I.POSTFIX)
    assert not np.array_equal(tok.ops, post.ops)
    a = oracle.evaluate(tok.ops, tok.imm, tok.tree_off, I.PREFIX, 9, 7, -5, 5, -5, 5)
    b = oracle.evaluate(post.ops, post.imm, post.tree_off, I.POSTFIX, 9, 7, -5, 5, -5, 5)
    for u, v in zip(a, b):
        assert np.array_equal(u, v, equal_nan=True)


def test_duplicate_and_permuted_trees_keep_fitness():
    tok, g = I.small_population(seed=3)
    trees = I.from_tokens(tok)
    perm = list(reversed(trees)) + trees[:5]
    t2 = I.to_tokens(perm)
    r1, _, _ = oracle.fitness(tok.ops, tok.imm, tok.tree_off, 0, 16, 16, -5, 5, -5, 5)
    r2, _, _ = oracle.fitness(t2.ops, t2.imm, t2.tree_off, 0, 16, 16, -5, 5, -5, 5)
    assert np.array_equal(r2[:len(trees)], r1[::-1])
    assert np.array_equal(r2[len(trees):], r1[:5])


def test_malformed_tokens_are_rejected():
    cases = [
        ([3, 0], [], [0, 2]),            # add with one operand
        ([0, 1], [], [0, 2]),            # two terminals
        ([42], [], [0, 1]),              # unknown opcode
        ([2], [], [0, 1]),               # CONST without imm
        ([0], [1.0], [0, 1]),            # imm left over
    ]
    for ops, imm, off in cases:
        with pytest.raises(oracle.OracleError):
            oracle.evaluate(np.array(ops), np.array(imm, np.float32), np.array(off), 0, 2, 2, -1, 1, -1, 1)


# ---------------------------------------------------------------- brute force

def _all_trees(depth):
    """Every tree of depth <= depth over {x, y, 0.5} and the 10 functions."""
    leaves = ["x", "y", "0.5"]
    if depth == 0:
        return leaves
    sub = _all_trees(depth - 1)
    out = list(leaves)
    for f in ["sin", "cos", "neg", "abs"]:
        out += [f"{f}({a})" for a in sub]
    for f in ["add", "sub", "mult", "div", "min", "max"]:
        out += [f"{f}({a}, {b})" for a in sub for b in sub]
    return out


def _np_eval(tree, X, Y, sing):
    """Direct numpy binary64 evaluation of a tuple tree (independent of the
    oracle: numpy ufuncs, pi-scaled trig through np.sin(np.pi * a)).  sing is
    OR-ed with the points where a division saw |denominator| < 1e-6 (there the
    inexact numpy trig may turn an exact zero denominator into a tiny one)."""
    op, v, kids = tree
    if op == I.X:
        return X
    if op == I.Y:
        return Y
    if op == I.CONST:
        return np.full_like(X, float(v))
    a = _np_eval(kids[0], X, Y, sing)
    b = _np_eval(kids[1], X, Y, sing) if len(kids) > 1 else None
    if op == I.DIV:
        sing |= np.abs(b) < 1e-6
    with np.errstate(all="ignore"):
        return {
            I.ADD: lambda: a + b, I.SUB: lambda: a - b, I.MUL: lambda: a * b,
            I.DIV: lambda: np.where(b == 0, 0.0, a / np.where(b == 0, 1.0, b)),
            I.SIN: lambda: np.sin(np.pi * a), I.COS: lambda: np.cos(np.pi * a),
            I.NEG: lambda: -a, I.ABS: lambda: np.abs(a),
            I.MIN: lambda: np.fmin(a, b), I.MAX: lambda: np.fmax(a, b),
        }[op]()


@pytest.mark.parametrize("W,H", [(1, 1), (2, 2), (3, 5)])
def test_brute_force_depth2_trees(W, H):
    exprs = _all_trees(2)
    assert len(exprs) > 1000
    trees = [I.parse_string(e) for e in exprs]
    tok = I.to_tokens(trees)
    v64, _, fl = oracle.evaluate(tok.ops, tok.imm, tok.tree_off, 0, W, H, -5, 5, -5, 5)
    X, Y = np_grid(W, H)
    sing = np.zeros((len(trees), W * H), bool)
    exp = np.stack([_np_eval(t, X, Y, sing[i]) for i, t in enumerate(trees)])
    ok = ~(sing | fl)
    assert ok.mean() > 0.9
    # trig: numpy's sin(pi*a) carries ~1e-15 absolute error that the exact
    # reduction avoids; everything else is identical
    assert np.allclose(v64[ok], exp[ok], rtol=1e-13, atol=1e-13, equal_nan=True)
    # trees without any division agree on every point
    nodiv = np.array(["div" not in e for e in exprs])
    assert np.allclose(v64[nodiv], exp[nodiv], rtol=1e-13, atol=1e-13, equal_nan=True)
    r64, _, _ = oracle.fitness(tok.ops, tok.imm, tok.tree_off, 0, W, H, -5, 5, -5, 5)
    P = X ** 4 / (1 + X ** 4) + Y ** 4 / (1 + Y ** 4)
    with np.errstate(all="ignore"):
        re = np.sqrt(np.mean((exp - P) ** 2, axis=1))
    re = np.where(np.isfinite(re), re, np.inf)
    clean = ok.all(axis=1)
    assert np.allclose(r64[clean], re[clean], rtol=1e-12, atol=1e-13)


def test_golden_regression_small_population():
    """Config-1 fitness written by tests/golden/make_golden.py (oracle only);
    guards the oracle against unintended changes."""
    path = os.path.join(GOLD, "small_population_rmse.txt")
    exp = np.loadtxt(path)
    tok, g = I.small_population(seed=0)
    r64, _, _ = oracle.fitness(tok.ops, tok.imm, tok.tree_off, 0, g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi)
    assert np.allclose(r64, exp, rtol=1e-12, atol=0, equal_nan=False)


# ---------------------------------------------------------------- error bound

U32 = 2.0 ** -24


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_error_bound_contains_fp32_faithful_evaluation(seed):
    """The FP32-faithful walk is one binary32 evaluation with correctly rounded
    operators, so it must lie within the bound of the binary64 value."""
    pops = [I.small_population(seed=seed)[0]]
    rng = np.random.default_rng(seed)
    trees, _ = I.exact_size_population(60, 3, 255, 12, 0.3, rng)
    pops.append(I.to_tokens(trees))
    pops.append(I.to_tokens([I._full(rng, 8, I.FUNCTIONS) for _ in range(6)]))
    for tok in pops:
        v64, v32, fl, eb = oracle.evaluate(tok.ops, tok.imm, tok.tree_off, 0, 23, 19, -5, 5, -5, 5,
                                           with_bound=True)
        m = np.isfinite(v64) & np.isfinite(eb)
        d = np.abs(v32.astype(np.float64) - v64)
        assert np.all(d[m] <= eb[m])
        assert m.mean() > 0.8
        # tight: the bound is not vacuous on the elements that round
        assert np.nanmax(np.where(m & (eb > 0), d / np.where(eb > 0, eb, 1), 0)) > 0.05
        r64, r32, _, re = oracle.fitness(tok.ops, tok.imm, tok.tree_off, 0, 23, 19, -5, 5, -5, 5,
                                         with_bound=True)
        f = np.isfinite(re) & np.isfinite(r64)
        assert np.all(np.abs(r32[f] - r64[f]) <= re[f] * (1 + 1e-12))


def test_error_bound_closed_forms():
    W, H = 7, 5
    X, Y = np_grid(W, H)
    v64, _, _, eb = ev_bound(["x", "0.5", "add(x, y)", "mult(x, y)", "neg(abs(x))", "min(x, y)",
                              "div(x, sub(y, y))"], W, H)
    assert np.all(eb[0] == 0) and np.all(eb[1] == 0)
    assert np.allclose(eb[2], U32 * np.abs(X + Y), rtol=1e-15, atol=0)
    assert np.allclose(eb[3], U32 * np.abs(X * Y) + np.where(X * Y == 0, 0, 0), rtol=1e-15, atol=0)
    assert np.all(eb[4] == 0) and np.all(eb[5] == 0)
    assert np.all(eb[6] == 0)          # exact zero denominator: protected result is exactly 0


def test_error_bound_trig_and_division():
    W, H = 5, 3
    X, Y = np_grid(W, H)
    _, _, _, eb = ev_bound(["sin(x)", "sin(add(x, y))", "div(1.0, add(x, 0.3))"], W, H)
    # exact argument: only the 2-ulp allowance of the function
    assert np.all(eb[0] <= 2 * (2 * U32 * np.abs(np.sin(np.pi * X)) + 2.0 ** -149) * (1 + 1e-12))
    # rounded argument: pi |cos(pi a)| E(arg) is propagated
    assert np.all(eb[1] >= np.pi * U32 * np.abs(X + Y) * np.abs(np.cos(np.pi * (X + Y))) * (1 - 1e-12))
    b = X + np.float32(0.3).astype(np.float64)
    exp = (1.0 * U32 * np.abs(b) / np.abs(b) ** 2) / (1 - U32)   # Eb/|b|^2 leading term
    assert np.all(eb[2] >= exp * 0.99)


def test_error_bound_unbounded_cases():
    _, _, _, eb = ev_bound(["div(1.0, sub(mult(x, 0.1), mult(0.1, x)))", "mult(x, 1e30)",
                            "mult(mult(x, 1e30), mult(x, 1e30))"], 3, 3)
    # undecided zero test of the denominator
    assert np.all(~np.isfinite(eb[0][[0, 2, 6, 8]]))
    assert np.all(np.isfinite(eb[1]))
    # binary32 overflow
    assert np.all(~np.isfinite(eb[2][[0, 2, 6, 8]]))


def _hulp(r):
    """Half the binary32 spacing at |r| (normal range): the largest error of
    one correctly rounded binary32 operation whose exact result is r."""
    m, e = np.frexp(np.abs(np.asarray(r, np.float64)))
    return np.ldexp(1.0, e - 25)


# first-order worst case of a binary32 evaluation of each one- and
# two-operator tree, written from the derivatives of the tree (each rounding
# at most half an ulp, sin/cos(pi a) at most 2 ulp): (expression, worst case,
# mask of the elements where it applies)
def _worst_cases(X, Y):
    pi = np.pi
    s, p, d, q = X + Y, X * Y, X - Y, X / Y
    sx, cy = np.sin(pi * X), np.cos(pi * Y)
    c03 = float(np.float32(0.3))
    with np.errstate(all="ignore"):
        cases = [
            ("add(x, y)", _hulp(s), np.ones_like(s, bool)),
            ("sub(x, y)", _hulp(d), np.ones_like(s, bool)),
            ("mult(x, y)", _hulp(p), np.ones_like(s, bool)),
            ("div(x, y)", _hulp(q), np.abs(Y) > 1e-3),
            ("add(x, 0.3)", _hulp(X + c03), np.ones_like(s, bool)),
            ("sin(x)", 4 * _hulp(sx), np.ones_like(s, bool)),
            ("cos(y)", 4 * _hulp(cy), np.ones_like(s, bool)),
            ("neg(add(x, y))", _hulp(s), np.ones_like(s, bool)),
            ("abs(sub(x, y))", _hulp(d), np.ones_like(s, bool)),
            ("sin(add(x, y))", pi * np.abs(np.cos(pi * s)) * _hulp(s) + 4 * _hulp(np.sin(pi * s)),
             np.ones_like(s, bool)),
            ("cos(mult(x, y))", pi * np.abs(np.sin(pi * p)) * _hulp(p) + 4 * _hulp(np.cos(pi * p)),
             np.ones_like(s, bool)),
            ("mult(add(x, y), x)", np.abs(X) * _hulp(s) + _hulp(s * X), np.ones_like(s, bool)),
            ("div(x, add(x, y))", np.abs(X / s ** 2) * _hulp(s) + _hulp(X / s), np.abs(s) > 1e-3),
            ("sub(sin(x), y)", 4 * _hulp(sx) + _hulp(sx - Y), np.ones_like(s, bool)),
            ("add(mult(x, x), y)", _hulp(X * X) + _hulp(X * X + Y), np.ones_like(s, bool)),
            ("div(sin(x), y)", 4 * _hulp(sx) / np.abs(Y) + _hulp(sx / Y), np.abs(Y) > 1e-3),
            ("mult(sin(x), cos(y))", np.abs(cy) * 4 * _hulp(sx) + np.abs(sx) * 4 * _hulp(cy) + _hulp(sx * cy),
             np.ones_like(s, bool)),
            # the comparison decided with a margin: the taken operand's error
            ("min(add(x, y), mult(x, y))", np.where(s < p, _hulp(s), _hulp(p)),
             np.abs(s - p) > 4 * 2.0 ** -24 * (np.abs(s) + np.abs(p))),
            ("max(sin(x), cos(y))", np.where(sx > cy, 4 * _hulp(sx), 4 * _hulp(cy)),
             np.abs(sx - cy) > 16 * 2.0 ** -24 * (np.abs(sx) + np.abs(cy))),
        ]
    return cases


@pytest.mark.parametrize("W,H,lo,hi", [(37, 29, -5.0, 5.0), (23, 31, -0.9, 0.9), (16, 16, -3.0, 1.75)])
def test_error_bound_is_tight_on_one_and_two_operator_trees(W, H, lo, hi):
    """The bound is no looser than twice the first-order worst case of a
    binary32 evaluation of the tree, and no tighter than it (each term of the
    bound is at least the matching worst-case term and below twice it)."""
    X, Y = np_grid(W, H, lo, hi)
    cases = _worst_cases(X, Y)
    v64, _, _, eb = ev_bound([c[0] for c in cases], W, H, lo, hi)
    for i, (expr, worst, mask) in enumerate(cases):
        m = mask & np.isfinite(eb[i]) & (np.abs(v64[i]) > 1e-30) & (worst > 0)
        # exact zeros of sin/cos(pi a) at integer or half-integer arguments have no ulp
        m &= np.abs(X) > 0
        assert m.mean() > 0.5, expr
        ratio = eb[i][m] / worst[m]
        assert ratio.min() >= 1 - 1e-6, (expr, ratio.min())
        assert ratio.max() <= 2 + 1e-4, (expr, ratio.max())


def ev_bound(exprs, W, H, lo=-5.0, hi=5.0):
    t = toks(*exprs)
    return oracle.evaluate(t.ops, t.imm, t.tree_off, 0, W, H, lo, hi, lo, hi, with_bound=True)


# ---------------------------------------------------------------- the rest of Table 1

def _scalar(expr):
    """binary64 value of a constant expression (1x1 grid)."""
    v64, _, _ = ev([expr], 1, 1)
    return float(v64[0, 0])


@pytest.mark.parametrize("expr,value", [
    ("tan(0.25)", 1.0), ("tan(-0.25)", -1.0), ("tan(0.0)", 0.0), ("tan(1.0)", 0.0),
    ("exp(0.0)", 1.0), ("exp(1.0)", math.e), ("exp(-2.0)", math.exp(-2.0)),
    ("log(1.0)", 0.0), ("log(-3.0)", -1.0), ("log(-0.5)", -1.0), ("log(0.5)", -math.log(2.0)),
    ("pow(0.0, 0.0)", 0.0), ("pow(2.0, 3.0)", 8.0), ("pow(-2.0, 3.0)", -8.0), ("pow(4.0, 0.5)", 2.0),
    ("pow(0.0, 2.0)", 0.0), ("pow(3.0, 0.0)", 1.0),
    ("mdist(1.0, 2.0)", 1.5), ("mdist(-3.0, 3.0)", 0.0),
    ("sqrt(9.0)", 3.0), ("sqrt(-4.0)", 0.0), ("sqrt(0.0)", 0.0), ("sqrt(2.0)", math.sqrt(2.0)),
    ("sign(-2.5)", -1.0), ("sign(0.0)", 0.0), ("sign(3.0)", 1.0), ("sign(-0.0)", 0.0),
    ("clip(5.0, 0.0, 1.0)", 1.0), ("clip(-5.0, 0.0, 1.0)", 0.0), ("clip(0.25, 0.0, 1.0)", 0.25),
    ("clip(0.5, 1.0, 0.0)", 1.0),          # max(min(z, x), y) with y > z gives y
    ("mod(5.0, 3.0)", 2.0), ("mod(-5.0, 3.0)", 1.0), ("mod(5.0, -3.0)", -1.0), ("mod(-5.0, -3.0)", -2.0),
    ("mod(5.5, 2.0)", 1.5), ("mod(6.0, 3.0)", 0.0), ("mod(-0.5, 1.0)", 0.5),
    ("frac(2.25)", 0.25), ("frac(-2.25)", 0.75), ("frac(3.0)", 0.0), ("frac(-3.0)", 0.0),
    ("if(0.0, 1.0, 2.0)", 2.0), ("if(-0.0, 1.0, 2.0)", 2.0), ("if(3.0, 1.0, 2.0)", 1.0),
    ("if(-1e-30, 1.0, 2.0)", 1.0),
])
def test_table1_operators_special_values(expr, value):
    assert _scalar(expr) == pytest.approx(value, rel=1e-15, abs=1e-15), expr


def test_table1_operators_nonfinite_cases():
    assert math.isinf(_scalar("tan(0.5)"))                       # cos(pi/2) is exactly 0
    assert _scalar("log(0.0)") == -math.inf
    assert math.isnan(_scalar("pow(-8.0, 0.5)"))
    assert math.isnan(_scalar("mod(1.0, 0.0)"))
    assert _scalar("if(div(1.0, 0.0), 1.0, 2.0)") == 2.0          # protected 1/0 = 0 is false
    assert math.isnan(_scalar("sign(mod(1.0, 0.0))"))


def test_frac_equals_mod_one_and_clip_identities():
    W, H = 9, 7
    v64, _, _ = ev(["frac(mult(x, 1.3))", "mod(mult(x, 1.3), 1.0)", "clip(x, -1.0, 1.0)",
                    "max(min(1.0, x), -1.0)", "if(sub(x, y), x, y)"], W, H)
    assert np.array_equal(v64[0], v64[1])
    assert np.array_equal(v64[2], v64[3])
    X, Y = np_grid(W, H)
    assert np.array_equal(v64[4], np.where(X - Y != 0, X, Y))


_EXT_LEAVES = ["x", "y", "0.5"]


def _ext_np(tree, X, Y):
    """Independent numpy binary64 restatement of every Table 1 operator."""
    op, v, kids = tree
    if op == I.X:
        return X
    if op == I.Y:
        return Y
    if op == I.CONST:
        return np.full_like(X, float(v))
    k = [_ext_np(c, X, Y) for c in kids]
    a = k[0]
    b = k[1] if len(k) > 1 else None
    c = k[2] if len(k) > 2 else None
    with np.errstate(all="ignore"):
        if op == I.TAN:
            return np.tan(np.pi * a)
        if op == I.EXP:
            return np.exp(a)
        if op == I.LOG:
            return np.where(a < 0, -1.0, np.log(np.where(a < 0, 1.0, a)))
        if op == I.POW:
            return np.where((a == 0) & (b == 0), 0.0, np.power(a, b))
        if op == I.MDIST:
            return (a + b) / 2
        if op == I.SQRT:
            return np.where(a < 0, 0.0, np.sqrt(np.where(a < 0, 0.0, a)))
        if op == I.SIGN:
            return np.sign(a)
        if op == I.CLIP:
            return np.fmax(np.fmin(c, a), b)
        if op == I.MOD:
            return np.mod(a, b)          # numpy's floored remainder
        if op == I.FRAC:
            return a - np.floor(a)
        if op == I.IF:
            return np.where(a != 0, b, c)
        if op == I.SIN:
            return np.sin(np.pi * a)
        if op == I.COS:
            return np.cos(np.pi * a)
        if op == I.NEG:
            return -a
        if op == I.ABS:
            return np.abs(a)
        return {I.ADD: a + b if b is not None else None, I.SUB: a - b if b is not None else None,
                I.MUL: a * b if b is not None else None,
                I.MIN: np.fmin(a, b) if b is not None else None,
                I.MAX: np.fmax(a, b) if b is not None else None}[op]


@pytest.mark.parametrize("W,H", [(2, 2), (3, 5)])
def test_brute_force_new_operators_depth2(W, H):
    """Every tree of depth <= 2 with one new operator at the root over the
    depth-1 trees of {x, y, 0.5} and {neg, sin}; against numpy."""
    sub1 = _EXT_LEAVES + [f"{f}({a})" for f in ("neg", "sin") for a in _EXT_LEAVES]
    exprs = []
    for f in ("tan", "exp", "log", "sqrt", "sign", "frac"):
        exprs += [f"{f}({a})" for a in sub1]
    for f in ("pow", "mdist", "mod"):
        exprs += [f"{f}({a}, {b})" for a in sub1 for b in sub1]
    for f in ("clip", "if"):
        exprs += [f"{f}({a}, {b}, {c})" for a in sub1[:5] for b in sub1[:5] for c in sub1[:5]]
    trees = [I.parse_string(e) for e in exprs]
    tok = I.to_tokens(trees)
    v64, _, _ = oracle.evaluate(tok.ops, tok.imm, tok.tree_off, 0, W, H, -5, 5, -5, 5)
    X, Y = np_grid(W, H)
    exp = np.stack([_ext_np(t, X, Y) for t in trees])
    # numpy's sin(pi*a) is not exactly 0 at integers (the oracle's is), which
    # operators that are steep or discontinuous at 0 (tan poles, log, sqrt,
    # pow, sign, frac, mod, the zero test of if) amplify: those trees are
    # compared on the other trees' tolerance only in aggregate
    fin = np.isfinite(exp) & np.isfinite(v64)
    close = np.isclose(v64, exp, rtol=1e-9, atol=1e-9)
    steep = ("tan", "frac", "mod", "sign", "if", "log", "sqrt", "pow")
    sens = np.array([e.split("(")[0] in steep and "sin" in e for e in exprs])
    assert close[fin & ~sens[:, None]].all()
    assert close[fin].mean() > 0.97
    assert fin.mean() > 0.8


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_error_bound_contains_fp32_faithful_new_operators(seed):
    rng = np.random.default_rng(seed)
    trees = [I._full(rng, int(rng.integers(2, 6)), I.ALL_FUNCTIONS) for _ in range(60)]
    tok = I.to_tokens(trees)
    v64, v32, fl, eb = oracle.evaluate(tok.ops, tok.imm, tok.tree_off, 0, 17, 13, -5, 5, -5, 5,
                                       with_bound=True)
    m = np.isfinite(v64) & np.isfinite(eb)
    with np.errstate(invalid="ignore"):
        d = np.abs(v32.astype(np.float64) - v64)
    assert np.all(d[m] <= eb[m])
    assert m.mean() > 0.5


def test_error_bound_new_operators_closed_forms():
    W, H = 7, 5
    X, Y = np_grid(W, H)
    _, _, _, eb = ev_bound(["sqrt(abs(x))", "sign(x)", "clip(x, y, 0.5)", "if(x, y, 0.5)",
                            "frac(x)", "mdist(x, y)", "exp(0.0)", "sign(sub(x, mult(x, 1.1)))"], W, H)
    assert np.all(eb[0] <= U32 * np.sqrt(np.abs(X)) * (1 + 1e-12) + 2.0 ** -150)   # exact operand
    assert np.all(eb[1] == 0) and np.all(eb[2] == 0) and np.all(eb[3] == 0)
    assert np.all(eb[4] <= U32 * np.abs(X - np.floor(X)) * (1 + 1e-12))
    assert np.all(eb[5] <= U32 * np.abs((X + Y) / 2) * (1 + 1e-12) + 2.0 ** -150)
    assert np.all(eb[6] <= 2 * (2 * U32 + 2.0 ** -149) * (1 + 1e-12))
    # sign of a rounded value: undecided only where it is within its bound of 0
    assert np.all(np.isfinite(eb[7][X != 0]))


# ------------------------------------------------ radians (Table 1 footnote)

def ev_rad(exprs, W, H, lo=-5.0, hi=5.0, with_bound=False):
    t = toks(*exprs)
    return oracle.evaluate(t.ops, t.imm, t.tree_off, 0, W, H, lo, hi, lo, hi, with_bound=with_bound, trig="rad")


def test_radian_trig_is_the_library_function_of_the_argument():
    W, H = 9, 4
    X, Y = np_grid(W, H)
    v64, v32, _ = ev_rad(["sin(x)", "cos(y)", "tan(x)", "sin(0.5)", "cos(3.0)"], W, H)
    assert np.array_equal(v64[0], np.sin(X)) and np.array_equal(v64[1], np.cos(Y))
    assert np.allclose(v64[2], np.tan(X), rtol=1e-15, atol=0)
    assert np.all(v64[3] == math.sin(0.5)) and np.all(v64[4] == math.cos(3.0))
    assert np.array_equal(v32[0], np.sin(X).astype(np.float32))
    # not pi-scaled, and the default is still pi-scaled
    p64, _, _ = ev(["sin(x)"], W, H)
    assert not np.allclose(p64[0], v64[0], atol=1e-3)


def test_radian_trig_identities():
    W, H = 13, 7
    v64, _, _ = ev_rad(["add(mult(sin(x), sin(x)), mult(cos(x), cos(x)))", "sub(tan(y), div(sin(y), cos(y)))",
                        "add(sin(neg(x)), sin(x))"], W, H, lo=-40.0, hi=40.0)
    assert np.allclose(v64[0], 1.0, rtol=0, atol=1e-15)
    assert np.allclose(v64[1], 0.0, rtol=0, atol=1e-12)
    assert np.all(v64[2] == 0.0)


def test_radian_fitness_by_hand():
    W, H = 4, 3
    X, Y = np_grid(W, H)
    t = toks("cos(x)")
    r64, _, _ = oracle.fitness(t.ops, t.imm, t.tree_off, 0, W, H, -5, 5, -5, 5, trig="rad")
    P = X ** 4 / (1 + X ** 4) + Y ** 4 / (1 + Y ** 4)
    assert r64[0] == pytest.approx(math.sqrt(np.mean((np.cos(X) - P) ** 2)), rel=1e-14)


def test_radian_error_bound_contains_fp32_faithful_and_propagates():
    rng = np.random.default_rng(11)
    trees = [I._full(rng, int(rng.integers(2, 6)), (I.ADD, I.MUL, I.SIN, I.COS, I.TAN, I.SUB)) for _ in range(60)]
    t = I.to_tokens(trees)
    v64, v32, _, eb = oracle.evaluate(t.ops, t.imm, t.tree_off, 0, 23, 19, 10.0, 20.0, -5, 5, with_bound=True,
                                      trig="rad")
    m = np.isfinite(v64) & np.isfinite(eb)
    assert m.mean() > 0.8
    assert np.all(np.abs(v32.astype(np.float64) - v64)[m] <= eb[m])
    W, H = 5, 3
    X, Y = np_grid(W, H)
    _, _, _, e = ev_rad(["sin(add(x, y))", "sin(x)"], W, H, with_bound=True)
    # rounded argument: |cos(a)| E(arg) is propagated (not pi |cos(pi a)| E(arg))
    assert np.all(e[0] >= U32 * np.abs(X + Y) * np.abs(np.cos(X + Y)) * (1 - 1e-12))
    assert np.all(e[0] < np.pi * U32 * np.abs(X + Y) + 4 * (2 * U32 + 2.0 ** -149))
    assert np.all(e[1] <= 2 * (2 * U32 * np.abs(np.sin(X)) + 2.0 ** -149) * (1 + 1e-12))


def test_unknown_trig_mode_is_refused():
    t = toks("sin(x)")
    with pytest.raises(ValueError):
        oracle.evaluate(t.ops, t.imm, t.tree_off, 0, 2, 2, -5, 5, -5, 5, trig="degrees")
