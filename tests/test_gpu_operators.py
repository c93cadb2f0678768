"""The rest of Table 1 on the device (tan, exp, log, pow, mdist, sqrt, sign,
clip, mod, frac, if): every element and fitness against the oracle, the
exactly rounded operators bitwise against the FP32-faithful oracle, special
values, and simplification still exact with every operator."""
import numpy as np
import pytest

import oracle
import paper_2103_07512_gb300 as tgp
from paper_2103_07512_gb300 import inputs as I
from parity import check_population

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EXACT = (I.ADD, I.SUB, I.MUL, I.DIV, I.NEG, I.ABS, I.MIN, I.MAX, I.MDIST, I.SQRT, I.SIGN, I.CLIP, I.FRAC, I.IF)


def device(ctx, tok, g):
    dom = ctx.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi)
    pop = ctx.compile_tokens(tok)
    out = torch.empty((tok.n_trees, g.N), dtype=torch.float32, device="cuda")
    ctx.evaluate(pop, dom, out)
    fit = ctx.fitness(pop, dom, tok.n_trees)
    torch.cuda.synchronize()
    return out.cpu().numpy(), fit


@pytest.mark.parametrize("K", [0, 1, 4, 8])
def test_all_operators_against_oracle(K):
    rng = np.random.default_rng(51)
    trees = [I._full(rng, int(rng.integers(2, 6)), I.ALL_FUNCTIONS) for _ in range(200)]
    trees += I.ramped_half_and_half(100, 2, 6, rng, I.ALL_FUNCTIONS)
    tok = I.to_tokens(trees)
    g = I.Grid(33, 17)
    with tgp.Context(points_per_thread=K) as ctx:
        ph, fit = device(ctx, tok, g)
        r = check_population(ctx, tok, g, fit, f"all operators K={K}", budget="operators")
    c = r["elements"]
    assert c["n_bound"] + c["n_unbounded"] < 0.4 * c["n"]


def test_exactly_rounded_operators_equal_fp32_faithful():
    rng = np.random.default_rng(52)
    trees = [I._full(rng, int(rng.integers(2, 7)), EXACT) for _ in range(200)]
    tok = I.to_tokens(trees)
    g = I.Grid(40, 30)
    with tgp.Context() as ctx:
        ph, _ = device(ctx, tok, g)
    _, v32, _ = oracle.evaluate(tok.ops, tok.imm, tok.tree_off, tok.order, g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi)
    # equal as binary32 values: NaN = NaN, zeros of either sign equal (min/max/if of zeros)
    assert np.array_equal(ph, v32, equal_nan=True)


@pytest.mark.parametrize("expr,expect", [
    ("tan(0.25)", 1.0), ("tan(0.0)", 0.0), ("exp(0.0)", 1.0), ("log(1.0)", 0.0), ("log(-3.0)", -1.0),
    ("pow(0.0, 0.0)", 0.0), ("pow(2.0, 10.0)", 1024.0), ("pow(-2.0, 3.0)", -8.0), ("mdist(1.0, 2.0)", 1.5),
    ("sqrt(-4.0)", 0.0), ("sqrt(9.0)", 3.0), ("sign(-2.5)", -1.0), ("sign(0.0)", 0.0), ("sign(7.0)", 1.0),
    ("clip(5.0, 0.0, 1.0)", 1.0), ("mod(-5.0, 3.0)", 1.0), ("mod(5.0, -3.0)", -1.0), ("frac(-2.25)", 0.75),
    ("if(0.0, 1.0, 2.0)", 2.0), ("if(-0.0, 1.0, 2.0)", 2.0), ("if(3.0, 1.0, 2.0)", 1.0),
])
def test_special_values_on_device(expr, expect):
    # a copy whose constants c become add(x, c), so nothing is folded on the
    # host (x = 0 on this grid), beside the expression as written
    def unfold(t):
        op, v, kids = t
        if op == I.CONST:
            return I.node(I.ADD, I.leaf(I.X), t)
        return (op, v, tuple(unfold(k) for k in kids))
    t = I.parse_string(expr)
    tok = I.to_tokens([unfold(t), t])
    e = I.to_string(unfold(t))
    g = I.Grid(1, 1, 0.0, 0.0, 0.0, 0.0)
    with tgp.Context() as ctx:
        ph, _ = device(ctx, tok, g)
    assert ph[0, 0] == np.float32(expect), (e, ph[0, 0])
    assert ph[1, 0] == np.float32(expect), (expr, ph[1, 0])


def test_nonfinite_results_on_device():
    tok = I.to_tokens([I.parse_string(e) for e in
                       ["tan(add(x, 0.5))", "log(mult(x, 0.0))", "pow(add(x, -8.0), 0.5)", "mod(1.0, mult(x, 0.0))",
                        "exp(add(x, 100.0))", "sign(mod(1.0, mult(x, 0.0)))"]])
    g = I.Grid(1, 1, 0.0, 0.0, 0.0, 0.0)
    with tgp.Context() as ctx:
        ph, fit = device(ctx, tok, g)
    v = ph[:, 0]
    assert np.isinf(v[0]) and v[1] == -np.inf and np.isnan(v[2]) and np.isnan(v[3])
    assert v[4] == np.inf and np.isnan(v[5])
    assert np.all(np.isinf(fit))


def test_simplified_equals_as_given_with_every_operator():
    rng = np.random.default_rng(53)

    def tree(d):
        if d == 0 or rng.random() < 0.2:
            r = rng.random()
            if r < 0.3:
                return I.leaf(I.X if r < 0.2 else I.Y)
            return I.leaf(I.CONST, (0.0, -0.0, 1.0, -1.0, 2.0, 0.5, 3.0)[int(rng.integers(7))])
        f = I.ALL_FUNCTIONS[int(rng.integers(len(I.ALL_FUNCTIONS)))]
        return I.node(f, *[tree(d - 1) for _ in range(I.ARITY[f])])

    tok = I.to_tokens([tree(int(rng.integers(2, 7))) for _ in range(300)])
    g = I.Grid(48, 40)
    with tgp.Context() as a, tgp.Context(simplify=False) as b:
        pa, fa = device(a, tok, g)
        pb, fb = device(b, tok, g)
        assert a.stats()["dag_internal"] < b.stats()["dag_internal"]

    def bits(x):
        y = x.view(np.int32).copy()
        y[np.isnan(x)] = 0x7FC00000
        return y
    assert np.array_equal(bits(pa), bits(pb))
    assert np.array_equal(fa.view(np.int64), fb.view(np.int64))


@pytest.mark.parametrize("lo,hi", [(-2.0, 2.0), (-1e-3, 1e-3), (999.0, 1003.0), (4194304.0, 4194368.0),
                                   (-3e7, 3e7), (0.49, 0.51), (-1e30, 1e30)])
def test_sin_cos_pi_within_one_ulp(lo, hi):
    """The device's sin(pi a) / cos(pi a) against the exactly reduced binary64
    values: within 1 ulp everywhere (the oracle's bound allows 2), 0 at the
    zeros."""
    W = 1 << 14
    g = I.Grid(W, 1, lo, hi, 0.0, 0.0)
    tok = I.to_tokens([I.parse_string("sin(x)"), I.parse_string("cos(x)")])
    with tgp.Context(simplify=False) as ctx:
        ph, _ = device(ctx, tok, g)
    xs = np.array([oracle.grid_point(W, 1, lo, hi, 0.0, 0.0, p)[0] for p in range(W)], np.float32)
    for row, f in ((0, oracle.sinpi), (1, oracle.cospi)):
        exact = np.array([f(float(v)) for v in xs])
        ulp = np.spacing(np.abs(exact).astype(np.float32)).astype(np.float64)
        err = np.abs(ph[row].astype(np.float64) - exact) / ulp
        assert err.max() <= 1.0, (row, float(err.max()), xs[int(err.argmax())])
        zero = exact == 0
        assert np.all(ph[row][zero] == 0)


@pytest.mark.parametrize("K", [1, 8])
def test_radian_trigonometry_against_oracle(K):
    """TGP_F_TRIG_RADIANS (the footnote of Table 1): sin, cos and tan of the
    argument itself, every element and fitness against the oracle's radian
    mode, and not the default pi-scaled values."""
    rng = np.random.default_rng(54)
    funcs = (I.ADD, I.SUB, I.MUL, I.DIV, I.SIN, I.COS, I.TAN, I.NEG, I.MIN)
    trees = [I._full(rng, int(rng.integers(2, 6)), funcs) for _ in range(150)]
    trees += [I.parse_string(e) for e in ("sin(x)", "cos(y)", "tan(x)", "sin(mult(x, 40.0))")]
    tok = I.to_tokens(trees)
    g = I.Grid(37, 21)
    with tgp.Context(points_per_thread=K, trig="rad") as ctx:
        ph, fit = device(ctx, tok, g)
        check_population(ctx, tok, g, fit, f"radians K={K}", budget="operators", trig="rad")
    xs = np.array([oracle.grid_point(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi, p)[0] for p in range(g.N)])
    assert np.allclose(ph[-4], np.sin(xs), rtol=0, atol=2e-7)
    with tgp.Context(points_per_thread=K) as ctx:
        pi_ph, _ = device(ctx, tok, g)
    assert not np.allclose(pi_ph[-4], ph[-4], atol=1e-3)


def test_radian_mode_with_cache_and_noalloc_paths():
    rng = np.random.default_rng(55)
    tok = I.to_tokens([I._full(rng, 4, I.FUNCTIONS) for _ in range(40)])
    g = I.Grid(64, 48)
    with tgp.Context(trig="rad", cache_budget_bytes=64 * g.N * 4, cache_min_cost=1) as ctx:
        dom = ctx.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi)
        pop = ctx.compile_tokens(tok)
        runs = [ctx.fitness(pop, dom, tok.n_trees) for _ in range(3)]
        out = torch.empty(tok.n_trees, dtype=torch.float64, device="cuda")
        ctx.fitness_noalloc(pop, dom, out)
        torch.cuda.synchronize()
        assert ctx.stats()["cache_hits"] > 0
        check_population(ctx, tok, g, runs[0], "radians, cached", pop=pop, dom=dom, budget="operators", trig="rad")
    for r in runs[1:]:
        assert np.array_equal(r.view(np.int64), runs[0].view(np.int64))
    assert np.array_equal(out.cpu().numpy().view(np.int64), runs[0].view(np.int64))
