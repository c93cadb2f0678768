"""Host side of the library, on CPU: the C ABI loads and exports what
include/tgp.h declares, token validation, hash-consing, and the bytecode the
compiler emits.  The bytecode is checked by running it through a small numpy
interpreter written here (test-only) and comparing with the CPU oracle."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_2103_07512_gb300 as tgp
from paper_2103_07512_gb300 import inputs as I
from parity import classify as parity_classify

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# decoded forms (order of the Form enum of the bytecode) and operand kinds
(F_END, F_AO, F_OA, F_TT, F_UA, F_UT, F_LD, F_ST, F_ROOT, F_CST, F_CLD, F_SEL) = range(12)
O_X, O_Y, O_C, O_S = range(4)


@pytest.fixture(scope="module")
def ctx():
    c = tgp.Context(host_only=True)
    yield c
    c.close()


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "tgp.h")).read()
    declared = set(re.findall(r"^\s*(?:int|const char\*)\s+(tgp_\w+)\s*\(", hdr, re.M))
    assert len(declared) >= 14
    L = tgp.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert declared == set(tgp.EXPORTS)


def test_layout():
    lay = tgp.debug_layout()
    assert lay["n_opnd"] == 4 and lay["n_forms"] == 14   # ... F_SEL, F_COL, F_ROW


def test_host_only_context_refuses_device_work(ctx):
    dom = ctx.load_domain(4, 4)          # a Pagie domain holds no device memory (planning only)
    pop = ctx.compile_tokens(I.to_tokens([I.parse_string("add(x, y)")]))
    for call in (lambda: ctx.fitness(pop, dom, 1),
                 lambda: ctx.load_domain(4, 4, target=np.zeros(16, np.float32))):
        with pytest.raises(tgp.TgpError) as e:
            call()
        assert e.value.code == tgp.E_INVALID


@pytest.mark.parametrize("columns", [False, True])
def test_plan_work_counts_evaluations(columns):
    """tgp_plan_work: every instruction counted once per point, per thread for
    values with no x below them, per column / row for tabled subtrees."""
    W, H, K = 16, 4, 8
    N, chunks = W * H, H * ((W + K - 1) // K)
    with tgp.Context(host_only=True, points_per_thread=K, threads_per_block=32, columns=columns) as c:
        dom = c.load_domain(W, H)
        pop = c.compile_tokens(I.to_tokens([I.parse_string("add(mult(x, y), sin(y))"),
                                            I.parse_string("div(cos(x), 0.5)")]))
        w, roots = c.plan_work(pop, dom)
    assert roots == 2 * N
    assert w[I.MUL] == N and w[I.ADD] == N
    # sin(y): no x below, once per thread; with tables, once per grid row
    assert w[I.SIN] == (H if columns else chunks)
    # cos(x): no y below, at every point; with tables, once per grid column (then div(cos(x), 0.5)
    # is tabled whole: the table holds the root's subtree)
    assert w[I.COS] == (W if columns else N)
    assert w[I.DIV] == (W if columns else N)
    assert w.sum() == w[[I.MUL, I.ADD, I.SIN, I.COS, I.DIV]].sum()


# ---------------------------------------------------------------- validation

@pytest.mark.parametrize("ops,imm,off,frag", [
    ([3, 0], [], [0, 2], "lacks operands"),
    ([0, 1], [], [0, 2], "exactly one expression"),
    ([42], [], [0, 1], "unknown opcode"),
    ([2], [], [0, 1], "beyond n_imm"),
    ([0], [1.0], [0, 1], "CONST tokens"),
    ([2], [float("nan")], [0, 1], "not finite"),
    ([2], [float("inf")], [0, 1], "not finite"),
    ([0, 0], [], [0, 1, 1], "empty"),
    ([0], [], [1, 1], "tree_off[0]"),
])
def test_malformed_tokens(ctx, ops, imm, off, frag):
    with pytest.raises(tgp.TgpError) as e:
        ctx.compile_population(np.array(ops), np.array(imm, np.float32), np.array(off))
    assert e.value.code == tgp.E_TOKENS
    assert frag in str(e.value)


def test_bad_arguments(ctx):
    with pytest.raises(tgp.TgpError) as e:
        ctx.compile_population(np.array([0]), np.array([], np.float32), np.array([0, 1]), order=7)
    assert e.value.code == tgp.E_INVALID


def test_depth_limit(ctx):
    t = I.leaf(I.X)
    for _ in range(1100):
        t = I.node(I.NEG, t)
    tok = I.to_tokens([t])
    with pytest.raises(tgp.TgpError) as e:
        ctx.compile_tokens(tok)
    assert "depth" in str(e.value)
    t = I.leaf(I.X)
    for _ in range(1000):
        t = I.node(I.NEG, t)
    ctx.compile_tokens(I.to_tokens([t]))


def test_empty_population(ctx):
    pop = ctx.compile_population(np.zeros(0, np.int32), np.zeros(0, np.float32), np.zeros(1, np.int64))
    ins, off = ctx.debug_plan(pop, 16)
    assert ins.shape[0] <= 1


# ---------------------------------------------------------------- hash-consing

def test_identical_subtrees_share_one_node(ctx):
    e = "add(mult(x, y), sin(mult(x, y)))"
    tok = I.to_tokens([I.parse_string(e), I.parse_string(e), I.parse_string("mult(x, y)")])
    ctx.compile_tokens(tok)
    st = ctx.stats()
    assert st["tree_nodes"] == 8 + 8 + 3
    # unique: x, y, mult(x,y), sin(.), add(.,.)
    assert st["dag_nodes"] == 5
    assert st["dag_internal"] == 3


def test_constants_are_identified_by_bits(ctx):
    tok = I.to_tokens([I.parse_string("add(x, 0.5)"), I.parse_string("add(x, 0.5)"),
                       I.parse_string("add(x, 0.25)")])
    ctx.compile_tokens(tok)
    assert ctx.stats()["dag_internal"] == 2


def test_prefix_and_postfix_give_same_dag(ctx):
    tok, _ = I.small_population(seed=0)
    ctx.compile_tokens(tok)
    a = ctx.stats()
    ctx.compile_tokens(I.convert_order(tok, I.POSTFIX))
    b = ctx.stats()
    assert a["dag_nodes"] == b["dag_nodes"] and a["tree_nodes"] == b["tree_nodes"]


# ---------------------------------------------------------------- bytecode

def _trigpi(a, shift):
    """sin(pi a) (shift 0) or cos(pi a) (shift 1) in binary64 with the
    argument reduced exactly to [-1/4, 1/4] around a multiple of 1/2, so zeros
    and +-1 at multiples of 1/2 are exact; rounded to binary32."""
    with np.errstate(invalid="ignore"):
        a64 = a.astype(np.float64)
        r = np.remainder(a64, 2.0)
        n = np.rint(2.0 * r)
        f = r - 0.5 * n
        q = (np.nan_to_num(n).astype(np.int64) + shift) % 4
        s, c = np.sin(np.pi * f), np.cos(np.pi * f)
        v = np.select([q == 0, q == 1, q == 2], [s, c, -s], -c)
        v = np.where(np.isfinite(a64), v, np.nan)
    return (v + 0.0).astype(np.float32)


def _sinpi32(a):
    return _trigpi(a, 0)


def _cospi32(a):
    return _trigpi(a, 1)


def _bin(fn, a, b):
    with np.errstate(all="ignore"):
        if fn == I.ADD:
            return a + b
        if fn == I.SUB:
            return a - b
        if fn == I.MUL:
            return a * b
        if fn == I.DIV:
            return np.where(b == 0, np.float32(0), a / np.where(b == 0, np.float32(1), b)).astype(np.float32)
        if fn == I.MIN:
            return np.fmin(a, b)
        if fn == I.MAX:
            return np.fmax(a, b)
        if fn == I.MDIST:
            return (a + b) * np.float32(0.5)
        if fn == I.MOD:
            r = np.fmod(a, b)
            return np.where((r != 0) & ((r < 0) != (b < 0)), r + b, r).astype(np.float32)
        if fn == I.POW:
            r = np.power(a.astype(np.float64), b.astype(np.float64)).astype(np.float32)
            return np.where((a == 0) & (b == 0), np.float32(0), r)
    raise AssertionError(fn)


def _un(fn, a):
    if fn == I.SIN:
        return _sinpi32(a)
    if fn == I.COS:
        return _cospi32(a)
    if fn == I.NEG:
        return -a
    if fn == I.ABS:
        return np.abs(a)
    with np.errstate(all="ignore"):
        if fn == I.SQRT:
            return np.where(a < 0, np.float32(0), np.sqrt(a))
        if fn == I.SIGN:
            return np.where(a > 0, np.float32(1), np.where(a < 0, np.float32(-1),
                                                            np.where(a == 0, np.float32(0), a)))
        if fn == I.FRAC:
            return a - np.floor(a)
        if fn == I.TAN:
            return (_sinpi32(a).astype(np.float64) / _cospi32(a).astype(np.float64)).astype(np.float32)
        if fn == I.EXP:
            return np.exp(a.astype(np.float64)).astype(np.float32)
        if fn == I.LOG:
            return np.where(a < 0, np.float32(-1), np.log(a.astype(np.float64)).astype(np.float32))
    raise AssertionError(fn)


def run_bytecode(ins, off, n_trees, X, Y):
    """Test-only numpy interpreter of the decoded bytecode (binary32)."""
    n = X.size
    out = np.full((n_trees, n), np.nan, np.float32)
    seen = np.zeros(n_trees, bool)
    for g in range(off.size - 1):
        A = np.zeros(n, np.float32)
        S = {}
        for i in range(off[g], off[g + 1]):
            form, fn, o1, o2, aux, immb = (int(v) for v in ins[i])
            imm = np.array([immb], np.int32).view(np.float32)[0]

            def opnd(o):
                if o == O_X:
                    return X
                if o == O_Y:
                    return Y
                if o == O_C:
                    return np.full(n, imm, np.float32)
                assert o == O_S and aux in S, "slot read before it was written"
                return S[aux]
            if form == F_END:
                assert i == off[g + 1] - 1
                break
            if form == F_AO:
                A = _bin(fn, A, opnd(o1))
            elif form == F_OA:
                assert fn in (I.SUB, I.DIV, I.POW, I.MOD)
                A = _bin(fn, opnd(o1), A)
            elif form == F_TT:
                assert o1 <= 2 and o2 <= 2 and not (o1 == 2 and o2 == 2)
                A = _bin(fn, opnd(o1), opnd(o2))
            elif form == F_UA:
                A = _un(fn, A)
            elif form == F_UT:
                assert o1 <= 2
                A = _un(fn, opnd(o1))
            elif form == F_LD:
                A = opnd(o1).copy()
            elif form == F_ST:
                S[aux] = A.copy()
            elif form == F_SEL:
                assert aux in S and immb in S, "select reads a slot before it was written"
                c = S[aux]
                A = np.where((c != 0) | np.isnan(c), S[immb], A).astype(np.float32)
            elif form == F_ROOT:
                assert not seen[aux], "tree emitted twice"
                seen[aux] = True
                out[aux] = A
            else:
                raise AssertionError(f"unexpected form {form}")
    assert seen.all(), "some tree never reached its root instruction"
    return out


def _check_population(ctx, tok, W=7, H=5, trig_free=False):
    pop = ctx.compile_tokens(tok)
    ins, off = ctx.debug_plan(pop, W * H)
    xs = np.array([oracle.grid_point(W, H, -5, 5, -5, 5, p) for p in range(W * H)], np.float32)
    got = run_bytecode(ins, off, tok.n_trees, xs[:, 0].copy(), xs[:, 1].copy())
    v64, v32, fl = oracle.evaluate(tok.ops, tok.imm, tok.tree_off, tok.order, W, H, -5, 5, -5, 5)
    if trig_free:
        assert np.array_equal(got, v32, equal_nan=True)
    else:
        ok = ~fl
        assert np.allclose(got[ok], v32[ok], rtol=1e-4, atol=1e-4, equal_nan=True)
    ctx.release_population(pop)
    return ins, off


def test_bytecode_small_population(ctx):
    tok, _ = I.small_population(seed=0)
    _check_population(ctx, tok)


def test_bytecode_postfix_input(ctx):
    tok, _ = I.small_population(seed=4)
    _check_population(ctx, I.convert_order(tok, I.POSTFIX))


def test_bytecode_trig_free_is_exact(ctx):
    rng = np.random.default_rng(11)
    funcs = (I.ADD, I.SUB, I.MUL, I.DIV, I.NEG, I.ABS, I.MIN, I.MAX)
    trees = I.ramped_half_and_half(40, 2, 7, rng, funcs)
    _check_population(ctx, I.to_tokens(trees), trig_free=True)


def test_bytecode_deep_trees_use_many_slots(ctx):
    rng = np.random.default_rng(3)
    funcs = (I.ADD, I.SUB, I.MUL, I.MIN, I.MAX)
    trees = [I._full(rng, 9, funcs) for _ in range(3)]   # full binary trees of depth 9: 8 slots
    ins, off = _check_population(ctx, I.to_tokens(trees), W=3, H=2, trig_free=True)
    assert ins[ins[:, 0] == F_ST, 4].max() == 7


def test_bytecode_shared_subtrees_are_evaluated_once(ctx):
    s = "sin(add(mult(x, y), 0.25))"
    trees = [f"add({s}, {s})", f"mult({s}, x)", f"div(y, {s})", s]
    tok = I.to_tokens([I.parse_string(e) for e in trees])
    ins, off = _check_population(ctx, tok)
    # the sin node is computed by exactly one unary instruction in the plan
    n_sin = int(((ins[:, 0] == F_UA) & (ins[:, 1] == I.SIN)).sum())
    n_sin += int(((ins[:, 0] == F_UT) & (ins[:, 1] == I.SIN)).sum())
    groups = off.size - 1
    assert n_sin <= groups


def test_bytecode_duplicated_trees_and_leaf_roots(ctx):
    trees = ["x", "y", "0.5", "x", "add(x, y)", "add(x, y)", "neg(0.5)", "sub(0.5, 0.25)"]
    tok = I.to_tokens([I.parse_string(e) for e in trees])
    _check_population(ctx, tok, trig_free=True)


def test_bytecode_exact_size_population_with_duplicates(ctx):
    rng = np.random.default_rng(2)
    trees, stats = I.exact_size_population(120, 3, 255, 12, 0.3, rng)
    assert 0.15 < stats["dup_fraction"] < 0.45
    _check_population(ctx, I.to_tokens(trees), W=4, H=3)


@pytest.mark.parametrize("n_points", [1, 100, 4096, 1 << 20])
def test_plan_group_offsets_are_consistent(ctx, n_points):
    tok, _ = I.small_population(seed=1)
    pop = ctx.compile_tokens(tok)
    ins, off = ctx.debug_plan(pop, n_points)
    assert off[0] == 0 and off[-1] == ins.shape[0]
    assert np.all(np.diff(off) > 0)
    assert np.all(ins[off[1:] - 1, 0] == F_END)
    roots = ins[ins[:, 0] == F_ROOT, 4]
    assert sorted(roots.tolist()) == list(range(tok.n_trees))


def test_server_needs_a_device_context():
    with tgp.Context(host_only=True) as c:
        with pytest.raises(tgp.TgpError) as e:
            tgp.Server(c)
        assert e.value.code == tgp.E_INVALID


# ---------------------------------------------------------------- simplification

CONSTS = (0.0, -0.0, 1.0, -1.0, 2.0, 0.5, 3.0)


def _const_heavy_tree(rng, d, funcs):
    """Random tree whose terminals are mostly small constants (rewrites fire)."""
    if d == 0 or rng.random() < 0.15:
        r = rng.random()
        if r < 0.25:
            return I.leaf(I.X)
        if r < 0.35:
            return I.leaf(I.Y)
        return I.leaf(I.CONST, CONSTS[int(rng.integers(len(CONSTS)))])
    f = funcs[int(rng.integers(len(funcs)))]
    return I.node(f, *[_const_heavy_tree(rng, d - 1, funcs) for _ in range(I.ARITY[f])])


def _nan_canonical_bits(a):
    b = np.asarray(a, np.float32).view(np.int32).copy()
    b[np.isnan(a)] = 0x7FC00000
    return b


@pytest.mark.parametrize("expr,simplified", [
    ("neg(neg(x))", "x"), ("abs(neg(y))", "abs(y)"), ("abs(abs(x))", "abs(x)"),
    ("mult(x, 1.0)", "x"), ("mult(1.0, y)", "y"), ("div(x, 1.0)", "x"), ("div(sin(x), 0.0)", "0.0"),
    ("add(x, -0.0)", "x"), ("sub(y, 0.0)", "y"), ("sub(-0.0, x)", "neg(x)"), ("min(x, x)", "x"),
    ("max(sin(y), sin(y))", "sin(y)"), ("add(0.5, 0.25)", "0.75"), ("mult(3.0, neg(0.5))", "-1.5"),
    ("div(1.0, 0.0)", "0.0"), ("abs(-2.0)", "2.0"), ("sub(1.0, 1.0)", "0.0"),
    ("add(x, neg(y))", "sub(x, y)"), ("add(neg(x), y)", "sub(y, x)"), ("sub(x, neg(y))", "add(x, y)"),
    ("mult(neg(x), neg(y))", "mult(x, y)"), ("div(neg(x), neg(y))", "div(x, y)"),
    ("mult(neg(x), 2.0)", "mult(x, -2.0)"), ("div(neg(y), 4.0)", "div(y, -4.0)"),
    ("div(3.0, neg(x))", "div(-3.0, x)"),
])
def test_simplification_rewrites(ctx, expr, simplified):
    a = I.to_tokens([I.parse_string(expr)])
    b = I.to_tokens([I.parse_string(simplified)])
    ctx.compile_tokens(a)
    sa = ctx.stats()
    ctx.compile_tokens(b)
    sb = ctx.stats()
    assert (sa["dag_nodes"], sa["dag_internal"]) == (sb["dag_nodes"], sb["dag_internal"])
    assert sa["tree_nodes"] == a.ops.size          # the token count is kept
    with tgp.Context(host_only=True, simplify=False) as raw:
        raw.compile_tokens(a)
        assert raw.stats()["dag_nodes"] > sa["dag_nodes"]


def test_commutative_operands_share_a_node(ctx):
    tok = I.to_tokens([I.parse_string("add(x, mult(y, 0.5))"), I.parse_string("add(mult(0.5, y), x)")])
    ctx.compile_tokens(tok)
    assert ctx.stats()["dag_internal"] == 2
    with tgp.Context(host_only=True, simplify=False) as raw:
        raw.compile_tokens(tok)
        assert raw.stats()["dag_internal"] == 4


def test_no_folding_of_trig_nan_or_subnormal_results(ctx):
    for e in ["sin(0.5)", "cos(1.0)", "mult(1e-20, 1e-20)", "min(0.0, -0.0)", "mult(3e38, 3e38)"]:
        tok = I.to_tokens([I.parse_string(e)])
        ctx.compile_tokens(tok)
        assert ctx.stats()["dag_internal"] == 1, e


def test_simplified_bytecode_equals_oracle_on_raw_trees(ctx):
    """The simplified plan, run by the numpy interpreter, gives exactly the
    binary32 values the oracle computes on the trees as given."""
    rng = np.random.default_rng(21)
    funcs = (I.ADD, I.SUB, I.MUL, I.DIV, I.NEG, I.ABS, I.MIN, I.MAX)
    trees = [_const_heavy_tree(rng, int(rng.integers(2, 7)), funcs) for _ in range(200)]
    tok = I.to_tokens(trees)
    W, H = 5, 4
    pop = ctx.compile_tokens(tok)
    st = ctx.stats()
    with tgp.Context(host_only=True, simplify=False) as raw:
        raw.compile_tokens(tok)
        assert st["dag_internal"] < raw.stats()["dag_internal"]
    ins, off = ctx.debug_plan(pop, W * H)
    xs = np.array([oracle.grid_point(W, H, -5, 5, -5, 5, p) for p in range(W * H)], np.float32)
    got = run_bytecode(ins, off, tok.n_trees, xs[:, 0].copy(), xs[:, 1].copy())
    v64, v32, fl = oracle.evaluate(tok.ops, tok.imm, tok.tree_off, tok.order, W, H, -5, 5, -5, 5)
    # equal as binary32 values (NaN = NaN; a zero of either sign = 0: fmin/fmax of
    # two zeros may return either, and operand order differs between the plans)
    assert np.array_equal(got, v32, equal_nan=True)


def test_absorbed_negations_keep_every_bit(ctx):
    """Negation-heavy trees over add, sub, mult, div, neg and abs with signed
    zeros among the constants: the simplified plan and the plan of the trees
    as given, both run by the numpy interpreter, agree bit for bit (signed
    zeros included; NaN canonical)."""
    rng = np.random.default_rng(22)
    funcs = (I.ADD, I.SUB, I.MUL, I.DIV, I.NEG, I.NEG, I.ABS)
    trees = [_const_heavy_tree(rng, int(rng.integers(2, 7)), funcs) for _ in range(300)]
    tok = I.to_tokens(trees)
    W, H = 7, 3
    xs = np.array([oracle.grid_point(W, H, -1, 1, -1, 1, p) for p in range(W * H)], np.float32)
    with tgp.Context(host_only=True, simplify=False) as raw:
        ins_r, off_r = raw.debug_plan(raw.compile_tokens(tok), W * H)
        n_raw = raw.stats()["dag_internal"]
    ins_s, off_s = ctx.debug_plan(ctx.compile_tokens(tok), W * H)
    assert ctx.stats()["dag_internal"] < n_raw
    with np.errstate(all="ignore"):
        a = run_bytecode(ins_s, off_s, tok.n_trees, xs[:, 0].copy(), xs[:, 1].copy())
        b = run_bytecode(ins_r, off_r, tok.n_trees, xs[:, 0].copy(), xs[:, 1].copy())
    assert np.array_equal(_nan_canonical_bits(a), _nan_canonical_bits(b))


# ---------------------------------------------------------------- the rest of Table 1

EXACT_FUNCS = (I.ADD, I.SUB, I.MUL, I.DIV, I.NEG, I.ABS, I.MIN, I.MAX, I.MDIST, I.SQRT, I.SIGN,
               I.CLIP, I.FRAC, I.IF)


def test_bytecode_new_exact_operators_equal_oracle(ctx):
    """mdist, sqrt, sign, clip, frac and if are exactly rounded steps: the
    plan, run by the numpy interpreter, gives the oracle's binary32 values."""
    rng = np.random.default_rng(41)
    trees = [I._full(rng, int(rng.integers(2, 6)), EXACT_FUNCS) for _ in range(120)]
    tok = I.to_tokens(trees)
    W, H = 6, 5
    pop = ctx.compile_tokens(tok)
    ins, off = ctx.debug_plan(pop, W * H)
    assert (ins[:, 0] == F_SEL).any()
    xs = np.array([oracle.grid_point(W, H, -5, 5, -5, 5, p) for p in range(W * H)], np.float32)
    got = run_bytecode(ins, off, tok.n_trees, xs[:, 0].copy(), xs[:, 1].copy())
    v64, v32, fl = oracle.evaluate(tok.ops, tok.imm, tok.tree_off, tok.order, W, H, -5, 5, -5, 5)
    assert np.array_equal(got, v32, equal_nan=True)


def test_bytecode_all_operators_close_to_oracle(ctx):
    rng = np.random.default_rng(42)
    trees = [I._full(rng, int(rng.integers(2, 5)), I.ALL_FUNCTIONS) for _ in range(150)]
    tok = I.to_tokens(trees)
    for order in (I.PREFIX, I.POSTFIX):
        t = I.convert_order(tok, order)
        W, H = 5, 4
        pop = ctx.compile_tokens(t)
        ins, off = ctx.debug_plan(pop, W * H)
        xs = np.array([oracle.grid_point(W, H, -5, 5, -5, 5, p) for p in range(W * H)], np.float32)
        got = run_bytecode(ins, off, t.n_trees, xs[:, 0].copy(), xs[:, 1].copy())
        v64, v32, fl, eb = oracle.evaluate(t.ops, t.imm, t.tree_off, order, W, H, -5, 5, -5, 5,
                                           with_bound=True)
        c = parity_classify(got, v64, v32, fl, eb)
        assert c["n_fail"] == 0, c["n_fail"]
        assert c["n_bound"] + c["n_unbounded"] < 0.3 * c["n"]


def test_clip_is_lowered_to_min_max(ctx):
    a = I.to_tokens([I.parse_string("clip(x, -1.0, 1.0)")])
    b = I.to_tokens([I.parse_string("max(min(1.0, x), -1.0)")])
    pa, pb = ctx.compile_tokens(a), ctx.compile_tokens(b)
    ia, _ = ctx.debug_plan(pa, 16)
    ib, _ = ctx.debug_plan(pb, 16)
    assert np.array_equal(ia, ib)


def test_three_operand_tokens_validate(ctx):
    bad = I.Tokens(np.array([I.IF, I.X, I.Y], np.int32), np.zeros(0, np.float32),
                   np.array([0, 3], np.int64), I.PREFIX)
    with pytest.raises(tgp.TgpError) as e:
        ctx.compile_tokens(bad)
    assert e.value.code == tgp.E_TOKENS


def test_unknown_context_flags_and_trig_mode_are_refused():
    import ctypes
    cfg = tgp.Config()
    cfg.flags = tgp.F_HOST_ONLY | 1024
    h = ctypes.c_void_p()
    assert tgp.lib().tgp_create(ctypes.byref(h), ctypes.byref(cfg)) == tgp.E_INVALID
    with pytest.raises(ValueError):
        tgp.Context(host_only=True, trig="degrees")
    with tgp.Context(host_only=True, trig="rad") as c:
        c.compile_tokens(I.to_tokens([I.parse_string("sin(x)")]))


@pytest.mark.parametrize("name", ["small", "at_scale", "batched"])
def test_concurrent_group_planning_gives_the_serial_bytecode(name):
    """Tree groups planned on the context's worker threads (the default) give
    the bytecode of serial planning (plan_threads = 1), group by group."""
    if name == "small":
        tok, g = I.small_population()
    elif name == "at_scale":
        tok, g = I.population_at_scale()
    else:
        tok, g = I.batched_uneven()[:2]
    with tgp.Context(host_only=True, plan_threads=1) as a, tgp.Context(host_only=True) as b:
        for n_points in (g.N, 4096, 1):
            ia, oa = a.debug_plan(a.compile_tokens(tok), n_points)
            ib, ob = b.debug_plan(b.compile_tokens(tok), n_points)
            assert np.array_equal(oa, ob) and np.array_equal(ia, ib)
            assert len(oa) > 2 or n_points == 1


@pytest.mark.parametrize("simplify", [True, False])
@pytest.mark.parametrize("order", [I.PREFIX, I.POSTFIX])
def test_parallel_parse_equals_serial(simplify, order):
    """A large population parsed in chunks of trees on the context's workers
    gives the serial parse's DAG: the same nodes with the same ids (so the
    same exported tokens and bytecode)."""
    tok, g = I.batched_uneven()[:2]
    tok = I.convert_order(tok, order)
    with tgp.Context(host_only=True, plan_threads=1, simplify=simplify) as a, \
            tgp.Context(host_only=True, simplify=simplify) as b:
        pa, pb = a.compile_tokens(tok), b.compile_tokens(tok)
        sa, sb = a.stats(), b.stats()
        assert sa["dag_nodes"] == sb["dag_nodes"] and sa["dag_internal"] == sb["dag_internal"]
        ta, tb = a.population_tokens(pa), b.population_tokens(pb)
        assert np.array_equal(ta.ops, tb.ops) and np.array_equal(ta.imm.view(np.int32), tb.imm.view(np.int32))
        ia, oa = a.debug_plan(pa, g.N)
        ib, ob = b.debug_plan(pb, g.N)
        assert np.array_equal(ia, ib) and np.array_equal(oa, ob)
    # a malformed tree deep in the stream gives the serial parse's message
    bad = I.Tokens(tok.ops.copy(), tok.imm, tok.tree_off, tok.order)
    t = 3000
    bad.ops[bad.tree_off[t]:bad.tree_off[t + 1]][0] = 99
    with tgp.Context(host_only=True, plan_threads=1) as a, tgp.Context(host_only=True) as b:
        msgs = []
        for c in (a, b):
            with pytest.raises(tgp.TgpError) as e:
                c.compile_tokens(bad)
            msgs.append(str(e.value))
        assert msgs[0] == msgs[1] and "tree 3000" in msgs[0]
    # one immediate too many: the constant count check of both parses
    extra = I.Tokens(tok.ops, np.append(tok.imm, np.float32(1.0)), tok.tree_off, tok.order)
    with tgp.Context(host_only=True, plan_threads=1) as a, tgp.Context(host_only=True) as b:
        msgs = []
        for c in (a, b):
            with pytest.raises(tgp.TgpError) as e:
                c.compile_tokens(extra)
            assert e.value.code == tgp.E_TOKENS
            msgs.append(str(e.value))
        assert msgs[0] == msgs[1] and "CONST tokens" in msgs[0]


def test_column_flag_is_accepted_and_debug_plans_have_no_column_loads():
    tok = I.to_tokens([I.parse_string("add(sin(x), mult(y, cos(x)))")])
    for cols in (True, False):
        with tgp.Context(host_only=True, columns=cols) as c:
            ins, off = c.debug_plan(c.compile_tokens(tok), 64 * 64)
            assert not (ins[:, 0] == 12).any()   # F_COL: column tables need a grid of several rows
    assert tgp.F_NO_COLUMNS == 32
