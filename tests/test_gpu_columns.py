"""Column and row tables (subtrees with x but no y below them evaluated once
per grid column, those with no x below them once per grid row, then loaded):
phenotypes and fitness bitwise equal to evaluating every subtree at every
point, on square, ragged, one-row and one-column grids, for every
points-per-thread value, with every operator, in radians, with a target tensor
and through a captured graph; and against the oracle."""
import numpy as np
import pytest

import oracle
import paper_2103_07512_gb300 as tgp
from paper_2103_07512_gb300 import inputs as I
from parity import check_population

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def run(ctx, tok, g, target=None):
    dom = ctx.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi, target=target)
    pop = ctx.compile_tokens(tok)
    out = torch.empty((tok.n_trees, g.N), dtype=torch.float32, device="cuda")
    ctx.evaluate(pop, dom, out)
    fit = ctx.fitness(pop, dom, tok.n_trees)
    torch.cuda.synchronize()
    return out.cpu().numpy(), fit


def bits(a):
    b = np.asarray(a, np.float32).view(np.int32).copy()
    b[np.isnan(a)] = 0x7FC00000
    return b


def y_free_heavy(rng, n, funcs=I.FUNCTIONS, main=I.X, other=I.Y):
    """Trees whose subtrees often have `main` but not `other` below them (and
    the mirror image for half of the trees)."""
    def tree(d, allow_other, a, b):
        if d == 0 or rng.random() < 0.15:
            r = rng.random()
            if r < 0.45:
                return I.leaf(a)
            if r < 0.6 and allow_other:
                return I.leaf(b)
            return I.leaf(I.CONST, float(rng.uniform(-1, 1)))
        f = funcs[int(rng.integers(len(funcs)))]
        ao = allow_other and rng.random() < 0.5
        return I.node(f, *[tree(d - 1, ao, a, b) for _ in range(I.ARITY[f])])
    return [tree(int(rng.integers(2, 7)), True, main, other) if i % 2 == 0 else
            tree(int(rng.integers(2, 7)), True, other, main) for i in range(n)]


@pytest.mark.parametrize("W,H", [(64, 48), (33, 17), (129, 65), (7, 5), (100, 1), (1, 100), (1024, 16)])
@pytest.mark.parametrize("K", [1, 4, 8, 16])
def test_columns_bitwise_equal_to_every_point(W, H, K):
    rng = np.random.default_rng(W * 131 + H + K)
    tok = I.to_tokens(y_free_heavy(rng, 120))
    g = I.Grid(W, H)
    with tgp.Context(points_per_thread=K) as a, tgp.Context(points_per_thread=K, columns=False) as b:
        pa, fa = run(a, tok, g)
        pb, fb = run(b, tok, g)
    assert np.array_equal(bits(pa), bits(pb))
    assert np.array_equal(fa.view(np.int64), fb.view(np.int64))


def test_columns_with_every_operator_in_radians_and_a_target_tensor():
    rng = np.random.default_rng(61)
    tok = I.to_tokens(y_free_heavy(rng, 150, I.ALL_FUNCTIONS))
    g = I.Grid(96, 40)
    target = torch.rand(g.N, device="cuda") * 2 - 1
    for trig in ("pi", "rad"):
        with tgp.Context(trig=trig) as a, tgp.Context(trig=trig, columns=False) as b:
            pa, fa = run(a, tok, g, target=target)
            pb, fb = run(b, tok, g, target=target)
        assert np.array_equal(bits(pa), bits(pb)), trig
        assert np.array_equal(fa.view(np.int64), fb.view(np.int64)), trig


def test_columns_against_the_oracle_and_through_a_graph():
    rng = np.random.default_rng(62)
    tok = I.to_tokens(y_free_heavy(rng, 100))
    g = I.Grid(80, 30)
    with tgp.Context() as ctx:
        ph, fit = run(ctx, tok, g)
        dom = ctx.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi)
        pop = ctx.compile_tokens(tok)
        st = torch.cuda.Stream()
        dev = torch.empty(tok.n_trees, dtype=torch.float64, device="cuda")
        for _ in range(3):
            ctx.fitness_graph(pop, dom, dev, stream=st)
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy().view(np.int64), fit.view(np.int64))
        check_population(ctx, tok, g, fit, "columns", pop=pop, dom=dom)


@pytest.mark.parametrize("expr,extra", [("add(sin(x), y)", 2), ("add(cos(y), x)", 2),
                                        ("mult(sin(x), cos(y))", 4), ("add(x, y)", 0)])
def test_table_launches_are_counted(expr, extra):
    tok = I.to_tokens([I.parse_string(expr)])
    g = I.Grid(64, 64)
    with tgp.Context() as a, tgp.Context(columns=False) as b:
        for c in (a, b):
            run(c, tok, g)
        # phenotype and fitness, each with a column and / or a row pass where there are tables
        assert a.stats()["launches"] == b.stats()["launches"] + extra


def test_graph_replays_count_their_table_launches():
    # a column and a row table: two table launches, the interpreter and the
    # finalize kernel in every replay, as in a direct call
    tok = I.to_tokens([I.parse_string("mult(sin(x), cos(y))")])
    g = I.Grid(64, 64)
    with tgp.Context() as c:
        dom = c.load_domain(g.W, g.H)
        pop = c.compile_tokens(tok)
        st = torch.cuda.Stream()
        out = torch.empty(1, dtype=torch.float64, device="cuda")
        c.fitness_graph(pop, dom, out, stream=st)      # captured, then launched
        n0 = c.stats()["launches"]
        for _ in range(3):
            c.fitness_graph(pop, dom, out, stream=st)
        n1 = c.stats()["launches"]
        c.fitness_dev(pop, dom, out, stream=st)
        st.synchronize()
        n2 = c.stats()["launches"]
    assert n2 - n1 == 4
    assert n1 - n0 == 3 * 4
