"""Column tables (subtrees with x but no y below them evaluated once per grid
column, then loaded): phenotypes and fitness bitwise equal to evaluating every
subtree at every point, on square, ragged and one-row grids, for every
points-per-thread value, with every operator, in radians, with a target tensor
and through a captured graph; and against the oracle."""
import numpy as np
import pytest

import oracle
import paper_2103_07512_gb300 as tgp
from paper_2103_07512_gb300 import inputs as I
from parity import assert_elements, assert_fitness

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


def y_free_heavy(rng, n, funcs=I.FUNCTIONS):
    """Trees whose subtrees often have x but no y below them."""
    def tree(d, allow_y):
        if d == 0 or rng.random() < 0.15:
            r = rng.random()
            if r < 0.45:
                return I.leaf(I.X)
            if r < 0.6 and allow_y:
                return I.leaf(I.Y)
            return I.leaf(I.CONST, float(rng.uniform(-1, 1)))
        f = funcs[int(rng.integers(len(funcs)))]
        ay = allow_y and rng.random() < 0.5
        return I.node(f, *[tree(d - 1, ay) for _ in range(I.ARITY[f])])
    return [tree(int(rng.integers(2, 7)), True) for _ in range(n)]


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
    v64, v32, fl, eb = oracle.evaluate(tok.ops, tok.imm, tok.tree_off, tok.order, g.W, g.H,
                                       g.xlo, g.xhi, g.ylo, g.yhi, with_bound=True)
    assert_elements(ph, v64, fl, eb, context="columns", v32=v32)
    r64, _, _, re = oracle.fitness(tok.ops, tok.imm, tok.tree_off, tok.order, g.W, g.H,
                                   g.xlo, g.xhi, g.ylo, g.yhi, with_bound=True)
    assert_fitness(fit, r64, re, g.N, "columns")


def test_column_launch_is_counted():
    rng = np.random.default_rng(63)
    tok = I.to_tokens([I.parse_string("add(sin(x), y)")] + y_free_heavy(rng, 20))
    g = I.Grid(64, 64)
    with tgp.Context() as a, tgp.Context(columns=False) as b:
        for c in (a, b):
            run(c, tok, g)
        # phenotype and fitness: two launches each, plus a column pass each with tables
        assert a.stats()["launches"] == b.stats()["launches"] + 2
