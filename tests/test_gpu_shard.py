"""Domains that hold a band of a grid's rows, and the sums of squared
residuals that the row-sharded fitness adds across GPUs (one GPU here: the
bands are evaluated one after the other; the exchange between ranks is
checked with gloo ranks on the CPU in test_shard.py).

A band's points, coordinates and values are bitwise those of the same rows of
the full grid; its sums, added over the bands, give the full grid's fitness.
"""
import numpy as np
import pytest

import oracle
import paper_2103_07512_gb300 as tgp
from paper_2103_07512_gb300 import inputs as I
from paper_2103_07512_gb300 import shard

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    c = tgp.Context()
    yield c
    c.close()


def phenotypes(ctx, pop, dom, n_trees, n_points):
    out = torch.empty((n_trees, n_points), dtype=torch.float32, device="cuda")
    ctx.evaluate(pop, dom, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def sse(ctx, pop, dom, n_trees):
    out = torch.full((n_trees,), float("nan"), dtype=torch.float64, device="cuda")
    ctx.fitness_sse_dev(pop, dom, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def bitwise(a, b):
    a = np.ascontiguousarray(a)
    b = np.ascontiguousarray(b)
    return a.shape == b.shape and np.array_equal(a.view(np.uint8), b.view(np.uint8))


@pytest.mark.parametrize("world", [2, 3, 5])
def test_band_phenotypes_are_the_full_grids_rows(ctx, world):
    """Every operator (with division, sin and cos) on ragged bands of a grid
    with a ragged row length: bitwise the rows of the full grid."""
    tok, _ = I.small_population(seed=7)
    g = I.Grid(96, 37)
    pop = ctx.compile_tokens(tok)
    full = phenotypes(ctx, pop, ctx.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi), tok.n_trees, g.N)
    for r in range(world):
        row0, n = shard.band_rows(g.H, r, world)
        dom = ctx.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi, rows=(row0, n))
        got = phenotypes(ctx, pop, dom, tok.n_trees, g.W * n)
        assert bitwise(got, full[:, row0 * g.W:(row0 + n) * g.W]), f"band {r} of {world}"
        ctx.release_domain(dom)


def test_band_is_bitwise_fp32_faithful_at_its_global_points(ctx):
    """The oracle's FP32-faithful values at the band's points of the full grid
    (a trig-free population: correctly rounded binary32 at every step)."""
    rng = np.random.default_rng(21)
    funcs = (I.ADD, I.SUB, I.MUL, I.DIV, I.NEG, I.ABS, I.MIN, I.MAX)
    tok = I.to_tokens(I.ramped_half_and_half(40, 2, 7, rng, funcs))
    g = I.Grid(41, 53)
    row0, n = 17, 19
    dom = ctx.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi, rows=(row0, n))
    got = phenotypes(ctx, ctx.compile_tokens(tok), dom, tok.n_trees, g.W * n)
    pts = np.arange(row0 * g.W, (row0 + n) * g.W)
    _, v32, _ = oracle.evaluate(tok.ops, tok.imm, tok.tree_off, 0, g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi, pts=pts)
    same = (got == v32) | (np.isnan(got) & np.isnan(v32))
    assert same.all(), f"{(~same).sum()} elements differ from the correctly rounded binary32 value"


def test_band_sums_add_up_to_the_full_grid(ctx):
    """Pagie target, the 1024x1024 population: the bands' sums add to the full
    grid's sum (binary64, different association: 1e-12 relative), and one
    band holding every row is the full grid bitwise."""
    tok, g = I.population_at_scale(seed=1)
    pop = ctx.compile_tokens(tok)
    T = tok.n_trees
    dfull = ctx.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi)
    s_full = sse(ctx, pop, dfull, T)
    rmse = torch.empty(T, dtype=torch.float64, device="cuda")
    ctx.fitness_dev(pop, dfull, rmse)
    torch.cuda.synchronize()
    rmse = rmse.cpu().numpy()
    # the sum under the square root, bitwise: sqrt(sum / N) in binary64
    assert bitwise(np.sqrt(s_full / float(g.N)), rmse)
    # a single band of every row: the same launch and sums
    dall = ctx.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi, rows=(0, g.H))
    assert bitwise(sse(ctx, pop, dall, T), s_full)
    # the sharded formula with one rank is the fitness, bitwise
    s_dev = torch.from_numpy(s_full).cuda()
    assert bitwise(shard.reduce_band_sse(s_dev, g.N).cpu().numpy(), rmse)
    for world in (2, 4):
        total = np.zeros(T)
        for r in range(world):
            row0, n = shard.band_rows(g.H, r, world)
            dom = ctx.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi, rows=(row0, n))
            total = total + sse(ctx, pop, dom, T)
            ctx.release_domain(dom)
        fin = np.isfinite(s_full)
        assert np.array_equal(np.isfinite(total), fin)
        np.testing.assert_allclose(total[fin], s_full[fin], rtol=1e-12, atol=0)


def test_band_targets_tensor_and_tokens(ctx):
    """A tensor target holds the band's values; a token target is evaluated
    on the band's points: both give the sums of the band of the full target."""
    rng = np.random.default_rng(44)
    target_tree = I._full(rng, 4, I.FUNCTIONS)
    tt = I.to_tokens([target_tree])
    tok, _ = I.small_population(seed=4)
    g = I.Grid(64, 45)
    pop = ctx.compile_tokens(tok)
    # the target tree's values on the full grid, as a tensor
    tpop = ctx.compile_tokens(tt)
    tfull = phenotypes(ctx, tpop, ctx.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi), 1, g.N)[0]
    row0, n = shard.band_rows(g.H, 1, 3)
    band_t = np.ascontiguousarray(tfull[row0 * g.W:(row0 + n) * g.W])
    d_tensor = ctx.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi, target=band_t, rows=(row0, n))
    d_tokens = ctx.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi, target_tokens=(tt.ops, tt.imm, tt.order),
                               rows=(row0, n))
    s_tensor = sse(ctx, pop, d_tensor, tok.n_trees)
    assert bitwise(sse(ctx, pop, d_tokens, tok.n_trees), s_tensor)
    # the band's own RMSE is the square root of its mean
    rmse = ctx.fitness(pop, d_tensor, tok.n_trees)
    assert bitwise(np.sqrt(s_tensor / float(g.W * n)), rmse)


def test_band_bounds_are_checked(ctx):
    for rows in [(-1, 3), (0, 0), (10, 36), (45, 1)]:
        with pytest.raises(tgp.TgpError) as e:
            ctx.load_domain(32, 45, rows=rows)
        assert e.value.code == tgp.E_INVALID
