"""Generations made by the library's variation step (tgp_evolve) scored on
the device: fitness against the oracle on the exported tokens, equal bitwise
to a fresh compile of those tokens, and with the subtree cache equal bitwise
to without it (every operator of Table 1, so ternary nodes are cached too)."""
import numpy as np
import pytest

import oracle
import paper_2103_07512_gb300 as tgp
from paper_2103_07512_gb300 import inputs as I
from paper_2103_07512_gb300.evolve import DeviceEvolution
from parity import assert_elements, assert_fitness

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def run(ctx, g, generations, seed, funcs=I.ALL_FUNCTIONS, pop_size=50):
    dom = ctx.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi)
    ev = DeviceEvolution(ctx, dom, pop_size=pop_size, generations=generations, seed=seed, funcs=funcs)
    rows, toks = [], []

    def keep(gen, rmse):
        rows.append(rmse.copy())
        toks.append(ctx.population_tokens(ev.pop))

    ev.run(keep)
    ev.close()
    return rows, toks, dom


def test_device_generations_match_oracle():
    g = I.Grid(64, 48)
    with tgp.Context() as c:
        rows, toks, _ = run(c, g, 8, seed=4)
    assert len({t.ops.tobytes() for t in toks}) == len(toks)   # the population changes every generation
    for gen in (0, 3, 7):
        tok = toks[gen]
        r64, _, _, re = oracle.fitness(tok.ops, tok.imm, tok.tree_off, tok.order, g.W, g.H,
                                       g.xlo, g.xhi, g.ylo, g.yhi, with_bound=True)
        assert_fitness(rows[gen], r64, re, g.N, context=f"generation {gen}")
    assert min(np.nanmin(r) for r in rows[1:]) <= np.nanmin(rows[0])   # elitism


def test_evolved_population_equals_a_fresh_compile_of_its_tokens():
    g = I.Grid(96, 80)
    with tgp.Context() as c, tgp.Context() as d:
        rows, toks, _ = run(c, g, 5, seed=6)
        dom = d.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi)
        for r, tok in zip(rows, toks):
            fresh = d.fitness(d.compile_tokens(tok), dom, tok.n_trees)
            assert np.array_equal(r.view(np.int64), fresh.view(np.int64))


@pytest.mark.parametrize("min_cost", [2, 8])
def test_device_evolution_with_cache_is_bitwise_equal_to_without(min_cost):
    g = I.Grid(128, 96)
    with tgp.Context(cache_budget_bytes=64 * g.N * 4, cache_min_cost=min_cost) as a, tgp.Context() as b:
        ra, _, _ = run(a, g, 12, seed=8)
        rb, _, _ = run(b, g, 12, seed=8)
        for i, (x, y) in enumerate(zip(ra, rb)):
            assert np.array_equal(x.view(np.int64), y.view(np.int64)), f"generation {i}"
        st = a.stats()
        assert st["cache_inserts"] > 0 and st["cache_hits"] > 0


def test_cached_ternary_nodes_are_told_apart_by_their_third_operand():
    # if(h, h2, x) and if(h, h2, y) differ only in the third operand; each is
    # seen twice (admitted on the second sighting), then the other is scored
    h = "sin(cos(sin(add(x, y))))"
    h2 = "cos(sin(cos(mult(x, y))))"
    g = I.Grid(64, 64)
    exprs = [f"if({h}, {h2}, x)", f"if({h}, {h2}, y)", f"clip({h}, {h2}, x)", f"clip({h}, {h2}, y)"]
    with tgp.Context(cache_budget_bytes=64 * g.N * 4, cache_min_cost=1) as a, tgp.Context() as b:
        da = a.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi)
        db = b.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi)
        for e in exprs:
            tok = I.to_tokens([I.parse_string(e)])
            for _ in range(3):
                got = a.fitness(a.compile_tokens(tok), da, 1)
            ref = b.fitness(b.compile_tokens(tok), db, 1)
            assert got.view(np.int64)[0] == ref.view(np.int64)[0], e
        assert a.stats()["cache_hits"] > 0


def _grid_target64(g, dev):
    """Eq. 1 in binary64 at the grid's binary32 coordinates (flat point order)."""
    f = torch.float32
    sx = (torch.tensor(g.xhi, dtype=f) - torch.tensor(g.xlo, dtype=f)) / torch.tensor(g.W - 1, dtype=f)
    sy = (torch.tensor(g.yhi, dtype=f) - torch.tensor(g.ylo, dtype=f)) / torch.tensor(g.H - 1, dtype=f)
    xs = (torch.tensor(g.xlo, dtype=f) + torch.arange(g.W, dtype=f) * sx).double().to(dev)
    ys = (torch.tensor(g.ylo, dtype=f) + torch.arange(g.H, dtype=f) * sy).double().to(dev)
    x4 = xs ** 4
    y4 = ys ** 4
    return ((y4 / (1 + y4))[:, None] + (x4 / (1 + x4))[None, :]).reshape(-1)


@pytest.mark.parametrize("arm", ["python", "library"])
def test_evolution_at_full_size_sampled(arm):
    """The generational workload at its full size (population 50 on the
    4096x4096 grid, seed 3, subtree cache on): after 6 generations, the
    phenotypes of the current population on 2048 sampled points against the
    oracle, and every tree's fitness against the binary64 RMSE of the device's
    own phenotype over all 2^24 points."""
    from paper_2103_07512_gb300.evolve import Evolution, gpu_fitness
    g = I.Grid(4096, 4096)
    with tgp.Context(cache_budget_bytes=4 * 10**9, cache_min_cost=8) as ctx:
        dom = ctx.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi)
        if arm == "library":
            ev = DeviceEvolution(ctx, dom, pop_size=50, generations=6, seed=3)
            ev.run()
            tok = ctx.population_tokens(ev.pop)
            ev.close()
        else:
            ev = Evolution(gpu_fitness(ctx, dom), pop_size=50, generations=6, seed=3)
            ev.run()
            tok = I.to_tokens(ev.population)
        pop = ctx.compile_tokens(tok)
        fit = ctx.fitness(pop, dom, tok.n_trees)
        assert ctx.stats()["cache_inserts"] > 0, ctx.stats()
        ph = torch.empty((tok.n_trees, g.N), dtype=torch.float32, device="cuda")
        ctx.evaluate(pop, dom, ph)
        torch.cuda.synchronize()
        rng = np.random.default_rng(7)
        pts = np.concatenate([np.sort(rng.choice(g.N, 2048, replace=False)), [0, g.N - 1]])
        got = ph[:, torch.from_numpy(pts).cuda()].cpu().numpy()
        v64, v32, fl, eb = oracle.evaluate(tok.ops, tok.imm, tok.tree_off, tok.order, g.W, g.H, g.xlo, g.xhi,
                                           g.ylo, g.yhi, pts=pts, with_bound=True)
        assert_elements(got, v64, fl, eb, context=f"evolution {arm}, 4096x4096", v32=v32)
        t64 = _grid_target64(g, ph.device)
        r = np.array([float(torch.sqrt(torch.mean((ph[t].double() - t64) ** 2))) for t in range(tok.n_trees)])
        r = np.where(np.isfinite(r), r, np.inf)
        fin = np.isfinite(r)
        assert fin.sum() >= tok.n_trees // 2, r
        assert np.all(np.isinf(fit[~fin])), (fit[~fin], r[~fin])
        # the per-warp binary32 sums of squared residuals may overflow where
        # the binary64 sum reaches the binary32 range
        big = fin & (g.N * r * r >= np.finfo(np.float32).max / 2)
        assert np.all(np.isfinite(fit[fin & ~big]) | big[fin & ~big])
        ok = fin & ~(big & np.isinf(fit))
        # binary32 target and per-warp binary32 sums on the device
        bad = ok & ~np.isclose(fit, r, rtol=1e-4, atol=1e-6)
        assert not bad.any(), (np.flatnonzero(bad), fit[bad], r[bad])
