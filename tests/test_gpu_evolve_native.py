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
from parity import check_population, oracle_pool

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
        rows, toks, dom = run(c, g, 8, seed=4)
        assert len({t.ops.tobytes() for t in toks}) == len(toks)   # the population changes every generation
        for gen in (0, 3, 7):
            check_population(c, toks[gen], g, rows[gen], f"generation {gen}", dom=dom, budget="operators")
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


@pytest.mark.parametrize("arm", ["python", "library"])
def test_evolution_at_full_size_generations_0_25_49(arm):
    """The generational workload at its full size: population 50, 50
    generations on the 4096x4096 grid (seed 3, subtree cache on), variation in
    Python on tuple trees or in the library on the DAG.  For generations 0,
    25 and 49: every tree on 65,536 sampled points against the oracle, and
    every tree's fitness, as the run computed it, against the oracle over all
    2^24 points (the oracle split over rows on all host cores)."""
    from paper_2103_07512_gb300.evolve import Evolution, gpu_fitness
    g = I.Grid(4096, 4096)
    oracle_pool()                       # spawned before the first device call
    keep = (0, 25, 49)
    rows, toks = {}, {}
    with tgp.Context(cache_budget_bytes=4 * 10**9, cache_min_cost=8) as ctx:
        dom = ctx.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi)
        if arm == "library":
            ev = DeviceEvolution(ctx, dom, pop_size=50, generations=50, seed=3)

            def on_gen(gen, rmse):
                if gen.index in keep:
                    rows[gen.index] = rmse.copy()
                    toks[gen.index] = ctx.population_tokens(ev.pop)
            ev.run(on_gen)
            ev.close()
        else:
            ev = Evolution(gpu_fitness(ctx, dom), pop_size=50, generations=50, seed=3)

            def on_gen(gen, rmse):
                if gen.index in keep:
                    rows[gen.index] = rmse.copy()
                    toks[gen.index] = I.to_tokens(ev.population)
            ev.run(on_gen)
        assert ctx.stats()["cache_inserts"] > 0, ctx.stats()
        rng = np.random.default_rng(7)
        pts = np.concatenate([np.sort(rng.choice(g.N, 65536, replace=False)), [0, g.N - 1]])
        for gen in keep:
            r = check_population(ctx, toks[gen], g, rows[gen], f"evolution {arm}, generation {gen}", dom=dom,
                                 budget="evolution", elem_pts=pts, point_chunks=16)
            assert r["fitness"]["trees"] == 50
