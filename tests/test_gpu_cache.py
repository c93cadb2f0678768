"""The cross-call subtree cache (HBM entries, Keijzer-style flush under a
budget): results with the cache on are bitwise those with it off, across the
generations of an evolutionary run, under budgets small enough to force
evictions, for phenotypes and fitness, and against the oracle."""
import numpy as np
import pytest

import oracle
import paper_2103_07512_gb300 as tgp
from paper_2103_07512_gb300 import inputs as I
from paper_2103_07512_gb300.evolve import Evolution, gpu_fitness
from parity import check_population

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def run_ga(ctx, g, generations, seed=5, pop_size=50):
    dom = ctx.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi)
    rows, toks = [], []
    ev = Evolution(gpu_fitness(ctx, dom), pop_size=pop_size, generations=generations, seed=seed)

    def keep(gen, rmse):
        rows.append(rmse.copy())
        toks.append(I.to_tokens(ev.population))

    ev.run(keep)
    return rows, toks, dom


@pytest.mark.parametrize("entries,min_cost", [(4, 4), (64, 4), (64, 0)])
def test_ga_with_cache_is_bitwise_equal_to_without(entries, min_cost):
    g = I.Grid(256, 192)
    budget = entries * g.N * 4
    with tgp.Context(cache_budget_bytes=budget, cache_min_cost=min_cost) as a, tgp.Context() as b:
        ra, _, _ = run_ga(a, g, 10)
        rb, _, _ = run_ga(b, g, 10)
        for i, (x, y) in enumerate(zip(ra, rb)):
            assert np.array_equal(x.view(np.int64), y.view(np.int64)), f"generation {i}"
        st = a.stats()
        assert st["cache_bytes"] <= budget
        if min_cost:   # with the default threshold the run may store nothing
            assert st["cache_inserts"] > 0 and st["cache_hits"] > 0
        if entries == 4:
            assert st["cache_evictions"] > 0
        assert b.stats()["cache_hits"] == 0


def test_cached_generation_matches_oracle():
    g = I.Grid(64, 48)
    with tgp.Context(cache_budget_bytes=32 * g.N * 4, cache_min_cost=4) as c:
        rows, toks, dom = run_ga(c, g, 6, seed=9)
        assert c.stats()["cache_hits"] > 0
        for gen in (3, 5):
            check_population(c, toks[gen], g, rows[gen], f"generation {gen}", dom=dom, budget="evolution")


def test_cached_phenotypes_bitwise():
    tok, _, _ = I.batched_uneven(seed=21, n_trees=200)
    g = I.Grid(100, 70)
    with tgp.Context(cache_budget_bytes=256 * g.N * 4, cache_min_cost=4) as a, tgp.Context() as b:
        da, db = a.load_domain(g.W, g.H), b.load_domain(g.W, g.H)
        pa, pb = a.compile_tokens(tok), b.compile_tokens(tok)
        ref = torch.empty((tok.n_trees, g.N), dtype=torch.float32, device="cuda")
        b.evaluate(pb, db, ref)
        for call in range(4):   # seen, stored, then loaded
            out = torch.full_like(ref, float("nan"))
            a.evaluate(pa, da, out)
            torch.cuda.synchronize()
            assert torch.equal(out.view(torch.int32), ref.view(torch.int32)), f"call {call}"
        st = a.stats()
        assert st["cache_inserts"] > 0 and st["cache_hits"] > 0
        # a second population sharing subtrees with the first reads them back
        trees = I.from_tokens(tok)
        tok2 = I.to_tokens(trees[100:] + trees[:50])
        p2a, p2b = a.compile_tokens(tok2), b.compile_tokens(tok2)
        fa = a.fitness(p2a, da, tok2.n_trees)
        fb = b.fitness(p2b, db, tok2.n_trees)
        assert np.array_equal(fa.view(np.int64), fb.view(np.int64))


def test_cache_is_per_domain_and_released_with_it():
    tok, _ = I.small_population(seed=22)
    g1, g2 = I.Grid(64, 64), I.Grid(40, 30, -1.0, 2.0, -3.0, 1.0)
    with tgp.Context(cache_budget_bytes=1 << 26, cache_min_cost=4) as a, tgp.Context() as b:
        pa, pb = a.compile_tokens(tok), b.compile_tokens(tok)
        d1 = a.load_domain(g1.W, g1.H, g1.xlo, g1.xhi, g1.ylo, g1.yhi)
        d2 = a.load_domain(g2.W, g2.H, g2.xlo, g2.xhi, g2.ylo, g2.yhi)
        e1 = b.load_domain(g1.W, g1.H, g1.xlo, g1.xhi, g1.ylo, g1.yhi)
        e2 = b.load_domain(g2.W, g2.H, g2.xlo, g2.xhi, g2.ylo, g2.yhi)
        for _ in range(3):
            for da, db in ((d1, e1), (d2, e2)):
                fa = a.fitness(pa, da, tok.n_trees)
                fb = b.fitness(pb, db, tok.n_trees)
                assert np.array_equal(fa.view(np.int64), fb.view(np.int64))
        st = a.stats()
        assert st["cache_entries"] > 0 and st["cache_bytes"] > 0
        a.release_domain(d1)
        a.release_domain(d2)
        st = a.stats()
        assert st["cache_entries"] == 0 and st["cache_bytes"] == 0


def test_non_blocking_calls_with_entries_in_flight():
    tok, _ = I.small_population(seed=23)
    g = I.Grid(512, 256)
    with tgp.Context(cache_budget_bytes=1 << 28, cache_min_cost=4) as a, tgp.Context() as b:
        da, db = a.load_domain(g.W, g.H), b.load_domain(g.W, g.H)
        pa, pb = a.compile_tokens(tok), b.compile_tokens(tok)
        ref = b.fitness(pb, db, tok.n_trees)
        s = torch.cuda.Stream()
        outs = [torch.full((tok.n_trees,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(4)]
        for o in outs:          # back to back: later calls may find entries still being written
            a.fitness_dev(pa, da, o, stream=s)
        s.synchronize()
        for o in outs:
            assert np.array_equal(o.cpu().numpy().view(np.int64), ref.view(np.int64))


@pytest.mark.parametrize("columns", [True, False])
def test_tabled_subtrees_are_not_stored(columns):
    """With column and row tables, a subtree with no x or no y below it is
    tabled, never stored, and counts as one add in the cost of the subtrees
    above it: add(A(x), B(y)) costs 3 there (A and B cost 49 each as trees),
    so with a store threshold of 4 only cos(add(x, y)) and sin(cos(add(x,
    y))) are stored.  Without tables every subtree of cost >= 4 is."""
    exprs = ["sin(cos(sin(mult(x, x))))", "cos(sin(cos(mult(y, y))))",
             "add(sin(cos(sin(mult(x, x)))), cos(sin(cos(mult(y, y)))))", "sin(cos(add(x, y)))"]
    tok = I.to_tokens([I.parse_string(e) for e in exprs])
    g = I.Grid(160, 96)
    with tgp.Context(cache_budget_bytes=64 * g.N * 4, cache_min_cost=4, columns=columns) as a, \
            tgp.Context(columns=columns) as b:
        da, db = a.load_domain(g.W, g.H), b.load_domain(g.W, g.H)
        pa, pb = a.compile_tokens(tok), b.compile_tokens(tok)
        ref = b.fitness(pb, db, tok.n_trees)
        for _ in range(3):      # seen, stored, loaded
            got = a.fitness(pa, da, tok.n_trees)
            assert np.array_equal(got.view(np.int64), ref.view(np.int64))
        st = a.stats()
    if columns:
        assert st["cache_inserts"] == 2 and st["cache_hits"] == 2, st
    else:
        assert st["cache_inserts"] == 9 and st["cache_hits"] == 9, st


def test_cache_ids_stay_bounded_and_the_cache_keeps_working():
    """The context-wide DAG that keys the cache is rebuilt from the live
    populations (a full flush of the cache) once it passes cache_ids_max:
    many populations adopted one after the other, two alive at a time, each
    evaluated three times (its subtrees are seen, then stored, then loaded).
    Every result is bitwise that of a context without the cache, the DAG
    stays near its bound, and loads keep happening after the rebuilds."""
    g = I.Grid(128, 96)
    cap = 1000   # about two populations' nodes
    with tgp.Context(cache_budget_bytes=256 * g.N * 4, cache_min_cost=4, cache_ids_max=cap) as a, \
            tgp.Context() as b:
        da = a.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi)
        db = b.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi)
        live = []
        hits_after = None
        for seed in range(14):
            tok, _ = I.small_population(seed=100 + seed)
            pa, pb = a.compile_tokens(tok), b.compile_tokens(tok)
            ref = b.fitness(pb, db, tok.n_trees)
            for call in range(3):
                got = a.fitness(pa, da, tok.n_trees)
                assert np.array_equal(got.view(np.int64), ref.view(np.int64)), f"population {seed} call {call}"
            b.release_population(pb)
            live.append(pa)
            if len(live) > 2:
                a.release_population(live.pop(0))
            st = a.stats()
            assert st["cache_id_nodes"] <= 2 * cap + 8 * tok.ops.size
            if st["cache_id_rebuilds"] >= 1 and hits_after is None:
                hits_after = st["cache_hits"]
        st = a.stats()
        assert st["cache_id_rebuilds"] >= 2
        assert hits_after is not None and st["cache_hits"] > hits_after
