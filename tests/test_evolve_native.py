"""The library's generational step (tgp_evolve) and token export
(tgp_population_tokens) on a host-only context: every offspring is one of the
trees the variation operators of Sec. 3 / Table 2 can make from the parents,
tournament selection draws ranks with the tournament law, the depth limit and
the function set hold, elitism keeps the best tree, and the same seed gives
the same generation."""
import math

import numpy as np
import pytest

import paper_2103_07512_gb300 as tgp
from paper_2103_07512_gb300 import evolve as E
from paper_2103_07512_gb300 import inputs as I


@pytest.fixture
def raw():
    with tgp.Context(host_only=True, simplify=False) as c:
        yield c


def trees_of(ctx, pop):
    return I.from_tokens(ctx.population_tokens(pop))


def at(t, path):
    for i in path:
        t = t[2][i]
    return t


def ops_of(t, out=None):
    out = set() if out is None else out
    out.add(t[0])
    for k in t[2]:
        ops_of(k, out)
    return out


def consts_of(t, out=None):
    out = [] if out is None else out
    if t[0] == I.CONST:
        out.append(float(t[1]))
    for k in t[2]:
        consts_of(k, out)
    return out


NOT_LOWERED = tuple(f for f in I.ALL_FUNCTIONS if f != I.CLIP)


@pytest.mark.parametrize("order", [I.PREFIX, I.POSTFIX])
def test_tokens_round_trip(raw, order):
    rng = np.random.default_rng(1)
    trees = I.ramped_half_and_half(40, 1, 6, rng, NOT_LOWERED)
    pop = raw.compile_tokens(I.to_tokens(trees, order))
    tok = raw.population_tokens(pop)
    ref = I.to_tokens(trees, I.PREFIX)
    assert tok.order == I.PREFIX
    assert np.array_equal(tok.ops, ref.ops) and np.array_equal(tok.tree_off, ref.tree_off)
    assert np.array_equal(tok.imm.view(np.int32), ref.imm.view(np.int32))


def test_clip_comes_back_as_its_definition(raw):
    # clip(x, y, z) is stored as max(min(z, x), y) (Table 1)
    tok = raw.population_tokens(raw.compile_tokens(I.to_tokens([I.parse_string("clip(x, -1.0, y)")])))
    assert I.to_string(I.from_tokens(tok)[0]) == "max(min(y, x), -1.0)"


def test_tokens_of_simplified_population_are_the_stored_trees():
    t = I.parse_string("sin(mult(x, 1.0))")
    with tgp.Context(host_only=True) as c:
        tok = c.population_tokens(c.compile_tokens(I.to_tokens([t])))
    assert I.to_string(I.from_tokens(tok)[0]) == "sin(x)"


def test_token_buffers_too_small_are_refused(raw):
    pop = raw.compile_tokens(I.to_tokens([I.parse_string("add(x, 0.5)")]))
    L = tgp.lib()
    import ctypes
    ops = np.empty(3, np.int32)
    imm = np.empty(1, np.float32)
    off = np.empty(2, np.int64)
    no, ni, nt = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    for cap in ((2, 1, 2), (3, 0, 2), (3, 1, 1)):
        rc = L.tgp_population_tokens(raw._h, pop, tgp._ptr(ops), cap[0], tgp._ptr(imm), cap[1], tgp._ptr(off), cap[2],
                                     ctypes.byref(no), ctypes.byref(ni), ctypes.byref(nt))
        assert rc == tgp.E_INVALID
        assert (no.value, ni.value, nt.value) == (3, 1, 1)


def test_same_seed_same_generation_and_parent_untouched(raw):
    rng = np.random.default_rng(2)
    tok = I.to_tokens(I.ramped_half_and_half(30, 2, 6, rng))
    pop = raw.compile_tokens(tok)
    r = rng.random(30)
    a = raw.population_tokens(raw.evolve(pop, r, seed=11))
    b = raw.population_tokens(raw.evolve(pop, r, seed=11))
    c = raw.population_tokens(raw.evolve(pop, r, seed=12))
    assert np.array_equal(a.ops, b.ops) and np.array_equal(a.imm, b.imm)
    assert not (np.array_equal(a.ops, c.ops) and np.array_equal(a.imm, c.imm))
    again = raw.population_tokens(pop)
    assert np.array_equal(again.ops, tok.ops) and np.array_equal(again.imm, tok.imm)


def test_elitism_keeps_the_best_finite_tree(raw):
    rng = np.random.default_rng(3)
    trees = I.ramped_half_and_half(20, 2, 5, rng)
    pop = raw.compile_tokens(I.to_tokens(trees))
    r = rng.random(20) + 1.0
    r[0] = np.nan
    r[1] = np.inf
    r[7] = 0.5
    r[12] = 0.75
    nxt = trees_of(raw, raw.evolve(pop, r, seed=1, elitism=2))
    assert nxt[0] == trees[7] and nxt[1] == trees[12]


def test_crossover_offspring_are_subtree_swaps_of_parents(raw):
    rng = np.random.default_rng(4)
    trees = I.ramped_half_and_half(8, 1, 3, rng)
    max_depth = 4
    pop = raw.compile_tokens(I.to_tokens(trees))
    swaps = set()
    for a in trees:
        for pa, _, da in E._nodes(a):
            for b in trees:
                for _, sb, _ in E._nodes(b):
                    if da + I.depth(sb) <= max_depth:
                        swaps.add(E._replace(a, pa, sb))
    made = 0
    for seed in range(20):
        kids = trees_of(raw, raw.evolve(pop, rng.random(8), seed=seed, p_crossover=1.0, p_mutation=-1,
                                        elitism=-1, max_depth=max_depth))
        assert len(kids) == 8
        for k in kids:
            assert k in swaps or k in trees, I.to_string(k)
            assert I.depth(k) <= max_depth
            made += k not in trees
    assert made > 50


def test_mutation_offspring_replace_one_subtree_by_a_grow_tree(raw):
    rng = np.random.default_rng(5)
    trees = I.ramped_half_and_half(10, 2, 4, rng)
    pop = raw.compile_tokens(I.to_tokens(trees))
    funcs = [I.ADD, I.SIN, I.IF]
    mdepth, max_depth, lo, hi = 2, 6, 2.0, 3.0

    def explained(k):
        for a in trees:
            for pa, _, da in E._nodes(a):
                try:
                    sub = at(k, pa)
                except IndexError:
                    continue
                if E._replace(a, pa, sub) != k or I.depth(sub) > mdepth or da + I.depth(sub) > max_depth:
                    continue
                if ops_of(sub) - set(funcs) - {I.X, I.Y, I.CONST}:
                    continue
                if all(lo <= v < hi for v in consts_of(sub)):
                    return True
        return False

    new = 0
    for seed in range(15):
        kids = trees_of(raw, raw.evolve(pop, rng.random(10), seed=seed, p_crossover=-1, p_mutation=1.0,
                                        elitism=-1, max_depth=max_depth, mutation_depth=mdepth, functions=funcs,
                                        const_range=(lo, hi)))
        for k in kids:
            assert k in trees or explained(k), I.to_string(k)
            new += k not in trees
    assert new > 60


def test_tournament_selection_follows_the_rank_law(raw):
    # distinct constant trees; with variation off every offspring is a
    # tournament winner: P(rank i) = ((T-i)^k - (T-i-1)^k) / T^k
    T, k = 10, 3
    trees = [I.leaf(I.CONST, float(i)) for i in range(T)]
    pop = raw.compile_tokens(I.to_tokens(trees))
    rmse = np.array([5.0, 1.0, 7.0, 3.0, 9.0, 0.5, 2.0, 8.0, 4.0, 6.0])
    rank_of_value = {float(i): int(np.argsort(np.argsort(rmse))[i]) for i in range(T)}
    counts = np.zeros(T)
    for seed in range(500):
        for t in trees_of(raw, raw.evolve(pop, rmse, seed=seed, tournament=k, p_crossover=-1, p_mutation=-1,
                                          elitism=-1)):
            counts[rank_of_value[float(t[1])]] += 1
    n = counts.sum()
    p = np.array([((T - i) ** k - (T - i - 1) ** k) / T ** k for i in range(T)])
    chi2 = float(((counts - n * p) ** 2 / (n * p)).sum())
    assert chi2 < 27.88, (chi2, counts)   # 0.999 quantile of chi-square with 9 degrees of freedom


def test_non_finite_rmse_loses_tournaments(raw):
    trees = [I.leaf(I.CONST, float(i)) for i in range(4)]
    pop = raw.compile_tokens(I.to_tokens(trees))
    rmse = np.array([np.nan, np.inf, 3.0, np.nan])
    wins = set()
    for seed in range(50):
        for t in trees_of(raw, raw.evolve(pop, rmse, seed=seed, tournament=4, p_crossover=-1, p_mutation=-1,
                                          elitism=-1)):
            wins.add(float(t[1]))
    # a tournament of 4 draws tree 2 with probability 1 - (3/4)^4; every other win needs all draws non-finite
    assert 2.0 in wins and wins <= {0.0, 1.0, 2.0, 3.0}


def test_depth_limit_and_function_set_hold_over_generations():
    rng = np.random.default_rng(6)
    funcs = [I.ADD, I.MUL, I.SIN, I.IF]
    with tgp.Context(host_only=True) as c:
        pop = c.compile_tokens(I.to_tokens(I.ramped_half_and_half(30, 2, 5, rng, funcs)))
        for g in range(25):
            nxt = c.evolve(pop, rng.random(30), seed=g, max_depth=7, functions=funcs)
            c.release_population(pop)
            pop = nxt
        for t in trees_of(c, pop):
            assert I.depth(t) <= 7
            assert not (ops_of(t) - set(funcs) - {I.X, I.Y, I.CONST})


def test_simplifying_context_offspring_equal_simplified_tokens():
    rng = np.random.default_rng(7)
    with tgp.Context(host_only=True) as c, tgp.Context(host_only=True) as d:
        pop = c.compile_tokens(I.to_tokens(I.ramped_half_and_half(30, 2, 6, rng)))
        for g in range(5):
            pop = c.evolve(pop, rng.random(30), seed=g)
        tok = c.population_tokens(pop)
        again = d.population_tokens(d.compile_tokens(tok))
        # offspring are already in simplified form: compiling them again folds
        # no node away (operands of commutative operators may come back
        # swapped, their canonical order being that of DAG ids, and with them
        # which of two negations an addition absorbs)
        assert np.array_equal(tok.tree_off, again.tree_off)


def test_invalid_arguments():
    with tgp.Context(host_only=True) as c:
        pop = c.compile_tokens(I.to_tokens([I.parse_string("add(x, y)")]))
        with pytest.raises(tgp.TgpError):
            c.evolve(pop, [1.0], seed=0, functions=[I.X])
        with pytest.raises(tgp.TgpError):
            c.evolve(pop + 999, [1.0], seed=0)
        with pytest.raises(tgp.TgpError):
            c.evolve(pop, [1.0], seed=0, max_depth=1025)
        with pytest.raises(tgp.TgpError):
            c.population_tokens(pop + 999)


def test_all_non_finite_rmse_still_gives_a_generation():
    rng = np.random.default_rng(8)
    with tgp.Context(host_only=True) as c:
        pop = c.compile_tokens(I.to_tokens(I.ramped_half_and_half(12, 2, 4, rng)))
        nxt = c.evolve(pop, np.full(12, math.inf), seed=3)
        assert c.population_tokens(nxt).n_trees == 12


def test_offspring_stay_within_the_token_limit(raw):
    """A tree whose written-out size doubles with every level (add(t, t),
    23 levels: 2^24 - 1 tokens, 23 DAG nodes): crossover that would graft a
    larger subtree deeper gives the parent instead, so every offspring stays
    within the 2^24-token limit of one tree."""
    seq = np.array([I.X], np.int32)
    for _ in range(23):
        seq = np.concatenate([np.array([I.ADD], np.int32), seq, seq])
    ops = np.concatenate([seq, np.array([I.Y], np.int32)])
    pop = raw.compile_population(ops, np.zeros(0, np.float32), np.array([0, seq.size, seq.size + 1], np.int64))
    assert raw.stats()["dag_internal"] == 23
    grew = 0
    for seed in range(4):
        tok = raw.population_tokens(raw.evolve(pop, np.array([0.0, 1.0]), seed=seed, p_crossover=1.0,
                                               p_mutation=-1, elitism=-1, max_depth=64))
        sizes = np.diff(tok.tree_off)
        assert sizes.max() <= (1 << 24)
        grew += int((sizes > 1).sum())
    assert grew > 0
