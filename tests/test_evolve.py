"""Host logic of the evolutionary driver (no GPU): variation operators keep
the depth limit and produce valid trees, elitism keeps the best individual,
and a run is a deterministic function of its seed.  Fitness here is the
oracle on a tiny grid."""
import numpy as np

import oracle
from paper_2103_07512_gb300 import inputs as I
from paper_2103_07512_gb300.evolve import Evolution, crossover, mutate, _nodes

G = I.Grid(6, 5)


def oracle_fitness(tok):
    r64, _, _ = oracle.fitness(tok.ops, tok.imm, tok.tree_off, tok.order, G.W, G.H, G.xlo, G.xhi, G.ylo, G.yhi)
    return r64


def test_crossover_and_mutation_respect_depth_and_arity():
    rng = np.random.default_rng(0)
    pop = I.ramped_half_and_half(40, 2, 6, rng)
    for i in range(400):
        a, b = pop[i % 40], pop[(7 * i + 3) % 40]
        c = crossover(a, b, rng, max_depth=7)
        m = mutate(a, rng, max_depth=7, mutation_depth=4)
        for t in (c, m):
            assert I.depth(t) <= max(7, I.depth(a))
            for _, n, _ in _nodes(t):
                assert len(n[2]) == I.ARITY[n[0]]
            # round trip through tokens
            assert I.to_string(I.from_tokens(I.to_tokens([t]))[0]) == I.to_string(t)


def test_crossover_takes_a_subtree_of_the_second_parent():
    rng = np.random.default_rng(1)
    a = I.parse_string("add(x, mult(y, y))")
    b = I.parse_string("sin(cos(0.5))")
    subs_b = {I.to_string(n) for _, n, _ in _nodes(b)}
    seen = set()
    for _ in range(200):
        c = crossover(a, b, rng, max_depth=12)
        s = I.to_string(c)
        seen.add(s)
        assert s == I.to_string(a) or any(sb in s for sb in subs_b)
    assert "sin(cos(0.5))" in seen      # the root of `a` replaced by the whole of `b`


def test_run_is_deterministic_and_elitist():
    runs = []
    for _ in range(2):
        best = []
        ev = Evolution(oracle_fitness, pop_size=20, generations=8, seed=3)
        ev.run(lambda g, r: best.append(g.best_rmse))
        runs.append((best, [I.to_string(t) for t in ev.population]))
    assert runs[0] == runs[1]
    best = runs[0][0]
    assert all(b2 <= b1 for b1, b2 in zip(best, best[1:]))   # elitism 1: never worse


def test_depth_limit_holds_over_a_run():
    ev = Evolution(oracle_fitness, pop_size=16, generations=12, seed=4, max_depth=6, init_depth=(2, 5))
    ev.run()
    assert all(I.depth(t) <= 6 for t in ev.population)
    assert len(ev.history) == 12
