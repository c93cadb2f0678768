"""Generational GP around the GPU fitness path.

Two drivers of the same algorithm (TensorGP, Sec. 3 and Table 2: tournament
selection, subtree crossover and subtree mutation, elitism):
  * Evolution: the population lives as Python trees; each generation is
    written as tokens, compiled into one population DAG and scored in one
    fitness call.  Any fitness callable works (the oracle, the GPU path).
  * DeviceEvolution: the population stays a library population; the
    variation step runs in the library on the population DAG (tgp_evolve),
    so unchanged subtrees are never re-parsed and no tokens cross the API
    between generations.
Their random streams differ (numpy here, splitmix64 in the library), so the
two produce different runs of the same algorithm.  With a context created with a
non-zero cache budget, subtrees that survive from one generation to the next
are read back from the device-resident subtree cache instead of being
evaluated again (Sec. 2, Handley's DAG caching across evaluations).

The variation operators follow the usual tree-GP definitions:
  * tournament of `tournament` individuals drawn with replacement, lowest RMSE
    wins (non-finite RMSE ranks last);
  * subtree crossover: a uniformly chosen node of the first parent is replaced
    by a uniformly chosen subtree of the second; an offspring deeper than
    `max_depth` is discarded and the first parent is copied instead;
  * subtree mutation: a uniformly chosen node is replaced by a *grow* tree of
    depth 0..`mutation_depth`, under the same depth limit;
  * `elitism` best individuals are copied unchanged.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math
import time

import numpy as np

from . import inputs as I


def _nodes(t, path=(), d=0, out=None):
    """(path, subtree, depth of the node) for every node, preorder."""
    if out is None:
        out = []
    out.append((path, t, d))
    for i, k in enumerate(t[2]):
        _nodes(k, path + (i,), d + 1, out)
    return out


def _replace(t, path, new):
    if not path:
        return new
    kids = list(t[2])
    kids[path[0]] = _replace(kids[path[0]], path[1:], new)
    return (t[0], t[1], tuple(kids))


def crossover(a, b, rng, max_depth):
    """Subtree crossover; returns the offspring of `a` or a copy of `a`."""
    na = _nodes(a)
    nb = _nodes(b)
    pa, _, da = na[int(rng.integers(len(na)))]
    _, sb, _ = nb[int(rng.integers(len(nb)))]
    if da + I.depth(sb) > max_depth:
        return a
    return _replace(a, pa, sb)


def mutate(a, rng, max_depth, mutation_depth, funcs=I.FUNCTIONS):
    """Subtree mutation with a grow tree; returns a copy of `a` on a depth overflow."""
    na = _nodes(a)
    pa, _, da = na[int(rng.integers(len(na)))]
    d = int(rng.integers(0, mutation_depth + 1))
    sub = I._grow(rng, d, funcs) if d > 0 else I._rand_terminal(rng)
    if da + I.depth(sub) > max_depth:
        return a
    return _replace(a, pa, sub)


def _rank_key(r):
    return r if math.isfinite(r) else math.inf


@dataclass
class Generation:
    index: int
    best_rmse: float
    mean_nodes: float
    nodes: int            # token count of the population
    seconds: float        # wall time of the fitness call
    stats: dict = field(default_factory=dict)


class Evolution:
    """Runs `generations` generations; `fitness(tokens) -> np.ndarray[T]` scores a
    population given as tokens (the GPU path, or any other evaluator)."""

    def __init__(self, fitness, pop_size=50, generations=50, seed=0, tournament=3, p_crossover=0.9,
                 p_mutation=0.1, elitism=1, max_depth=12, init_depth=(2, 6), mutation_depth=4,
                 funcs=I.FUNCTIONS):
        self.fitness = fitness
        self.pop_size = pop_size
        self.generations = generations
        self.rng = np.random.default_rng(seed)
        self.tournament = tournament
        self.p_crossover = p_crossover
        self.p_mutation = p_mutation
        self.elitism = elitism
        self.max_depth = max_depth
        self.mutation_depth = mutation_depth
        self.funcs = funcs
        self.population = I.ramped_half_and_half(pop_size, init_depth[0], init_depth[1], self.rng, funcs)
        self.history: list[Generation] = []
        self.best = None

    def _select(self, rmse):
        idx = self.rng.integers(0, len(rmse), size=self.tournament)
        return int(min(idx, key=lambda i: (_rank_key(rmse[i]), i)))

    def step(self, on_generation=None):
        tok = I.to_tokens(self.population)
        t0 = time.perf_counter()
        rmse = np.asarray(self.fitness(tok), dtype=np.float64)
        dt = time.perf_counter() - t0
        order = sorted(range(len(rmse)), key=lambda i: (_rank_key(rmse[i]), i))
        best = order[0]
        if self.best is None or _rank_key(rmse[best]) < _rank_key(self.best[1]):
            self.best = (self.population[best], float(rmse[best]))
        g = Generation(len(self.history), float(rmse[best]),
                       float(np.mean(tok.node_counts())), int(len(tok.ops)), dt)
        if on_generation:
            on_generation(g, rmse)
        self.history.append(g)
        nxt = [self.population[i] for i in order[:self.elitism]]
        while len(nxt) < self.pop_size:
            a = self.population[self._select(rmse)]
            u = self.rng.random()
            if u < self.p_crossover:
                b = self.population[self._select(rmse)]
                child = crossover(a, b, self.rng, self.max_depth)
            elif u < self.p_crossover + self.p_mutation:
                child = mutate(a, self.rng, self.max_depth, self.mutation_depth, self.funcs)
            else:
                child = a
            nxt.append(child)
        self.population = nxt
        return rmse

    def run(self, on_generation=None):
        for _ in range(self.generations):
            self.step(on_generation)
        return self.history


class DeviceEvolution:
    """The generational loop with selection and variation in the library
    (tgp_evolve); `ctx` is a library context and `domain` a loaded domain.
    The initial population is the same ramped half-and-half draw as
    Evolution's for the same seed."""

    def __init__(self, ctx, domain, pop_size=50, generations=50, seed=0, tournament=3, p_crossover=0.9,
                 p_mutation=0.1, elitism=1, max_depth=12, init_depth=(2, 6), mutation_depth=4,
                 funcs=I.FUNCTIONS):
        self.ctx = ctx
        self.domain = domain
        self.pop_size = pop_size
        self.generations = generations
        self.seed = seed
        self.params = dict(tournament=tournament, p_crossover=p_crossover, p_mutation=p_mutation,
                           elitism=elitism, max_depth=max_depth, mutation_depth=mutation_depth,
                           functions=list(funcs))
        rng = np.random.default_rng(seed)
        self.pop = ctx.compile_tokens(I.to_tokens(I.ramped_half_and_half(pop_size, init_depth[0], init_depth[1],
                                                                         rng, funcs)))
        self.history: list[Generation] = []
        self.variation_seconds = 0.0
        self.best = None

    def step(self, on_generation=None):
        ctx = self.ctx
        t0 = time.perf_counter()
        rmse = ctx.fitness(self.pop, self.domain, self.pop_size)
        dt = time.perf_counter() - t0
        st = ctx.stats()
        best = min(range(len(rmse)), key=lambda i: (_rank_key(rmse[i]), i))
        if self.best is None or _rank_key(rmse[best]) < _rank_key(self.best[1]):
            tok = ctx.population_tokens(self.pop)
            self.best = (I.from_tokens(tok)[best], float(rmse[best]))
        g = Generation(len(self.history), float(rmse[best]), st["tree_nodes"] / self.pop_size,
                       int(st["tree_nodes"]), dt)
        if on_generation:
            on_generation(g, rmse)
        self.history.append(g)
        t1 = time.perf_counter()
        gen_seed = (self.seed * 1000003 + len(self.history)) & 0xFFFFFFFFFFFFFFFF
        nxt = ctx.evolve(self.pop, rmse, seed=gen_seed, **self.params)
        ctx.release_population(self.pop)
        self.pop = nxt
        self.variation_seconds += time.perf_counter() - t1
        return rmse

    def run(self, on_generation=None):
        for _ in range(self.generations):
            self.step(on_generation)
        return self.history

    def close(self):
        if self.pop is not None:
            self.ctx.release_population(self.pop)
            self.pop = None


def gpu_fitness(ctx, domain):
    """Fitness callable for Evolution on a library context and loaded domain:
    compiles the generation's tokens, scores them, releases the population."""
    def f(tok):
        pop = ctx.compile_tokens(tok)
        try:
            return ctx.fitness(pop, domain, tok.n_trees)
        finally:
            ctx.release_population(pop)
    return f


def main(argv=None):
    """Command line: one evolutionary run on the GPU, one line per generation."""
    import argparse
    from . import Context

    ap = argparse.ArgumentParser(prog="python -m paper_2103_07512_gb300.evolve")
    ap.add_argument("--grid", type=int, default=4096, help="side of the square grid over [-5,5]^2")
    ap.add_argument("--population", type=int, default=50)
    ap.add_argument("--generations", type=int, default=50)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--cache-gb", type=float, default=20.0, help="subtree cache budget (0: off)")
    ap.add_argument("--min-cost", type=int, default=0, help="store threshold of the cache (0: default)")
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--variation", choices=("host", "library"), default="host",
                    help="selection and variation in Python (host) or in the library on the DAG (library)")
    ap.add_argument("--no-tables", action="store_true",
                    help="evaluate every subtree at every point (no column or row tables)")
    a = ap.parse_args(argv)
    with Context(device=a.device, cache_budget_bytes=int(a.cache_gb * 1e9), cache_min_cost=a.min_cost,
                 columns=not a.no_tables) as ctx:
        dom = ctx.load_domain(a.grid, a.grid)
        if a.variation == "library":
            ev = DeviceEvolution(ctx, dom, pop_size=a.population, generations=a.generations, seed=a.seed)
        else:
            ev = Evolution(gpu_fitness(ctx, dom), pop_size=a.population, generations=a.generations, seed=a.seed)

        def report(g, rmse):
            st = ctx.stats()
            print(f"gen {g.index:3d}  best {g.best_rmse:.6g}  nodes {g.nodes:6d}  {1e3 * g.seconds:8.3f} ms  "
                  f"cache hits {st['cache_hits']} inserts {st['cache_inserts']} evictions {st['cache_evictions']}",
                  flush=True)

        ev.run(report)
        print(f"best {ev.best[1]:.6g}: {I.to_string(ev.best[0])}")


if __name__ == "__main__":
    main()
