"""Seeded synthetic inputs: GP populations as token arrays.

This module holds no evaluation arithmetic.  It only draws random trees and
writes them as prefix or postfix token streams, so that the CUDA path and the
CPU oracle can be fed the very same inputs.

Token format (the library's boundary):
  ops      int32[n_tokens]  opcodes (below), all trees back to back
  imm      float32[n_const] one value per CONST token, in stream order
  tree_off int64[T+1]       tree t owns ops[tree_off[t]:tree_off[t+1]]

Opcodes: terminals X=0, Y=1, CONST=2; functions of Table 1 (TensorGP, arXiv
2103.07512) ADD=3, SUB=4, MUL=5, DIV=6, SIN=7, COS=8, NEG=9, ABS=10, MIN=11,
MAX=12, TAN=13, EXP=14, LOG=15, POW=16, MDIST=17, SQRT=18, SIGN=19, CLIP=20
(arity 3), MOD=21, FRAC=22, IF=23 (arity 3).

Generators:
  * ramped half-and-half (Sec. 4.1, Table 2): depths ramp evenly from dmin to
    dmax across the population, half of each depth built with *grow*, half with
    *full*; the root alone has depth 0; terminals are drawn uniformly from
    {x, y, const} with const ~ U[-1, 1] rounded to binary32;
  * exact-size trees with a shared-subtree pool, for batched uneven
    populations with a controlled fraction of duplicated subtrees.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

X, Y, CONST = 0, 1, 2
ADD, SUB, MUL, DIV, SIN, COS, NEG, ABS, MIN, MAX = range(3, 13)
TAN, EXP, LOG, POW, MDIST, SQRT, SIGN, CLIP, MOD, FRAC, IF = range(13, 24)
PREFIX, POSTFIX = 0, 1

ARITY = {X: 0, Y: 0, CONST: 0, ADD: 2, SUB: 2, MUL: 2, DIV: 2,
         SIN: 1, COS: 1, NEG: 1, ABS: 1, MIN: 2, MAX: 2,
         TAN: 1, EXP: 1, LOG: 1, POW: 2, MDIST: 2, SQRT: 1, SIGN: 1, CLIP: 3, MOD: 2, FRAC: 1, IF: 3}
NAMES = {X: "x", Y: "y", CONST: "const", ADD: "add", SUB: "sub", MUL: "mult", DIV: "div",
         SIN: "sin", COS: "cos", NEG: "neg", ABS: "abs", MIN: "min", MAX: "max",
         TAN: "tan", EXP: "exp", LOG: "log", POW: "pow", MDIST: "mdist", SQRT: "sqrt", SIGN: "sign",
         CLIP: "clip", MOD: "mod", FRAC: "frac", IF: "if"}
BY_NAME = {v: k for k, v in NAMES.items()}
BY_NAME["mul"] = MUL

# the function set of the benchmark configurations
FUNCTIONS = (ADD, SUB, MUL, DIV, SIN, COS, NEG, ABS, MIN, MAX)
# every mathematical and conditional operator of Table 1
ALL_FUNCTIONS = FUNCTIONS + (TAN, EXP, LOG, POW, MDIST, SQRT, SIGN, CLIP, MOD, FRAC, IF)
TERMINALS = (X, Y, CONST)
UNARY = tuple(f for f in FUNCTIONS if ARITY[f] == 1)
BINARY = tuple(f for f in FUNCTIONS if ARITY[f] == 2)


# A tree node is a tuple (op, imm, kids): imm is a float for CONST, else None.
def leaf(op, imm=None):
    return (op, None if op != CONST else np.float32(imm), ())


def node(op, *kids):
    assert len(kids) == ARITY[op]
    return (op, None, tuple(kids))


def size(t) -> int:
    return 1 + sum(size(k) for k in t[2])


def depth(t) -> int:
    return 0 if not t[2] else 1 + max(depth(k) for k in t[2])


def _rand_terminal(rng):
    op = TERMINALS[int(rng.integers(len(TERMINALS)))]
    if op == CONST:
        return leaf(CONST, np.float32(rng.uniform(-1.0, 1.0)))
    return leaf(op)


def _full(rng, d, funcs):
    if d == 0:
        return _rand_terminal(rng)
    f = funcs[int(rng.integers(len(funcs)))]
    return node(f, *[_full(rng, d - 1, funcs) for _ in range(ARITY[f])])


def _grow(rng, d, funcs, at_root=True):
    if d == 0:
        return _rand_terminal(rng)
    if at_root:
        f = funcs[int(rng.integers(len(funcs)))]
    else:
        pick = int(rng.integers(len(funcs) + len(TERMINALS)))
        if pick >= len(funcs):
            return _rand_terminal(rng)
        f = funcs[pick]
    return node(f, *[_grow(rng, d - 1, funcs, False) for _ in range(ARITY[f])])


def ramped_half_and_half(n_trees: int, dmin: int, dmax: int, rng, funcs=FUNCTIONS):
    """Ramped half-and-half initial population (Table 2 generation method)."""
    depths = list(range(dmin, dmax + 1))
    trees = []
    for i in range(n_trees):
        d = depths[i % len(depths)]
        full = (i // len(depths)) % 2 == 0
        trees.append(_full(rng, d, funcs) if full else _grow(rng, d, funcs))
    return trees


def _cap(d):
    """Largest node count of a tree of depth <= d (binary fan-out)."""
    return (1 << (d + 1)) - 1


def _exact(rng, n, dmax, funcs, pool, budget, stats, at_root):
    """Random tree of exactly n nodes and depth <= dmax (n <= _cap(dmax)).

    budget[0] is the number of nodes this tree may still take from the pool of
    earlier trees' subtrees; a non-root subtree of size >= 3 that fits the
    budget is taken from the pool with probability 1/2 when the pool holds one
    of that exact size and a fitting depth."""
    if n == 1:
        return _rand_terminal(rng)
    if not at_root and 3 <= n <= budget[0] and rng.random() < 0.5:
        cands = pool.get(n)
        if cands:
            ok = [c for c in cands if c[1] <= dmax]
            if ok:
                t = ok[int(rng.integers(len(ok)))][0]
                budget[0] -= n
                stats["dup_nodes"] += n
                stats["dup_subtrees"] += 1
                return t
    unary_ok = n - 1 <= _cap(dmax - 1)
    bin_lo = max(1, n - 1 - _cap(dmax - 1))
    bin_hi = min(n - 2, _cap(dmax - 1))
    binary_ok = n >= 3 and bin_lo <= bin_hi
    un = [f for f in funcs if ARITY[f] == 1]
    bi = [f for f in funcs if ARITY[f] == 2]
    choices = (un if unary_ok else []) + (bi if binary_ok else [])
    f = choices[int(rng.integers(len(choices)))]
    if ARITY[f] == 1:
        return node(f, _exact(rng, n - 1, dmax - 1, funcs, pool, budget, stats, False))
    a = int(rng.integers(bin_lo, bin_hi + 1))
    return node(f, _exact(rng, a, dmax - 1, funcs, pool, budget, stats, False),
                _exact(rng, n - 1 - a, dmax - 1, funcs, pool, budget, stats, False))


def _add_to_pool(t, pool, limit=64):
    n = size(t)
    if n >= 3:
        lst = pool.setdefault(n, [])
        if len(lst) < limit:
            lst.append((t, depth(t)))
    for k in t[2]:
        _add_to_pool(k, pool, limit)


def exact_size_population(n_trees, size_lo, size_hi, max_depth, dup_p, rng, funcs=FUNCTIONS):
    """Trees with node counts ~ U{size_lo..size_hi}, depth <= max_depth.

    About a fraction dup_p of each tree's nodes is taken, as whole subtrees of
    size >= 3, from a pool of subtrees of earlier trees (a per-tree budget of
    round(dup_p * n) nodes).  Returns (trees, stats); stats counts the reused
    subtrees, the nodes inside them and their fraction of all nodes.
    """
    pool: dict = {}
    stats = {"dup_nodes": 0, "dup_subtrees": 0}
    trees = []
    for _ in range(n_trees):
        n = int(rng.integers(size_lo, size_hi + 1))
        n = min(n, _cap(max_depth))
        budget = [int(round(dup_p * n))]
        t = _exact(rng, n, max_depth, funcs, pool, budget, stats, True)
        trees.append(t)
        _add_to_pool(t, pool)
    total = sum(size(t) for t in trees)
    stats["total_nodes"] = total
    stats["dup_fraction"] = stats["dup_nodes"] / max(total, 1)
    return trees, stats


# ------------------------------------------------------------ serialisation

def _emit_prefix(t, ops, imm):
    stack = [t]
    while stack:
        cur = stack.pop()
        ops.append(cur[0])
        if cur[0] == CONST:
            imm.append(cur[1])
        stack.extend(reversed(cur[2]))


def _emit_postfix(t, ops, imm):
    # iterative post-order: children left to right, then the node
    stack = [(t, False)]
    while stack:
        cur, done = stack.pop()
        if done or not cur[2]:
            ops.append(cur[0])
            if cur[0] == CONST:
                imm.append(cur[1])
            continue
        stack.append((cur, True))
        for k in reversed(cur[2]):
            stack.append((k, False))


@dataclass
class Tokens:
    ops: np.ndarray       # int32
    imm: np.ndarray       # float32
    tree_off: np.ndarray  # int64, T+1
    order: int

    @property
    def n_trees(self) -> int:
        return int(self.tree_off.size - 1)

    def node_counts(self) -> np.ndarray:
        return np.diff(self.tree_off)


def to_tokens(trees, order=PREFIX) -> Tokens:
    ops: list = []
    imm: list = []
    off = [0]
    emit = _emit_prefix if order == PREFIX else _emit_postfix
    for t in trees:
        emit(t, ops, imm)
        off.append(len(ops))
    return Tokens(np.asarray(ops, np.int32), np.asarray(imm, np.float32),
                  np.asarray(off, np.int64), order)


def from_tokens(tok: Tokens):
    """Rebuilds the tuple trees from a token stream (no validation beyond arity)."""
    trees = []
    ip = 0
    for t in range(tok.n_trees):
        seq = tok.ops[tok.tree_off[t]:tok.tree_off[t + 1]]
        if tok.order == PREFIX:
            pos = 0

            def rec():
                nonlocal pos, ip
                op = int(seq[pos])
                pos += 1
                if op == CONST:
                    v = tok.imm[ip]
                    ip += 1
                    return leaf(CONST, v)
                return (op, None, tuple(rec() for _ in range(ARITY[op])))
            trees.append(rec())
        else:
            st = []
            for op in seq:
                op = int(op)
                if op == CONST:
                    st.append(leaf(CONST, tok.imm[ip]))
                    ip += 1
                    continue
                ar = ARITY[op]
                kids = tuple(st[len(st) - ar:]) if ar else ()
                del st[len(st) - ar:]
                st.append((op, None, kids))
            trees.append(st[0])
    return trees


def convert_order(tok: Tokens, order: int) -> Tokens:
    return to_tokens(from_tokens(tok), order)


def to_string(t) -> str:
    op, v, kids = t
    if op == CONST:
        return repr(float(v))
    if not kids:
        return NAMES[op]
    return f"{NAMES[op]}(" + ", ".join(to_string(k) for k in kids) + ")"


def parse_string(s: str):
    """Parses 'add(x, mult(y, 0.5))' into a tuple tree (test tooling)."""
    s = s.replace(" ", "")
    pos = 0

    def rec():
        nonlocal pos
        j = pos
        while j < len(s) and s[j] not in "(),":
            j += 1
        word = s[pos:j]
        pos = j
        if word in BY_NAME and BY_NAME[word] not in (X, Y, CONST) and pos < len(s) and s[pos] == "(":
            op = BY_NAME[word]
            pos += 1
            kids = [rec()]
            while s[pos] == ",":
                pos += 1
                kids.append(rec())
            assert s[pos] == ")"
            pos += 1
            return node(op, *kids)
        if word in ("x", "y"):
            return leaf(BY_NAME[word])
        return leaf(CONST, np.float32(float(word)))
    t = rec()
    assert pos == len(s), s
    return t


# ------------------------------------------------------------ workloads

@dataclass(frozen=True)
class Grid:
    W: int
    H: int
    xlo: float = -5.0
    xhi: float = 5.0
    ylo: float = -5.0
    yhi: float = 5.0

    @property
    def N(self) -> int:
        return self.W * self.H


def small_population(seed=0, order=PREFIX):
    """50 RHH trees, depth 2-6, the 10-function set; 64x64 grid over [-5,5]^2."""
    rng = np.random.default_rng(seed)
    return to_tokens(ramped_half_and_half(50, 2, 6, rng), order), Grid(64, 64)


def population_at_scale(seed=1, order=PREFIX):
    """100 RHH trees, depth 2-8; 1024x1024 grid over [-5,5]^2."""
    rng = np.random.default_rng(seed)
    return to_tokens(ramped_half_and_half(100, 2, 8, rng), order), Grid(1024, 1024)


def batched_uneven(seed=2, order=PREFIX, n_trees=4096, dup_p=0.3):
    """4096 trees of U{3..255} nodes, depth <= 12, shared-subtree pool p=0.3;
    256x256 grid over [-5,5]^2.  Returns (tokens, grid, stats)."""
    rng = np.random.default_rng(seed)
    trees, stats = exact_size_population(n_trees, 3, 255, 12, dup_p, rng)
    return to_tokens(trees, order), Grid(256, 256), stats


def serving_jobs(n_jobs, seed=4, trees=(10, 1000), depth=(2, 10), side_log2=(6.0, 11.0), pool=None,
                 order=PREFIX):
    """Evaluation jobs for the serving loop: each has U{trees} RHH trees of
    depth U{depth} ramp, a square grid of side round(2^u), u ~ U[side_log2]
    (log-uniform point counts, sides that are not powers of two included),
    over [-5,5]^2, and the Pagie target or a random full depth-4 target tree
    with probability 1/2 each.  With `pool`, job i takes population i % pool
    (drawn once), so long streams need not draw thousands of populations.
    Returns a list of dicts {tok, W, H, target_tokens (None for Pagie)}."""
    rng = np.random.default_rng(seed)
    pops = []
    jobs = []
    for i in range(n_jobs):
        if pool is None or len(pops) < pool:
            n = int(rng.integers(trees[0], trees[1] + 1))
            pops.append(to_tokens(ramped_half_and_half(n, depth[0], depth[1], rng), order))
            tok = pops[-1]
        else:
            tok = pops[i % pool]
        side = int(round(2.0 ** rng.uniform(side_log2[0], side_log2[1])))
        target = None
        if rng.random() < 0.5:
            tt = to_tokens([_full(rng, 4, FUNCTIONS)], PREFIX)
            target = (tt.ops, tt.imm, tt.order)
        jobs.append({"tok": tok, "W": side, "H": side, "target_tokens": target})
    return jobs
