"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every element and every fitness is judged by the rules of tests/parity.py:
the stated tolerance against binary64, or (counted, budgeted) the oracle's
binary32 error bound where it shows the tolerance cannot be met; every tree's
fitness against the oracle's over the elements it finds comparable, and the
kernel's reduction against the device phenotype.  Sizes span several tiles
and ragged tails; the full-size workloads are checked on sampled points for
elements and over all points for fitness (the oracle in a spawn process pool).
"""
import numpy as np
import pytest

import oracle
import paper_2103_07512_gb300 as tgp
from paper_2103_07512_gb300 import inputs as I
from parity import check_population, oracle_pool

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def subset(tok, idx):
    trees = I.from_tokens(tok)
    return I.to_tokens([trees[i] for i in idx], tok.order)


@pytest.fixture(scope="module")
def ctx():
    c = tgp.Context()
    yield c
    c.close()


def load(ctx, g, **kw):
    return ctx.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi, **kw)


def phenotype(ctx, tok, g, pop=None, dom=None):
    dom = load(ctx, g) if dom is None else dom
    pop = ctx.compile_tokens(tok) if pop is None else pop
    out = torch.empty((tok.n_trees, g.N), dtype=torch.float32, device="cuda")
    ctx.evaluate(pop, dom, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def full_check(ctx, tok, g, context="", budget="default"):
    """Every element and every fitness against the oracle."""
    dom = load(ctx, g)
    pop = ctx.compile_tokens(tok)
    fit = ctx.fitness(pop, dom, tok.n_trees)
    r = check_population(ctx, tok, g, fit, context, pop=pop, dom=dom, budget=budget)
    ctx.release_population(pop)
    ctx.release_domain(dom)
    return fit, r


# ---------------------------------------------------------------- small configs

@pytest.mark.parametrize("K,threads", [(0, 0), (1, 128), (2, 64), (4, 128), (8, 128), (8, 32)])
def test_small_population_every_element(K, threads):
    """50 RHH trees (depth 2-6) on the 64x64 grid, Pagie target."""
    tok, g = I.small_population(seed=0)
    with tgp.Context(points_per_thread=K, threads_per_block=threads) as c:
        full_check(c, tok, g, f"K={K} threads={threads}", budget="small")


@pytest.mark.parametrize("W,H", [(1, 1), (2, 3), (7, 5), (33, 17), (1, 100), (100, 1), (129, 65)])
@pytest.mark.parametrize("K", [1, 8])
def test_odd_grids_and_ragged_tails(W, H, K):
    tok, _ = I.small_population(seed=5)
    # no category budgets on a few dozen points: one element is several percent
    with tgp.Context(points_per_thread=K, threads_per_block=64) as c:
        full_check(c, tok, I.Grid(W, H), f"{W}x{H} K={K}", budget=None)


@pytest.mark.parametrize("K,threads", [(1, 32), (2, 64), (4, 128), (8, 128), (16, 128)])
def test_residual_squares_beyond_binary32_and_root_batches(K, threads):
    """Trees whose values stay finite in binary32 but whose squared residuals
    do not (|v| up to 1e26, squares up to 1e52): the sums are formed from
    residuals scaled by 2^-80, in warps that mix scaled and unscaled threads
    (max(x, 0) is 0 on half the grid), next to ordinary trees, in batches of
    roots that end at every place of the group (10 trees: two full batches and
    one of two), on a grid with ragged chunks.  Every RMSE is the oracle's
    binary64 one within 1e-5 (binary32 squares and sums: below 2^-19)."""
    X, Y = I.leaf(I.X), I.leaf(I.Y)

    def C(v):
        return I.leaf(I.CONST, np.float32(v))
    n = I.node
    trees = [n(I.MUL, X, C(1e25)), n(I.ADD, X, Y), n(I.MUL, n(I.MAX, X, C(0.0)), C(3e25)),
             n(I.MUL, n(I.MUL, X, Y), C(4e24)), n(I.SUB, X, C(0.25)), n(I.MUL, n(I.SIN, X), C(1e21)),
             n(I.MUL, Y, C(2e19)), n(I.DIV, X, C(7.0)), n(I.MUL, n(I.MIN, Y, C(0.5)), C(-6e25)), Y]
    tok = I.to_tokens(trees)
    g = I.Grid(37, 29)
    with tgp.Context(points_per_thread=K, threads_per_block=threads) as c:
        dom = load(c, g)
        pop = c.compile_tokens(tok)
        fit = c.fitness(pop, dom, tok.n_trees)
    r64, _, _ = oracle.fitness(tok.ops, tok.imm, tok.tree_off, tok.order, g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi)
    assert np.all(np.isfinite(fit)) and np.all(np.isfinite(r64))
    np.testing.assert_allclose(fit, r64, rtol=1e-5, atol=0)


def test_other_domain_bounds():
    tok, _ = I.small_population(seed=6)
    with tgp.Context() as c:
        full_check(c, tok, I.Grid(40, 24, -1.0, 1.0, 0.5, 3.0), "bounds")


def test_trig_free_population_is_bitwise_fp32_faithful(ctx):
    rng = np.random.default_rng(21)
    funcs = (I.ADD, I.SUB, I.MUL, I.DIV, I.NEG, I.ABS, I.MIN, I.MAX)
    tok = I.to_tokens(I.ramped_half_and_half(60, 2, 8, rng, funcs))
    g = I.Grid(37, 29)
    got = phenotype(ctx, tok, g)
    _, v32, _ = oracle.evaluate(tok.ops, tok.imm, tok.tree_off, 0, g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi)
    same = (got == v32) | (np.isnan(got) & np.isnan(v32))
    assert same.all(), f"{(~same).sum()} elements differ from the correctly rounded binary32 value"


def test_deep_trees_use_many_slots(ctx):
    rng = np.random.default_rng(7)
    trees = [I._full(rng, 10, (I.ADD, I.SUB, I.MUL, I.MIN, I.MAX, I.DIV, I.SIN)) for _ in range(4)]
    tok = I.to_tokens(trees)
    full_check(ctx, tok, I.Grid(31, 9), "deep", budget=None)   # full trees of depth 10: divisions everywhere
    assert ctx.stats()["slots"] > 4


def test_closed_forms_on_device(ctx):
    g = I.Grid(64, 64)
    exprs = ["add(x, y)", "mult(x, x)", "sin(0.5)", "cos(1.0)", "div(x, sub(y, y))",
             "neg(neg(x))", "abs(neg(x))", "x", "0.25"]
    tok = I.to_tokens([I.parse_string(e) for e in exprs])
    got = phenotype(ctx, tok, g)
    xs = np.array([oracle.grid_point(g.W, g.H, -5, 5, -5, 5, p) for p in range(g.N)], np.float32)
    X, Y = xs[:, 0], xs[:, 1]
    assert np.array_equal(got[0], X + Y)
    assert np.array_equal(got[1], X * X)
    assert np.all(got[2] == 1.0) and np.all(got[3] == -1.0)
    assert np.all(got[4] == 0.0)
    assert np.array_equal(got[5], X) and np.array_equal(got[6], np.abs(X))
    assert np.array_equal(got[7], X) and np.all(got[8] == np.float32(0.25))


def test_pagie_tree_fits_pagie_target(ctx):
    e = ("add(div(mult(mult(x, x), mult(x, x)), add(1.0, mult(mult(x, x), mult(x, x)))),"
         " div(mult(mult(y, y), mult(y, y)), add(1.0, mult(mult(y, y), mult(y, y)))))")
    tok = I.to_tokens([I.parse_string(e)])
    g = I.Grid(256, 256)
    dom = load(ctx, g)
    pop = ctx.compile_tokens(tok)
    fit = ctx.fitness(pop, dom, 1)
    assert fit[0] < 1e-6   # binary32 round-off only


# ---------------------------------------------------------------- invariants

def test_cached_equals_uncached_bitwise():
    tok, g, _ = I.batched_uneven(seed=12, n_trees=300)
    g = I.Grid(96, 80)
    with tgp.Context() as a, tgp.Context(dedup=False) as b:
        pa = phenotype(a, tok, g)
        pb = phenotype(b, tok, g)
        assert np.array_equal(pa.view(np.int32), pb.view(np.int32))
        fa = a.fitness(a.compile_tokens(tok), load(a, g), tok.n_trees)
        fb = b.fitness(b.compile_tokens(tok), load(b, g), tok.n_trees)
        assert np.array_equal(fa, fb)
        assert a.stats()["code_instrs"] < b.stats()["code_instrs"]


def test_prefix_equals_postfix(ctx):
    tok, g = I.small_population(seed=9)
    post = I.convert_order(tok, I.POSTFIX)
    a = phenotype(ctx, tok, g)
    b = phenotype(ctx, post, g)
    assert np.array_equal(a.view(np.int32), b.view(np.int32))


def test_duplicated_and_permuted_trees(ctx):
    tok, g = I.small_population(seed=3)
    trees = I.from_tokens(tok)
    perm = list(reversed(trees)) + trees[:7]
    t2 = I.to_tokens(perm)
    dom = load(ctx, g)
    f1 = ctx.fitness(ctx.compile_tokens(tok), dom, tok.n_trees)
    f2 = ctx.fitness(ctx.compile_tokens(t2), dom, t2.n_trees)
    T = tok.n_trees
    # phenotypes are bitwise identical; the partial sums are ordered identically
    assert np.array_equal(f2[:T], f1[::-1])
    assert np.array_equal(f2[T:], f1[:7])


def test_launch_shapes_give_identical_phenotypes():
    tok, g = I.small_population(seed=2)
    g = I.Grid(150, 70)
    ref = None
    for K, thr, G in [(1, 32, 1), (2, 64, 3), (4, 128, 50), (8, 128, 7), (8, 64, 1)]:
        with tgp.Context(points_per_thread=K, threads_per_block=thr, n_groups=G) as c:
            p = phenotype(c, tok, g)
        if ref is None:
            ref = p
        assert np.array_equal(ref.view(np.int32), p.view(np.int32)), (K, thr, G)


def test_fitness_is_deterministic_and_matches_phenotype(ctx):
    tok, _ = I.small_population(seed=8)
    g = I.Grid(300, 200)
    dom = load(ctx, g)
    pop = ctx.compile_tokens(tok)
    f1 = ctx.fitness(pop, dom, tok.n_trees)
    f2 = ctx.fitness(pop, dom, tok.n_trees)
    assert np.array_equal(f1, f2)
    ph = phenotype(ctx, tok, g, pop, dom).astype(np.float64)
    xs = np.array([oracle.grid_point(g.W, g.H, -5, 5, -5, 5, p) for p in range(g.N)], np.float64)
    # target in binary32 as the kernel forms it
    x32, y32 = xs[:, 0].astype(np.float32), xs[:, 1].astype(np.float32)
    x4, y4 = (x32 * x32) * (x32 * x32), (y32 * y32) * (y32 * y32)
    P = (x4 / (np.float32(1) + x4) + y4 / (np.float32(1) + y4)).astype(np.float64)
    with np.errstate(all="ignore"):
        r = np.sqrt(np.mean((ph - P) ** 2, axis=1))
    r = np.where(np.isfinite(r), r, np.inf)
    fin = np.isfinite(r) & (r < 1e15)
    assert np.allclose(f1[fin], r[fin], rtol=2e-6, atol=0)


def test_fitness_dev_and_nonblocking(ctx):
    tok, g = I.small_population(seed=1)
    dom = load(ctx, g)
    pop = ctx.compile_tokens(tok)
    ref = ctx.fitness(pop, dom, tok.n_trees)
    out = torch.empty(tok.n_trees, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    ctx.fitness_dev(pop, dom, out, stream=s)
    s.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)
    host = torch.empty(tok.n_trees, dtype=torch.float64).pin_memory()
    ctx.fitness(pop, dom, tok.n_trees, stream=s, blocking=False, out=host.numpy())
    s.synchronize()
    assert np.array_equal(host.numpy(), ref)


# ---------------------------------------------------------------- targets

def test_target_tensor_host_and_device(ctx):
    tok, g = I.small_population(seed=4)
    g = I.Grid(48, 40)
    rng = np.random.default_rng(0)
    target = rng.uniform(-2, 2, g.N).astype(np.float32)
    pop = ctx.compile_tokens(tok)
    dh = ctx.load_domain(g.W, g.H, target=target)
    fh = ctx.fitness(pop, dh, tok.n_trees)
    fd = ctx.fitness(pop, ctx.load_domain(g.W, g.H, target=torch.from_numpy(target).cuda()), tok.n_trees)
    assert np.array_equal(fh, fd)
    check_population(ctx, tok, g, fh, "tensor target", pop=pop, dom=dh, target=target)


def test_target_tokens_random_tree(ctx):
    rng = np.random.default_rng(44)
    target_tree = I._full(rng, 4, I.FUNCTIONS)
    tt = I.to_tokens([target_tree])
    tok, _ = I.small_population(seed=4)
    g = I.Grid(50, 30)
    dom = ctx.load_domain(g.W, g.H, target_tokens=(tt.ops, tt.imm, tt.order))
    pop = ctx.compile_tokens(tok)
    fit = ctx.fitness(pop, dom, tok.n_trees)
    # the device forms the target tree in binary32; its error bound adds (L2)
    # to every tree's fitness bound
    check_population(ctx, tok, g, fit, "token target", pop=pop, dom=dom, target_tokens=(tt.ops, tt.imm, tt.order))


# ---------------------------------------------------------------- full size

def test_population_at_scale_sampled_elements_and_full_fitness(ctx):
    """100 RHH trees (depth 2-8) on 1024x1024: phenotypes on 8192 sampled
    points, fitness of every tree against the oracle over all 2^20 points."""
    tok, g = I.population_at_scale(seed=1)
    oracle_pool()   # created before the first device call of this test
    dom = load(ctx, g)
    pop = ctx.compile_tokens(tok)
    fit = ctx.fitness(pop, dom, tok.n_trees)
    rng = np.random.default_rng(123)
    pts = np.concatenate([np.sort(rng.choice(g.N, 8192, replace=False)), [0, g.N - 1]])
    r = check_population(ctx, tok, g, fit, "at scale", pop=pop, dom=dom, budget="at_scale", elem_pts=pts,
                         point_chunks=4)
    assert r["fitness"]["trees"] == tok.n_trees


def test_batched_uneven_sampled(ctx):
    """4096 trees of 3..255 nodes with ~30% duplicated subtrees on 256x256:
    every tree on 256 sampled points; 256 sampled trees on every point, and
    their fitness from the 4096-tree launch against the oracle over all points."""
    tok, g, stats = I.batched_uneven(seed=2)
    assert 0.2 < stats["dup_fraction"] < 0.4
    oracle_pool()
    dom = load(ctx, g)
    pop = ctx.compile_tokens(tok)
    fit = ctx.fitness(pop, dom, tok.n_trees)
    rng = np.random.default_rng(5)
    pts = np.sort(rng.choice(g.N, 256, replace=False))
    check_population(ctx, tok, g, fit, "batched, all trees", pop=pop, dom=dom, budget="batched", elem_pts=pts,
                     fit_trees=[])
    idx = np.sort(rng.choice(tok.n_trees, 256, replace=False))
    sub = subset(tok, idx)
    r = check_population(ctx, sub, g, fit[idx], "batched, 256 trees on all points", dom=dom, budget="batched")
    assert r["fitness"]["trees"] == 256


# ---------------------------------------------------------------- edge cases

def test_empty_and_leaf_populations(ctx):
    g = I.Grid(10, 10)
    dom = load(ctx, g)
    empty = ctx.compile_population(np.zeros(0, np.int32), np.zeros(0, np.float32), np.zeros(1, np.int64))
    assert ctx.fitness(empty, dom, 0).size == 0
    tok = I.to_tokens([I.parse_string(e) for e in ["x", "y", "0.5"]])
    full_check(ctx, tok, g, "leaves")


def test_bad_handles_and_shapes(ctx):
    g = I.Grid(8, 8)
    dom = load(ctx, g)
    tok, _ = I.small_population()
    pop = ctx.compile_tokens(tok)
    with pytest.raises(tgp.TgpError):
        ctx.fitness(pop + 1000, dom, tok.n_trees)
    with pytest.raises(tgp.TgpError):
        ctx.fitness(pop, dom + 1000, tok.n_trees)
    with pytest.raises(tgp.TgpError):
        ctx.load_domain(0, 5)
    with tgp.Context(points_per_thread=3) as c:
        with pytest.raises(tgp.TgpError):
            c.fitness(c.compile_tokens(tok), c.load_domain(4, 4), tok.n_trees)


# ---------------------------------------------------------------- division

def _division_operands(rng, n):
    """binary32 operands over the whole range: random magnitudes 2^-149..2^127,
    powers of two, values next to 1, subnormals, the largest values, zeros."""
    f = np.float32
    mag = np.exp2(rng.uniform(-149, 127.9, n)).astype(f) * rng.choice([-1, 1], n).astype(f)
    special = np.array([0.0, -0.0, 1.0, -1.0, 2.0, 0.5, 3.0, 1.0 / 3.0, np.nextafter(f(1), f(2)),
                        np.nextafter(f(1), f(0)), np.finfo(f).max, -np.finfo(f).max, np.finfo(f).tiny,
                        np.finfo(f).smallest_subnormal, -np.finfo(f).smallest_subnormal, 2.0 ** -60,
                        2.0 ** 61, 2.0 ** -100, 1e-30, 7.0, 0.1, 1e30, 2.0 ** 126, 2.0 ** -126], f)
    return np.concatenate([mag, special]).astype(f)


def test_division_is_bitwise_ieee(ctx):
    """The interpreter's division (self-checked fast path with an IEEE
    fallback) equals numpy's correctly rounded binary32 quotient bitwise, with
    the protection 0 for a zero denominator."""
    rng = np.random.default_rng(77)
    a = _division_operands(rng, 3000)
    b = _division_operands(rng, 3000)
    rng.shuffle(b)
    n = min(a.size, b.size)
    a, b = a[:n], b[:n]
    # div(a, b) with constants (load then divide) and div(a, x-free expression)
    trees = [I.node(I.DIV, I.leaf(I.CONST, a[i]), I.leaf(I.CONST, b[i])) for i in range(n)]
    tok = I.to_tokens(trees)
    got = phenotype(ctx, tok, I.Grid(2, 1))[:, 0]
    with np.errstate(all="ignore"):
        exp = np.where(b == 0, np.float32(0), a / np.where(b == 0, np.float32(1), b)).astype(np.float32)
    same = (got.view(np.int32) == exp.view(np.int32)) | (np.isnan(got) & np.isnan(exp))
    assert same.all(), list(zip(a[~same][:5], b[~same][:5], got[~same][:5], exp[~same][:5]))


def test_division_forms_on_grid(ctx):
    """A / F and F / A forms with coordinates, constants and slot operands."""
    g = I.Grid(97, 61, -3.0, 7.0, -2.0, 2.0)
    exprs = ["div(x, y)", "div(y, x)", "div(0.37, x)", "div(x, -0.37)", "div(mult(x, y), sub(y, 0.5))",
             "div(sub(y, 0.5), mult(x, y))", "div(add(x, 1.5), add(x, 1.5))", "div(x, sub(y, y))"]
    tok = I.to_tokens([I.parse_string(e) for e in exprs])
    got = phenotype(ctx, tok, g)
    _, v32, _ = oracle.evaluate(tok.ops, tok.imm, tok.tree_off, 0, g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi)
    same = (got == v32) | (np.isnan(got) & np.isnan(v32))
    assert same.all()


# ---------------------------------------------------------------- graph + autotuner

def test_graph_replay_equals_direct_launch(ctx):
    tok, g = I.small_population(seed=11)
    dom = load(ctx, g)
    pop = ctx.compile_tokens(tok)
    ref = torch.empty(tok.n_trees, dtype=torch.float64, device="cuda")
    ctx.fitness_dev(pop, dom, ref)
    s = torch.cuda.Stream()
    out = torch.full((tok.n_trees,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(3):                       # capture, then two replays
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        ctx.fitness_graph(pop, dom, out, stream=s)
        s.synchronize()
        assert torch.equal(out, ref)
    with pytest.raises(tgp.TgpError) as e:   # the legacy default stream cannot be captured
        ctx.fitness_graph(pop, dom, out)
    assert e.value.code == tgp.E_INVALID
    ctx.release_population(pop)              # frees the graph


def test_autotune_picks_a_shape_and_keeps_results(ctx):
    tok, g = I.small_population(seed=12)
    g = I.Grid(256, 256)
    with tgp.Context() as c:
        dom = c.load_domain(g.W, g.H)
        pop = c.compile_tokens(tok)
        before = c.fitness(pop, dom, tok.n_trees)
        K, G, ms = c.autotune(pop, dom)
        assert K in (2, 4, 8, 16) and 1 <= G <= tok.n_trees and ms > 0
        after = c.fitness(pop, dom, tok.n_trees)
        assert c.stats()["points_per_thread"] == K and c.stats()["n_groups"] == G
        fin = np.isfinite(before)
        assert np.allclose(after[fin], before[fin], rtol=2e-6, atol=0)
        assert np.array_equal(np.isinf(after), np.isinf(before))
        # another population of the same size bucket reuses the choice
        tok2, _ = I.small_population(seed=13)
        pop2 = c.compile_tokens(tok2)
        c.fitness(pop2, dom, tok2.n_trees)
        assert c.stats()["points_per_thread"] == K
