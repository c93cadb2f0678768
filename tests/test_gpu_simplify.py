"""Simplification while hash-consing is exact on the device: simplified and
as-given populations give the same binary32 values bit for bit (NaNs
compared as NaN), and both match the oracle."""
import numpy as np
import pytest

import oracle
import paper_2103_07512_gb300 as tgp
from paper_2103_07512_gb300 import inputs as I
from parity import check_population

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CONSTS = (0.0, -0.0, 1.0, -1.0, 2.0, 0.5, 3.0)


def const_heavy(rng, d, funcs):
    if d == 0 or rng.random() < 0.15:
        r = rng.random()
        if r < 0.25:
            return I.leaf(I.X)
        if r < 0.35:
            return I.leaf(I.Y)
        return I.leaf(I.CONST, CONSTS[int(rng.integers(len(CONSTS)))])
    f = funcs[int(rng.integers(len(funcs)))]
    return I.node(f, *[const_heavy(rng, d - 1, funcs) for _ in range(I.ARITY[f])])


def bits(a):
    b = np.asarray(a, np.float32).view(np.int32).copy()
    b[np.isnan(a)] = 0x7FC00000
    return b


def phenotypes(ctx, tok, g):
    dom = ctx.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi)
    pop = ctx.compile_tokens(tok)
    out = torch.empty((tok.n_trees, g.N), dtype=torch.float32, device="cuda")
    ctx.evaluate(pop, dom, out)
    fit = ctx.fitness(pop, dom, tok.n_trees)
    return out.cpu().numpy(), fit


def test_min_max_of_signed_zeros_do_not_depend_on_operand_order():
    z, nz = "sub(x, x)", "neg(sub(x, x))"      # +0 and -0 at every (finite) point
    exprs = [f"min({z}, {nz})", f"min({nz}, {z})", f"max({z}, {nz})", f"max({nz}, {z})"]
    tok = I.to_tokens([I.parse_string(e) for e in exprs])
    g = I.Grid(8, 4)
    with tgp.Context(simplify=False) as ctx:
        ph, _ = phenotypes(ctx, tok, g)
    b = ph.view(np.int32)
    assert np.array_equal(b[0], b[1]) and np.array_equal(b[2], b[3])


@pytest.mark.parametrize("seed", [31, 32])
def test_simplified_equals_as_given_bitwise(seed):
    rng = np.random.default_rng(seed)
    trees = [const_heavy(rng, int(rng.integers(2, 8)), I.FUNCTIONS) for _ in range(300)]
    tok = I.to_tokens(trees)
    g = I.Grid(96, 40)
    with tgp.Context() as a, tgp.Context(simplify=False) as b:
        pa, fa = phenotypes(a, tok, g)
        pb, fb = phenotypes(b, tok, g)
        sa, sb = a.stats(), b.stats()
    assert sa["dag_internal"] < sb["dag_internal"]
    assert np.array_equal(bits(pa), bits(pb))
    assert np.array_equal(fa.view(np.int64), fb.view(np.int64))


def test_simplified_population_matches_oracle():
    rng = np.random.default_rng(33)
    trees = [const_heavy(rng, int(rng.integers(2, 7)), I.FUNCTIONS) for _ in range(120)]
    tok = I.to_tokens(trees)
    g = I.Grid(33, 17)
    with tgp.Context() as ctx:
        ph, fit = phenotypes(ctx, tok, g)
        check_population(ctx, tok, g, fit, "simplified")
