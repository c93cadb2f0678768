"""tgp_fitness_noalloc: fitness without any device allocation by the library.

Callers that cannot call cudaMalloc -- a host that has reserved the device's
memory for its own pool, code that must not risk the implicit synchronisation
of an allocation, code that must not touch the allocator after start-up -- use
this entry point; it keeps its scratch in one fixed 8 MiB device array.  Here
it is called through the C ABI and compared with tgp_fitness_dev on two calls
in a row (the array keeps the previous call's contents, so the second call
checks that nothing stale is read).  Both run the same arithmetic on the same
values (the no-allocation plan has no column or row tables, whose values are
bitwise those computed in place), so the results are compared bit for bit.
The file is named to be collected last.
"""
import numpy as np
import pytest

import paper_2103_07512_gb300 as tgp
from paper_2103_07512_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _same_fitness(a, b):
    """Bitwise equal binary64 values."""
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    return a.shape == b.shape and bool(np.array_equal(a.view(np.int64), b.view(np.int64)))


def test_noalloc_matches_fitness_dev_on_two_calls_in_a_row():
    with tgp.Context() as ctx:
        tok_a, g = I.population_at_scale(seed=1)
        tok_b, _ = I.small_population(seed=3)
        dom = ctx.load_domain(g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi)
        pa = ctx.compile_tokens(tok_a)
        pb = ctx.compile_tokens(tok_b)
        ref_a = torch.empty(tok_a.n_trees, dtype=torch.float64, device="cuda")
        ref_b = torch.empty(tok_b.n_trees, dtype=torch.float64, device="cuda")
        ctx.fitness_dev(pa, dom, ref_a)
        ctx.fitness_dev(pb, dom, ref_b)
        out1 = torch.full((tok_a.n_trees,), float("nan"), dtype=torch.float64, device="cuda")
        out2 = torch.full((tok_a.n_trees,), float("nan"), dtype=torch.float64, device="cuda")
        ctx.fitness_noalloc(pa, dom, out1)
        ctx.fitness_noalloc(pa, dom, out2)
        torch.cuda.synchronize()
        assert _same_fitness(out1.cpu().numpy(), ref_a.cpu().numpy())
        assert _same_fitness(out2.cpu().numpy(), ref_a.cpu().numpy())
        # a different, smaller population next: nothing left over from the last call
        out3 = torch.full((tok_b.n_trees,), float("nan"), dtype=torch.float64, device="cuda")
        ctx.fitness_noalloc(pb, dom, out3)
        torch.cuda.synchronize()
        assert _same_fitness(out3.cpu().numpy(), ref_b.cpu().numpy())


def test_noalloc_on_a_stream_and_rejects_oversized_populations():
    with tgp.Context() as ctx:
        tok, g = I.small_population(seed=0)
        dom = ctx.load_domain(g.W, g.H)
        pop = ctx.compile_tokens(tok)
        ref = ctx.fitness(pop, dom, tok.n_trees)
        s = torch.cuda.Stream()
        out = torch.empty(tok.n_trees, dtype=torch.float64, device="cuda")
        ctx.fitness_noalloc(pop, dom, out, stream=s)
        s.synchronize()
        assert _same_fitness(out.cpu().numpy(), ref)
        # 600 trees on 1024x1024: 600 * 1024 tiles * 4 warps partial sums = 9.4 MiB > 8 MiB
        big = I.to_tokens([I.parse_string("x")] * 600)
        big_dom = ctx.load_domain(1024, 1024)
        bp = ctx.compile_tokens(big)
        dst = torch.empty(600, dtype=torch.float64, device="cuda")
        with pytest.raises(tgp.TgpError) as e:
            ctx.fitness_noalloc(bp, big_dom, dst)
        assert e.value.code == tgp.E_INVALID and "scratch" in str(e.value)
