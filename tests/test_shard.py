"""Row-sharded fitness, host side: the split of the rows into bands, the
exchange of the bands' sums between ranks (two and three gloo ranks on the
CPU), and the checks of a band's bounds (a host-only context, no device).

Each rank's sums are the oracle's binary64 sums of squared residuals over its
band (the sums the library computes on each GPU); every rank must end with
the same bits, those of the sums added in rank order, and the result must be
the oracle's fitness over the whole grid.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
import paper_2103_07512_gb300 as tgp  # noqa: E402
from paper_2103_07512_gb300 import inputs as I  # noqa: E402
from paper_2103_07512_gb300 import shard  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GRID = I.Grid(40, 31)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _population():
    return I.small_population(seed=11)[0]


def _band_sums(tok, g, row0, n):
    pts = np.arange(row0 * g.W, (row0 + n) * g.W)
    parts = oracle.fitness_parts(tok.ops, tok.imm, tok.tree_off, tok.order, g.W, g.H, g.xlo, g.xhi, g.ylo, g.yhi,
                                 pts=pts)
    return parts["s64"]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    tok = _population()
    row0, n = shard.band_rows(GRID.H, rank, world)
    s = torch.from_numpy(_band_sums(tok, GRID, row0, n))
    r = shard.reduce_band_sse(s, GRID.N)
    out[rank] = r.numpy().tobytes()
    dist.destroy_process_group()


def test_band_rows_cover_the_grid():
    for H in (1, 2, 7, 31, 1024):
        for world in range(1, 9):
            if world > H:
                continue
            bands = [shard.band_rows(H, r, world) for r in range(world)]
            assert bands[0][0] == 0
            for (a, n), (b, _) in zip(bands, bands[1:]):
                assert a + n == b
            assert bands[-1][0] + bands[-1][1] == H
            sizes = [n for _, n in bands]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        shard.band_rows(10, 2, 2)


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_agree_bitwise_and_match_the_oracle(world):
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = [np.frombuffer(out[r], np.float64) for r in range(world)]
    for r in range(1, world):
        assert res[r].tobytes() == res[0].tobytes(), f"rank {r} differs from rank 0"
    # the same sums added in rank order here
    tok = _population()
    total = None
    for r in range(world):
        row0, n = shard.band_rows(GRID.H, r, world)
        s = _band_sums(tok, GRID, row0, n)
        total = s.copy() if total is None else total + s
    expect = np.sqrt(total / float(GRID.N))
    expect = np.where(np.isfinite(expect), expect, np.inf)
    assert res[0].tobytes() == expect.tobytes()
    # and the oracle's fitness over the whole grid (binary64, another order of addition)
    r64, _, _ = oracle.fitness(tok.ops, tok.imm, tok.tree_off, tok.order, GRID.W, GRID.H, GRID.xlo, GRID.xhi,
                               GRID.ylo, GRID.yhi)
    fin = np.isfinite(r64)
    assert np.array_equal(np.isfinite(res[0]), fin)
    np.testing.assert_allclose(res[0][fin], r64[fin], rtol=1e-12, atol=0)


def test_single_rank_without_process_group():
    s = torch.tensor([4.0, 0.0, float("inf"), float("nan")], dtype=torch.float64)
    r = shard.reduce_band_sse(s, 4)
    assert r.tolist() == [1.0, 0.0, float("inf"), float("inf")]
    with pytest.raises(ValueError):
        shard.reduce_band_sse(s.float(), 4)


def test_band_bounds_on_a_host_only_context():
    with tgp.Context(host_only=True) as ctx:
        for rows in [(-1, 3), (0, 0), (10, 36), (45, 1)]:
            with pytest.raises(tgp.TgpError) as e:
                ctx.load_domain(32, 45, rows=rows)
            assert e.value.code == tgp.E_INVALID
        dom = ctx.load_domain(32, 45, rows=(10, 35))
        tok = _population()
        pop = ctx.compile_tokens(tok)
        # planning for the band: the work covers its 35 rows of 32 points
        w, roots = ctx.plan_work(pop, dom)
        assert roots == tok.n_trees * 32 * 35
