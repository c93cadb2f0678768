"""The serving loop: jobs of different populations, grids and targets give
the same RMSE values alone and in a mix (fused launches, overlapping
streams), match the oracle, respect the HBM budget, and report a timeline."""
import numpy as np
import pytest

import oracle
import paper_2103_07512_gb300 as tgp
from paper_2103_07512_gb300 import inputs as I
from parity import check_population, oracle_pool

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def small_jobs(n, seed):
    return I.serving_jobs(n, seed=seed, trees=(10, 60), depth=(2, 6), side_log2=(3.0, 8.0))


def submit(srv, job):
    return srv.submit(job["tok"], job["W"], job["H"], target_tokens=job["target_tokens"])


def test_alone_equals_in_mix():
    jobs = small_jobs(14, seed=40)
    # repeat some domains so that queued jobs share a launch
    jobs += [dict(j, tok=k["tok"]) for j, k in zip(jobs[:6], jobs[6:12])]
    # four heavy jobs first (1,000 trees on 2048 x 2048 points each) keep every
    # stream busy while the rest queue
    heavy = I.to_tokens(I.ramped_half_and_half(1000, 2, 8, np.random.default_rng(46)))
    jobs = [{"tok": heavy, "W": 2048, "H": 2048 - 8 * k, "target_tokens": None} for k in range(4)] + jobs
    with tgp.Context() as ctx:
        with tgp.Server(ctx, streams=1) as srv:      # alone: one job at a time
            alone = []
            for j in jobs:
                r, info = srv.wait(submit(srv, j))
                assert info["batch_jobs"] == 1
                alone.append(r)
        with tgp.Server(ctx, streams=4) as srv:      # mix: all queued at once
            ids = [submit(srv, j) for j in jobs]
            mixed = [srv.wait(i) for i in ids]
            st = srv.stats()
        assert st["completed"] == len(jobs) and st["failed"] == 0
        assert st["batches"] < len(jobs) and st["max_batch_jobs"] > 1
        assert st["max_batch_domains"] > 1          # launches fused jobs of different domains
        for k, (a, (m, info)) in enumerate(zip(alone, mixed)):
            assert np.array_equal(a.view(np.int64), m.view(np.int64)), f"job {k}"
            assert info["submit_ns"] <= info["launch_ns"] <= info["done_ns"]


def test_fused_domains_alone_equals_in_mix():
    """Jobs on many different grids of one launch shape (K = 8: 2^18 points
    and more) and both target kinds, queued at once behind a long first job
    (2,000 trees on 2048 x 2048 points, so that the others are all queued
    when it ends): fused across domains into few launches, each result
    bitwise that of the job alone."""
    rng = np.random.default_rng(47)
    jobs = [{"tok": I.to_tokens(I.ramped_half_and_half(2000, 2, 10, rng)), "W": 2048, "H": 2048,
             "target_tokens": None}]
    for k in range(12):
        side = int(rng.integers(512, 800))
        tok = I.to_tokens(I.ramped_half_and_half(int(rng.integers(10, 40)), 2, 6, rng))
        target = None
        if k % 3 == 0:
            tt = I.to_tokens([I._full(rng, 3, I.FUNCTIONS)])
            target = (tt.ops, tt.imm, tt.order)
        jobs.append({"tok": tok, "W": side, "H": side + k, "target_tokens": target})
    with tgp.Context() as ctx:
        with tgp.Server(ctx, streams=1) as srv:
            alone = [srv.wait(submit(srv, j))[0] for j in jobs]
        with tgp.Server(ctx, streams=1) as srv:    # one slot: the queue builds up behind the first launch
            ids = [submit(srv, j) for j in jobs]
            mixed = [srv.wait(i) for i in ids]
            st = srv.stats()
    assert st["completed"] == len(jobs) and st["max_batch_domains"] >= 3, st
    for k, (a, (m, info)) in enumerate(zip(alone, mixed)):
        assert np.array_equal(a.view(np.int64), m.view(np.int64)), f"job {k}"
    assert max(info["batch_jobs"] for _, info in mixed) >= 3


def test_server_large_job_matches_oracle():
    """A job at the serving workload's upper end (1,000 RHH trees of depth
    2-10 on 2048x2048 = 2^22 points) through the server: every tree on 16,384
    sampled points, and 48 sampled trees' fitness over all points, against the
    oracle."""
    rng = np.random.default_rng(48)
    tok = I.to_tokens(I.ramped_half_and_half(1000, 2, 10, rng))
    g = I.Grid(2048, 2048)
    oracle_pool()
    with tgp.Context() as ctx:
        with tgp.Server(ctx, streams=2) as srv:
            r, info = srv.wait(submit(srv, {"tok": tok, "W": g.W, "H": g.H, "target_tokens": None}))
        pts = np.concatenate([np.sort(rng.choice(g.N, 16384, replace=False)), [0, g.N - 1]])
        trees = np.sort(rng.choice(tok.n_trees, 48, replace=False))
        c = check_population(ctx, tok, g, r, "serving, 1000 trees on 2^22 points", budget="serving", elem_pts=pts,
                             fit_trees=trees, point_chunks=8)
    assert c["fitness"]["trees"] == 48


def test_server_results_match_oracle():
    jobs = small_jobs(6, seed=41)
    with tgp.Context() as ctx, tgp.Server(ctx, streams=3) as srv:
        ids = [submit(srv, j) for j in jobs]
        res = [srv.wait(i)[0] for i in ids]
    with tgp.Context() as ctx:
        for k, (j, r) in enumerate(zip(jobs, res)):
            g = I.Grid(j["W"], j["H"])
            check_population(ctx, j["tok"], g, r, f"job {k}", target_tokens=j["target_tokens"], budget="serving")


def test_server_with_subtree_cache_is_bitwise_equal():
    jobs = small_jobs(8, seed=42)
    jobs = jobs + jobs + jobs     # stored on the second round, loaded on the third
    with tgp.Context() as c0, tgp.Server(c0, streams=1) as s0:
        ref = [s0.wait(submit(s0, j))[0] for j in jobs]
    with tgp.Context(cache_budget_bytes=1 << 26, cache_min_cost=4) as c1, tgp.Server(c1, streams=4) as s1:
        ids = [submit(s1, j) for j in jobs]
        got = [s1.wait(i)[0] for i in ids]
        assert c1.stats()["cache_inserts"] > 0
    for a, b in zip(ref, got):
        assert np.array_equal(a.view(np.int64), b.view(np.int64))


def test_hbm_budget_admission_and_domain_release():
    jobs = I.serving_jobs(10, seed=43, trees=(10, 30), depth=(2, 5), side_log2=(7.0, 7.0))
    rng = np.random.default_rng(43)
    for k, j in enumerate(jobs):     # distinct domains, each with a target tree (device memory)
        j["xlo"] = -5.0 - 0.25 * k
        if j["target_tokens"] is None:
            tt = I.to_tokens([I._full(rng, 3, I.FUNCTIONS)])
            j["target_tokens"] = (tt.ops, tt.imm, tt.order)
    N = jobs[0]["W"] * jobs[0]["H"]
    budget = 3 * N * 4 + (200 << 10)   # about three resident targets plus the launches
    with tgp.Context() as ctx:
        with tgp.Server(ctx, streams=1) as s0:
            ref = [s0.wait(s0.submit(j["tok"], j["W"], j["H"], xlo=j["xlo"], target_tokens=j["target_tokens"]))[0]
                   for j in jobs]
        with tgp.Server(ctx, streams=4, hbm_budget_bytes=budget) as srv:
            ids = [srv.submit(j["tok"], j["W"], j["H"], xlo=j["xlo"], target_tokens=j["target_tokens"])
                   for j in jobs]
            got = [srv.wait(i)[0] for i in ids]
            st = srv.stats()
        assert st["max_bytes_in_use"] <= budget
        assert st["domains_loaded"] == len(jobs)
        assert st["domains_released"] >= len(jobs) - 5
        for a, b in zip(ref, got):
            assert np.array_equal(a.view(np.int64), b.view(np.int64))


def test_submit_errors_and_wait_timeout():
    tok, _ = I.small_population(seed=44)
    with tgp.Context() as ctx, tgp.Server(ctx, streams=2, hbm_budget_bytes=1 << 16) as srv:
        with pytest.raises(tgp.TgpError) as e:       # cannot fit the budget at all
            srv.submit(tok, 1024, 1024)
        assert e.value.code == tgp.E_BUDGET
        bad = I.Tokens(np.array([I.ADD, I.X], np.int32), np.zeros(0, np.float32),
                       np.array([0, 2], np.int64), tgp.PREFIX)
        with pytest.raises(tgp.TgpError) as e:       # add with one operand
            srv.submit(bad, 8, 8)
        assert e.value.code == tgp.E_TOKENS
        with pytest.raises(tgp.TgpError) as e:
            srv.submit(tok, 0, 8)
        assert e.value.code == tgp.E_INVALID
        i = srv.submit(tok, 16, 16)
        r, info = srv.wait(i)
        assert r.shape == (tok.n_trees,) and info["status"] == 0
        with pytest.raises(tgp.TgpError) as e:       # already collected
            srv.wait(i)
        assert e.value.code == tgp.E_INVALID


def test_destroy_finishes_submitted_jobs():
    jobs = small_jobs(6, seed=45)
    with tgp.Context() as ctx:
        srv = tgp.Server(ctx, streams=2)
        for j in jobs:
            submit(srv, j)
        srv.close()                                   # returns after the jobs ran
        assert ctx.stats()["launches"] > 0
