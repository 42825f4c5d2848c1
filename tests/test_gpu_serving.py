"""Serving (continuous batching, Hutch++ proxy): queries admitted by HBM
budget and slots at every tick, a tick being one Lanczos step of every
active query at its own step; each result is bit-identical alone and in the
mix and matches the oracle's Hutch++ with N_r = 4 sketch columns and the
served number of projected Hutchinson vectors on the same probes (mixed
path, 1e-5 relative)."""
import numpy as np
import pytest

from oracle import density, estimators
from paper_2212_09642_gb300 import graphs, vne

pytestmark = pytest.mark.gpu

M_STEPS = 30


def _graphs():
    return [graphs.erdos_renyi(3000, 8 / 2999, 31), graphs.barabasi_albert(5000, 3, 32),
            graphs.watts_strogatz(2000, 6, 0.1, 33), graphs.barabasi_albert(1500, 3, 34),
            graphs.erdos_renyi(7000, 8 / 6999, 35)]


def _run(vctx, mats, schedule, budget, max_active, eps=2e-3, cap=1024, opt=None):
    """schedule: list of (tick, matrix index, seed); returns per-request results and
    the largest number of queries active in one tick.  Checks that the bytes
    held by admitted queries never exceed the budget."""
    srv = vne.vne_server_create(vctx, budget, max_active=max_active, krylov_steps=M_STEPS, block_vectors=64,
                                opt=opt if opt is not None else vne.options(reorth=0, panel=8))
    tickets = {}
    most = 0
    try:
        tick = 0
        pending = list(schedule)
        while True:
            while pending and pending[0][0] <= tick:
                _, mi, seed = pending.pop(0)
                tickets[(mi, seed)] = vne.vne_server_submit(vctx, srv, mats[mi], eps, seed, cap)
            done, active = vne.vne_server_step(vctx, srv)
            most = max(most, active)
            q, a, used = vne.vne_server_info(srv)
            assert used <= budget
            tick += 1
            if not pending and q == 0 and a == 0:
                break
            assert tick < 100000
        res = {k: vne.vne_server_result(srv, t) for k, t in tickets.items()}
    finally:
        vne.vne_server_destroy(srv)
    return res, most


def test_serving_same_alone_and_in_mix(vctx):
    gs = _graphs()
    mats = [vne.matrix_from_graph(vctx, g, fp64=False) for g in gs]
    try:
        # arrivals in the middle of other queries' blocks
        mix = [(0, 0, 11), (0, 1, 12), (7, 2, 13), (31, 3, 14), (45, 0, 15), (50, 4, 16), (93, 1, 17)]
        mixed, most = _run(vctx, mats, mix, budget=1 << 36, max_active=8)
        assert most >= 3  # queries really overlapped
        for (mi, seed), r in mixed.items():
            assert r["state"] == 2
            # a free slot admits a query at the tick after its submission, and a
            # query then takes one tick per Lanczos step of each of its blocks
            assert r["admit_tick"] == r["submit_tick"]
            assert r["done_tick"] - r["admit_tick"] == (r["vectors"] // 64) * M_STEPS
            alone, _ = _run(vctx, mats, [(0, mi, seed)], budget=1 << 36, max_active=8)
            ra = alone[(mi, seed)]
            assert ra["estimate"] == r["estimate"] and ra["vectors"] == r["vectors"]
            A, _ = density.density_matrix(gs[mi])
            ref = estimators.hutchpp(A, 4, r["vectors"], M_STEPS, seed=seed, reorth="none")
            assert abs(r["estimate"] - ref) <= 1e-5 * ref
            conv = 2.576 * r["std_error"] <= 0.5 * 2e-3 * r["estimate"]
            assert conv or r["vectors"] >= 1024
    finally:
        for m in mats:
            vne.vne_matrix_destroy(m)


def test_serving_admission_respects_budget_and_slots(vctx):
    gs = _graphs()
    mats = [vne.matrix_from_graph(vctx, g, fp64=False) for g in gs]
    try:
        sched = [(0, i % 5, 100 + i) for i in range(8)]
        # slots: at most 2 queries per tick
        res, most = _run(vctx, mats, sched, budget=1 << 36, max_active=2)
        assert most <= 2 and all(r["state"] == 2 for r in res.values())
        # budget: room for about two of the larger queries only
        biggest = max(g.n for g in gs)
        budget = int(2.2 * (3 * biggest * 64 * 4 + 4 * 80000))
        res2, most2 = _run(vctx, mats, sched, budget=budget, max_active=8)
        assert most2 < 8 and all(r["state"] == 2 for r in res2.values())
        for k in res:
            assert res[k]["estimate"] == res2[k]["estimate"]
        with pytest.raises(vne.VneError):  # a query larger than the whole budget
            srv = vne.vne_server_create(vctx, 1000, max_active=2, krylov_steps=30, block_vectors=64)
            try:
                vne.vne_server_submit(vctx, srv, mats[0], 1e-3, 1)
            finally:
                vne.vne_server_destroy(srv)
    finally:
        for m in mats:
            vne.vne_matrix_destroy(m)


def test_serving_fp64_one_at_a_time(vctx):
    """An FP64 server with one slot serves the same Hutch++ proxy one query at
    a time; its estimates match the oracle's to 1e-10."""
    gs = _graphs()[:3]
    mats = [vne.matrix_from_graph(vctx, g, fp64=True) for g in gs]
    try:
        sched = [(0, i, 200 + i) for i in range(3)]
        res, most = _run(vctx, mats, sched, budget=1 << 34, max_active=1)
        assert most == 1
        for (mi, seed), r in res.items():
            A, _ = density.density_matrix(gs[mi])
            ref = estimators.hutchpp(A, 4, r["vectors"], M_STEPS, seed=seed, reorth="none")
            assert abs(r["estimate"] - ref) <= 1e-10 * ref
    finally:
        for m in mats:
            vne.vne_matrix_destroy(m)


CHECK = 3


@pytest.mark.parametrize("fp64", [False, True])
def test_serving_krylov_stopping(vctx, fp64):
    """quad_tol < 0: every query's blocks (the basis vectors' quadratic forms
    at admission, then the deflated probe blocks) stop their Lanczos runs at
    the first multiple of check_every where every column's Theorem 4.4
    estimate is within half the query's accuracy (Section 5.2); the FP32
    server also takes a short sketch (sketch_steps).  Each result is
    bit-identical alone and in the mix; it is the oracle's served estimator
    with the same rule (1e-5 mixed, 1e-10 FP64): the same probes, the same
    Lanczos steps (the ticks a query took are the oracle's block steps) and
    the same estimate."""
    gs = _graphs()[:4] if not fp64 else _graphs()[:2]
    mats = [vne.matrix_from_graph(vctx, g, fp64=fp64) for g in gs]
    eps = 2e-3
    sketch = M_STEPS if fp64 else 8  # FP32: a short sketch (Hutch++ stays unbiased)
    opt = vne.options(reorth=0, panel=8, quad_tol=-1.0, check_every=CHECK, sketch_steps=0 if fp64 else sketch)
    try:
        if fp64:
            sched = [(0, i, 300 + i) for i in range(len(gs))]
            res, most = _run(vctx, mats, sched, budget=1 << 34, max_active=1, eps=eps, opt=opt)
        else:
            sched = [(0, 0, 41), (0, 1, 42), (5, 2, 43), (17, 3, 44), (20, 0, 45)]
            res, most = _run(vctx, mats, sched, budget=1 << 36, max_active=8, eps=eps, opt=opt)
            assert most >= 3
        for (mi, seed), r in res.items():
            assert r["state"] == 2
            if not fp64:
                alone, _ = _run(vctx, mats, [(0, mi, seed)], budget=1 << 36, max_active=8, eps=eps, opt=opt)
                assert alone[(mi, seed)]["estimate"] == r["estimate"]
            A, _ = density.density_matrix(gs[mi])
            ref, _, nv, steps, _ = estimators.served_hutchpp(A, eps, 64, M_STEPS, seed, max_vectors=1024,
                                                             quad_tol=0.5 * eps, check_every=CHECK,
                                                             sketch_steps=sketch)
            assert r["vectors"] == nv
            assert r["done_tick"] - r["admit_tick"] == sum(steps), (steps, r)
            assert max(steps) < M_STEPS  # the blocks stopped early
            tol = 1e-10 if fp64 else 1e-5
            assert abs(r["estimate"] - ref) <= tol * ref
    finally:
        for m in mats:
            vne.vne_matrix_destroy(m)


def test_serving_work_tables_reused_and_grown(vctx):
    """The server's work tables (CTAs, long rows, tiles) are device tables in
    which each admitted query takes first-fit ranges and frees them at
    completion.  Queries of very different sizes through three slots make
    the ranges fragment, get reused by other queries and the tables grow
    mid-run; every result is still bit-identical to the query served alone,
    and within the mixed-path tolerance of the oracle for two of them."""
    # the large ones need more than the tables' first 1024 CTAs together
    gs = [graphs.barabasi_albert(300_000, 3, 61), graphs.erdos_renyi(1500, 8 / 1499, 62),
          graphs.watts_strogatz(150_000, 6, 0.1, 63), graphs.barabasi_albert(900, 3, 64),
          graphs.erdos_renyi(250_000, 8 / 249_999, 65)]
    mats = [vne.matrix_from_graph(vctx, g, fp64=False) for g in gs]
    opt = vne.options(reorth=0, panel=8, quad_tol=-1.0, check_every=CHECK, sketch_steps=8)
    eps = 4e-3
    try:
        sched = [(t, i % 5, 700 + i) for i, t in enumerate([0, 0, 0, 3, 9, 15, 22, 30, 41, 55, 60, 75])]
        mixed, most = _run(vctx, mats, sched, budget=1 << 36, max_active=3, eps=eps, cap=512, opt=opt)
        assert most == 3
        for (mi, seed), r in mixed.items():
            assert r["state"] == 2
            alone, _ = _run(vctx, mats, [(0, mi, seed)], budget=1 << 36, max_active=3, eps=eps, cap=512, opt=opt)
            assert alone[(mi, seed)]["estimate"] == r["estimate"], (mi, seed)
        for mi, seed in [(1, 701), (3, 703)]:
            A, _ = density.density_matrix(gs[mi])
            ref, _, nv, steps, _ = estimators.served_hutchpp(A, eps, 64, M_STEPS, seed, max_vectors=512,
                                                             quad_tol=0.5 * eps, check_every=CHECK, sketch_steps=8)
            r = mixed[(mi, seed)]
            assert r["vectors"] == nv and abs(r["estimate"] - ref) <= 1e-5 * ref
    finally:
        for m in mats:
            vne.vne_matrix_destroy(m)
