"""GPU parity of the multi-query, batched and serving entry points against the oracle.

Every traversal result, however it was scheduled (several queries in one
level loop, instances in disjoint-union groups inside one graph launch,
queries admitted into a running server), must equal the oracle's BFS levels /
Dijkstra distances from the same source bit for bit. The serving test also
checks that a query's result is the same alone (np_bfs / np_sssp) and in the
mix.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle
from gpu_util import DevGraph
from paper_2201_02789_gb300 import gen
from paper_2201_02789_gb300 import nestpar as npb

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def ctx():
    from paper_2201_02789_gb300 import build as nbuild
    nbuild.build()
    nbuild.build_gen()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = npb.Context(0)
    yield c
    c.close()


def _ref(g, kind, src):
    return oracle.bfs(g.row_ptr, g.col, src) if kind == 0 else oracle.sssp(g.row_ptr, g.col, g.w, src)


# ------------------------------------------------------------------ multi-query

MULTI_FORMS = [("nodp", npb.config("nodp")), ("tca", npb.config("tca")),
               ("tca-T1-C1", npb.config("tca", threshold=1, cfactor=1)),
               ("cdp-chunk", npb.config("cdp")),
               ("block", npb.config("tca", granularity="block", threshold=4)),
               ("mb3-lb", npb.config("tca", granularity="multiblock", group_blocks=3, scan=npb.NP_SCAN_LOOKBACK)),
               # swept frontier over every query's state: every grid level, or levels of 100+ parents
               ("sweep", npb.config("tca", sweep_parents=1, small_parents=0)),
               ("sweep-mixed", npb.config("tca", sweep_parents=100))]


@pytest.mark.parametrize("name,cfg", MULTI_FORMS, ids=[f[0] for f in MULTI_FORMS])
def test_multi_source_rows_equal_single_solves(ctx, name, cfg):
    g = gen.rmat(11, 12, seed=21, n=1500)
    dg = DevGraph(g)
    srcs = gen.random_sources(g, 9, seed=22)
    srcs[3] = srcs[1]                       # two queries from one source
    ld = npb.multi_stride(g.n)
    assert ld == 2048 and ld > g.n
    lv = torch.full((len(srcs), ld), 7, dtype=torch.int32, device=DEV)
    dist = torch.full((len(srcs), ld), 7, dtype=torch.int32, device=DEV)
    _, st = npb.np_bfs_multi(ctx.handle, dg.csr, srcs, lv, ld, cfg, stats=True)
    assert st["error"] == 0
    npb.np_sssp_multi(ctx.handle, dg.csr, srcs, dist, ld, cfg)
    lv_h = lv.cpu().numpy()
    d_h = dist.cpu().numpy().view(np.uint32)
    for q, s in enumerate(srcs):
        np.testing.assert_array_equal(lv_h[q, :g.n], oracle.bfs(g.row_ptr, g.col, int(s)))
        np.testing.assert_array_equal(d_h[q, :g.n], oracle.sssp(g.row_ptr, g.col, g.w, int(s)))
        assert (lv_h[q, g.n:] == -1).all() and (d_h[q, g.n:] == 0xFFFFFFFF).all()
    assert st["parents"] == sum(int((oracle.bfs(g.row_ptr, g.col, int(s)) >= 0).sum()) for s in srcs)


@pytest.mark.parametrize("sweep", [0, 1, 5000], ids=["append", "sweep", "sweep-large-levels"])
def test_multi_source_larger_graph(ctx, sweep):
    """16 queries on an R-MAT scale-16 graph (2^20 state elements: many sweep CTAs and
    parent tiles per level), every row against the oracle."""
    g = gen.rmat(16, 16, seed=23)
    dg = DevGraph(g)
    srcs = gen.random_sources(g, 16, seed=24)
    ld = npb.multi_stride(g.n)
    cfg = npb.config("tca", sweep_parents=sweep)
    lv = torch.full((len(srcs), ld), 7, dtype=torch.int32, device=DEV)
    dist = torch.full((len(srcs), ld), 7, dtype=torch.int32, device=DEV)
    _, st = npb.np_bfs_multi(ctx.handle, dg.csr, srcs, lv, ld, cfg, stats=True)
    assert st["error"] == 0
    _, st = npb.np_sssp_multi(ctx.handle, dg.csr, srcs, dist, ld, cfg, stats=True)
    assert st["error"] == 0
    lv_h = lv.cpu().numpy()
    d_h = dist.cpu().numpy().view(np.uint32)
    with ThreadPoolExecutor(8) as ex:
        refs = list(ex.map(lambda s: (oracle.bfs(g.row_ptr, g.col, int(s)), oracle.sssp(g.row_ptr, g.col, g.w, int(s))),
                           srcs))
    for q, (rl, rd) in enumerate(refs):
        np.testing.assert_array_equal(lv_h[q, :g.n], rl)
        np.testing.assert_array_equal(d_h[q, :g.n], rd)
        assert (lv_h[q, g.n:] == -1).all() and (d_h[q, g.n:] == 0xFFFFFFFF).all()


def test_multi_source_argument_errors(ctx):
    g = gen.rmat(8, 4, seed=23)
    dg = DevGraph(g)
    out = torch.empty(4 * 256, dtype=torch.int32, device=DEV)
    for ld, srcs in ((255, [0, 1]), (384, [0, 1]), (256, [0, 256]), (256, [-1])):
        s = npb.np_bfs_multi(ctx.handle, dg.csr, srcs, out, ld, npb.config("tca"), check=False)
        assert s == npb.NP_ERR_INVALID, (ld, srcs)


# ---------------------------------------------------------------------- batched

def _batch_inputs(count, lo, hi, seed, kind):
    specs = gen.batch_specs(count, seed=seed, log2_lo=lo, log2_hi=hi)
    graphs = gen.batch_graphs(specs, weights=(1, 255))
    srcs = np.zeros(count, dtype=np.int32)          # source 0, per the batched recipe
    devs = [DevGraph(g) for g in graphs]
    return specs, graphs, srcs, devs


def _check_batch(graphs, srcs, out_h, offs, kind, sample=None):
    idx = range(len(graphs)) if sample is None else sample
    with ThreadPoolExecutor(8) as ex:
        refs = list(ex.map(lambda i: _ref(graphs[i], kind, int(srcs[i])), idx))
    for i, ref in zip(idx, refs):
        got = out_h[offs[i]:offs[i] + graphs[i].n]
        np.testing.assert_array_equal(got, ref, err_msg=f"instance {i}")


@pytest.mark.parametrize("kind", [npb.NP_BATCH_BFS, npb.NP_BATCH_SSSP])
@pytest.mark.parametrize("form", ["tca", "nodp", "tca-T1", "tca-sweep", "tca-sweep-mixed"])
def test_batch_matches_oracle(ctx, kind, form):
    # (swept frontier: every grid level, or only levels of at least 50 parents)
    cfg = {"tca": npb.config("tca"), "nodp": npb.config("nodp"),
           "tca-T1": npb.config("tca", threshold=1, cfactor=2, child_block=64),
           "tca-sweep": npb.config("tca", sweep_parents=1, small_parents=0),
           "tca-sweep-mixed": npb.config("tca", sweep_parents=50)}[form]
    specs, graphs, srcs, devs = _batch_inputs(48, 6.0, 14.0, 40 + kind, kind)
    # small groups: several groups per class, and classes of width 2
    b = npb.np_batch_create(ctx.handle, [d.csr for d in devs], srcs, kind, cfg, max_group_edges=40000)
    try:
        offs, total = npb.np_batch_layout(b, len(graphs))
        assert total == sum(g.n for g in graphs)
        classes = npb.np_batch_classes(b)
        assert sum(c["instances"] for c in classes) == len(graphs)
        assert sum(c["edges"] for c in classes) == sum(g.m for g in graphs)
        assert any(c["groups"] > 1 for c in classes)
        out = torch.full((total,), 5, dtype=torch.int32, device=DEV)
        _, st = npb.np_batch_run(b, out, stats=True)
        assert st["error"] == 0
        oh = out.cpu().numpy() if kind == 0 else out.cpu().numpy().view(np.uint32)
        _check_batch(graphs, srcs, oh, offs, kind)
        # a second run into another buffer (graph rebuilt) gives the same bytes
        out2 = torch.zeros((total,), dtype=torch.int32, device=DEV)
        npb.np_batch_run(b, out2)
        torch.cuda.synchronize()
        assert torch.equal(out, out2)
    finally:
        npb.np_batch_destroy(b)


def test_batch_tune_then_run(ctx):
    kind = npb.NP_BATCH_SSSP
    specs, graphs, srcs, devs = _batch_inputs(24, 8.0, 15.0, 44, kind)
    b = npb.np_batch_create(ctx.handle, [d.csr for d in devs], srcs, kind, npb.config("tca"))
    try:
        offs, total = npb.np_batch_layout(b, len(graphs))
        out = torch.zeros((total,), dtype=torch.int32, device=DEV)
        npb.np_batch_tune(b, out, reps=2)
        classes = npb.np_batch_classes(b)
        for c in classes:
            # 17 candidates, and the pick with a swept frontier when its form can sweep
            assert c["tuned_ms"] > 0 and c["candidates"] in (17, 18)
            cfg = c["config"]
            assert cfg["variant"] == npb.NP_VARIANT_NODP or cfg["granularity"] == npb.NP_GRAN_GRID_HOST
            # (the candidates keep the class's own value, the library default here)
            assert cfg["sweep_parents"] in (npb.np_config_default().sweep_parents, 1)
        out.fill_(3)
        _, st = npb.np_batch_run(b, out, stats=True)
        assert st["error"] == 0
        _check_batch(graphs, srcs, out.cpu().numpy().view(np.uint32), offs, kind)
        # forms with device-side launches cannot sit in the batch graph
        s = npb.np_batch_set_config(b, 0, npb.config("cdp"), check=False)
        assert s == npb.NP_ERR_UNSUPPORTED
        npb.np_batch_set_config(b, 0, npb.config("tca", threshold=64))
        npb.np_batch_run(b, out)
        _check_batch(graphs, srcs, out.cpu().numpy().view(np.uint32), offs, kind)
        npb.np_batch_set_config(b, 0, npb.config("tca", sweep_parents=1))
        out.fill_(3)
        npb.np_batch_run(b, out)
        _check_batch(graphs, srcs, out.cpu().numpy().view(np.uint32), offs, kind)
    finally:
        npb.np_batch_destroy(b)


def test_create_checks_graphs_on_device(ctx):
    """A column index outside [0, n) or a row_ptr that breaks its contract is refused by
    np_batch_create / np_server_create before any traversal reads it."""
    g = gen.rmat(9, 8, seed=45)
    good = DevGraph(g)
    bad_col = g.col.copy()
    bad_col[17] = g.n                      # one past the last vertex
    bad = DevGraph(gen.Csr(g.n, g.row_ptr, bad_col, g.w))
    bad_rp = g.row_ptr.copy()
    bad_rp[5], bad_rp[6] = bad_rp[6], bad_rp[5] - 1     # decreasing
    bad2 = DevGraph(gen.Csr(g.n, bad_rp, g.col, g.w))
    for dg in (bad, bad2):
        with pytest.raises(npb.NestparError) as e:
            npb.np_batch_create(ctx.handle, [good.csr, dg.csr], [0, 0], npb.NP_BATCH_BFS, npb.config("tca"))
        assert e.value.status == npb.NP_ERR_INVALID
        s = npb.np_server_create(ctx.handle, [good.csr, dg.csr], check=False)
        assert s == npb.NP_ERR_INVALID
    b = npb.np_batch_create(ctx.handle, [good.csr], [0], npb.NP_BATCH_BFS, npb.config("tca"))
    npb.np_batch_destroy(b)


@pytest.mark.slow
def test_batch_full_size_sampled(ctx):
    """512 instances, n log-uniform in [2^10, 2^20], edge factor 8..32 (about 1.7e9 edges),
    in the launch configuration the batched benchmark uses; the oracle checks a sample of
    instances (the 6 smallest, 6 spread through the middle, the 4 largest)."""
    kind = npb.NP_BATCH_SSSP
    specs = gen.batch_specs()
    graphs = gen.batch_graphs(specs)
    srcs = np.zeros(len(specs), dtype=np.int32)
    devs = [DevGraph(g) for g in graphs]
    b = npb.np_batch_create(ctx.handle, [d.csr for d in devs], srcs, kind, npb.config("tca"))
    try:
        offs, total = npb.np_batch_layout(b, len(graphs))
        del devs                                        # the batch owns its copies
        torch.cuda.empty_cache()
        out = torch.empty((total,), dtype=torch.int32, device=DEV)
        _, st = npb.np_batch_run(b, out, stats=True)
        assert st["error"] == 0
        oh = out.cpu().numpy().view(np.uint32)
        order = np.argsort([g.n for g in graphs], kind="stable")
        sample = sorted(set(order[:6].tolist() + order[len(order) // 2 - 3:len(order) // 2 + 3].tolist()
                            + order[-4:].tolist()))
        _check_batch(graphs, srcs, oh, offs, kind, sample=sample)
        # every instance: the source is at distance 0 and reached vertices are a subset of [0, n)
        for i, g in enumerate(graphs):
            assert oh[offs[i]] == 0
    finally:
        npb.np_batch_destroy(b)


# ---------------------------------------------------------------------- serving

@pytest.fixture(scope="module")
def serve_graphs():
    graphs = [gen.rmat(s, 16, seed=50 + s) for s in (9, 11, 13)]
    return graphs, [DevGraph(g) for g in graphs]


# (swept frontier: the default's levels of 4096+ parents, or every level; the scale-9 pool's slots
# are smaller than a sweep chunk, so it sweeps every slot, the others skip the idle ones)
@pytest.mark.parametrize("sweep", [{}, dict(sweep_parents=1)], ids=["default", "sweep-every-level"])
def test_server_alone_equals_mix(ctx, serve_graphs, sweep):
    graphs, devs = serve_graphs
    sv = npb.np_server_create(ctx.handle, [d.csr for d in devs], max_slots=3, levels_per_step=2,
                              bfs_cfg=npb.config("tca", **sweep), sssp_cfg=npb.config("tca", threshold=8, **sweep))
    try:
        rng = np.random.default_rng(0)   # order of arrivals only; sources come from gen
        queries = []
        for gi, g in enumerate(graphs):
            for kind in (0, 1):
                for s in gen.random_sources(g, 6, seed=60 + 2 * gi + kind):
                    queries.append((gi, kind, int(s)))
        order = rng.permutation(len(queries))
        outs, tickets = {}, {}
        pending = list(order)
        steps = 0
        while pending or any(not npb.np_server_poll(sv, t)["done"] for t in tickets.values()):
            # a few arrivals per step, while earlier queries are still resident
            for _ in range(3):
                if pending:
                    qi = int(pending.pop(0))
                    gi, kind, s = queries[qi]
                    outs[qi] = torch.full((graphs[gi].n,), 9, dtype=torch.int32, device=DEV)
                    tickets[qi] = npb.np_server_submit(sv, gi, kind, s, outs[qi])
            npb.np_server_step(sv)
            steps += 1
            assert steps < 10000
        infos = {qi: npb.np_server_poll(sv, t) for qi, t in tickets.items()}
        fin = npb.np_server_finished(sv)
        assert sorted(fin) == sorted(tickets.values())        # every ticket reported once
        assert npb.np_server_finished(sv) == []
        # queries overlapped: some were admitted while others were resident
        assert any(i["admit_step"] > i["submit_step"] for i in infos.values())
        for qi, (gi, kind, s) in enumerate(queries):
            got = outs[qi].cpu().numpy()
            g, dg = graphs[gi], devs[gi]
            alone = torch.empty((g.n,), dtype=torch.int32, device=DEV)
            if kind == 0:
                npb.np_bfs(ctx.handle, dg.csr, s, alone, npb.config("tca"))
            else:
                npb.np_sssp(ctx.handle, dg.csr, s, alone, npb.config("tca"))
            np.testing.assert_array_equal(got, alone.cpu().numpy(), err_msg=f"query {qi} mix vs alone")
            ref = _ref(g, kind, s)
            np.testing.assert_array_equal(got.view(np.uint32) if kind else got, ref, err_msg=f"query {qi}")
    finally:
        npb.np_server_destroy(sv)


def test_server_memory_admission(ctx, serve_graphs):
    graphs, devs = serve_graphs
    csrs = [d.csr for d in devs]
    # a budget below one slot of the largest pool is refused
    s = npb.np_server_create(ctx.handle, csrs, memory_budget=1 << 20, check=False)
    assert s == npb.NP_ERR_NOMEM
    budget = 256 << 20
    sv = npb.np_server_create(ctx.handle, csrs, memory_budget=budget, max_slots=1024)
    try:
        share = budget // (2 * len(csrs))
        for gi, g in enumerate(graphs):
            npad = npb.multi_stride(g.n)
            for kind in (0, 1):
                slots, per = npb.np_server_pool_info(sv, gi, kind)
                assert 1 <= slots <= 1024
                if slots < 1024:
                    # per = the bytes of a one-slot pool, at least a slot's marginal cost; a slot
                    # costs at least 36 bytes per element (state, two frontiers, stamp, record, offset)
                    assert share // per <= slots <= share // (36 * npad) + 1
        # more queries than slots on the smallest pool: all finish, by admission as slots free up
        slots, _ = npb.np_server_pool_info(sv, 0, 0)
        g = graphs[0]
        srcs = gen.random_sources(g, slots + 5, seed=70)
        outs = [torch.empty((g.n,), dtype=torch.int32, device=DEV) for _ in srcs]
        ts = [npb.np_server_submit(sv, 0, 0, int(s), o) for s, o in zip(srcs, outs)]
        for _ in range(1000):
            if npb.np_server_step(sv) == 0:
                break
        for s, o, t in zip(srcs, outs, ts):
            assert npb.np_server_poll(sv, t)["done"] == 1
            np.testing.assert_array_equal(o.cpu().numpy(), oracle.bfs(g.row_ptr, g.col, int(s)))
    finally:
        npb.np_server_destroy(sv)


def test_server_rejects_device_launch_forms(ctx, serve_graphs):
    _, devs = serve_graphs
    s = npb.np_server_create(ctx.handle, [devs[0].csr], bfs_cfg=npb.config("cdp"), check=False)
    assert s == npb.NP_ERR_UNSUPPORTED


@pytest.mark.slow
def test_server_full_size_sampled(ctx):
    """The serving workload's graphs (R-MAT scales 16..22, edge factor 16): a mix of BFS and
    SSSP queries submitted in waves while others are resident; a sample checked against the
    oracle (queries on the largest graphs included) and against single solves."""
    from concurrent.futures import ThreadPoolExecutor
    graphs = [gen.rmat(s, 16, seed=5 * 1000 + s) for s in range(16, 23)]
    devs = [DevGraph(g) for g in graphs]
    sv = npb.np_server_create(ctx.handle, [d.csr for d in devs], max_slots=16, levels_per_step=2,
                              bfs_cfg=npb.config("tca"), sssp_cfg=npb.config("tca"))
    try:
        qs = []
        for gi, g in enumerate(graphs):
            for kind in (0, 1):
                for s in gen.random_sources(g, 3, seed=500 + 2 * gi + kind):
                    qs.append((gi, kind, int(s)))
        outs, ticks, pending = {}, {}, list(range(len(qs)))
        for step in range(100000):
            for _ in range(4):
                if pending:
                    q = pending.pop(0)
                    gi, kind, s = qs[q]
                    outs[q] = torch.empty((graphs[gi].n,), dtype=torch.int32, device=DEV)
                    ticks[q] = npb.np_server_submit(sv, gi, kind, s, outs[q])
            if npb.np_server_step(sv) == 0 and not pending:
                break
        assert all(npb.np_server_poll(sv, t)["done"] for t in ticks.values())
        sample = [q for q in range(len(qs)) if q % 3 == 0]
        with ThreadPoolExecutor(8) as ex:
            refs = list(ex.map(lambda q: _ref(graphs[qs[q][0]], qs[q][1], qs[q][2]), sample))
        for q, ref in zip(sample, refs):
            gi, kind, s = qs[q]
            got = outs[q].cpu().numpy()
            np.testing.assert_array_equal(got.view(np.uint32) if kind else got, ref, err_msg=f"query {q}")
        for q in range(0, len(qs), 7):
            gi, kind, s = qs[q]
            alone = torch.empty((graphs[gi].n,), dtype=torch.int32, device=DEV)
            (npb.np_sssp if kind else npb.np_bfs)(ctx.handle, devs[gi].csr, s, alone, npb.config("tca"))
            assert torch.equal(alone, outs[q]), q
    finally:
        npb.np_server_destroy(sv)
