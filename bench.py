#!/usr/bin/env python3
"""Benchmark of the B2SR hot path on the R-MAT scale-20 workload.

One step is one pass of the hot path over the workload: CSR -> B2SR
conversion (tile_dim 4, direct SpMV schedule: the autotuner's choice for
the step's dominant scheme on this graph), one Boolean SpMV, BFS from 16
seeded sources (one batched sequence over 32-lane frontier words), PageRank
(fp32, d = 0.85, 50 iterations) and connected components.  Throughput is
GTEPS: the edges the step's queries must touch -- nnz for the SpMV, nnz per
BFS source, nnz per PageRank iteration and nnz for CC, i.e. 68 * nnz per
step -- divided by the step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--extra NAME ...] [--no-extras] [--permute SEED]

N > 1 runs under torchrun, one replica per GPU (the path has no exchange
step); rank 0 prints one JSON line.  --impl reference times whole steps of
the same workload on the CPU oracle, on all host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "B2SR SpMV/BFS GTEPS & % HBM peak; TC edges/s; batched BFS queries/s vs plain"
SCALE, EDGE_FACTOR, SEED = 20, 16, 1
TILE = 4                 # B2SR tile_dim of the main workload ...
SCHEDULE = 2             # ... and its SpMV schedule (b2sr_schedule DIRECT); see workload_desc
SERVE_TILE = 4           # tile_dim of the served graphs (direct schedule, as the main workload)
EXTRA_TILE = 8           # tile_dim of the grid SSSP, triangle-count and arena extras
NSRC, PR_ITERS, DAMP = 16, 50, 0.85
QUERIES_PER_STEP = 1 + NSRC + PR_ITERS + 1  # edge passes counted per step (x nnz)
PERMUTE = None           # seed of a vertex relabelling of the main workload (None: R-MAT's own ids)
FAMILIES = ["spmv_bool", "spmv_count", "spmv_plus", "spmv_minplus", "spmv_min_i32", "spmm_or64", "spmm_or32",
            "spmm_plus4", "spmv_max", "spmv_maxkey"]


def ids_desc():
    return "unpermuted ids" if PERMUTE is None else f"ids permuted (seed {PERMUTE})"


def workload_desc(n, nnz):
    return {
        "workload": f"R-MAT scale {SCALE} ef{EDGE_FACTOR} a/b/c/d=0.57/0.19/0.19/0.05 seed {SEED}, symmetrised, "
                    f"no self-loops/duplicates, {ids_desc()}; B2SR tile {TILE}x{TILE}; step = CSR->B2SR + Boolean SpMV + "
                    f"BFS from {NSRC} seeded sources (batched) + fp32 PageRank {PR_ITERS} iters + CC",
        "n": int(n), "nnz": int(nnz), "tile_dim": TILE, "schedule": "direct" if SCHEDULE == 2 else "staged",
        "tile_choice": "tile_dim sweep 4/8/16/32 by b2sr_autotune for the step's dominant scheme (plus-times, "
                       "PageRank); its live choice is reported in extra.autotune_main",
        "sources": NSRC, "pagerank_iters": PR_ITERS,
        "edges_per_step": int(QUERIES_PER_STEP * nnz),
        "cache": "inputs larger than L2 (tile stream 272 MiB vs 129 MB L2); no flush",
    }


def make_graph():
    from paper_2201_08560_gb300 import graphs
    g = graphs.rmat(SCALE, EDGE_FACTOR, seed=SEED)
    if PERMUTE is not None:
        g = graphs.permute(g, PERMUTE)
    srcs = graphs.sources(g, NSRC, seed=7)
    xbits = graphs.random_bits(g.n, 0.05, seed=3)
    return g, srcs, xbits


# ---------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------

def oracle_step(g, srcs, xbits, threads):
    """One whole step of the workload on the CPU oracle with `threads` host
    threads: CSR -> B2SR (one thread), the Boolean SpMV (row loop on all
    threads), BFS from the 16 sources (one source per thread), PageRank for
    50 iterations (row loops on all threads) and CC (one thread, union-find).
    Returns (seconds, per-part seconds)."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    oracle.set_threads(threads)
    t = {}
    a = time.perf_counter(); oracle.b2sr(g, TILE); t["convert"] = time.perf_counter() - a
    a = time.perf_counter(); oracle.spmv_bool(g, xbits); t["spmv"] = time.perf_counter() - a
    a = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda s: oracle.bfs(g, int(s)), srcs))
    t["bfs_16_sources"] = time.perf_counter() - a
    a = time.perf_counter(); oracle.pagerank(g, DAMP, PR_ITERS); t["pagerank_50"] = time.perf_counter() - a
    a = time.perf_counter(); oracle.cc(g); t["cc"] = time.perf_counter() - a
    return sum(t.values()), t


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    """The CPU oracle on the same workload and metric: whole steps (no
    extrapolation) on all of the host's cores, W untimed then K timed."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    g, srcs, xbits = make_graph()
    import oracle
    oracle.build()
    cores = host_cores()
    edges = QUERIES_PER_STEP * g.nnz
    for _ in range(args.warmup):
        oracle_step(g, srcs, xbits, cores)
    times, parts = [], []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        st, p = oracle_step(g, srcs, xbits, cores)
        times.append(st)
        parts.append(p)
    wall = time.perf_counter() - t_all
    total = sum(times)
    value = args.steps * edges / total / 1e9
    sample = (f"whole steps of the workload on the oracle (plain C): CSR->B2SR k={TILE} and CC on one thread, "
              f"the Boolean SpMV and PageRank's row loops on {cores} OpenMP threads, the {NSRC} BFS sources "
              f"{cores} at a time; {args.steps} timed steps after {args.warmup} untimed")
    line = {
        "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": int(args.gpus), "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8/f64", "data": "synthetic", "impl": "reference",
        "config": dict(workload_desc(g.n, g.nnz), parallelism=f"replicas x{args.gpus}"),
        "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": cores, "kind": "oracle", "sample": sample,
                         "nproc": os.cpu_count(), "timed_wall_s": wall,
                         "parts_s_median": {k: statistics.median(p[k] for p in parts) for k in parts[0]}},
        "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# serving: resident R-MAT graphs and a Poisson stream of mixed queries
# ---------------------------------------------------------------------------
SERVE_GRAPHS, SERVE_SCALES = 32, (14, 20)
SERVE_QUERIES, SERVE_RATE, SERVE_PR_ITERS = 10000, 2000.0, 20
SERVE_BUDGET = 64 << 30
SERVE_SOLO_QUERIES = 300
SERVE_FIFO_QUERIES = 1000


def _serve_graph(scale, seed):
    from paper_2201_08560_gb300 import graphs
    g = graphs.rmat(scale, EDGE_FACTOR, seed=seed)
    deg = np.diff(g.rowptr)
    return g.n, g.rowptr, g.colind, np.flatnonzero(deg > 0).astype(np.int32)


def serving_extra(B, dev, gs, t_gen):
    """32 resident graphs (scales 14..20, k = 8); 10,000 queries, half BFS from
    a random non-isolated source and half personalised PageRank (20 iterations,
    all teleport mass on a random non-isolated source), arriving as a Poisson
    stream at 2,000 queries/s.  Reports the server's latency percentiles and
    throughput for that stream, its throughput when all queries are queued at
    once, and the throughput of one query per driver call on a sample of the
    same mix."""
    import torch
    lo, hi = SERVE_SCALES
    mats = []
    for n, rp, ci, _ in gs:
        mats.append(B.b2sr_from_csr(n, torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev), SERVE_TILE))
        B.b2sr_set_schedule(mats[-1], SCHEDULE)
    rng = np.random.default_rng(11)
    plan = []
    for _ in range(SERVE_QUERIES):
        gi = int(rng.integers(SERVE_GRAPHS))
        cand = gs[gi][3]
        src = int(cand[rng.integers(cand.size)])
        plan.append(("bfs" if rng.random() < 0.5 else "pr", gi, src))
    arrivals = np.cumsum(rng.exponential(1.0 / SERVE_RATE, SERVE_QUERIES))
    # every query's output preallocated (one slab), so submission is one C call
    sizes = [gs[gi][0] for _, gi, _ in plan]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    slab = torch.empty(int(offs[-1]), dtype=torch.int32, device=dev)
    outs_i = [slab[offs[i]:offs[i + 1]] for i in range(SERVE_QUERIES)]
    outs_f = [o.view(torch.float32) for o in outs_i]
    torch.cuda.synchronize()

    def run(srv, gids, queries, times=None):
        srv.reset_stats()
        t0 = time.perf_counter()
        ids = []
        for i, (kind, gi, src) in enumerate(queries):
            if times is not None:
                due = t0 + times[i]
                while True:
                    now = time.perf_counter()
                    if now >= due:
                        break
                    if due - now > 3e-4:
                        time.sleep(due - now - 2e-4)
            if kind == "bfs":
                ids.append(srv.submit_bfs(gids[gi], src, outs_i[i])[0])
            else:
                ids.append(srv.submit_pagerank(gids[gi], src, DAMP, SERVE_PR_ITERS, outs_f[i])[0])
        srv.drain(600.0)
        wall = time.perf_counter() - t0
        st = srv.stats()
        return {"queries": len(queries), "wall_s": wall, "queries_per_s": len(queries) / wall,
                "p50_ms": st["p50_us"] / 1e3, "p99_ms": st["p99_us"] / 1e3, "max_ms": st["max_us"] / 1e3,
                "device_steps": st["steps"], "failed": st["failed"]}

    res = {}
    with B.Server(SERVE_BUDGET, 64, 2) as srv:
        gids = [srv.add_graph(m) for m in mats]
        resident = sum(srv.graph_bytes(g)[0] for g in gids)
        run(srv, gids, plan[:200])                                     # warm-up
        res["poisson"] = run(srv, gids, plan, arrivals)
        res["saturated"] = run(srv, gids, plan)
        bfs_only = [q for q in plan if q[0] == "bfs"]
        res["saturated_bfs_only"] = run(srv, gids, bfs_only)
    # one query per driver call in arrival order (a FIFO) on the same Poisson stream's first queries
    nf = SERVE_FIFO_QUERIES
    tele = torch.zeros(max(n for n, _, _, _ in gs), dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    lat = []
    t0 = time.perf_counter()
    for i, (kind, gi, src) in enumerate(plan[:nf]):
        due = t0 + arrivals[i]
        now = time.perf_counter()
        if now < due:
            time.sleep(due - now)
        m = mats[gi]
        if kind == "bfs":
            B.b2sr_bfs(m, src, outs_i[i])
        else:
            t = tele[: m.n]
            t[src] = 1.0
            B.b2sr_pagerank(m, DAMP, SERVE_PR_ITERS, t, outs_f[i])
            t[src] = 0.0
        torch.cuda.synchronize()
        lat.append(time.perf_counter() - due)
    wall = time.perf_counter() - t0
    lat_ms = np.sort(np.array(lat) * 1e3)
    res["fifo_one_query_per_call"] = {"queries": nf, "queries_per_s": nf / wall,
                                      "p50_ms": float(lat_ms[int(np.ceil(0.5 * nf)) - 1]),
                                      "p99_ms": float(lat_ms[int(np.ceil(0.99 * nf)) - 1]),
                                      "note": f"the first {nf} queries of the same Poisson stream, one driver call each"}
    # one query per driver call, same mix
    base = plan[:SERVE_SOLO_QUERIES]
    for kind, gi, src in base[:20]:   # warm-up
        if kind == "bfs":
            B.b2sr_bfs(mats[gi], src, outs_i[0])
        else:
            B.b2sr_pagerank(mats[gi], DAMP, 2, None, outs_f[0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nb = 0
    for i, (kind, gi, src) in enumerate(base):
        m = mats[gi]
        if kind == "bfs":
            B.b2sr_bfs(m, src, outs_i[i])
            nb += 1
        else:
            t = tele[: m.n]
            t[src] = 1.0
            B.b2sr_pagerank(m, DAMP, SERVE_PR_ITERS, t, outs_f[i])
            t[src] = 0.0
    torch.cuda.synchronize()
    base_wall = time.perf_counter() - t0
    t0 = time.perf_counter()
    bq = [q for q in plan if q[0] == "bfs"][:SERVE_SOLO_QUERIES]
    for i, (kind, gi, src) in enumerate(bq):
        B.b2sr_bfs(mats[gi], src, outs_i[i])
    torch.cuda.synchronize()
    base_bfs_wall = time.perf_counter() - t0
    res["one_query_per_call"] = {"queries": len(base), "queries_per_s": len(base) / base_wall}
    res["one_query_per_call_bfs_only"] = {"queries": len(bq), "queries_per_s": len(bq) / base_bfs_wall}
    res["speedup_saturated_vs_one_per_call"] = res["saturated"]["queries_per_s"] / res["one_query_per_call"]["queries_per_s"]
    res["speedup_bfs_saturated_vs_one_per_call"] = (res["saturated_bfs_only"]["queries_per_s"] /
                                                     res["one_query_per_call_bfs_only"]["queries_per_s"])
    res["config"] = (f"{SERVE_GRAPHS} R-MAT graphs, scales {lo}..{hi} (scale {lo} + i mod {hi - lo + 1}), ef{EDGE_FACTOR}, "
                     f"seeds 1000+i, k={SERVE_TILE} direct schedule, {resident / 2**30:.2f} GiB resident; {SERVE_QUERIES} queries, 50% BFS "
                     f"(random non-isolated source) / 50% personalised PageRank ({SERVE_PR_ITERS} iters, d={DAMP}), "
                     f"Poisson arrivals at {SERVE_RATE:.0f}/s; budget {SERVE_BUDGET >> 30} GiB, 64 BFS lanes and 2 "
                     f"four-column PageRank blocks per graph; graphs generated on the host before any timing ({t_gen:.1f} s)")
    for m in mats:
        m.close()
    return res


# ---------------------------------------------------------------------------
# the other workloads: weighted grid SSSP and triangle counting; batching
# ---------------------------------------------------------------------------
GRID_SIDE, GRID_WSEED, SSSP_DELTA = 4096, 5, 400.0
SSSP_DELTA_SWEEP = (50.0, 100.0, 200.0, 400.0, 800.0, 1600.0)  # bucket widths timed beside the default
TC_SCALE, TC_EF = 18, 32
MS_SCALE, MS_SOURCES = 22, 64
ARENA_GRAPHS, ARENA_SCALES = 256, (8, 16)
PERM_SEED = 2
ALU_PEAK_TOPS = 152 * 4 * 32 * 2.07e9 / 3 / 1e12   # AND-popc word operations per second at issue bound


def _grid_weighted():
    from paper_2201_08560_gb300 import graphs
    g = graphs.grid2d(GRID_SIDE, GRID_SIDE)
    return g.n, g.rowptr, g.colind, graphs.symmetric_weights(g, GRID_WSEED)


def _rmat_plain(scale, ef, seed):
    from paper_2201_08560_gb300 import graphs
    g = graphs.rmat(scale, ef, seed=seed)
    return g.n, g.rowptr, g.colind


def _timed(fn, reps=1):
    import torch
    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    b.synchronize()
    return a.elapsed_time(b) / reps


def tc_extra(B, dev, tc):
    """Triangle count of R-MAT scale 18 ef32 (tile_dim 8): the whole driver,
    the lower-triangle extraction and the masked-count kernel alone."""
    import torch
    out = {}
    n, rp, ci = tc
    rp_d, ci_d = torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev)
    with B.b2sr_from_csr(n, rp_d, ci_d, EXTRA_TILE) as m:
        cnt = {}
        ms = _timed(lambda: cnt.__setitem__("t", B.b2sr_tc(m)), reps=3)
        ms_lower = _timed(lambda: B.b2sr_lower(m).close(), reps=3)
        with B.b2sr_lower(m) as L:
            count = torch.empty(1, dtype=torch.int64, device=dev)
            B.b2sr_spgemm_masked_count(L, L, L, count)
            torch.cuda.synchronize()
            B.b2sr_timing_reset()
            B.b2sr_timing_enable(True)
            for _ in range(5):
                B.b2sr_spgemm_masked_count(L, L, L, count)
            torch.cuda.synchronize()
            tk, nk, _ = B.b2sr_timing_read("spgemm_masked")
            B.b2sr_timing_enable(False)
            B.b2sr_timing_reset()
            _, pairs = B.b2sr_spgemm_masked_count_work(L, L, L)
            pairs = int(pairs.item())
            l_tiles = L.n_tiles
        kern_ms = tk / nk
        ops = pairs / (kern_ms / 1e3)
        out = {
            "tile_dim": EXTRA_TILE, "ms": ms, "lower_ms": ms_lower, "kernel_ms": kern_ms,
            "nnz": int(ci.size), "l_edges": int(ci.size) // 2, "l_tiles": int(l_tiles),
            "edges_per_s": (ci.size // 2) / (ms / 1e3), "kernel_edges_per_s": (ci.size // 2) / (kern_ms / 1e3),
            "edges_counted": "|L|, the strictly lower triangle's entries",
            "triangles": int(cnt["t"].item()), "n": int(n),
            "roofline": {"bound": "alu", "kernel": f"masked_count_kernel (k={EXTRA_TILE})",
                         "achieved": ops / 1e12, "peak": ALU_PEAK_TOPS, "unit": "T AND-popc ops/s",
                         "frac": ops / 1e12 / ALU_PEAK_TOPS, "algorithmic_ops_per_launch": pairs,
                         "peak_source": "issue bound: 3 integer instructions (LOP3, POPC, IADD) per AND-popc "
                                        "of one row word, 152 SMs x 4 schedulers x 32 lanes x 2.07 GHz / 3",
                         "traffic": None}}
    return out


def grid_sssp_extra(B, dev, grid):
    """SSSP from the corner of a 4096 x 4096 4-neighbour grid with fp32
    weights on the 1/16 lattice in [1, 100) (tile_dim 8): the push driver at
    the default bucket width, its rounds, and a sweep of bucket widths."""
    import torch
    n, rp, ci, w = grid
    rp_d, ci_d = torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev)
    with B.b2sr_from_csr(n, rp_d, ci_d, EXTRA_TILE) as m:
        wb = B.b2sr_weights_from_csr(m, rp_d, ci_d, torch.from_numpy(w).to(dev))
        dist = torch.empty(n, dtype=torch.float32, device=dev)
        # push rounds over the frontier (the grid is symmetric: the handle is its own transpose),
        # delta-stepping buckets of 4x the largest weight
        ms = _timed(lambda: B.b2sr_sssp_push(m, 0, wb, dist, delta=SSSP_DELTA), reps=3)
        rounds, rows = B.b2sr_sssp_push_rounds(with_rows=True)
        far = float(dist[-1].item())
        sweep = {}
        for delta in SSSP_DELTA_SWEEP:
            t = _timed(lambda: B.b2sr_sssp_push(m, 0, wb, dist, delta=delta), reps=1)
            r = B.b2sr_sssp_push_rounds()
            sweep[str(delta)] = {"ms": t, "rounds": r, "us_per_round": t * 1e3 / r}
        out = {"driver": "b2sr_sssp_push", "delta": SSSP_DELTA, "ms": ms, "nnz": int(ci.size),
               "gteps": ci.size / (ms / 1e3) / 1e9, "rounds": rounds,
               "us_per_round": ms * 1e3 / rounds, "active_tile_rows_per_round": rows / rounds,
               "dist_far_corner": far, "n": int(n),
               "delta_sweep": sweep}
    return out


def batching_extra(B, dev, big, arena_gs, arena_scales):
    """64-source BFS on R-MAT scale 22 (tile_dim and schedule from the
    autotuner) against 64 single-source BFS calls; 256 R-MAT graphs (scales
    8..16) in one block-diagonal arena, one BFS each in one captured level loop,
    against one BFS call per separately converted graph."""
    import torch
    from paper_2201_08560_gb300 import graphs
    out = {}
    n, rp, ci = big
    rp_d, ci_d = torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev)
    rng = np.random.default_rng(17)
    deg = np.diff(rp)
    cand = np.flatnonzero(deg > 0)
    srcs = [int(v) for v in cand[rng.integers(0, cand.size, MS_SOURCES)]]
    smp = rng.integers(0, n, 8192).astype(np.int32)
    t0 = time.perf_counter()
    m, rep = B.b2sr_autotune(n, rp_d, ci_d, smp, B.BOOL_OR_AND, B.VEC_BITS64, keep_ratio=0.0, trials=3)
    t_tune = time.perf_counter() - t0
    with m:
        lv = torch.empty((MS_SOURCES, n), dtype=torch.int32, device=dev)
        t_multi = _timed(lambda: B.b2sr_bfs_multi(m, srcs, lv))
        lv1 = torch.empty(n, dtype=torch.int32, device=dev)

        def plain():
            for s in srcs:
                B.b2sr_bfs(m, s, lv1)
        t_plain = _timed(plain)
        out["bfs64_rmat22"] = {"tile_dim": rep["tile_dim"], "schedule": rep["schedule"],
                               "autotune_s": t_tune, "trial_us": rep["trial_us"], "est_ratio": rep["est_ratio"],
                               "batched_ms": t_multi, "plain_ms": t_plain,
                               "batched_queries_per_s": MS_SOURCES / (t_multi / 1e3),
                               "plain_queries_per_s": MS_SOURCES / (t_plain / 1e3),
                               "speedup": t_plain / t_multi, "nnz": int(ci.size),
                               "batched_gteps": MS_SOURCES * ci.size / (t_multi / 1e3) / 1e9}
    del rp_d, ci_d
    # the arena and the separate graphs run at the tile size and schedule the
    # autotuner chose above for the same scheme (Boolean BFS) on R-MAT graphs
    a_tile, a_sched = int(rep["tile_dim"]), int(rep["schedule"])
    gs = arena_gs
    csrs = [(gn, torch.from_numpy(grp).to(dev), torch.from_numpy(gci).to(dev)) for gn, grp, gci in gs]
    arena, bases = B.b2sr_from_csr_batch(csrs, a_tile)
    B.b2sr_set_schedule(arena, a_sched)
    srcs_a = [int(bases[i]) for i in range(len(gs))]  # vertex 0 of every graph (its hub)
    with arena:
        lva = torch.empty(arena.n, dtype=torch.int32, device=dev)
        t_arena = _timed(lambda: B.b2sr_bfs_sources(arena, srcs_a, lva))
        mats = [B.b2sr_from_csr(gn, grp, gci, a_tile) for gn, grp, gci in csrs]
        for mm in mats:
            B.b2sr_set_schedule(mm, a_sched)
        outs = [torch.empty(gn, dtype=torch.int32, device=dev) for gn, _, _ in csrs]

        def per_graph():
            for mm, o in zip(mats, outs):
                B.b2sr_bfs(mm, 0, o)
        t_each = _timed(per_graph)
        # the arena's per-graph slices equal the separate runs
        same = all(torch.equal(lva[b0:b0 + gn], o) for (gn, _, _), b0, o in zip(csrs, bases, outs))
        for mm in mats:
            mm.close()
        out["arena_256_graphs"] = {"graphs": len(gs), "scales": arena_scales, "arena_n": int(arena.n),
                                   "tile_dim": a_tile, "schedule": a_sched,
                                   "arena_ms": t_arena, "per_graph_ms": t_each,
                                   "graphs_per_s_arena": len(gs) / (t_arena / 1e3),
                                   "graphs_per_s_per_graph": len(gs) / (t_each / 1e3),
                                   "speedup": t_each / t_arena, "same_levels": bool(same)}
    return out


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        self.gpu_id = gpu_id

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", self.gpu_id],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def traffic_key(permute):
    """Names the graph a traffic figure was taken on."""
    return f"rmat{SCALE}" + ("" if permute is None else f"_perm{permute}")


def traffic_for(family, tile, kname, graph):
    """dram bytes per launch from the committed ncu summary, if it was taken on
    the same kernel, tile_dim, graph and kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    src = os.path.join(ROOT, "paper_2201_08560_gb300", "csrc", "spmv.cu")
    try:
        rec = json.load(open(path))
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        for ent in rec.values():
            if (ent.get("family") == family and ent.get("tile_dim") == tile and ent.get("kernel", "").startswith(kname)
                    and ent.get("graph") == graph and ent.get("kernel_source_sha256") == sha):
                return float(ent["dram_bytes_per_launch"]), ent
    except Exception:
        pass
    return None, None


def aggregate_replicas(ms_total, e2e_ms, edges_per_step, steps, world, device):
    """Whole-job throughput of `world` independent replicas (the graph does not
    shard: every query reads all of it): the slowest rank's times (all-reduce
    MAX) over the edges all ranks processed.  Returns (ms_total, e2e_ms,
    GTEPS, end-to-end GTEPS), the same on every rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_total, e2e_ms], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_total, e2e_ms = float(t[0]), float(t[1])
    value = world * edges_per_step * steps / (ms_total / 1e3) / 1e9
    e2e_value = world * edges_per_step * steps / (e2e_ms / 1e3) / 1e9
    return ms_total, e2e_ms, value, e2e_value


EXTRAS = ("config2", "serving", "tc", "grid_sssp", "batching")


def generate_extra_graphs(which):
    """Every graph the chosen extras use, generated on the host by a
    spawn-started process pool before any timed region starts (so no timing
    overlaps host generation work).  Returns a dict of plain arrays and the
    wall time."""
    import multiprocessing as mp
    t0 = time.perf_counter()
    lo, hi = SERVE_SCALES
    serve_specs = [(lo + i % (hi - lo + 1), 1000 + i) for i in range(SERVE_GRAPHS)]
    rng = np.random.default_rng(23)
    a_scales = [int(v) for v in rng.integers(ARENA_SCALES[0], ARENA_SCALES[1] + 1, ARENA_GRAPHS)]
    out = {}
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        jobs = {}
        if "serving" in which:
            jobs["serve"] = pool.starmap_async(_serve_graph, serve_specs)
        if "grid_sssp" in which:
            jobs["grid"] = pool.apply_async(_grid_weighted)
        if "tc" in which:
            jobs["tc"] = pool.apply_async(_rmat_plain, (TC_SCALE, TC_EF, 2))
        if "batching" in which:
            jobs["big"] = pool.apply_async(_rmat_plain, (MS_SCALE, EDGE_FACTOR, 3))
            jobs["arena"] = pool.starmap_async(_rmat_plain, [(sc, EDGE_FACTOR, 5000 + i) for i, sc in enumerate(a_scales)])
        if "config2" in which:
            jobs["perm"] = pool.apply_async(_rmat_perm, (SCALE, EDGE_FACTOR, SEED, PERM_SEED))
        for key, job in jobs.items():
            out[key] = job.get()
    return out, time.perf_counter() - t0


def _rmat_perm(scale, ef, seed, perm_seed):
    from paper_2201_08560_gb300 import graphs
    g = graphs.permute(graphs.rmat(scale, ef, seed=seed), perm_seed)
    return g.n, g.rowptr, g.colind


def timed_steps(B, step, args, barrier, uuid=None):
    """W untimed then K timed steps (CUDA events on the launching stream, a
    synchronising barrier on both sides), with the library's per-family SpMV
    launch timing on and, if `uuid` is given, clocks sampled meanwhile.
    Returns (ms over the K steps, per-family timing, launches, clocks)."""
    import torch
    for _ in range(args.warmup):
        step()
    barrier()
    B.b2sr_timing_reset()
    B.b2sr_timing_enable(True)
    launches0 = B.b2sr_launch_count()
    clk = ClockSampler(uuid) if uuid is not None else None
    if clk is not None:
        clk.__enter__()
    try:
        barrier()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(args.steps):
            step()
        ev1.record()
        barrier()
    finally:
        if clk is not None:
            clk.__exit__()
    launches = B.b2sr_launch_count() - launches0
    B.b2sr_timing_enable(False)
    fam = {}
    for f in FAMILIES:
        t, n, by = B.b2sr_timing_read(f)
        if n:
            fam[f] = {"ms": t, "launches": n, "bytes": by}
    B.b2sr_timing_reset()
    return ev0.elapsed_time(ev1), fam, launches, (clk.summary() if clk is not None else None)


def roofline_of(fam, ms_total, peak, peak_src, tile, schedule, graph):
    """Roofline entry of the family with the most device time in a timed
    region: algorithmic bytes per launch over its average CUDA-event launch
    time, against the measured copy bandwidth."""
    if not fam:
        return None
    dom = max(fam, key=lambda f: fam[f]["ms"])
    d = fam[dom]
    achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
    kname = spmv_kernel_name(dom, tile, schedule)
    traffic, _ = traffic_for(dom, tile, kname, graph)
    return {"bound": "hbm", "kernel": f"{kname} ({dom}, k={tile})", "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
            "algorithmic_bytes_per_launch": d["bytes"] / d["launches"],
            "avg_launch_us": d["ms"] / d["launches"] * 1e3, "launches": d["launches"],
            "share_of_step": d["ms"] / ms_total, "traffic": traffic}


def spmv_kernel_name(family, tile, schedule):
    """The SpMV kernel a family runs at this tile_dim and schedule (the
    library's dispatch: at k = 4 the tile_dim-4 kernel for the bit-vector
    schemes and, under the direct schedule, for the unweighted 4-byte value
    schemes; the staged gather kernel for the value schemes under the staged
    schedule at k <= 16; the chunk kernel otherwise)."""
    bits = family in ("spmv_bool", "spmv_count")
    k4_values = family in ("spmv_plus", "spmv_min_i32", "spmv_max", "spmm_or32")
    if tile == 4 and (bits or (k4_values and schedule == 2)):
        return "spmv_k4_kernel"
    if not bits and tile <= 16 and schedule != 2:
        return "spmv_gather_kernel"
    return "spmv_chunks_kernel"


def measured_peak():
    peak, src = 6800.0, "fallback 6.8 TB/s"
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak, src = float(pk["hbm_gbs"]), "measured hbm_gbs (MEASURED_PEAKS.json)"
    except Exception:
        pass
    return peak, src


def tile_sweep(B, dev, graphs_by_name, x_bits, peak):
    """Boolean and plus-times SpMV kernel time at tile_dim 4/8/16/32 (both
    schedules of the value scheme where it has two) on each graph: kernel us,
    algorithmic GB/s and the fraction of the measured copy bandwidth."""
    import torch
    out = {}
    for name, (n, rp, ci) in graphs_by_name.items():
        rows = {}
        rp_d, ci_d = torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev)
        x = torch.from_numpy(x_bits.view(np.int32)).to(dev)
        y = torch.empty(B.bitset_words(n), dtype=torch.int32, device=dev)
        xf = torch.from_numpy(np.random.default_rng(5).random(n).astype(np.float32)).to(dev)
        yf = torch.empty(n, dtype=torch.float32, device=dev)
        for k in (4, 8, 16, 32):
            ent = {}
            with B.b2sr_from_csr(n, rp_d, ci_d, k) as m:
                ent["tiles"] = m.n_tiles
                for label, sched, call, fam in (
                        ("bool", 2, lambda: B.b2sr_spmv(m, B.BOOL_OR_AND, B.VEC_BITS, x, B.VEC_BITS, y), "spmv_bool"),
                        ("plus_staged", 1, lambda: B.b2sr_spmv(m, B.PLUS_TIMES, B.VEC_F32, xf, B.VEC_F32, yf), "spmv_plus"),
                        ("plus_direct", 2, lambda: B.b2sr_spmv(m, B.PLUS_TIMES, B.VEC_F32, xf, B.VEC_F32, yf), "spmv_plus")):
                    if k == 32 and label == "plus_staged":
                        continue  # one schedule at tile_dim 32
                    B.b2sr_set_schedule(m, sched)
                    for _ in range(3):
                        call()
                    torch.cuda.synchronize()
                    B.b2sr_timing_reset()
                    B.b2sr_timing_enable(True)
                    for _ in range(10):
                        call()
                    torch.cuda.synchronize()
                    t, nl, by = B.b2sr_timing_read(fam)
                    B.b2sr_timing_enable(False)
                    B.b2sr_timing_reset()
                    us = t / nl * 1e3
                    gbs = by / nl / (us / 1e6) / 1e9
                    ent[label] = {"kernel": spmv_kernel_name(fam, k, sched), "us": us, "gbs": gbs,
                                  "frac": gbs / peak, "gteps": int(ci.size) / (us / 1e6) / 1e9}
            rows[f"k{k}"] = ent
        out[name] = rows
        del rp_d, ci_d
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the extras (config 2 sweep, serving, grid/TC, batching)")
    ap.add_argument("--extra", action="append", choices=EXTRAS, default=None,
                    help="run only these extras (repeatable; default all)")
    ap.add_argument("--tile", type=int, default=None, help="override the main workload's tile_dim")
    ap.add_argument("--schedule", type=int, default=None, help="override its SpMV schedule (1 staged, 2 direct)")
    ap.add_argument("--permute", type=int, default=None,
                    help="relabel the main workload's vertices by the random permutation of this seed")
    args = ap.parse_args()
    global TILE, SCHEDULE, PERMUTE
    if args.permute is not None:
        PERMUTE = args.permute
    if args.tile:
        TILE = args.tile
    if args.schedule:
        SCHEDULE = args.schedule
    if args.impl == "reference":
        return run_reference(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # the extras' graphs are generated before any GPU timing (rank 0 only)
    pre, t_gen = (None, 0.0)
    which = () if args.no_extras else tuple(args.extra or EXTRAS)
    if rank == 0 and which:
        pre, t_gen = generate_extra_graphs(which)

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2201_08560_gb300 import binding as B

    g, srcs, xbits = make_graph()
    rp_h = torch.from_numpy(g.rowptr).pin_memory()
    ci_h = torch.from_numpy(g.colind).pin_memory()
    x_h = torch.from_numpy(xbits.view(np.int32)).pin_memory()
    rp = rp_h.to(dev)
    ci = ci_h.to(dev)
    x = x_h.to(dev)
    words = B.bitset_words(g.n)
    y = torch.empty(words, dtype=torch.int32, device=dev)
    levels = torch.empty((NSRC, g.n), dtype=torch.int32, device=dev)
    pr = torch.empty(g.n, dtype=torch.float32, device=dev)
    labels = torch.empty(g.n, dtype=torch.int32, device=dev)
    srcs_l = [int(s) for s in srcs]

    def step(rp_=rp, ci_=ci, x_=x, y_=y, levels_=levels, pr_=pr, labels_=labels, n=g.n, srcs_=srcs_l):
        m = B.b2sr_from_csr(n, rp_, ci_, TILE)
        B.b2sr_set_schedule(m, SCHEDULE)
        B.b2sr_spmv(m, B.BOOL_OR_AND, B.VEC_BITS, x_, B.VEC_BITS, y_)
        B.b2sr_bfs_multi(m, srcs_, levels_)
        B.b2sr_pagerank(m, DAMP, PR_ITERS, None, pr_)
        B.b2sr_cc(m, labels_)
        m.close()

    # ---- device-resident timed region ----
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = str(local)
    ms_total, fam, launches, clocks = timed_steps(B, step, args, barrier, uuid)

    # ---- end to end through the C ABI with host buffers ----
    # Every step copies its CSR and input vector in from pinned host memory and
    # its results (levels, PageRank, labels, SpMV output) back out.  The copies
    # run on two copy streams with double buffers, so step i+1's input copy and
    # step i's result copy overlap step i's kernels; events order each buffer's
    # reuse.  The library runs on the default stream.
    comp = torch.cuda.current_stream()
    cin, cout = torch.cuda.Stream(), torch.cuda.Stream()
    ins_d = [tuple(torch.empty_like(t) for t in (rp, ci, x)) for _ in range(2)]
    outs_d = [(y, levels, pr, labels), tuple(torch.empty_like(t) for t in (y, levels, pr, labels))]
    outs_h = [tuple(torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in outs_d[0]) for _ in range(2)]
    h2d = sum(t.numel() * t.element_size() for t in (rp_h, ci_h, x_h))
    d2h = sum(t.numel() * t.element_size() for t in outs_h[0])
    in_ready = [torch.cuda.Event() for _ in range(2)]
    in_free = [torch.cuda.Event() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    out_free = [torch.cuda.Event() for _ in range(2)]

    def copy_in(i):
        b = i % 2
        cin.wait_event(in_free[b])        # step i-2 is done reading this buffer
        with torch.cuda.stream(cin):
            for dst, src in zip(ins_d[b], (rp_h, ci_h, x_h)):
                dst.copy_(src, non_blocking=True)
        in_ready[b].record(cin)

    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(comp)
    copy_in(0)
    for i in range(args.steps):
        b = i % 2
        if i + 1 < args.steps:
            copy_in(i + 1)
        comp.wait_event(in_ready[b])
        comp.wait_event(out_free[b])      # step i-2's results have left this buffer
        step(*ins_d[b], *outs_d[b])
        in_free[b].record(comp)
        done[b].record(comp)
        cout.wait_event(done[b])
        with torch.cuda.stream(cout):
            for dst, src in zip(outs_h[b], outs_d[b]):
                dst.copy_(src, non_blocking=True)
        out_free[b].record(cout)
    for b in range(2):
        comp.wait_event(out_free[b])
    e1.record(comp)
    e1.synchronize()
    barrier()
    e2e_ms = e0.elapsed_time(e1)

    # ---- max over ranks ----
    edges = QUERIES_PER_STEP * g.nnz
    ms_total, e2e_ms, value, e2e_value = aggregate_replicas(ms_total, e2e_ms, edges, args.steps, world, dev)
    ms_step = ms_total / args.steps
    del ins_d, outs_d, outs_h

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    peak, peak_src = measured_peak()
    roofline = roofline_of(fam, ms_total, peak, peak_src, TILE, SCHEDULE, traffic_key(PERMUTE))
    extra = {}

    # ---- extras: batched vs plain BFS, Boolean SpMV alone ----
    with B.b2sr_from_csr(g.n, rp, ci, TILE) as m:
        B.b2sr_set_schedule(m, SCHEDULE)
        for _ in range(2):
            B.b2sr_bfs_multi(m, srcs_l, levels)
            B.b2sr_bfs(m, srcs_l[0], levels[0])
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
        a.record(); B.b2sr_bfs_multi(m, srcs_l, levels); b.record(); b.synchronize()
        t_batched = a.elapsed_time(b)
        a.record()
        for i, s in enumerate(srcs_l):
            B.b2sr_bfs(m, s, levels[i])
        b.record(); b.synchronize()
        t_plain = a.elapsed_time(b)
        # Graph500-style TEPS: undirected edges with both endpoints reached (a symmetric
        # graph: every neighbour of a reached vertex is reached) over the search time
        deg = (rp[1:] - rp[:-1]).to(torch.int64)
        edges_src = [int((deg * (levels[i] >= 0)).sum().item()) // 2 for i in range(NSRC)]
        teps, teps_do = [], []
        for i, s in enumerate(srcs_l):
            a.record(); B.b2sr_bfs(m, s, levels[i]); b.record(); b.synchronize()
            teps.append(edges_src[i] / (a.elapsed_time(b) / 1e3))
            a.record(); B.b2sr_bfs_diropt(m, s, None, levels[i]); b.record(); b.synchronize()
            teps_do.append(edges_src[i] / (a.elapsed_time(b) / 1e3))
        hmean = len(teps) / sum(1.0 / t for t in teps)
        hmean_do = len(teps_do) / sum(1.0 / t for t in teps_do)
        extra["bfs_graph500_teps"] = {"sources": NSRC, "pull_harmonic_mean_gteps": hmean / 1e9,
                                      "direction_optimising_harmonic_mean_gteps": hmean_do / 1e9,
                                      "batched_gteps": sum(edges_src) / (t_batched / 1e3) / 1e9,
                                      "edges_counted": "undirected edges with both endpoints reached, per source"}
        extra["bfs_16_sources"] = {"batched_ms": t_batched, "plain_ms": t_plain,
                                   "batched_queries_per_s": NSRC / (t_batched / 1e3),
                                   "plain_queries_per_s": NSRC / (t_plain / 1e3),
                                   "speedup": t_plain / t_batched}
        B.b2sr_timing_enable(True)
        for _ in range(10):
            B.b2sr_spmv(m, B.BOOL_OR_AND, B.VEC_BITS, x, B.VEC_BITS, y)
        torch.cuda.synchronize()
        tb, nb, byb = B.b2sr_timing_read("spmv_bool")
        B.b2sr_timing_enable(False)
        B.b2sr_timing_reset()
        extra["spmv_bool"] = {"tile_dim": TILE, "kernel_us": tb / nb * 1e3, "gteps": g.nnz / (tb / nb / 1e3) / 1e9,
                              "gbs": byb / nb / (tb / nb / 1e3) / 1e9, "frac": byb / nb / (tb / nb / 1e3) / 1e9 / peak}
        # CSR -> B2SR alone: the rows as generated (column order: ranking
        # conversion) and the same CSR with its longest row reversed (radix sort)
        def convert(cd):
            B.b2sr_from_csr(g.n, rp, cd, TILE).close()
        ci_u = ci.clone()
        ilong = int(torch.argmax(rp[1:] - rp[:-1]).item())
        a0, a1 = int(rp[ilong].item()), int(rp[ilong + 1].item())
        ci_u[a0:a1] = torch.flip(ci_u[a0:a1], [0])
        extra["conversion"] = {"tile_dim": TILE, "sorted_rows_ms": _timed(lambda: convert(ci), reps=5),
                               "one_row_reversed_ms": _timed(lambda: convert(ci_u), reps=5),
                               "includes": "validation, keys in order, tiles, B2SR arrays, SpMV schedule"}
        del ci_u
        # max-times (Table 4): the SpMV alone, then MIS and colouring by rounds of local maxima
        xf = torch.from_numpy(np.random.default_rng(37).normal(size=g.n).astype(np.float32)).to(dev)
        yf = torch.empty(g.n, dtype=torch.float32, device=dev)
        B.b2sr_timing_enable(True)
        for _ in range(10):
            B.b2sr_spmv(m, B.MAX_TIMES, B.VEC_F32, xf, B.VEC_F32, yf)
        torch.cuda.synchronize()
        tm, nm, bym = B.b2sr_timing_read("spmv_max")
        B.b2sr_timing_enable(False)
        B.b2sr_timing_reset()
        prio = torch.from_numpy(np.random.default_rng(31).permutation(g.n).astype(np.float32) + 1.0).to(dev)
        ins = torch.empty(g.n, dtype=torch.int32, device=dev)
        cols = torch.empty(g.n, dtype=torch.int32, device=dev)
        t_mis = _timed(lambda: B.b2sr_mis(m, prio, ins), reps=3)
        t_col = _timed(lambda: B.b2sr_color(m, prio, cols, method=B.COLOR_PUSH), reps=3)
        t_col_mt = _timed(lambda: B.b2sr_color(m, prio, cols, method=B.COLOR_MAX_TIMES), reps=1)
        # B2SR of the transpose (Sec. III-A) and 8-bit weights as bit-planes (Sec. VII)
        t_tr = _timed(lambda: B.b2sr_transpose(m).close(), reps=3)
        wq = torch.from_numpy(np.random.default_rng(41).integers(0, 256, g.nnz).astype(np.int32)).to(dev)
        t_pl = _timed(lambda: B.b2sr_planes_from_csr(m, rp, ci, wq, 8), reps=1)
        planes = B.b2sr_planes_from_csr(m, rp, ci, wq, 8)
        yl = torch.empty(g.n, dtype=torch.int64, device=dev)
        B.b2sr_timing_enable(True)
        for _ in range(10):
            B.b2sr_spmv_planes(m, planes, 8, B.VEC_BITS, x, B.VEC_I64, yl)
            B.b2sr_spmv_planes(m, planes, 8, B.VEC_F32, xf, B.VEC_F32, yf)
        torch.cuda.synchronize()
        tpc, npc, bpc = B.b2sr_timing_read("spmv_planes_count")
        tpp, npp, bpp = B.b2sr_timing_read("spmv_planes_plus")
        B.b2sr_timing_enable(False)
        B.b2sr_timing_reset()
        del planes
        extra["transpose_and_bit_planes"] = {
            "tile_dim": TILE, "transpose_ms": t_tr, "weights": "uniform 8-bit integers (seed 41)",
            "planes_from_csr_ms": t_pl, "planes_count_us": tpc / npc * 1e3,
            "planes_count_gbs": bpc / npc / (tpc / npc / 1e3) / 1e9, "planes_plus_us": tpp / npp * 1e3,
            "planes_plus_gbs": bpp / npp / (tpp / npp / 1e3) / 1e9}
        extra["max_times_mis_colouring"] = {
            "tile_dim": TILE, "spmv_max_kernel_us": tm / nm * 1e3, "spmv_max_gbs": bym / nm / (tm / nm / 1e3) / 1e9,
            "priority": "random permutation of 1..n (seed 31)", "mis_ms": t_mis, "mis_size": int(ins.sum().item()),
            "colouring_push_ms": t_col, "colouring_max_times_rounds_ms": t_col_mt,
            "colours": int(cols.max().item()) + 1}
    del levels

    if pre is not None and "config2" in which:
        # config 2's permuted ids: the same step on the permuted graph
        pn, prp, pci = pre["perm"]
        prp_d, pci_d = torch.from_numpy(prp).to(dev), torch.from_numpy(pci).to(dev)
        psrcs = [int(v) for v in graphs_sources(pn, prp, NSRC, 7)]
        plev = torch.empty((NSRC, pn), dtype=torch.int32, device=dev)

        def pstep():
            step(prp_d, pci_d, x, y, plev, pr, labels, pn, psrcs)
        pms, pfam, _, _ = timed_steps(B, pstep, args, barrier)
        extra["step_rmat20_permuted"] = {
            "workload": f"R-MAT scale {SCALE} ef{EDGE_FACTOR} seed {SEED}, ids permuted (seed {PERM_SEED}); "
                        f"the same step, tile_dim {TILE}", "nnz": int(pci.size),
            "gteps": QUERIES_PER_STEP * int(pci.size) * args.steps / (pms / 1e3) / 1e9,
            "ms_per_step": pms / args.steps, "roofline": roofline_of(pfam, pms, peak, peak_src, TILE, SCHEDULE,
                                                                 traffic_key(PERM_SEED)),
            "kernel_breakdown_ms_per_step": {f: pfam[f]["ms"] / args.steps for f in pfam}}
        del plev
        # config 2's tile_dim sweep of the Boolean and plus-times SpMVs, unpermuted and permuted
        try:
            extra["tile_sweep"] = tile_sweep(B, dev, {"rmat20": (g.n, g.rowptr, g.colind), "rmat20_perm": (pn, prp, pci)},
                                             xbits, peak)
        except Exception as e:
            extra["tile_sweep"] = {"failed": repr(e)}
        del prp_d, pci_d
        torch.cuda.empty_cache()
        try:
            smp = np.random.default_rng(29).integers(0, g.n, 8192).astype(np.int32)
            mt, rep = B.b2sr_autotune(g.n, rp, ci, smp, B.PLUS_TIMES, B.VEC_F32, keep_ratio=0.0, trials=5)
            mt.close()
            extra["autotune_main"] = {"scheme": "plus-times fp32 (PageRank)", "choice_tile_dim": rep["tile_dim"],
                                      "choice_schedule": rep["schedule"], "trial_us": rep["trial_us"],
                                      "est_ratio": rep["est_ratio"], "used": {"tile_dim": TILE, "schedule": SCHEDULE}}
        except Exception as e:
            extra["autotune_main"] = {"failed": repr(e)}
    if pre is not None:
        for name, fn in (("serving", lambda: serving_extra(B, dev, pre["serve"], t_gen)),
                         ("tc", lambda: tc_extra(B, dev, pre["tc"])),
                         ("grid_sssp", lambda: grid_sssp_extra(B, dev, pre["grid"])),
                         ("batching", lambda: batching_extra(B, dev, pre["big"], pre["arena"],
                                                             f"{ARENA_SCALES[0]}..{ARENA_SCALES[1]} uniform, seed 23"))):
            if name not in which:
                continue
            try:
                extra[name] = fn()
            except Exception as e:  # reported, never fatal to the main line
                extra[name] = {"failed": repr(e)}
            torch.cuda.empty_cache()
        extra["graph_generation_s"] = t_gen

    cpu = None
    if not args.no_cpu_baseline:
        try:
            import oracle
            oracle.build()
            cores = host_cores()
            s_all, p_all = oracle_step(g, srcs, xbits, cores)
            s_one, p_one = oracle_step(g, srcs, xbits, 1)
            cpu = {"value": edges / s_all / 1e9, "unit": "GTEPS", "cores": cores, "kind": "oracle",
                   "nproc": os.cpu_count(),
                   "sample": (f"one whole step of the workload on the oracle (plain C) with {cores} host threads "
                              f"(CSR->B2SR and CC on one thread, SpMV and PageRank row loops on all, the BFS "
                              f"sources {cores} at a time), then the same step on one thread"),
                   "step_s": s_all, "parts_s": p_all,
                   "single_thread": {"value": edges / s_one / 1e9, "unit": "GTEPS", "cores": 1, "step_s": s_one,
                                     "parts_s": p_one}}
        except Exception as e:  # the baseline is reported, never required
            cpu = {"value": None, "unit": "GTEPS", "cores": None, "kind": "oracle", "sample": f"failed: {e}"}

    line = {
        "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8/f32", "data": "synthetic",
        "config": dict(workload_desc(g.n, g.nnz), parallelism=f"replicas x{world}"),
        "e2e": {"value": e2e_value, "unit": "GTEPS", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": e2e_ms / args.steps},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "kernel_breakdown_ms_per_step": {f: fam[f]["ms"] / args.steps for f in fam},
        "extra": extra,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def graphs_sources(n, rowptr, count, seed):
    from paper_2201_08560_gb300 import graphs
    return graphs.sources(graphs.CSR(n, rowptr, np.zeros(0, np.int32)), count, seed)


if __name__ == "__main__":
    sys.exit(main())
