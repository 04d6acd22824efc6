#!/usr/bin/env python3
"""Benchmark: one full compressive-PCA pass per step on the 10304 x 1000
workload (rank 10, 10 clusters, 5% gross errors, K = 10 graphs, 1/4 of the
rows and columns sampled, 300 FISTA iterations, PCG decoder to 1e-6).

A step runs every hot-path stage through the C ABI: the two full kNN graphs
and Laplacians, sampling + gather, the two compressed graphs, the power
iterations for lambda, 300 FISTA iterations, and the approximate decoder
(partial SVD, PCG upsampling of U and V, rank-k output X).

Prints ONE JSON line (rank 0). ``--impl reference`` times the FP64 oracle
on the host instead (bounded sample of the same workload).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cpca|reference]
Multi-GPU (torchrun): every rank runs an independent replica (the workload
is one instance; there is no data exchange), value = total FISTA iterations
of all ranks / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

# The oracle baseline is single-threaded by construction; pin BLAS threads
# before numpy loads so the reported core count is what ran.
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gen  # noqa: E402

METRIC = "wall-time to 1e-4 rel err vs plain GPU; FISTA/CG iters/s; % of HBM peak"
UNIT = "FISTA iters/s"
WORKLOAD = "bench_10304x1000"
L2_FLUSH_BYTES = 256 << 20


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# ----------------------------------------------------------- clock sampling
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------- oracle arm
def oracle_step_seconds(Y, cfg, n_query: int, dec_graphs, rng_seed: int = 0):
    """Seconds the FP64 oracle needs for one full pipeline step, measured on
    a bounded sample: the two full-graph kNN searches are timed on n_query
    sampled query points each and scaled to all points; sampling, the
    compressed graphs, the power iterations, all FISTA iterations and the
    decoder (SVD + PCG + output) run in full."""
    import oracle as O
    p, n = Y.shape
    K, J = cfg["K"], cfg["J"]
    rng = np.random.default_rng(rng_seed)
    t_knn = 0.0
    Yd = Y.astype(np.float64)
    for P in (Yd, Yd.T):
        N = P.shape[0]
        qs = rng.choice(N, size=min(n_query, N), replace=False)
        t0 = time.perf_counter()
        O.knn_bruteforce(P, K, queries=qs)
        t_knn += (time.perf_counter() - t0) * N / len(qs)
    rr, rc = int(p * cfg["fr"] + 0.5), int(n * cfg["fc"] + 0.5)
    t0 = time.perf_counter()
    # Laplacians of the full graphs: same O(N K) construction as below, timed
    # on the compressed kNN lists and scaled by the point count
    om_r, om_c = O.sample_indices(0, p, rr, 0), O.sample_indices(0, n, rc, 1)
    Yt = Yd[np.ix_(om_r, om_c)]
    Lrt, _, ir, dr, _ = O.knn_graph(Yt, K)
    Lct, _, ic, dc, _ = O.knn_graph(Yt.T, K)
    t_small = time.perf_counter() - t0
    t0 = time.perf_counter()
    O.laplacian_from_knn(ir, dr, rr, O.sigma2_mean(dr))
    t_lap = (time.perf_counter() - t0) * (p + n) / rr
    t0 = time.perf_counter()
    lam = O.fista_step(cfg["gamma_r"], cfg["gamma_c"], O.power_norm(Lrt, 200, 0, 2),
                       O.power_norm(Lct, 200, 0, 3))
    Xt, _ = O.frpcag_fista(Yt, Lrt, Lct, cfg["gamma_r"], cfg["gamma_c"], lam, J)
    t_fista = time.perf_counter() - t0
    Lr, Lc = dec_graphs
    t0 = time.perf_counter()
    O.approx_decode(Xt, om_r, om_c, p, n, Lr, Lc, tol=cfg["cg_tol"])
    t_dec = time.perf_counter() - t0
    return t_knn + t_lap + t_small + t_fista + t_dec


def decoder_graphs_for_timing(Y, K):
    """Full-size graphs for timing the oracle's decoder (setup, untimed):
    exact kNN lists from a blocked matmul ranking, then the oracle's own
    Laplacian construction. Only a timing input, never a parity input."""
    import oracle as O
    out = []
    Yd = Y.astype(np.float64)
    for P in (Yd, Yd.T):
        N = P.shape[0]
        nrm = np.einsum("ij,ij->i", P, P)
        idx = np.empty((N, K), dtype=np.int64)
        d2 = np.empty((N, K))
        for a in range(0, N, 1024):
            D = nrm[a:a + 1024, None] + nrm[None, :] - 2.0 * (P[a:a + 1024] @ P.T)
            D[np.arange(D.shape[0]), np.arange(a, a + D.shape[0])] = np.inf
            part = np.argpartition(D, K, axis=1)[:, :K]
            dd = np.take_along_axis(D, part, 1)
            o = np.argsort(dd, axis=1)
            idx[a:a + 1024] = np.take_along_axis(part, o, 1)
            d2[a:a + 1024] = np.take_along_axis(dd, o, 1)
        L, _ = O.laplacian_from_knn(idx, np.maximum(d2, 0), N, float(np.mean(np.maximum(d2, 0))))
        out.append(L)
    return out


def cpu_sample_text(nq):
    return (f"full-graph kNN brute force timed on {nq} sampled query points per graph and scaled to "
            "all points; Laplacian construction timed on the compressed graph and scaled by point "
            "count; sampling, compressed kNN graphs, power iterations, all 300 FISTA iterations and "
            "the decoder (SVD, PCG, output) in full")


def run_reference(args, cfg, Y):
    dec = decoder_graphs_for_timing(Y, cfg["K"])
    nq = 8
    for _ in range(args.warmup):
        oracle_step_seconds(Y, cfg, nq, dec)
    secs = [oracle_step_seconds(Y, cfg, nq, dec, rng_seed=s + 1) for s in range(args.steps)]
    tot = float(sum(secs))
    value = cfg["J"] * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(cfg),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": cpu_sample_text(nq)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def config_dict(cfg):
    return {"workload": f"CPCA {cfg['p']}x{cfg['n']} rank {cfg['r']}, {cfg['C']} clusters, "
                        f"{int(cfg['frac'] * 100)}% gross errors, K={cfg['K']}, sample "
                        f"{cfg['fr']}x{cfg['fc']}, {cfg['J']} FISTA iterations, PCG tol {cfg['cg_tol']}",
            "p": cfg["p"], "n": cfg["n"], "rank": cfg["r"], "K": cfg["K"],
            "rho_r": int(cfg["p"] * cfg["fr"] + 0.5), "rho_c": int(cfg["n"] * cfg["fc"] + 0.5),
            "fista_iters": cfg["J"], "gamma_r": cfg["gamma_r"], "gamma_c": cfg["gamma_c"],
            "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
            "parallelism": "replicas"}


# ------------------------------------------------------------------- GPU arm
def batched_comparison(M, torch, J=300, reps=3):
    """64 uneven instances (sizes, ranks and gamma pairs of the batched
    workload) solved to the same J FISTA iterations two ways: one batched,
    autotuned, graph-captured launch vs 64 sequential plain solves."""
    specs = gen.batched_instances(64)
    probs = []
    for sp in specs:
        Y = gen.make_instance_torch(sp["seed"], sp["p"], sp["n"], sp["r"], sp["C"], sp["frac"])
        rr, rc = M.rho_of(sp["p"], sp["fr"]), M.rho_of(sp["n"], sp["fc"])
        _, _, Yt = M.cpca_sample(sp["seed"], sp["p"], sp["n"], rr, rc, Y)
        del Y
        Lr, _, _ = M.cpca_knn_graph(Yt, sp["K"])
        Lc, _, _ = M.cpca_knn_graph(Yt, sp["K"], transposed=True)
        probs.append(dict(Yt=Yt, Lr=Lr, Lc=Lc, gamma_r=sp["gamma_r"], gamma_c=sp["gamma_c"]))
    B = M.Batch(probs)
    blocks, _ = B.tune()
    prm = M.frpcag_params(max_iter=J, blocks=blocks)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        B.solve(prm)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        B.solve(prm)
    stream = torch.cuda.current_stream()

    def timed(fn):
        best = 1e30
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        return best

    t_batched = timed(graph.replay)
    lib = M.lib()
    outs = [torch.empty_like(q["Yt"]) for q in probs]
    wss = [torch.empty(lib.cpca_frpcag_workspace_size(*q["Yt"].shape), dtype=torch.uint8,
                       device="cuda") for q in probs]

    def sequential():
        for q, X, ws in zip(probs, outs, wss):
            M.cpca_frpcag_solve(q["Yt"], q["Lr"], q["Lc"], gamma_r=q["gamma_r"],
                                gamma_c=q["gamma_c"], max_iter=J, want_info=False, out=X, ws=ws)

    t_seq = timed(sequential)
    diff = max(float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) for a, b in zip(B.X, outs))
    entries = sum(q["Yt"].shape[0] * q["Yt"].shape[1] for q in probs)
    return {"instances": len(probs), "entries": entries, "fista_iters": J,
            "batched_graph_ms": t_batched, "sequential_ms": t_seq, "speedup": t_seq / t_batched,
            "max_rel_fro_diff": diff, "autotuned_blocks": blocks}


def adjoint_comparison(M, torch, Yd, cfg, n_heldout=10000, reps=3, h=1e-3):
    """The differentiation workload: gradient of the held-out reconstruction
    loss 1/2 sum_e (X_e - Y_e)^2 (10^4 entries outside the sampled block)
    with respect to gamma_r, gamma_c, the sampled entries Y~ and the edge
    weights of all four graphs, through torch.autograd on the library's
    adjoints (FISTA reverse sweep checkpointed every 20 of 300 iterations;
    also with the whole trajectory kept), against central differences in
    gamma_r and gamma_c with four plain GPU pipeline solves (FISTA + decoder)."""
    from paper_1602_02070_gb300 import autograd as AG
    p, n = Yd.shape
    K, J = cfg["K"], cfg["J"]
    rr, rc = M.rho_of(p, cfg["fr"]), M.rho_of(n, cfg["fc"])
    Lr, _, _ = M.cpca_knn_graph(Yd, K)
    Lc, _, _ = M.cpca_knn_graph(Yd, K, transposed=True)
    om_r, om_c, Yt = M.cpca_sample(0, p, n, rr, rc, Yd)
    Lrt, _, _ = M.cpca_knn_graph(Yt, K)
    Lct, _, _ = M.cpca_knn_graph(Yt, K, transposed=True)
    hr_np, hc_np = gen.heldout_entries(7, p, n, n_heldout, om_r.cpu().numpy(), om_c.cpu().numpy())
    hr = torch.as_tensor(hr_np, device=Yd.device)
    hc = torch.as_tensor(hc_np, device=Yd.device)
    target = Yd[hr.long(), hc.long()]
    Ytc = Yt.contiguous()
    pats = {"r": Lr, "c": Lc, "rt": Lrt, "ct": Lct}
    dprm = M.decode_params(cg_tol=cfg["cg_tol"])

    def gradient(ck):
        w = {k_: G.weight.clone().requires_grad_(True) for k_, G in pats.items()}
        Y_ = Ytc.clone().requires_grad_(True)
        g_r = torch.tensor(cfg["gamma_r"], dtype=torch.float64, device=Yd.device, requires_grad=True)
        g_c = torch.tensor(cfg["gamma_c"], dtype=torch.float64, device=Yd.device, requires_grad=True)
        L = {k_: AG.laplacian(pats[k_].rowptr, pats[k_].col, w[k_]) for k_ in pats}
        Xt = AG.frpcag(Y_, g_r, g_c, L["rt"], L["ct"], Lrt, Lct, max_iter=J, power_iters=200,
                       ckpt_every=ck)
        vals = AG.decode_entries(Xt, L["r"], L["c"], Lr, Lc, om_r, om_c, p, n, hr, hc, dprm)
        loss = 0.5 * ((vals - target) ** 2).sum()
        loss.backward()
        n_grad = 2 + Y_.numel() + sum(x.numel() for x in w.values())
        return g_r.grad.item(), g_c.grad.item(), n_grad

    def fd():
        out = []
        for a, b in ((1 + h, 1.0), (1 - h, 1.0), (1.0, 1 + h), (1.0, 1 - h)):
            X, _ = M.cpca_frpcag_solve(Yt, Lrt, Lct, gamma_r=a * cfg["gamma_r"],
                                       gamma_c=b * cfg["gamma_c"], max_iter=J, want_info=False)
            dec = M.cpca_decode(X, om_r, om_c, p, n, Lr, Lc, dprm, want_X=False)
            v = M.capi.decode_entries(dec["U"], dec["V"], dec["sigma"], dec["k"], hr, hc)
            out.append(0.5 * float(((v.double() - target.double()) ** 2).sum()))
        return ((out[0] - out[1]) / (2 * h * cfg["gamma_r"]),
                (out[2] - out[3]) / (2 * h * cfg["gamma_c"]))

    def timed(fn):
        fn()
        best, res = 1e30, None
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = fn()
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        return best * 1000.0, res

    t_adj, (gr, gc, n_grad) = timed(lambda: gradient(20))
    t_all, _ = timed(lambda: gradient(J))
    t_fd, (fr, fc) = timed(fd)
    return {"heldout_entries": int(n_heldout), "fista_iters": J, "checkpoint_every": 20,
            "adjoint_ms": t_adj, "adjoint_whole_trajectory_ms": t_all,
            "fd_gamma_4_solves_ms": t_fd, "speedup_vs_fd": t_fd / t_adj,
            "gradient_entries": int(n_grad),
            "dgamma_adjoint": [gr, gc], "dgamma_fd_fp32": [fr, fc],
            "note": "wall time (host clock, synchronised) for the whole gradient; the finite "
                    "differences give the two gamma derivatives only, from FP32 losses"}


def alternate_measure(M, torch, Yd, cfg, peaks, reps=3, gamma=1.0):
    """The alternate decoder (Eq. alternatedecoder) on the full matrix of the
    workload: X~ from the step's FISTA solve, the full row/column graphs,
    gamma-bars = 1, PCG to the step's tolerance. Kernel time from the
    library's CUDA-event profile; algorithmic bytes per CG iteration: 52 per
    entry of X (phase A reads z, q, p and writes q, p; phase B reads x, r,
    p, q and writes x, r, z and its transposed copy) plus 8 per CSR entry of
    both Laplacians (column index and value)."""
    p, n = Yd.shape
    K, J = cfg["K"], cfg["J"]
    rr, rc = M.rho_of(p, cfg["fr"]), M.rho_of(n, cfg["fc"])
    Lr, _, _ = M.cpca_knn_graph(Yd, K)
    Lc, _, _ = M.cpca_knn_graph(Yd, K, transposed=True)
    om_r, om_c, Yt = M.cpca_sample(0, p, n, rr, rc, Yd)
    Lrt, _, _ = M.cpca_knn_graph(Yt, K)
    Lct, _, _ = M.cpca_knn_graph(Yt, K, transposed=True)
    Xt, _ = M.cpca_frpcag_solve(Yt, Lrt, Lct, gamma_r=cfg["gamma_r"], gamma_c=cfg["gamma_c"], max_iter=J,
                                want_info=False)
    prm = M.alt_params(gamma_r=gamma, gamma_c=gamma, tol=cfg["cg_tol"], max_iter=20000)
    ws = M.capi._workspace(M.lib().cpca_alternate_decode_workspace_size(p, n), Yd.device)
    out = torch.empty(p, n, dtype=torch.float32, device=Yd.device)
    _, info, _ = M.cpca_alternate_decode(Xt, om_r, om_c, p, n, Lr, Lc, prm, out=out, ws=ws)
    torch.cuda.synchronize()
    M.profile_enable(True, "alt_cg")
    for _ in range(reps):
        out.zero_()
        _, info, _ = M.cpca_alternate_decode(Xt, om_r, om_c, p, n, Lr, Lc, prm, out=out, ws=ws)
    torch.cuda.synchronize()
    prof = M.profile_read()
    M.profile_enable(False, "")
    ms = prof["alt_cg"][0] / reps
    iters = int(info.iters)
    byts = 52.0 * p * n + 8.0 * (Lr.nnz + Lc.nnz)
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    gbs = byts * iters / (ms / 1000.0) / 1e9
    return {"workload": f"alternate decoder on the {p}x{n} matrix, gamma-bars {gamma}, PCG to {cfg['cg_tol']}",
            "cg_iters": iters, "rel_res": float(info.rel_res), "kernel_ms": ms,
            "cg_iters_per_s": iters / (ms / 1000.0), "us_per_iter": 1000.0 * ms / max(iters, 1),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                         "bytes_per_iter": byts,
                         "peak_source": "measured" if peaks else "fallback"}}


def _event_ms(torch, fn, reps):
    """Best of reps CUDA-event times (ms) of fn on the current stream, after one
    untimed call; L2 is flushed before each timed call."""
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    res = fn()
    best = 1e30
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        res = fn()
        b.record(stream)
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best, res


def other_decoders_measure(M, torch, Yd, out, cfg, peaks, reps=3):
    """The clustering decoder (Algorithm 3) and approximate decoders 2 and 3
    (X = U U^T Y, X = Y V V^T) on the step's own outputs: X~ from FISTA, the
    full column graph, the upsampled basis of Algorithm 2. The projections
    are HBM-bound: Y is read once for the skinny product and X written once
    (8 B per entry), plus the basis."""
    p, n = Yd.shape
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    src = "measured" if peaks else "fallback"
    k = out["k"]
    res = {}
    for side, name, basis in ((0, "U U^T Y", out["U"]), (1, "Y V V^T", out["V"])):
        X = torch.empty(p, n, dtype=torch.float32, device=Yd.device)
        ws = M.capi._workspace(M.lib().cpca_subspace_project_workspace_size(p, n, basis.stride(0)), Yd.device)
        ms, _ = _event_ms(torch, lambda: M.cpca_subspace_project(side, basis, k, Yd, out=X, ws=ws), reps)
        byts = 8.0 * p * n + 4.0 * basis.shape[0] * k
        gbs = byts / (ms / 1000.0) / 1e9
        res[f"decoder_{2 + side}"] = {
            "computes": f"X = {name}, k = {k}, {p}x{n}", "ms": ms,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                         "bytes": byts, "peak_source": src}}
    C = cfg["C"]
    Xt, om_c, Lc = out["Xt"], out["omega_c"], out["Lc"]
    rr, rc = Xt.shape
    ws = M.capi._workspace(M.lib().cpca_cluster_decode_workspace_size(rr, rc, n, C, Lc.nnz), Yd.device)
    ms, dec = _event_ms(torch, lambda: M.cpca_cluster_decode(Xt, om_c, n, Lc, C, seed=1, ws=ws), reps)
    res["clustering_decoder"] = {
        "computes": f"k-means (k = {C}) on the {rc} columns of X~ ({rr}x{rc}), harmonic extension of the "
                    f"labels on the {n}-node column graph (PCG to 1e-6), row argmax",
        "ms": ms, "kmeans_steps": int(dec["info"].kmeans_steps), "cg_iters": int(dec["info"].cg_iters),
        "note": "latency-bound: every operand is L2-resident (X~ 2.6 MB); the call synchronises once "
                "after k-means to read its status"}
    return res


def kron_measure(M, torch, out, cfg, peaks, reps=3):
    """Kron-reduced compressed Laplacians (Sec. IV-A) on the step's own full
    graphs and sampled sets, then the step's FISTA (J iterations, lambda by
    power iteration) on them instead of on the kNN graphs of Y~. The reduced
    Laplacians are dense, so each FISTA iteration's products are dense
    contractions: 2 (nnz_r rc + nnz_c rr) flops on the FP32 pipes (no tensor
    cores: FP32 parity), with 8 B per stored entry and 20 B per entry of Y~."""
    Lr, Lc, om_r, om_c, Yt = out["Lr"], out["Lc"], out["omega_r"], out["omega_c"], out["Yt"]
    rr, rc = Yt.shape
    res = {}

    def reduce_both():
        a = M.cpca_kron_reduce(Lr, om_r, tol=cfg["cg_tol"])
        b = M.cpca_kron_reduce(Lc, om_c, tol=cfg["cg_tol"])
        return a, b

    ms_red, (a, b) = _event_ms(torch, reduce_both, reps)
    res["reduction"] = {"computes": f"Schur complements {Lr.n} -> {rr} rows and {Lc.n} -> {rc} columns",
                        "ms": ms_red, "pcg_launches": int(a["info"].chunks + b["info"].chunks),
                        "cg_iters_max": int(max(a["info"].cg_iters, b["info"].cg_iters)),
                        "note": "latency-bound: one synchronising PCG launch per 48 columns"}
    Lrt, Lct = a["csr"], b["csr"]
    J = cfg["J"]
    X = torch.empty_like(Yt)
    ws = M.capi._workspace(M.lib().cpca_frpcag_workspace_size(rr, rc), Yt.device)
    prm = M.frpcag_params(gamma_r=cfg["gamma_r"], gamma_c=cfg["gamma_c"], max_iter=J)
    M.cpca_frpcag_solve(Yt, Lrt, Lct, prm, want_info=False, out=X, ws=ws)
    torch.cuda.synchronize()
    M.profile_enable(True, "fista_")
    for _ in range(reps):
        M.cpca_frpcag_solve(Yt, Lrt, Lct, prm, want_info=False, out=X, ws=ws)
    torch.cuda.synchronize()
    prof = M.profile_read()
    M.profile_enable(False, "")
    kname = "fista_dense" if "fista_dense" in prof else "fista_persistent"
    ms, nl = prof.get(kname, (0.0, 0))
    ms = ms / max(nl, 1)
    flops = 2.0 * (Lrt.nnz * rc + Lct.nnz * rr)
    byts = 20.0 * rr * rc + 8.0 * (Lrt.nnz + Lct.nnz)
    tfl = flops * J / (ms / 1000.0) / 1e12
    pk = 152 * 128 * 2 * 2.07e9 / 1e12
    res["fista"] = {"computes": f"{J} FISTA iterations on {rr}x{rc} with dense reduced Laplacians "
                                f"({Lrt.nnz} + {Lct.nnz} entries)",
                    "kernel": kname, "kernel_ms": ms, "us_per_iter": 1000.0 * ms / J,
                    "roofline": {"bound": "alu", "achieved": tfl, "peak": pk, "unit": "TFLOP/s", "frac": tfl / pk,
                                 "flops_per_iter": flops, "bytes_per_iter": byts,
                                 "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"}}
    return res


def fista_large_measure(M, torch, peaks, J=300, reps=3):
    """FISTA on the sampled matrix of the 8 GB workload (Y 20000 x 100000,
    rank 20, 50 clusters, 2% gross errors, 1/10 x 1/10 sampling: Y~ 2000 x
    10000, K = 10 graphs of Y~), J iterations. The 400 MB state does not fit
    in L2, so this is the size where the kernel meets the HBM roofline:
    20 B per entry of Y~ (read Y~, S_{j-1}, S_{j-2}, write S_j and Z) plus
    8 B per CSR entry and the row pointers, per iteration."""
    cfg = gen.CONFIGS["large_20000x100000"]
    p, n, K = cfg["p"], cfg["n"], cfg["K"]
    Y = gen.make_instance_torch(0, p, n, cfg["r"], cfg["C"], cfg["frac"])
    rr, rc = M.rho_of(p, cfg["fr"]), M.rho_of(n, cfg["fc"])
    _, _, Yt = M.cpca_sample(0, p, n, rr, rc, Y)
    del Y
    torch.cuda.empty_cache()
    Lrt, _, _ = M.cpca_knn_graph(Yt, K)
    Lct, _, _ = M.cpca_knn_graph(Yt, K, transposed=True)
    X = torch.empty_like(Yt)
    ws = M.capi._workspace(M.lib().cpca_frpcag_workspace_size(rr, rc), Yt.device)
    prm = M.frpcag_params(gamma_r=cfg["gamma_r"], gamma_c=cfg["gamma_c"], max_iter=J)
    M.cpca_frpcag_solve(Yt, Lrt, Lct, prm, want_info=False, out=X, ws=ws)
    torch.cuda.synchronize()
    M.profile_enable(True, "fista_persistent")
    for _ in range(reps):
        M.cpca_frpcag_solve(Yt, Lrt, Lct, prm, want_info=False, out=X, ws=ws)
    torch.cuda.synchronize()
    prof = M.profile_read()
    M.profile_enable(False, "")
    ms, nl = prof.get("fista_persistent", (0.0, 0))
    ms = ms / max(nl, 1)
    byts = 20.0 * rr * rc + 8.0 * (Lrt.nnz + Lct.nnz) + 8.0 * (rr + rc + 2)
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    gbs = byts * J / (ms / 1000.0) / 1e9
    return {"workload": f"FISTA on Y~ {rr}x{rc} (sampled from the 20000x100000 matrix), K={K} graphs "
                        f"({Lrt.nnz} + {Lct.nnz} entries), {J} iterations",
            "kernel_ms": ms, "us_per_iter": 1000.0 * ms / J, "fista_iters_per_s": J / (ms / 1000.0),
            "roofline": {"kernel": "fista_persistent", "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                         "frac": gbs / hbm, "bytes_per_iter": byts,
                         "peak_source": "measured" if peaks else "fallback"}}


def profiled_dram_bytes(summary):
    """DRAM bytes per launch recorded in a committed ncu summary under
    profiles/ (the 'dram_bytes_per_launch:' line), or None."""
    try:
        for line in open(os.path.join(ROOT, "profiles", summary)):
            if line.startswith("dram_bytes_per_launch:"):
                return int(line.split(":")[1])
    except OSError:
        pass
    return None


def roofline_for(name, ms, launches, ctx, peaks):
    """Algorithmic work of the named kernel over the timed region / its time."""
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    src = "measured" if peaks else "fallback"
    sec = ms / 1000.0
    if name == "fista_persistent":
        byts = ctx["fista_bytes_per_iter"] * ctx["fista_iters"] * launches
        a = byts / sec / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s",
                "frac": a / hbm, "traffic": profiled_dram_bytes("fista_batch_kernel_2576x250.md"),
                "traffic_unit": "bytes per launch (ncu dram read + write)", "peak_source": src,
                "note": "20 B per entry of Y~ + CSR bytes, per FISTA iteration; the working set "
                        "(13 MB) is L2-resident at this size, so the kernel is latency-bound"}
    if name.startswith("knn_candidates"):
        fl = ctx["knn_flops_per_step"] * ctx["steps"]
        a = fl / sec / 1e12
        if name.endswith("_tc"):
            pk = (peaks["bf16_tflops"] if peaks else 1900.0) * (1.1 / 2.25)
            return {"kernel": name, "bound": "tensor", "achieved": a, "peak": pk, "unit": "TFLOP/s",
                    "frac": a / pk, "traffic": None, "peak_source": f"tf32 = {src} bf16 x 1.1/2.25"}
        pk = ctx["fp32_simt_tflops"]
        return {"kernel": name, "bound": "alu", "achieved": a, "peak": pk, "unit": "TFLOP/s",
                "frac": a / pk, "traffic": None,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"}
    if name == "cg_pcg":
        byts = ctx["cg_bytes_per_iter"] * ctx["cg_iters"] * ctx["steps"]
        a = byts / sec / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s",
                "frac": a / hbm, "traffic": None, "peak_source": src}
    if name == "decode_output":
        a = ctx["out_bytes"] * launches / sec / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s",
                "frac": a / hbm, "traffic": None, "peak_source": src}
    return {"kernel": name, "bound": "hbm", "achieved": None, "peak": hbm, "unit": "GB/s",
            "frac": None, "traffic": None, "peak_source": src}


# ------------------------------------------------------- replicas (N > 1)
def max_over_ranks(dist, values, device):
    """Each value's maximum over all ranks (the slowest replica's times);
    the values themselves when there is no process group."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def whole_job_rate(units_per_rank, world, seconds):
    """Units all replicas processed per second of the slowest replica."""
    return units_per_rank * world / seconds


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cpca", choices=["cpca", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-alternate", action="store_true")
    ap.add_argument("--cpu-queries", type=int, default=32)
    ap.add_argument("--no-large", action="store_true", help="skip FISTA on the 8 GB workload's Y~")
    ap.add_argument("--fista-large-only", action="store_true",
                    help="only FISTA on the 8 GB workload's Y~ (one JSON object; for profiling)")
    ap.add_argument("--fista-large-iters", type=int, default=300)
    ap.add_argument("--kron-only", action="store_true",
                    help="only the Kron-reduced graphs and FISTA on them (one JSON object; for profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 0)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cfg = dict(gen.CONFIGS[WORKLOAD])
    Y, _, _ = gen.make_instance(0, cfg["p"], cfg["n"], cfg["r"], cfg["C"], cfg["frac"])

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, cfg, Y)
        return

    import torch
    import paper_1602_02070_gb300 as M

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    M.lib()
    if args.fista_large_only:
        print(json.dumps(fista_large_measure(M, torch, load_peaks(), J=args.fista_large_iters, reps=1)))
        return

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    Yh = torch.from_numpy(Y).pin_memory()
    Yd = Yh.to(dev)
    if args.kron_only:
        out = M.cpca_pipeline(Yd, K=cfg["K"], fr=cfg["fr"], fc=cfg["fc"], seed=0, J=cfg["J"], cg_tol=cfg["cg_tol"])
        print(json.dumps(kron_measure(M, torch, out, cfg, load_peaks(), reps=1)))
        return
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    kw = dict(K=cfg["K"], fr=cfg["fr"], fc=cfg["fc"], seed=0, J=cfg["J"], cg_tol=cfg["cg_tol"])
    info = {}

    def step(Yin):
        return M.cpca_pipeline(Yin, **kw)

    for _ in range(args.warmup):
        out = step(Yd)
    torch.cuda.synchronize()
    # one profiled step (outside the timed region) names the dominant kernel
    M.profile_enable(True, "")
    out = step(Yd)
    prof0 = M.profile_read()
    M.profile_enable(False, "")
    dominant = max(prof0.items(), key=lambda kv: kv[1][0])[0]
    rr, rc = out["Yt"].shape
    k = out["k"]
    dinfo = out["info"]
    cg_iters = max(dinfo.cg_iters_u, dinfo.cg_iters_v)
    nnz_t = out["Lrt"].nnz + out["Lct"].nnz
    m_u, m_v = cfg["p"] - rr, cfg["n"] - rc
    ctx = {
        "steps": args.steps,
        "fista_bytes_per_iter": 20 * rr * rc + 8 * nnz_t + 8 * (rr + rc + 2),
        "fista_iters": cfg["J"],
        "knn_flops_per_step": 2.0 * (cfg["p"] ** 2 * cfg["n"] + cfg["n"] ** 2 * cfg["p"]
                                     + rr ** 2 * rc + rc ** 2 * rr),
        "fp32_simt_tflops": 152 * 128 * 2 * 2.07e9 / 1e12,
        "cg_bytes_per_iter": 44 * (m_u + m_v) * k + 8 * (out["Lr"].nnz + out["Lc"].nnz),
        "cg_iters": cg_iters,
        "out_bytes": 4 * cfg["p"] * cfg["n"],
    }

    # ---------------- timed region: device-resident input
    clocks = ClockSampler(local)
    clocks.start()
    M.profile_enable(True, dominant)
    launches0 = M.launch_count()
    barrier()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    t_wall0 = time.perf_counter()
    for s in range(args.steps):
        flush.zero_()
        ev[s][0].record(stream)
        out = step(Yd)
        ev[s][1].record(stream)
    barrier()
    t_wall = time.perf_counter() - t_wall0
    gpu_launches = M.launch_count() - launches0
    prof = M.profile_read()
    M.profile_enable(False, "")
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1000.0
    clk = clocks.stop()

    # ---------------- end to end: pinned host input, result read back
    Xh = torch.empty(cfg["p"], cfg["n"], dtype=torch.float32).pin_memory()
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier()
    for s in range(args.steps):
        flush.zero_()
        ev2[s][0].record(stream)
        Yin = Yh.to(dev, non_blocking=True)
        o = step(Yin)
        Xh.copy_(o["X"], non_blocking=True)
        ev2[s][1].record(stream)
    barrier()
    e2e_s = sum(a.elapsed_time(b) for a, b in ev2) / 1000.0

    total_s, e2e_s = max_over_ranks(dist, [total_s, e2e_s], dev)
    units = cfg["J"] * args.steps * world
    value = whole_job_rate(cfg["J"] * args.steps, world, total_s)
    peaks = load_peaks()
    dom_ms, dom_n = prof.get(dominant, (0.0, 0))
    roof = roofline_for(dominant, dom_ms, dom_n, ctx, peaks) if dom_n else None
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": config_dict(cfg),
        "e2e": {"value": units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(Yh.numel() * 4),
                "d2h_bytes_per_step": int(Xh.numel() * 4)},
        "gpu_launches": int(gpu_launches),
        "roofline": roof,
        "clocks": clk,
        "phases_ms_one_step": {k_: round(v[0], 4) for k_, v in sorted(prof0.items(), key=lambda kv: -kv[1][0])},
        "fista_iters_per_step": cfg["J"], "cg_iters_per_step": cg_iters, "rank_k": k,
        "wall_s_timed": t_wall,
    }
    if not args.no_batched:
        line["batched_64"] = batched_comparison(M, torch)
    if not args.no_adjoint:
        line["adjoint"] = adjoint_comparison(M, torch, Yd, cfg)
    if not args.no_alternate:
        line["alternate_decoder"] = alternate_measure(M, torch, Yd, cfg, peaks)
        line["other_decoders"] = other_decoders_measure(M, torch, Yd, out, cfg, peaks)
        line["kron_graphs"] = kron_measure(M, torch, out, cfg, peaks)
    if not args.no_large:
        line["fista_8gb_workload"] = fista_large_measure(M, torch, peaks)
    if world == 1 and not args.no_cpu_baseline:
        dec = decoder_graphs_for_timing(Y, cfg["K"])
        secs = oracle_step_seconds(Y, cfg, args.cpu_queries, dec)
        line["cpu_baseline"] = {"value": cfg["J"] / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": cpu_sample_text(args.cpu_queries),
                                "seconds_per_step_extrapolated": secs}
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
