"""Benchmark: codon-constrained inside+outside DP on one synthetic 300-aa protein.

One step = the whole hot path on the 900-nt workload: inside (log Z) and the
adjoint outside (pair probabilities, codon marginals, codon-pair gradients)
in binary32 with per-diagonal power-of-two scaling.  The binary64 form, the
accuracy of the binary32 form against it, sampling throughput, an end-to-end
number through the public API with host buffers, the roofline of the
dominant kernel and the CPU oracle are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank runs its own replica (a single protein does not
shard): whole-job throughput = ranks x cells / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

import synth  # noqa: E402

METRIC = "DP cells/s & proteins/s (inside+outside) vs plain FP64 GPU at |ΔlogZ|≤1e-6"
WORKLOAD = "p300_dirichlet"
NS = 6


def codon_counts(res):
    per_aa = [4, 6, 2, 2, 2, 2, 2, 4, 2, 3, 6, 2, 1, 2, 4, 6, 4, 1, 2, 4]  # ARNDCQEGHILKMFPSTWYV
    return np.repeat(np.array([per_aa[int(r)] for r in res], dtype=np.int64), 3)


def state_cells(res):
    """sum over cells (i <= j) of M_i M_j: the codon-state entries of one table."""
    M = codon_counts(res).astype(np.float64)
    tot = np.sum(M) ** 2
    return float((tot + np.sum(M * M)) / 2)


def algorithmic_flops(res):
    """Analytic count of the inside and outside floating-point operations of
    the recursions in their documented contraction order (2 per FMA), from
    the protein's actual codon-state counts M_p."""
    M = codon_counts(res).astype(np.float64)
    n = M.size
    inside = 0.0
    # bifurcation: sum over cells (x,y) and split points k of Mx*Mk*My
    Mc = np.concatenate([[0.0], np.cumsum(M)])
    for x in range(n):
        ys = np.arange(x + 9, n)
        if ys.size == 0:
            continue
        # sum_{k=x+5}^{y-4} M_k for each y
        sk = Mc[ys - 3] - Mc[x + 5]
        inside += np.sum(M[x] * sk * M[ys])
    # per-cell local work: chain, XI, 29 interior partial sums, 60 bulges,
    # QB (transfers + stack + 4 multiloop products), 5 derived tables
    local = 0.0
    for d in range(1, n):
        x = np.arange(0, n - d)
        mx, my = M[x], M[x + d]
        m1 = M[x + 1]
        L_int = max(0, min(30, d - 4) - 1)
        L_bul = 2 * max(0, min(30, d - 4))
        cell = mx * m1 * my  # chain
        cell += (2 * mx * m1 * my) * (d >= 6) + L_int * 2 * mx * m1 * my
        cell += L_bul * mx * m1 * my
        cell += (4 + 8) * mx * m1 * my * (d >= 4) + 10 * mx * m1 * my * (d >= 5)
        local += np.sum(cell)
    inside = 2.0 * (inside + local)
    # the adjoint runs two transposed bifurcations (hG along rows, hQB along
    # columns) and the reverse of each local statement, which reads two
    # operands per forward product: twice the inside count
    outside = 2.0 * inside
    return inside, outside




def bf16_peak_tflops():
    """Measured dense BF16 burst throughput of the B300s (cuBLAS),
    else the recipe's fallback."""
    try:
        return float(json.loads((ROOT / "MEASURED_PEAKS.json").read_text())["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1800.0


def sm_peak_tflops(clock_mhz, sms=148):
    return sms * 128 * 2 * clock_mhz * 1e6 / 1e12


class Clocks:
    """nvidia-smi sampling while the timed region runs."""

    def __init__(self):
        self.rows, self.proc = [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, device=0):
        rows = [r for r in self.rows if r and r[0] == str(device)] or self.rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if len(r) > 5 + k and r[5 + k] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(backend="nccl"):
    """Rank layout from the torchrun environment; a process group for N > 1
    (NCCL on the GPU machine; the tests use gloo on CPU)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend, init_method="env://")
    return ws, rank, local


def barrier(ws, cuda=True):
    if ws > 1:
        import torch
        import torch.distributed as dist
        dist.barrier()
        if cuda:
            torch.cuda.synchronize()


def max_over_ranks(v, ws, device="cuda"):
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_rate(res, lw, pb, budget_m=60):
    """The oracle as it stands on a prefix of the workload (bounded CPU time)."""
    import oracle
    sub = res[:budget_m]
    n = 3 * len(sub)
    t = time.time()
    oracle.outside(synth.nn_params(0), sub, None if lw is None else lw[:budget_m], pb)
    dt = time.time() - t
    cells = n * (n + 1) / 2
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": cells / dt, "unit": "cells/s", "cores": threads, "kind": "oracle",
            "sample": f"PREFIX FIGURE: inside+outside of the first {len(sub)} residues ({n} nt) of the 300-aa "
                      f"workload, {dt:.1f} s; inside OpenMP over the cells of a diagonal, outside single-threaded. "
                      "The oracle's cost per cell grows with n, so this overstates its rate on the full 900 nt"}


def run_reference(args):
    ws, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return
    res, lw, pb = synth.workload(WORKLOAD)
    import oracle
    m = 40
    sub = res[:m]
    n = 3 * m
    params = synth.nn_params(0)
    for _ in range(args.warmup):
        oracle.outside(params, sub, lw, pb)
    t = time.time()
    for _ in range(args.steps):
        oracle.outside(params, sub, lw, pb)
    dt = time.time() - t
    cells = n * (n + 1) / 2
    val = args.steps * cells / dt
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "cells/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f80",
           "data": "synthetic",
           "config": {"workload": f"{WORKLOAD} (first {m} of 300 residues per step: bounded CPU sample)"},
           "cpu_baseline": {"value": val, "unit": "cells/s", "cores": threads, "kind": "oracle",
                            "sample": f"oracle inside+outside on the first {m} residues ({n} nt) per step"},
           "e2e": {"value": val, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def bench_windows(stream):
    """Batched fixed-sequence DP: the 200,000-window labelling batch."""
    from paper_2604_19718_b300 import screen
    ex = screen.Windows(synth.nn_params(0), stream=stream)
    res, slots, bases, off = synth.windows(200_000, seed=3)
    ex.logz(bases[:off[64]], off[:65])  # warm-up
    t = time.perf_counter()
    G = ex.free_energy(bases, off)
    wall = time.perf_counter() - t
    ms = ex.last_ms()
    n = np.diff(off).astype(np.float64)
    cells = float(np.sum(n * (n + 1) / 2))
    out = {"windows": len(n), "kernel_ms": ms, "windows_per_s": len(n) / (ms * 1e-3),
           "cells_per_s": cells / (ms * 1e-3),
           "e2e_windows_per_s": len(n) / wall, "lengths_nt": [int(n.min()), int(n.max())]}
    return out, ex, (res, slots, bases, off, G)


def bench_surrogate(ex, data, stream):
    """Surrogate training on the exact labels, prediction throughput and the
    design gain of surrogate pre-screening over the DP-only method."""
    import paper_2604_19718_b300 as cf
    from paper_2604_19718_b300 import screen
    res, slots, bases, off, G = data
    nw = len(res)
    tr, held = np.arange(nw - 2000), np.arange(nw - 2000, nw)
    b_tr, o_tr = screen.gather(bases, off, tr)
    sur = cf.Surrogate(synth.surrogate_init(0), stream=stream, max_batch=256)
    t = time.perf_counter()
    hist = screen.train(sur, b_tr, o_tr, G[tr], epochs=6, batch=256, lr=1e-3)
    train_s = time.perf_counter() - t
    b_h, o_h = screen.gather(bases, off, held)
    big = cf.Surrogate(sur.params(), stream=stream, max_batch=4096)
    # prediction throughput on the whole 200,000-window batch, both paths
    b_all, o_all = bases, off
    import torch
    paths, resident = {}, {}
    b_dev, o_dev = torch.tensor(b_all, device="cuda"), torch.tensor(o_all, device="cuda")
    g_dev = torch.empty(len(o_all) - 1, dtype=torch.float32, device="cuda")
    for path, key in ((0, "cuda_cores"), (1, "tensor_cores")):
        cf.cf_surrogate_set_path(big.h, path)
        big.predict(b_all[:o_all[4096]], o_all[:4097])
        p_all = big.predict(b_all, o_all)
        ms_all = cf.cf_surrogate_last_ms(big.h)
        paths[key] = {"ms": ms_all, "windows_per_s": (len(o_all) - 1) / (ms_all * 1e-3), "pred": p_all}
        # the same batch with the windows already resident in device memory
        cf.cf_surrogate_predict(big.h, b_dev, o_dev, g_dev)
        ms_r = []
        for _ in range(3):
            cf.cf_surrogate_predict(big.h, b_dev, o_dev, g_dev)
            ms_r.append(cf.cf_surrogate_last_ms(big.h))
        resident[key] = min(ms_r)
    n_all = np.diff(o_all).astype(np.float64)
    flops_all = float(np.sum(2 * 64 * (4 + 3 * 64) * 5 * n_all)) + float(np.sum(2 * 64 * n_all))
    tc_vs_cc = float(np.max(np.abs(paths["tensor_cores"]["pred"] - paths["cuda_cores"]["pred"])
                            / np.maximum(1.0, np.abs(paths["cuda_cores"]["pred"]))))
    cf.cf_surrogate_set_path(big.h, 1)
    big.predict(b_h, o_h)
    pred = big.predict(b_h, o_h)
    pred_ms = cf.cf_surrogate_last_ms(big.h)
    n_h = np.diff(o_h)
    base = n_h * np.mean(G[tr] / np.diff(off)[tr])
    mse, mse_b = float(np.mean((pred - G[held]) ** 2)), float(np.mean((base - G[held]) ** 2))
    flops_fwd = float(np.sum(2 * 64 * (4 + 3 * 64) * 5 * n_h)) + float(np.sum(2 * 64 * n_h))
    rng = np.random.default_rng(11)
    g_eval, g_time, ks = [], [], []
    for w in held[:16]:
        cands = screen.uniform_candidates(res[w], 1024, rng)
        s = screen.prescreen(big, ex, res[w], cands, top=32)
        t_s = s["seconds"]
        d_all = screen.dp_only(ex, res[w], cands)
        per = d_all["seconds"] / len(cands)
        k = max(1, min(len(cands), int(t_s / per)))
        d32 = screen.dp_only(ex, res[w], cands[:32])
        dk = screen.dp_only(ex, res[w], cands[:k])
        g_eval.append(d32["best_G"] - s["best_G"])
        g_time.append(dk["best_G"] - s["best_G"])
        ks.append(k)
    sur.close()
    big.close()
    return {"train_windows": len(tr), "epochs": 6, "train_s": train_s,
            "train_windows_per_s": 6 * len(tr) / train_s, "loss_per_epoch": [round(h, 6) for h in hist],
            "heldout_mse_kcal2": mse, "length_only_mse_kcal2": mse_b,
            "predict_windows_per_s": len(held) / (pred_ms * 1e-3),
            "predict_tflops": flops_fwd / (pred_ms * 1e-3) / 1e12,
            "predict_all_200k": {k: {"ms": v["ms"], "windows_per_s": v["windows_per_s"],
                                     "tflops": flops_all / (v["ms"] * 1e-3) / 1e12} for k, v in paths.items()},
            "predict_all_200k_resident": {
                k: {"ms": ms, "windows_per_s": (len(o_all) - 1) / (ms * 1e-3),
                    "tflops": flops_all / (ms * 1e-3) / 1e12,
                    # the tensor cores multiply both BF16 parts of each activation: twice the counted MMA work
                    "frac_of_measured_bf16_peak": (flops_all / (ms * 1e-3) / 1e12) / bf16_peak_tflops()}
                for k, ms in resident.items()},
            "predict_tensor_vs_cuda_cores_max_rel": tc_vs_cc,
            "prescreen": {"windows": 16, "candidates": 1024, "top": 32, "candidates_kind": "uniform codons",
                          "gain_kcal_equal_exact_evals": float(np.mean(g_eval)),
                          "gain_kcal_equal_wall_time": float(np.mean(g_time)),
                          "dp_only_candidates_at_equal_time": float(np.mean(ks))}}


def bench_adjoint(stream):
    """Autograd form on the 300-aa soft-weighted protein and 50 ascent steps."""
    import torch

    import paper_2604_19718_b300 as cf
    from paper_2604_19718_b300 import adjoint
    res, lw, pb = synth.workload("p300_weighted")
    f = cf.CodonFold(synth.nn_params(0), stream=stream)
    f.set_protein(res)
    lw_t = torch.tensor(lw, device="cuda", requires_grad=True)
    pb_t = torch.tensor(pb, device="cuda", requires_grad=True)
    for _ in range(2):
        adjoint.LogZ.apply(lw_t, pb_t, f, cf.CF_FP32_SCALED).backward()
    torch.cuda.synchronize()
    t = time.perf_counter()
    k = 5
    for _ in range(k):
        adjoint.LogZ.apply(lw_t, pb_t, f, cf.CF_FP32_SCALED).backward()
    torch.cuda.synchronize()
    step_s = (time.perf_counter() - t) / k
    aa = synth.to_string(res)
    fstar = adjoint.frequency_targets(aa, synth.ascent_targets(300))
    # one untimed step first: torch loads its own kernels on their first use
    adjoint.weight_ascent(f, aa, fstar, steps=1, lw0=lw, pb=pb, device="cuda")
    torch.cuda.synchronize()
    t = time.perf_counter()
    _, hist = adjoint.weight_ascent(f, aa, fstar, steps=50, lw0=lw, pb=pb, device="cuda")
    asc_s = time.perf_counter() - t
    f.close()
    return {"workload": "p300_weighted (lw ~ N(0,0.5), pb ~ N(0,0.2))", "forward_backward_ms": 1e3 * step_s,
            "ascent_steps": 50, "ascent_s": asc_s, "max_gap_first": hist[0]["max_gap"],
            "max_gap_last": hist[-1]["max_gap"]}


def bench_small_batch(nstreams=32, count=4096):
    """Proteins/s on the 4,096-protein batch of 8-residue (24-nt) proteins,
    inside + outside (pair probabilities and codon marginals) per protein,
    in the binary64 and binary32 forms.  Batched: the whole batch in one
    launch per kernel (cf_batch_*), timed on the device and end to end
    (proteins uploaded from a (count, 8) residue-index array, pair
    probabilities and codon marginals copied back into the caller's pinned
    host arrays, reused from run to run).  Per problem, for comparison:
    each worker thread with its own problem on its own stream (a new protein
    of the same length reuses the problem's tables and graphs)."""
    import torch

    import paper_2604_19718_b300 as cf
    prots = synth.batch_p8(count)
    params = synth.nn_params(0)
    out = {"proteins": count, "nt": 24, "streams": nstreams}
    idx = np.asarray(prots)
    Ph = torch.empty((count, 24, 24), dtype=torch.float32, pin_memory=True)
    cmh = torch.empty((count, 8, 6), dtype=torch.float64, pin_memory=True)
    for prec, key in ((cf.CF_FP64, "fp64"), (cf.CF_FP32_SCALED, "fp32")):
        b = cf.Batch(params, count, 8, prec)
        b.set_proteins(idx)
        b.run(Ph.numpy(), cmh.numpy())  # warm-up: graphs
        t = time.perf_counter()
        b.set_proteins(idx)
        lz, P, cm = b.run(Ph.numpy(), cmh.numpy())
        wall = time.perf_counter() - t
        ms = b.last_ms()
        b.close()
        out[key + "_batched_proteins_per_s"] = count / (ms * 1e-3)
        out[key + "_batched_e2e_proteins_per_s"] = count / wall
        out[key + "_batched_logZ_first"] = float(lz[0])
    streams = [torch.cuda.Stream() for _ in range(nstreams)]
    folds = [cf.CodonFold(params, stream=s.cuda_stream) for s in streams]
    for prec, key in ((cf.CF_FP64, "fp64"), (cf.CF_FP32_SCALED, "fp32")):
        lz = np.zeros(count)

        def work(k):
            f = folds[k]
            for i in range(k, count, nstreams):
                f.set_protein(prots[i])
                lz[i] = f.inside(prec)
                f.outside(True, True, False)

        for k in range(nstreams):  # warm-up: tables and graphs of every problem
            folds[k].set_protein(prots[k])
            folds[k].inside(prec)
            folds[k].outside(True, True, False)
        torch.cuda.synchronize()
        t = time.perf_counter()
        threads = [threading.Thread(target=work, args=(k,)) for k in range(nstreams)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        out[key + "_per_problem_proteins_per_s"] = count / dt
        out[key + "_per_problem_logZ_first"] = float(lz[0])
    for f in folds:
        f.close()
    return out


def bench_concurrent(nprob=4, rounds=5):
    """Proteins/s of the 900-nt workload with nprob independent problems at
    once, each on its own stream and worker thread (one protein is a
    latency-bound wavefront that leaves most SMs idle on its long diagonals)."""
    import torch

    import paper_2604_19718_b300 as cf
    res, _, _ = synth.workload(WORKLOAD)
    params = synth.nn_params(0)
    streams = [torch.cuda.Stream() for _ in range(nprob)]
    folds = [cf.CodonFold(params, stream=s.cuda_stream) for s in streams]
    n = 3 * len(res)
    lz = np.zeros(nprob)
    for k, f in enumerate(folds):  # warm-up: tables and graphs of every problem
        f.set_protein(res)
        f.inside(cf.CF_FP32_SCALED)
        f.outside(True, True, False)

    def work(k):
        f = folds[k]
        for _ in range(rounds):
            lz[k] = f.inside(cf.CF_FP32_SCALED)
            f.outside(True, True, False)

    torch.cuda.synchronize()
    t = time.perf_counter()
    threads = [threading.Thread(target=work, args=(k,)) for k in range(nprob)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    for f in folds:
        f.close()
    return {"problems": nprob, "rounds": rounds, "nt": n, "proteins_per_s": nprob * rounds / dt,
            "cells_per_s": nprob * rounds * n * (n + 1) / 2 / dt, "logZ_equal": bool(np.all(lz == lz[0]))}


def bench_mfe(stream):
    """Minimum free energy (min-sum recursions on exact integer costs) with
    traceback, on the 300-aa soft-weighted protein and the 1000-aa protein."""
    import paper_2604_19718_b300 as cf
    out = {}
    for name in ("p300_weighted", "p1000_weighted"):
        res, lw, pb = synth.workload(name)
        f = cf.CodonFold(synth.nn_params(0), stream=stream)
        f.set_protein(res, lw, pb)
        f.mfe()  # warm-up: tables and graph
        q, kc, cod, par = f.mfe()
        ms_tb = cf.cf_mfe_last_ms(f.prob)
        cf.cf_mfe(f.prob)
        ms = cf.cf_mfe_last_ms(f.prob)
        n = 3 * len(res)
        f.close()
        out[name] = {"mfe_kcal": kc, "ms": ms, "ms_with_traceback": ms_tb,
                     "cells_per_s": n * (n + 1) / 2 / (ms * 1e-3), "pairs": int((par >= 0).sum() // 2)}
    return out


def bench_subopt(stream):
    """Every configuration within a gap of the minimum free energy (cf_subopt:
    min-sum tables, then a depth-first search on the device), on the 300-aa
    soft-weighted protein, at most 10,000 outputs per call."""
    import paper_2604_19718_b300 as cf
    res, lw, pb = synth.workload("p300_weighted")
    f = cf.CodonFold(synth.nn_params(0), stream=stream)
    f.set_protein(res, lw, pb)
    f.subopt(0.0, 10)  # warm-up: tables
    cf.cf_mfe(f.prob)
    ms_tables = cf.cf_mfe_last_ms(f.prob)
    out = {"workload": "p300_weighted: 300 aa / 900 nt, lw ~ N(0,0.5), pb ~ N(0,0.2)", "ms_tables": ms_tables}
    for gap in (0.5, 2.0):
        cnt, cost, _, _ = f.subopt(gap, 10_000)
        ms = cf.cf_mfe_last_ms(f.prob)
        k = min(cnt, 10_000)
        out[f"gap_{gap}"] = {"count": cnt, "truncated": cnt > 10_000, "ms": ms, "steps": cf.cf_subopt_steps(f.prob),
                             "configs_per_s": k / max(ms - ms_tables, 1e-3) * 1e3,
                             "cost_span_kcal": float((cost.max() - cost.min()) / 2**32) if k else 0.0}
    f.close()
    return out


def bench_frequency(stream):
    """Frequency matching with Anderson mixing on the 900-nt workload: per-codon
    target bonuses exp(N(0,1)) (seed 3), r_tol = 0.002, binary32."""
    import paper_2604_19718_b300 as cf
    from paper_2604_19718_b300 import frequency as fq
    res, _, _ = synth.workload(WORKLOAD)
    aa = synth.to_string(res)
    fstar = np.exp(np.random.default_rng(3).normal(0.0, 1.0, 61))
    f = cf.CodonFold(synth.nn_params(0), stream=stream)
    f.set_protein(res)
    fq.fold_marginals(f)(np.zeros((len(res), 6)))  # warm-up: tables and graphs
    t = time.perf_counter()
    x, hist = fq.match_frequencies(fq.fold_marginals(f), aa, fstar, rtol=0.002, depth=5)
    dt = time.perf_counter() - t
    f.close()
    return {"evaluations": len(hist), "seconds": dt, "max_log_ratio_first": hist[0], "max_log_ratio_last": hist[-1],
            "r_tol": 0.002, "anderson_depth": 5}


def tm_flops(states, gamma):
    """Algorithmic flops of the tensor-model recursion (2 per FMA) with the
    protein's actual block sides gamma * M_p (M_p = states[p], the states of
    position p in the layout used): per cell [i, j+1) the unpaired
    extension Q[i, j] X_j and one block product per split point k = i..j-4,
    per pair (k, j) the two transfer products of the fold and its traces."""
    M = np.asarray(states, dtype=np.float64) * gamma
    n = M.size
    C = np.concatenate([[0.0], np.cumsum(M)])  # C[q] = sum of M[0..q-1]
    tot = 0.0
    for i in range(n):
        j = np.arange(i + 1, n)
        tot += 2 * np.sum(M[i] * M[j - 1] * M[j])
        j = np.arange(i + 4, n)  # split points: k = i (side M[i]) and k = i+1..j-4
        tot += 2 * np.sum(M[i] * M[j] * (M[i] + C[j - 3] - C[i + 1]))
    for k in range(n - 4):
        j = np.arange(k + 4, n)
        tot += np.sum(2 * (M[k] * M[k + 1] * M[j - 1] + M[k] * M[j - 1] * M[j]) + 4 * M[k] * M[j] * gamma)
    return float(tot)


def bench_tm(stream):
    """The paper's tensor-based model (synthetic gamma 4, two pair
    conformations, renormalised) under the codon constraints of the first
    100 and 300 residues of the 900-nt workload, both precisions."""
    import paper_2604_19718_b300 as cf
    V, B, S = synth.tm_params(0, 4, 2)
    model = cf.TensorModel(V, B, S)
    res_all, _, _ = synth.workload(WORKLOAD)
    out = {"model": "synthetic tensor model (seed 0): gamma 4, 2 pair conformations, spectral-radius renormalised",
           "workload": f"{WORKLOAD} prefixes, no codon weights"}
    for m in (100, 300):
        res = res_all[:m]
        f = cf.CodonFold(synth.nn_params(0), stream=stream)
        f.set_protein(res)
        f.tm_inside(model, cf.CF_FP32_SCALED)  # warm-up: tables and graph
        l32 = f.tm_inside(model, cf.CF_FP32_SCALED)
        ms32 = cf.cf_tm_last_ms(f.prob)
        f.tm_inside(model, cf.CF_FP64)
        l64 = f.tm_inside(model, cf.CF_FP64)
        ms64 = cf.cf_tm_last_ms(f.prob)
        f.close()
        n = 3 * m
        cells = n * (n + 1) / 2
        fl = tm_flops(codon_counts(res), 4)
        out[f"m{m}"] = {"nt": n, "fp32_ms": ms32, "fp64_ms": ms64, "cells_per_s_fp32": cells / (ms32 * 1e-3),
                        "algorithmic_tflops_fp32": fl / (ms32 * 1e-3) / 1e12,
                        "abs_dlogZ_fp32_vs_fp64": abs(l32 - l64), "rel_dlogZ": abs(l32 - l64) / abs(l64),
                        "logZ": l64}
    # the 900-nt prefix in the single-codon layout (paper Eq. single-tt)
    res = res_all[:300]
    f = cf.CodonFold(synth.nn_params(0), stream=stream)
    cf.cf_set_layout(f.prob, 1)
    f.set_protein(res)
    f.tm_inside(model, cf.CF_FP32_SCALED)
    l32 = f.tm_inside(model, cf.CF_FP32_SCALED)
    ms32 = cf.cf_tm_last_ms(f.prob)
    f.tm_inside(model, cf.CF_FP64)
    l64 = f.tm_inside(model, cf.CF_FP64)
    ms64 = cf.cf_tm_last_ms(f.prob)
    _, st = cf.cf_layout_states(f.prob, f.n)
    f.close()
    fl = tm_flops(st, 4)
    out["m300_single_codon"] = {"nt": 900, "states_per_position": float(np.mean(st)), "fp32_ms": ms32, "fp64_ms": ms64,
                                "algorithmic_tflops_fp32": fl / (ms32 * 1e-3) / 1e12,
                                "abs_dlogZ_vs_codon_states": abs(l64 - out["m300"]["logZ"]),
                                "abs_dlogZ_fp32_vs_fp64": abs(l32 - l64)}
    model.close()
    return out


def bench_layout(stream, steps=10):
    """The 900-nt step (binary32 inside + outside) in the single-codon layout
    (paper Eq. single-tt; the workload has no codon-pair bonuses), against
    the codon-state layout on the same GPU."""
    import torch

    import paper_2604_19718_b300 as cf
    res, lw, pb = synth.workload(WORKLOAD)
    out = {}
    for layout, key in ((0, "codon_states"), (1, "single_codon")):
        f = cf.CodonFold(synth.nn_params(0), stream=stream)
        cf.cf_set_layout(f.prob, layout)
        f.set_protein(res, lw, pb)
        for _ in range(3):
            lz = f.inside(cf.CF_FP32_SCALED)
            f.outside(False, True, False)
        tin = tout = 0.0
        for _ in range(steps):
            lz = f.inside(cf.CF_FP32_SCALED)
            f.outside(False, True, False)
            a, b, _, _ = f.timing()
            tin, tout = tin + a, tout + b
        _, st = cf.cf_layout_states(f.prob, f.n)
        f.sample(1000, 3)  # warm-up
        torch.cuda.synchronize()
        t = time.perf_counter()
        f.sample(10_000, 7)
        torch.cuda.synchronize()
        sps = 10_000 / (time.perf_counter() - t)
        f.mfe()  # warm-up: tables and graph
        f.mfe()
        mfe_ms = cf.cf_mfe_last_ms(f.prob)
        f.close()
        out[key] = {"inside_ms": tin / steps, "outside_ms": tout / steps, "ms_per_step": (tin + tout) / steps,
                    "mean_states_per_position": float(np.mean(st)), "logZ": lz, "samples_per_s": sps,
                    "mfe_ms_with_traceback": mfe_ms}
    torch.cuda.synchronize()
    out["speedup"] = out["codon_states"]["ms_per_step"] / out["single_codon"]["ms_per_step"]
    return out


def bench_large(stream, nsamples=10_000):
    """The 1000-aa / 3000-nt soft-weighted protein in binary32."""
    import paper_2604_19718_b300 as cf
    res, lw, pb = synth.workload("p1000_weighted")
    f = cf.CodonFold(synth.nn_params(0), stream=stream)
    f.set_protein(res, lw, pb)
    f.inside(cf.CF_FP32_SCALED)
    f.outside(False, True, False)
    lz = f.inside(cf.CF_FP32_SCALED)
    f.outside(False, True, False)
    tin, tout, lin, lout = f.timing()
    t = time.perf_counter()
    f.sample(nsamples, 7)
    ts = time.perf_counter() - t
    f.close()
    n = 3000
    cells = n * (n + 1) / 2
    return {"workload": "p1000_weighted: 1000 aa / 3000 nt, Dirichlet(1) (seed 4), lw ~ N(0,0.5)",
            "logZ": lz, "inside_ms": tin, "outside_ms": tout, "cells_per_s": cells / ((tin + tout) * 1e-3),
            "samples": nsamples, "samples_per_s": nsamples / ts, "launches": lin + lout}


def profile_form(form, steps, m=0):
    """One form on a small case, repeated `steps` times (profiler captures)."""
    import torch

    import paper_2604_19718_b300 as cf
    from paper_2604_19718_b300 import screen
    params = synth.nn_params(0)
    out = {"profile_form": form}
    if form == "surrogate":  # 4,096 windows: one batch of the tensor-core prediction path
        _, _, bases, off = synth.windows(4096, seed=3)
        sur = cf.Surrogate(synth.surrogate_init(0), max_batch=4096)
        for _ in range(steps):
            sur.predict(bases, off)
        out["ms"] = cf.cf_surrogate_last_ms(sur.h)
        sur.close()
    elif form == "surrogate_train":  # training steps on one batch of 4,096 windows (own forward and backward kernels)
        _, _, bases, off = synth.windows(4096, seed=3)
        G = np.random.default_rng(3).normal(0.0, 1.0, 4096).astype(np.float32)
        sur = cf.Surrogate(synth.surrogate_init(0), max_batch=4096)
        for _ in range(steps):
            out["loss"] = sur.train_step(bases, off, G, 1e-3)
        out["ms"] = cf.cf_surrogate_last_ms(sur.h)
        sur.close()
    elif form in ("mfe", "sample", "checkpoint"):
        res, lw, pb = synth.workload("p300_weighted")
        f = cf.CodonFold(params)
        if form == "checkpoint":
            cf.cf_set_checkpoint(f.prob, 1)
        f.set_protein(res, lw, pb)
        for _ in range(steps):
            if form == "mfe":
                f.mfe()
                out["ms"] = cf.cf_mfe_last_ms(f.prob)
            elif form == "sample":
                f.inside(cf.CF_FP32_SCALED)
                f.sample(10000, 2)
            else:
                f.inside(cf.CF_FP32_SCALED)
                f.outside(False, True, False)
                out["ms"] = f.timing()[:2]
        f.close()
    elif form == "tm":  # the tensor-model pass on the first 100 residues (300 nt), or the first m
        V, B, S = synth.tm_params(0, 4, 2)
        model = cf.TensorModel(V, B, S)
        res, _, _ = synth.workload(WORKLOAD)
        f = cf.CodonFold(params)
        f.set_protein(res[:m or 100])
        for _ in range(steps):
            f.tm_inside(model, cf.CF_FP32_SCALED)
        out["ms"] = cf.cf_tm_last_ms(f.prob)
        f.close()
        model.close()
    elif form == "subopt":  # every configuration within 1 kcal/mol, first 60 residues (or m) of p300_weighted
        res, lw, pb = synth.workload("p300_weighted")
        mm = m or 60
        f = cf.CodonFold(params)
        f.set_protein(res[:mm], lw[:mm], pb)
        for _ in range(steps):
            cnt, _, _, _ = f.subopt(1.0, 100_000)
        out["ms"] = cf.cf_mfe_last_ms(f.prob)
        out["count"] = cnt
        out["steps"] = cf.cf_subopt_steps(f.prob)
        f.close()
    elif form == "batch":  # the 4,096-protein batch of 24-nt proteins, binary32, run `steps` times
        b = cf.Batch(params, 4096, 8, cf.CF_FP32_SCALED)
        prots = synth.batch_p8(4096)
        for _ in range(steps):
            b.set_proteins(prots)
            b.run()
        out["ms"] = b.last_ms()
        b.close()
    elif form == "windows":
        ex = screen.Windows(params)
        _, _, bases, off = synth.windows(8000, seed=3)
        for _ in range(steps):
            ex.logz(bases, off)
        out["ms"] = ex.last_ms()
        ex.close()
    torch.cuda.synchronize()
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--samples", type=int, default=10000)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="binary32 inside+outside steps only (for profiler captures); prints timings")
    ap.add_argument("--m", type=int, default=0, help="use only the first M residues (profiling)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the window, surrogate, adjoint and 3000-nt measurements")
    ap.add_argument("--profile-form", default="", choices=["", "surrogate", "surrogate_train", "mfe", "sample", "windows", "checkpoint", "tm", "subopt", "batch"],
                    help="run one form on a small case (for profiler captures) and print its timing")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_form:
        return profile_form(args.profile_form, args.steps, args.m)
    if not args.profile:
        args.warmup = max(args.warmup, 3)

    ws, rank, local = dist_setup()
    import torch
    torch.cuda.set_device(local)
    import paper_2604_19718_b300 as cf

    params = synth.nn_params(0)
    res, lw, pb = synth.workload(WORKLOAD)
    if args.m:
        res = res[:args.m]
        lw = None if lw is None else lw[:args.m]
    n = 3 * len(res)
    cells = n * (n + 1) // 2
    stream = torch.cuda.Stream()
    f = cf.CodonFold(params, device=local, stream=stream.cuda_stream)
    f.set_protein(res, lw, pb)
    Pd = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    cmd = torch.zeros((len(res), 6), dtype=torch.float64, device="cuda")
    pgd = torch.zeros((61, 61), dtype=torch.float64, device="cuda")

    def step(prec):
        lz = cf.cf_inside(f.prob, prec)
        cf.cf_outside(f.prob, Pd, cmd, pair_grad=pgd)
        return lz

    if args.profile:
        for _ in range(args.warmup + args.steps):
            step(cf.CF_FP32_SCALED)
        torch.cuda.synchronize()
        print(json.dumps({"profile": True, "n": n, "timing_ms": cf.cf_last_timing(f.prob)}), flush=True)
        return

    # ---- binary32 form: the timed value
    for _ in range(args.warmup):
        step(cf.CF_FP32_SCALED)
    torch.cuda.synchronize()
    barrier(ws)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tin = tout = 0.0
    lin = lout = 0
    with Clocks() as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            lz32 = step(cf.CF_FP32_SCALED)
            a, b, c, d = cf.cf_last_timing(f.prob)
            tin, tout, lin, lout = tin + a, tout + b, lin + c, lout + d
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(ms, ws)
    P32 = Pd.cpu().numpy().copy()
    cm32 = cmd.cpu().numpy().copy()
    far_info = cf.cf_far_band_info(f.prob)
    value = ws * args.steps * cells / (ms * 1e-3)

    # ---- binary64 form on the same GPU
    for _ in range(2):
        step(cf.CF_FP64)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k64 = max(2, args.steps // 3)
    e0.record(stream)
    for _ in range(k64):
        lz64 = step(cf.CF_FP64)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1) / k64
    P64 = Pd.cpu().numpy().copy()
    cm64 = cmd.cpu().numpy().copy()

    # ---- sampling throughput (binary32 tables)
    step(cf.CF_FP32_SCALED)
    cod = torch.zeros((args.samples, len(res)), dtype=torch.int32, device="cuda")
    par = torch.zeros((args.samples, n), dtype=torch.int32, device="cuda")
    cf.cf_sample(f.prob, 64, 1, cod, par)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    cf.cf_sample(f.prob, args.samples, 2024, cod, par)
    s1.record(stream)
    torch.cuda.synchronize()
    samples_per_s = args.samples / (s0.elapsed_time(s1) * 1e-3)

    # ---- end to end through the public API with host buffers (the caller's
    # pinned output arrays, reused from step to step)
    Pt = torch.zeros((n, n), dtype=torch.float32, pin_memory=True)
    cmt = torch.zeros((len(res), 6), dtype=torch.float64, pin_memory=True)
    pgt = torch.zeros((61, 61), dtype=torch.float64, pin_memory=True)
    Ph, cmh, pgh = Pt.numpy(), cmt.numpy(), pgt.numpy()
    letters = cf.to_letters(res)
    ke = max(2, args.steps // 3)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(ke):
        cf.cf_set_protein(f.prob, letters, lw, pb)
        cf.cf_inside(f.prob, cf.CF_FP32_SCALED)
        cf.cf_outside(f.prob, Ph, cmh, pair_grad=pgh)
    e2e_s = (time.perf_counter() - t) / ke
    h2d = len(letters) + (0 if lw is None else lw.nbytes) + (0 if pb is None else pb.nbytes)
    d2h = Ph.nbytes + cmh.nbytes + pgh.nbytes

    forms = {}
    if not args.no_forms and rank == 0:
        forms["windows"], ex, wdata = bench_windows(stream.cuda_stream)
        forms["surrogate"] = bench_surrogate(ex, wdata, stream.cuda_stream)
        ex.close()
        del wdata
        forms["adjoint"] = bench_adjoint(stream.cuda_stream)
        forms["large"] = bench_large(stream.cuda_stream)
        forms["small_batch"] = bench_small_batch()
        forms["concurrent"] = bench_concurrent()
        forms["frequency_matching"] = bench_frequency(stream.cuda_stream)
        forms["mfe"] = bench_mfe(stream.cuda_stream)
        forms["subopt"] = bench_subopt(stream.cuda_stream)
        forms["tensor_model"] = bench_tm(stream.cuda_stream)
        forms["single_codon_layout"] = bench_layout(stream.cuda_stream)

    if rank != 0:
        return
    flops_in, flops_out = algorithmic_flops(res)
    clocks = clk.summary(local)
    clock = clocks["sm_mhz"] or 2032.0
    # the outside pass (the larger share of the step) is one CUDA graph whose
    # light and bifurcation kernels overlap, so it is timed as a unit
    achieved = flops_out / (tout / args.steps * 1e-3) / 1e12
    peak = sm_peak_tflops(clock)
    acc = {"abs_dlogZ_fp32_vs_fp64": abs(lz32 - lz64), "rel_dlogZ": abs(lz32 - lz64) / abs(lz64),
           "max_abs_dP": float(np.abs(P32 - P64).max()), "max_abs_dcodon": float(np.abs(cm32 - cm64).max())}
    out = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: 300 aa / {n} nt, Dirichlet(1) composition (seed 1), "
                               "synthetic nearest-neighbour parameters (seed 0), inside+outside, "
                               "binary32 tables with per-diagonal power-of-two exponents",
                   "cells_per_step": cells, "l2": "working set ~3 GB > 126 MB L2; no flush needed",
                   "parallelism": f"replicas x{ws}"},
        "proteins_per_s": ws * args.steps / (ms * 1e-3),
        "state_cells_per_s": ws * args.steps * state_cells(res) / (ms * 1e-3),
        "fp64_form": {"value": ws * cells / (ms64 * 1e-3), "unit": "cells/s", "ms_per_step": ms64,
                      "speedup_fp32_over_fp64": ms64 / (ms / args.steps)},
        "accuracy": acc,
        "samples_per_s": samples_per_s,
        "inside_ms": tin / args.steps, "outside_ms": tout / args.steps,
        "roofline": {"bound": "alu",
                     "kernel": "outside pass (one CUDA graph: k_out_light, k_out_off = bifurcation gathers + side work, k_out_far, k_out_tg)",
                     "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     # DRAM counters are taken per kernel on single launches of the 600-nt prefix
                     # (profiles/); a capture of the whole 900-nt pass's ~1,900 launches with
                     # counters beyond the launch time is not taken
                     "traffic": None,
                     "peak_basis": f"FP32 FFMA 148 SM x 128 lanes x 2 x {clock:.0f} MHz (median SM clock "
                                   "sampled during the timed region)"},
        "e2e": {"value": cells / e2e_s, "unit": "cells/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(lin + lout),
        "far_bands": dict(zip(("inside_max_departure_log2", "inside_bands_term_by_term",
                               "outside_max_departure_log2", "outside_term_by_term", "range_spread_log2"),
                              far_info)),
        "clocks": clocks,
    }
    out.update(forms)
    if not args.no_cpu:
        out["cpu_baseline"] = cpu_oracle_rate(res, lw, pb)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
