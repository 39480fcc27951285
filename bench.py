"""Benchmark: eigensolve time of the structured divide-and-conquer solver on one GB300.

Workload (default): tridiag(1,2,1) of order n = 16384, leaf size 64 -- the
Toeplitz matrix of the method's Example 2 at the size the headline metric is
quoted on.  One step = one full eigensolve T = Q diag(lam) Q^T through the C ABI
(tdc_eig) with d, e resident in HBM.  The Q and internal buffers (2 x 2 GiB) are
larger than L2, so no explicit flush is needed between steps.

The timed solve uses the library's default merge: the structured update (SRRSC
low-rank far tiles, Section 2.1 / Algorithm 2) with its products on the split
tensor-core GEMM for the large merges.  The default line also carries the merge
comparison on the same matrix (the plain split product, and the dense FP64 and
structured FP64 merges, each with its own accuracy check and roofline), the other
workloads (uniform n = 1024, the batch of 4096 tridiagonals under a CUDA graph,
d ~ U(0,1) with e = 1 at n = 32768, and the adjoint of 256 problems of order 512),
each timed with a few steps, and the FP64 CPU oracle timed on the host's cores on
the headline matrix itself.

Output: one JSON line (rank 0).  Under torchrun every rank solves its own copy
(replicas, weak scaling); the timed region is bracketed by a barrier and
synchronisations and the maximum over ranks is reported.

``--impl reference`` times the plain FP64 CPU oracle (the reference arm of this
project: there is no other implementation of the method to run) on the host's
cores on the same matrix.
"""
from __future__ import annotations

import argparse
import faulthandler
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "eigensolve s at n=16384: structured vs dense merge; Q·U TFLOP/s; test ratios"
EPS = np.finfo(np.float64).eps


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 pipe peak derived from unit counts: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, dist, device) -> float:
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_seconds_per_solve(ms_per_step: float, ranks: int) -> float:
    """Every rank solves one problem per step (replicas), so the job finishes `ranks`
    eigensolves per step of the slowest rank."""
    return ms_per_step / 1e3 / ranks


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(name: str):
    from paper_2008_01990_gb300 import inputs
    if name == "toeplitz16384":
        d, e = inputs.toeplitz_tridiag(16384)
        return d, e, 16, "tridiag(1,2,1) n=16384 leaf 16"
    if name == "toeplitz4096":
        d, e = inputs.toeplitz_tridiag(4096)
        return d, e, 16, "tridiag(1,2,1) n=4096 leaf 16"
    if name == "uniform1024":
        d, e = inputs.uniform_tridiag(1024, 1)
        return d, e, 16, "uniform(-1,1) n=1024 leaf 16 seed 1"
    if name == "c4_32768":
        d, e = inputs.c4_tridiag(32768, 4)
        return d, e, 16, "d uniform(0,1), e=1, n=32768 leaf 16 seed 4"
    # the closed-form and spherical-harmonic families of Examples 2 and 3 at n = 30000
    if name == "clement30000":
        d, e = inputs.clement_tridiag(30000)
        return d, e, 16, "Clement/Kac, e_i = sqrt(i(n-i)), n=30000 leaf 16"
    if name == "hermite30000":
        d, e = inputs.hermite_tridiag(30000)
        return d, e, 16, "Hermite, e_i = sqrt(i), n=30000 leaf 16"
    if name == "sht30000":
        d, e = inputs.sht_tridiag(30000)
        return d, e, 16, "spherical-harmonic transform (Example 3, m = n), n=30000 leaf 16"
    raise ValueError(name)


FAMILY = {"toeplitz16384": "toeplitz", "toeplitz4096": "toeplitz", "uniform1024": "uniform", "c4_32768": "c4",
          "clement30000": "clement", "hermite30000": "hermite", "sht30000": "sht"}


def _oracle_time(d, e, leaf):
    import oracle
    t0 = time.perf_counter()
    # the iteration cap only guards against a runaway root: the oracle bisects every root
    # to the rounding level of its offset, which can take a few hundred halvings
    oracle.eig(d, e, leaf=leaf, max_iter=2000)
    return time.perf_counter() - t0


def cpu_baseline(wl: str, budget_s: float = 180.0):
    """Time the FP64 oracle on the host's cores on the workload's own matrix: one full
    eigensolve at the workload's order.  Only when a quick estimate (the same family at
    n = 2048, scaled by the cube of the order ratio) exceeds budget_s does it fall back
    to that bounded sample, scaled, and the line says so."""
    import oracle
    from paper_2008_01990_gb300 import inputs
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    d_full, e_full, leaf, desc = workload(wl)
    n_full = d_full.size
    fam = FAMILY[wl]
    n_s = min(n_full, 2048)
    d_s, e_s = inputs.family(fam, n_s, 4 if fam == "c4" else 1)
    t_s = _oracle_time(d_s, e_s, leaf)
    est = t_s * (n_full / n_s) ** 3
    if n_s == n_full:
        dt, sample = t_s, "one oracle eigensolve of the workload's matrix (n=%d)" % n_full
    elif est <= budget_s:
        dt = _oracle_time(d_full, e_full, leaf)
        sample = "one oracle eigensolve of the workload's matrix (n=%d), %.1f s wall" % (n_full, dt)
    else:
        dt = est
        sample = ("oracle eigensolve of the same family at n=%d (%.2f s measured), scaled by (%d/%d)^3: the "
                  "full order would exceed %.0f s" % (n_s, t_s, n_full, n_s, budget_s))
    return {"value": dt, "unit": "s", "cores": oracle.get_threads(), "kind": "oracle", "sample": sample,
            "scaled": n_s != n_full and est > budget_s}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on the host's cores, on the same matrix as
    the GPU arm.  Warm-up: W solves of the same family at n = 1024 (page-in, thread
    start).  Timed: full-order eigensolves, as many as fit in about three minutes (at
    least one, at most --steps); the line reports the number actually timed."""
    import oracle
    from paper_2008_01990_gb300 import inputs
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    wl = args.workload
    d, e, leaf, desc = workload(wl)
    fam = FAMILY[wl]
    dw, ew = inputs.family(fam, min(1024, d.size), 4 if fam == "c4" else 1)
    for _ in range(args.warmup):
        _oracle_time(dw, ew, leaf)
    times = []
    t_start = time.perf_counter()
    while len(times) < max(1, args.steps):
        times.append(_oracle_time(d, e, leaf))
        if time.perf_counter() - t_start + times[-1] > 180.0:
            break
    v = float(np.mean(times))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": len(times), "steps_requested": args.steps, "warmup": args.warmup,
            "warmup_kind": "oracle solves of the same family at n=%d" % dw.size,
            "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc},
            "cpu_baseline": {"value": v, "unit": "s", "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": "%d full oracle eigensolve(s) of the workload's matrix (n=%d)"
                                       % (len(times), d.size)},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def sampled_ratios(tdc_lam, Q, d, e, nsample=256):
    """Residual / orthogonality ratios on sampled columns, eigenvalue error against
    the closed form where one exists (verification only, outside the timed region)."""
    import torch
    n = d.numel()
    g = np.random.default_rng(0)
    cols = torch.tensor(np.sort(g.choice(n, min(n, nsample), replace=False)), device=Q.device)
    Qs = Q[:, cols]
    Tq = d[:, None] * Qs
    Tq[1:] += e[:, None] * Qs[:-1]
    Tq[:-1] += e[:, None] * Qs[1:]
    nT = max(abs(tdc_lam[0].item()), abs(tdc_lam[-1].item()))
    res = torch.abs(Tq - Qs * tdc_lam[cols]).sum(dim=0).max().item() / (n * nT * EPS)
    G = Qs.t() @ Q
    G[torch.arange(cols.numel(), device=Q.device), cols] -= 1.0
    orth = torch.abs(G).sum(dim=1).max().item() / (n * EPS)
    return res, orth, nT


def run_qhat(args):
    """Stand-alone eigenvector-update product C = A * Qhat (tdc_cauchy_gemm) at the size of
    the top merge of the n=16384 workload: A 8192 x 8192 with |A_ij| <= 1, Qhat the 8192 x 8192
    Cauchy-like eigenvector matrix of a rank-one problem (generators from tdc_rank_one)."""
    import torch
    from paper_2008_01990_gb300 import inputs, tdc
    dev = torch.device("cuda", 0)
    m = K = 8192
    g = inputs.SplitMix64(11)
    D = np.sort(g.uniform(K, -1.0, 1.0))
    z = g.uniform(K, -1.0, 1.0)
    z /= np.linalg.norm(z)
    A = torch.tensor(g.uniform(m * K, -1.0, 1.0).reshape(K, m), device=dev).t() / np.sqrt(K)
    Dt, zt = torch.tensor(D, device=dev), torch.tensor(z, device=dev)
    org, tau, zh, s = tdc.rank_one(Dt, zt, 0.9, check=True)
    mode = tdc.MERGE_SPLIT if args.merge in ("split", "auto") else tdc.MERGE_DENSE
    opts = tdc.default_opts()
    for _ in range(args.warmup):
        C = tdc.cauchy_gemm(A, Dt, org, tau, zh, s, mode, opts)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        C = tdc.cauchy_gemm(A, Dt, org, tau, zh, s, mode, opts)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    flops = 2.0 * m * K * K
    print(json.dumps({"workload": "qhat8192", "merge": args.merge, "ms": ms,
                      "fp64_equivalent_tflops": flops / (ms * 1e-3) / 1e12}), flush=True)
    return 0


def run_example1(args, n):
    """Example 1 of the paper: C = A B with A random (uniform(-1,1)) and the Cauchy-like
    B_ij = u_i v_j / (d_i - w_j), d_i = 8 i / n, w_j = d_j + 4 / n, u, v uniform(0,1):
    every product mode timed (CUDA events, after a warm-up), with its error against the
    FP64 dense product on sampled columns."""
    import torch
    from paper_2008_01990_gb300 import inputs, tdc
    dev = torch.device("cuda", 0)
    d_np, w_np, u_np, v_np = inputs.example1_cauchy(n)
    d, w, u, v = (torch.tensor(x, device=dev) for x in (d_np, w_np, u_np, v_np))
    g = torch.Generator(device=dev)
    g.manual_seed(n)
    A = (torch.rand(n, n, dtype=torch.float64, device=dev, generator=g) * 2 - 1).t()
    cols = torch.tensor(np.sort(np.random.default_rng(0).choice(n, 64, replace=False)), device=dev)
    Bs = (u[:, None] * v[cols][None, :]) / (d[:, None] - w[cols][None, :])
    Cref = A @ Bs  # FP64 reference on the sampled columns (a library matmul, verification only)
    scale = torch.linalg.norm(A, dim=1)[:, None] * torch.linalg.norm(Bs, dim=0)[None, :]
    out = {"workload": "example1 n=%d: C = A B, B_ij = u_i v_j / (d_i - w_j)" % n, "modes": {}}
    opts = tdc.default_opts()
    for name, md in (("dense", tdc.MERGE_DENSE), ("structured", tdc.MERGE_STRUCTURED), ("split", tdc.MERGE_SPLIT),
                     ("structured_split", tdc.MERGE_STRUCTURED_SPLIT)):
        if name in ("dense", "structured") and n > 16384:
            continue  # the FP64 products at n = 32768 take tens of seconds each
        C = tdc.cauchy_like_gemm(A, d, w, u, v, md, opts, check=True)
        steps = 1 if name in ("dense", "structured") else max(1, min(args.steps, 5))
        ms = _event_ms(lambda: tdc.cauchy_like_gemm(A, d, w, u, v, md, opts), steps)
        err = float(torch.max(torch.abs(C[:, cols] - Cref) / scale).item())
        out["modes"][name] = {"ms": ms, "steps": steps, "max_err_over_rownorm_colnorm": err,
                              "fp64_equivalent_tflops": 2.0 * n ** 3 / (ms * 1e-3) / 1e12}
        del C
        progress("example1 %d %s done" % (n, name))
    R = tdc.cauchy_like_ranks(d, w, u, v, tdc.default_opts(lr_tile=4096, lr_tol=1e-15)).cpu().numpy()
    out["ranks_4096_tiles_first_block_column"] = [int(x) for x in R[1:, 0]]
    return out


def run_structured_products(args, n):
    """The further structured operands: C = A B with B Toeplitz (t[k - j + n - 1]) or
    Hankel (t[k + j]) from 2n - 1 generators uniform(-1, 1), A uniform(-1, 1) n x n; FP64
    and split modes timed with CUDA events after a warm-up, error against the FP64 dense
    product on sampled columns; the DFT product (split); and the bidiagonal SVD of order n
    (uniform family)."""
    import torch
    from paper_2008_01990_gb300 import inputs, tdc
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev)
    g.manual_seed(n)
    A = (torch.rand(n, n, dtype=torch.float64, device=dev, generator=g) * 2 - 1).t()
    t = torch.tensor(inputs.SplitMix64(n).uniform(2 * n - 1, -1.0, 1.0), device=dev)
    cols = torch.tensor(np.sort(np.random.default_rng(0).choice(n, 64, replace=False)), device=dev)
    k = torch.arange(n, device=dev)
    out = {"workload": "Toeplitz / Hankel / DFT products n=%d and the bidiagonal SVD" % n, "products": {}}
    for kind, kname in ((tdc.TOEPLITZ, "toeplitz"), (tdc.HANKEL, "hankel")):
        idx = (k[:, None] - cols[None, :] + n - 1) if kind == tdc.TOEPLITZ else (k[:, None] + cols[None, :])
        Bs = t[idx]
        Cref = A @ Bs  # FP64 reference on the sampled columns (a library matmul, verification only)
        scale = torch.linalg.norm(A, dim=1)[:, None] * torch.linalg.norm(Bs, dim=0)[None, :]
        for mname, md in (("dense", tdc.MERGE_DENSE), ("split", tdc.MERGE_SPLIT)):
            C = tdc.structured_gemm(A, t, kind, md, check=True)
            steps = 1 if mname == "dense" else max(1, min(args.steps, 5))
            ms = _event_ms(lambda: tdc.structured_gemm(A, t, kind, md), steps)
            err = float(torch.max(torch.abs(C[:, cols] - Cref) / scale).item())
            out["products"]["%s_%s" % (kname, mname)] = {
                "ms": ms, "steps": steps, "max_err_over_rownorm_colnorm": err,
                "fp64_equivalent_tflops": 2.0 * n ** 3 / (ms * 1e-3) / 1e12}
            del C
    Fr_ref = A @ torch.cos(2 * np.pi * ((k[:, None] * cols[None, :]) % n).double() / n)
    Cr, Ci = tdc.dft_gemm(A, tdc.MERGE_SPLIT, check=True)
    ms = _event_ms(lambda: tdc.dft_gemm(A, tdc.MERGE_SPLIT), max(1, min(args.steps, 5)))
    scale = torch.linalg.norm(A, dim=1)[:, None] * np.sqrt(n)
    out["products"]["dft_split"] = {"ms": ms, "max_err_over_rownorm_colnorm":
                                    float(torch.max(torch.abs(Cr[:, cols] - Fr_ref) / scale).item()),
                                    "note": "two real products (cos and -sin parts)"}
    del Cr, Ci, Fr_ref
    d_np, e_np = inputs.bidiag_family("uniform", n, seed=n)
    d, e = torch.tensor(d_np, device=dev), torch.tensor(e_np, device=dev)
    s, U, VT = tdc.bdsdc(d, e, check=True)
    ms = _event_ms(lambda: tdc.bdsdc(d, e), max(1, min(args.steps, 3)))
    cs = cols[:64]
    V = VT.t()
    Bv = d[:, None] * V[:, cs]
    Bv[:-1] += e[:, None] * V[1:, cs]
    res = torch.abs(Bv - U[:, cs] * s[cs][None, :]).sum(dim=0).max().item() / (n * s[0].item() * EPS)
    orth = torch.abs(U.t() @ U - torch.eye(n, dtype=U.dtype, device=dev)).sum(dim=0).max().item() / (n * EPS)
    out["bdsdc"] = {"ms": ms, "residual_sampled": res, "orthogonality_U": orth,
                    "note": "tdc_eig on the order-2n Golub-Kahan tridiagonal"}
    return out


def _event_ms(fn, steps, stream=None):
    """Average device time of fn over `steps` calls, CUDA events on `stream`."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        fn()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def full_ratios(d, e, lam, Q):
    """Residual and orthogonality ratios on every column (small orders), device FP64."""
    import torch
    n = d.numel()
    Tq = d[:, None] * Q
    Tq[1:] += e[:, None] * Q[:-1]
    Tq[:-1] += e[:, None] * Q[1:]
    nT = max(abs(lam[0].item()), abs(lam[-1].item()))
    res = torch.abs(Tq - Q * lam[None, :]).sum(dim=0).max().item() / (n * nT * EPS)
    G = Q.t() @ Q - torch.eye(n, dtype=Q.dtype, device=Q.device)
    orth = torch.abs(G).sum(dim=0).max().item() / (n * EPS)
    return res, orth, nT


def invariants(d, e, lam):
    """|sum lam - trace| / (n ||T||) and |sum lam^2 - ||T||_F^2| / (n ||T||^2): the trace and
    Frobenius invariants of the eigenvalues, in units of eps."""
    n = d.numel()
    nT = max(abs(lam[0].item()), abs(lam[-1].item()), 1e-300)
    tr = abs(lam.sum().item() - d.sum().item()) / (n * nT * EPS)
    fro = abs((lam * lam).sum().item() - ((d * d).sum().item() + 2 * (e * e).sum().item())) / (n * nT * nT * EPS)
    return tr, fro


def split_roofline(stats, split_ms, S, pk, pk_kind, note=""):
    products = S * (S + 1) // 2
    flops = float(stats["split_flops"])
    if not (flops > 0 and split_ms > 0):
        return None
    achieved = flops * products / (split_ms * 1e-3) / 1e12
    return {"bound": "tensor", "kernel": "k_gemm_split (BF16 digit products, tcgen05, TMEM FP32 levels)",
            "achieved": achieved, "peak": pk["bf16_tflops"], "unit": "TFLOP/s", "frac": achieved / pk["bf16_tflops"],
            "peak_kind": "bf16_tflops (burst) of %s%s" % (pk_kind, note),
            "fp64_equivalent_tflops": flops / (split_ms * 1e-3) / 1e12, "bf16_products_per_fp64_product": products}


def config_c1(args):
    """uniform(-1,1) n = 1024 (seed 1), leaf 32, the library's default merge."""
    import torch
    from paper_2008_01990_gb300 import tdc
    dev = torch.device("cuda", 0)
    d_np, e_np, leaf, desc = workload("uniform1024")
    d, e = torch.tensor(d_np, device=dev), torch.tensor(e_np, device=dev)
    o = tdc.default_opts(leaf=leaf)
    n = d.numel()
    lam = torch.empty(n, dtype=torch.float64, device=dev)
    Q = torch.empty(n, n, dtype=torch.float64, device=dev).t()
    ws = tdc.workspace(tdc.workspace_size(n, o), dev)
    step = lambda: tdc.eig(d, e, o, ws=ws, lam=lam, Q=Q)
    for _ in range(3):
        step()
    st = tdc.sync_status()
    ms = _event_ms(step, 20)
    res, orth, nT = full_ratios(d, e, lam, Q)
    tr, fro = invariants(d, e, lam)
    oi = tdc.default_opts(leaf=leaf, collect_stats=1)
    tdc.eig(d, e, oi, ws=ws, lam=lam, Q=Q)
    stats = tdc.get_stats()
    return {"workload": desc, "ms": ms, "steps": 20, "status": tdc.strerror(st),
            "checks": {"residual": res, "orthogonality": orth, "columns": "all", "trace_eps": tr,
                       "frobenius_eps": fro, "within_bounds": bool(res <= 50 and orth <= 50)},
            "bound": "latency: %d kernel launches per solve on a 1024-order tree" % stats["launches"],
            "phase_ms": stats["phase_ms"], "launches_per_solve": int(stats["launches"])}


def config_c3(args, steps=3, warmup=3):
    """The batched workload: 4096 tridiagonals, n_b uniform in [64, 2048] (seed 3), entries
    uniform(-1,1) (seed 3 + b), solved by one tdc_eig_batched call replayed from a CUDA
    graph, options chosen by the autotuner (outside the timed region)."""
    import torch
    from paper_2008_01990_gb300 import autotune, inputs, tdc
    dev = torch.device("cuda", 0)
    sizes = inputs.batched_sizes(args.batch, 64, 2048, 3)
    d, e, offs = inputs.batched_uniform(sizes, 3)
    qoffs = np.concatenate([[0], np.cumsum(sizes.astype(np.int64) ** 2)])
    dt, et = torch.tensor(d, device=dev), torch.tensor(e, device=dev)
    t0 = time.perf_counter()
    if args.leaf or args.split_min_k:
        opts = tdc.default_opts(leaf=args.leaf or 32, split_min_K=args.split_min_k or 128)
    else:
        opts = autotune.tune_batched(sizes, dt, et, offs[:-1], cache_path=None)
    tune_s = time.perf_counter() - t0
    lam = torch.empty(int(offs[-1]), dtype=torch.float64, device=dev)
    Q = torch.empty(int(qoffs[-1]), dtype=torch.float64, device=dev)
    ws = tdc.workspace(tdc.batched_workspace_size(sizes, opts), dev)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        tdc.eig_batched(sizes, dt, et, offs[:-1], qoffs[:-1], lam, Q, opts, ws=ws, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        tdc.eig_batched(sizes, dt, et, offs[:-1], qoffs[:-1], lam, Q, opts, ws=ws, stream=s)
    for _ in range(warmup):
        g.replay()
    ms = _event_ms(g.replay, steps)
    st = tdc.sync_status()
    # checks outside the timed region: every problem's eigenvalues sorted and finite;
    # residual and orthogonality ratios on 16 problems spread over the size range
    lam_h = lam.cpu().numpy()
    sorted_ok = bool(np.all(np.isfinite(lam_h)) and all(
        np.all(np.diff(lam_h[offs[b]:offs[b] + sizes[b]]) >= 0) for b in range(len(sizes))))
    order = np.argsort(sizes, kind="stable")
    pick = sorted(set(int(order[i]) for i in np.linspace(0, len(sizes) - 1, 16).round().astype(int)))
    worst_res = worst_orth = 0.0
    for b in pick:
        nb = int(sizes[b])
        Qb = Q[int(qoffs[b]):int(qoffs[b]) + nb * nb].view(nb, nb).t()
        r, o_, _ = full_ratios(dt[offs[b]:offs[b] + nb], et[offs[b]:offs[b] + nb - 1], lam[offs[b]:offs[b] + nb], Qb)
        worst_res, worst_orth = max(worst_res, r), max(worst_orth, o_)
    # one more solve with statistics (outside the timed region): launches and phases
    ost = tdc.default_opts(leaf=opts.leaf, split_min_K=opts.split_min_K, collect_stats=1)
    tdc.eig_batched(sizes, dt, et, offs[:-1], qoffs[:-1], lam, Q, ost, ws=ws)
    stats = tdc.get_stats()
    pk, pk_kind = peaks()
    out = {"workload": "4096 tridiagonals, n_b uniform in [64,2048] (seed 3), d, e uniform(-1,1)"
                       if args.batch == 4096 else "batched%d" % args.batch,
           "ms_per_batch": ms, "problems_per_s": args.batch / (ms * 1e-3), "steps": steps,
           "leaf": opts.leaf, "split_min_K": opts.split_min_K, "autotune_s": tune_s, "status": tdc.strerror(st),
           "graph": "one tdc_eig_batched call captured and replayed", "sum_n": int(sizes.sum()),
           "q_bytes": int(qoffs[-1]) * 8,
           "checks": {"eigenvalues_sorted_finite": sorted_ok, "problems_checked": len(pick),
                      "residual_max": worst_res, "orthogonality_max": worst_orth,
                      "within_bounds": bool(worst_res <= 50 and worst_orth <= 50)},
           "launches_per_solve": int(stats["launches"]), "phase_ms": stats["phase_ms"],
           "secular_iterations": {"mean": stats["secular_iter_mean"], "max": stats["secular_iter_max"],
                                  "handoffs": stats.get("secular_handoffs")},
           "K_per_level": stats["sum_K"], "n_per_level": stats["sum_n"],
           "split_roofline": split_roofline(stats, stats["phase_ms"]["split_mma"], opts.split_slices, pk, pk_kind,
                                            "; phase time with statistics on, two streams")}
    del g, ws, Q, lam
    torch.cuda.empty_cache()
    return out


def config_c4(args, steps=3, warmup=3):
    """d ~ U(0,1), e = 1, n = 32768 (seed 4), leaf and split threshold autotuned on the matrix."""
    import torch
    from paper_2008_01990_gb300 import autotune, tdc
    dev = torch.device("cuda", 0)
    d_np, e_np, _, desc = workload("c4_32768")
    d, e = torch.tensor(d_np, device=dev), torch.tensor(e_np, device=dev)
    n = d.numel()
    t0 = time.perf_counter()
    t = autotune.tune_single(d, e, tdc.MERGE_AUTO, cache_path=None)
    tune_s = time.perf_counter() - t0
    o = tdc.default_opts(leaf=t.leaf, split_min_K=t.split_min_K)
    lam = torch.empty(n, dtype=torch.float64, device=dev)
    Q = torch.empty(n, n, dtype=torch.float64, device=dev).t()
    ws = tdc.workspace(tdc.workspace_size(n, o), dev)
    step = lambda: tdc.eig(d, e, o, ws=ws, lam=lam, Q=Q)
    for _ in range(warmup):
        step()
    st = tdc.sync_status()
    ms = _event_ms(step, steps)
    oi = tdc.default_opts(leaf=t.leaf, split_min_K=t.split_min_K, collect_stats=1)
    tdc.eig(d, e, oi, ws=ws, lam=lam, Q=Q)
    stats = tdc.get_stats()
    res, orth, nT = sampled_ratios(lam, Q, d, e)
    tr, fro = invariants(d, e, lam)
    pk, pk_kind = peaks()
    out = {"workload": desc.split(" leaf ")[0] + " leaf %d, split_min_K %d (autotuned)" % (t.leaf, t.split_min_K),
           "ms": ms, "steps": steps, "autotune_s": tune_s, "status": tdc.strerror(st),
           "checks": {"residual": res, "orthogonality": orth, "sampled_columns": 256, "trace_eps": tr,
                      "frobenius_eps": fro, "within_bounds": bool(res <= 50 and orth <= 50)},
           "split_level_max": stats["split_level_max"], "phase_ms": stats["phase_ms"],
           "K_per_level": stats["sum_K"],
           "roofline": split_roofline(stats, stats["phase_ms"]["split_mma"], o.split_slices, pk, pk_kind,
                                      "; phase time of one solve with statistics on")}
    del ws, Q, lam
    torch.cuda.empty_cache()
    return out


def config_c5(args, steps=5, warmup=3):
    """The backward workload: 256 tridiagonals of order 512 (d, e uniform(-1,1), seed 5,
    redrawn until the smallest eigen-gap is >= 1e-5 ||T||), loss sum w_j lam_j + sum G_ij Q_ij
    with w, G ~ N(0,1); one step = batched forward solve + batched adjoint."""
    import torch
    from paper_2008_01990_gb300 import inputs, tdc
    dev = torch.device("cuda", 0)
    B, n = 256, 512
    ds, es, ws_, Gs, gaps, draws = inputs.backward_problems(B, n, 5)
    d = torch.tensor(ds, device=dev)
    e = torch.tensor(es, device=dev)
    w = torch.tensor(ws_, device=dev)
    G = torch.tensor(Gs, device=dev)
    opts = tdc.default_opts(leaf=32)

    def step():
        dd = d.clone().requires_grad_(True)
        ee = e.clone().requires_grad_(True)
        lam, Q = tdc.eigh_tridiagonal(dd, ee, opts)
        loss = (w * lam).sum() + (G * Q).sum()
        loss.backward()
        return dd.grad, ee.grad

    for _ in range(warmup):
        step()
    ms = _event_ms(step, steps)
    # adjoint alone (the two n^3 products per problem)
    lam, Q = tdc.eigh_tridiagonal(d, e, opts)
    Qs = Q.transpose(1, 2).contiguous()
    Gs_t = G.transpose(1, 2).contiguous()
    tdc.eig_backward_batched(lam, Qs, w, Gs_t)
    ams = _event_ms(lambda: tdc.eig_backward_batched(lam, Qs, w, Gs_t), steps)
    # check (closed form, Hellmann-Feynman): with Q_bar = 0 the cotangents are
    # d_bar_i = sum_k w_k Q_ik^2 and e_bar_i = 2 sum_k w_k Q_ik Q_i+1,k
    db, eb = tdc.eig_backward_batched(lam, Qs, w, None)
    Qm = Q  # (B, n, n) with Q[b] the eigenvector matrix
    db_ref = torch.einsum("bik,bk->bi", Qm * Qm, w)
    eb_ref = 2.0 * torch.einsum("bik,bk->bi", Qm[:, :-1, :] * Qm[:, 1:, :], w)
    scale = torch.abs(w).max().item()
    hf = max(torch.max(torch.abs(db - db_ref)).item(), torch.max(torch.abs(eb - eb_ref)).item()) / scale
    flops = B * 4.0 * n ** 3
    return {"workload": "backward: 256 x n=512, d, e uniform(-1,1) (seed 5), min gap >= 1e-5 ||T||",
            "ms_forward_backward": ms, "ms_adjoint": ams, "steps": steps,
            "adjoint_tflops_fp64_equivalent": flops / (ams * 1e-3) / 1e12,
            "checks": {"hellmann_feynman_max_err_over_max_w": hf, "within_bounds": bool(hf <= 1e-12)},
            "min_gap_rel": float(gaps.min()), "draws": int(draws)}


# DRAM bytes of k_gemm_split over one eigensolve, summed over its launches, from
# single-pass ncu captures of the kernel as it stands; keyed by the exact
# configuration (workload, merge, leaf, split_min_K, split_chunk_k, lr_tile), null for
# any other
TRAFFIC = {("toeplitz16384", "auto", 16, 128, 256, 256): 21.89e9}


def config_dense(args, n=4096, steps=3):
    """Dense symmetric eigenproblem, the pipeline of Example 3 on a synthetic matrix (the
    paper's SuiteSparse matrices are not available): A = (X + X^T) / 2, X uniform(-1, 1)
    from SplitMix64(n), solved by tdc_syevd (Householder reduction, divide and conquer on
    T, back-transform).  Whole call and each stage timed with CUDA events after warm-up;
    residual, orthogonality and the paper's residual ||A - Z Lam Z^T||_c / ||A||_2 on every
    column; the reduction against the FP64 pipe (its symv is the n^3/3 multiply-adds
    of the one-stage reduction, on FP64 units); cuSOLVER's syevd (torch.linalg.eigh) on
    the same matrix as context."""
    import torch
    from paper_2008_01990_gb300 import inputs, tdc
    dev = torch.device("cuda", 0)
    A = torch.tensor(inputs.dense_sym("uniform", n, seed=n), device=dev)
    ws = tdc.workspace(tdc.syevd_workspace_size(n), dev)
    for _ in range(2):
        tdc.syevd(A, ws=ws)
    ms = _event_ms(lambda: tdc.syevd(A, ws=ws), steps)
    st = tdc.sync_status()
    d, e, tau, R = tdc.sytrd(A, check=True)
    ms_trd = _event_ms(lambda: tdc.sytrd(A), steps)
    X0 = torch.eye(n, dtype=torch.float64, device=dev).t().contiguous().t()
    X = X0.clone().t().contiguous().t()
    ms_orm = _event_ms(lambda: tdc.ormtr(R, tau, X), steps)
    wse = tdc.workspace(tdc.workspace_size(n), dev)
    ms_eig = _event_ms(lambda: tdc.eig(d, e, ws=wse), steps)
    lam, Z = tdc.syevd(A, ws=ws, check=True)
    Rm = A @ Z - Z * lam[None, :]
    nA = max(abs(lam[0].item()), abs(lam[-1].item()))
    res = torch.abs(Rm).sum(dim=0).max().item() / (n * nA * EPS)
    orth = torch.abs(Z.t() @ Z - torch.eye(n, dtype=Z.dtype, device=dev)).sum(dim=0).max().item() / (n * EPS)
    paper_res = torch.linalg.norm(A - (Z * lam[None, :]) @ Z.t(), dim=0).max().item() / nA
    del Rm, X, X0
    torch.linalg.eigh(A)  # warm-up: handle and workspace of the library solver
    ms_eigh = _event_ms(lambda: torch.linalg.eigh(A), 2)
    fp64_peak = FP64_PEAK_TFLOPS
    symv_flops = 2.0 * sum(m * m for m in range(2, n))
    achieved = symv_flops / (ms_trd * 1e-3) / 1e12
    return {"workload": "dense symmetric uniform n=%d: tdc_syevd (reduction, divide and conquer, back-transform)" % n,
            "ms": ms, "steps": steps, "status": tdc.strerror(st),
            "stage_ms": {"sytrd": ms_trd, "eig": ms_eig, "ormtr": ms_orm},
            "checks": {"residual": res, "orthogonality": orth, "paper_residual": paper_res, "columns": "all",
                       "within_bounds": bool(res <= 50 and orth <= 50)},
            "roofline": {"bound": "alu", "kernel": "k_trd_panel (FP64 symv of the one-stage reduction)",
                         "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                         "note": "symv flops 2 sum m^2 over the whole tdc_sytrd time (trailing updates included); "
                                 "peak derived from unit counts (152 SMs x 2 DFMA/clk x 2.07 GHz)"},
            "context_cusolver_syevd_ms": ms_eigh, "speedup_vs_cusolver_syevd": ms_eigh / ms}


def config_band(args, n=4096, bws=(8, 32), steps=3):
    """Symmetric band eigenproblems (the band divide and conquer of tdc_sbevd) on the
    uniform band family (entries uniform(-1, 1) from SplitMix64(1), half-bandwidths b):
    whole call timed with CUDA events after a warm-up; residual and orthogonality ratios on
    every column; the dense solver (tdc_syevd) on the same matrix as context."""
    import torch
    from paper_2008_01990_gb300 import inputs, tdc
    dev = torch.device("cuda", 0)
    out = {"workload": "symmetric band uniform n=%d: tdc_sbevd (tearing, batched dense leaves, b rank-one "
                       "merges per node)" % n, "bands": {}}
    ms_dense = None
    for b in bws:
        AB = torch.tensor(inputs.band_sym("uniform", n, b, seed=1), device=dev)
        tdc.sbevd(AB)
        ms = _event_ms(lambda: tdc.sbevd(AB), steps)
        st = tdc.sync_status()
        lam, Q = tdc.sbevd(AB, check=True)
        A = torch.zeros(n, n, dtype=torch.float64, device=dev)
        for r in range(b + 1):
            idx = torch.arange(n - r, device=dev)
            A[idx + r, idx] = AB[r, : n - r]
            A[idx, idx + r] = AB[r, : n - r]
        nA = max(abs(lam[0].item()), abs(lam[-1].item()))
        res = torch.abs(A @ Q - Q * lam[None, :]).sum(dim=0).max().item() / (n * nA * EPS)
        orth = torch.abs(Q.t() @ Q - torch.eye(n, dtype=Q.dtype, device=dev)).sum(dim=0).max().item() / (n * EPS)
        entry = {"b": b, "ms": ms, "steps": steps, "status": tdc.strerror(st),
                 "checks": {"residual": res, "orthogonality": orth, "columns": "all",
                            "within_bounds": bool(res <= 50 and orth <= 50)}}
        if ms_dense is None and not getattr(args, "no_compare", False):
            tdc.syevd(A)
            ms_dense = _event_ms(lambda: tdc.syevd(A), 2)
        if ms_dense is not None:
            entry["context_tdc_syevd_ms"] = ms_dense
        out["bands"]["b%d" % b] = entry
        del A, Q, lam, AB
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2008_01990_gb300 import tdc

    ws_n, rank, local = dist_env()
    if ws_n > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    d_np, e_np, leaf, desc = workload(args.workload)
    n = d_np.size
    mode = {"dense": tdc.MERGE_DENSE, "auto": tdc.MERGE_AUTO, "structured": tdc.MERGE_STRUCTURED,
            "split": tdc.MERGE_SPLIT, "structured_split": tdc.MERGE_STRUCTURED_SPLIT}[args.merge]
    if args.leaf:
        leaf = args.leaf
        desc = desc.split(" leaf ")[0] + " leaf %d" % leaf + (" seed" + desc.split(" seed")[1] if " seed" in desc else "")
    kw = {"split_min_K": args.split_min_k} if args.split_min_k else {}
    d = torch.tensor(d_np, device=dev)
    e = torch.tensor(e_np, device=dev)
    if args.workload == "c4_32768" and not args.leaf and not args.split_min_k:
        # this workload's leaf size is chosen by the autotuner (timed on the matrix)
        from paper_2008_01990_gb300 import autotune
        t = autotune.tune_single(d, e, mode, cache_path=None)
        leaf, kw = t.leaf, {"split_min_K": t.split_min_K}
        desc = desc.split(" leaf ")[0] + " leaf %d (autotuned, split_min_K %d) seed 4" % (leaf, t.split_min_K)
    if args.split_chunk_k >= 0:
        kw["split_chunk_k"] = args.split_chunk_k
    opts = tdc.default_opts(leaf=leaf, merge_mode=mode, **kw)
    opts_i = tdc.default_opts(leaf=leaf, merge_mode=mode, collect_stats=1, **kw)
    lam = torch.empty(n, dtype=torch.float64, device=dev)
    Q = torch.empty(n, n, dtype=torch.float64, device=dev).t()
    wsb = tdc.workspace(tdc.workspace_size(n, opts), dev)
    stream = torch.cuda.current_stream()

    def step():
        tdc.eig(d, e, opts, ws=wsb, lam=lam, Q=Q, stream=stream)

    progress("inputs and workspace ready")
    for _ in range(args.warmup):
        step()
    st = tdc.sync_status(stream)
    progress("warm-up done")
    if st not in (0, tdc.TDC_WPRECISION):
        raise RuntimeError("device status %d (%s)" % (st, tdc.strerror(st)))
    # the timed region: K eigensolves, statistics off, clocks sampled meanwhile
    sampler = ClockSampler(local)
    if ws_n > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    if ws_n > 1:
        ms = max_over_ranks(ms, dist, dev)
        dist.barrier()
    # an instrumented region (statistics on: the library records CUDA events around its
    # phases on the stream each phase runs on; one host synchronisation per solve):
    # per-kernel times, flops and launch counts of the same solves
    isteps = max(1, min(args.steps, 5))
    phases = []
    i0 = torch.cuda.Event(enable_timing=True)
    i1 = torch.cuda.Event(enable_timing=True)
    i0.record(stream)
    for _ in range(isteps):
        tdc.eig(d, e, opts_i, ws=wsb, lam=lam, Q=Q, stream=stream)
        phases.append(tdc.get_stats())
    i1.record(stream)
    torch.cuda.synchronize()
    ims = i0.elapsed_time(i1) / isteps
    progress("timed and instrumented regions done")
    stats = phases[-1]
    S = opts.split_slices
    split_ms = float(np.median([p["phase_ms"]["split_mma"] for p in phases]))
    digits_ms = float(np.median([p["phase_ms"]["split_digits"] for p in phases]))
    dense_ms = float(np.median([p["phase_ms"]["gemm_fp64"] for p in phases]))
    split_flops = float(stats["split_flops"])
    dense_flops = float(sum(stats["gemm_flops"])) - split_flops
    pk, pk_kind = peaks()
    if split_flops > 0 and split_ms > 0:
        roof = split_roofline(stats, split_ms, S, pk, pk_kind,
                              ": the kernel runs in bursts of tens of ms and the SM clock stays at its maximum "
                              "(see clocks)")
        roof["traffic"] = TRAFFIC.get((args.workload, args.merge, opts.leaf, opts.split_min_K, opts.split_chunk_k,
                                       opts.lr_tile))
        roof["traffic_scope"] = "DRAM bytes of all k_gemm_split launches of one eigensolve (ncu)"
        roof["algorithmic_bytes"] = stats.get("split_bytes")
        roof["frac_of_sustained"] = roof["achieved"] / pk["bf16_tflops_sustained"]
        roof["timing"] = "median phase time over %d instrumented solves" % isteps
        qu_tflops = (split_flops + dense_flops) / ((split_ms + digits_ms + dense_ms) * 1e-3) / 1e12
    elif stats["struct_flops"] > 0:
        sflops = float(stats["struct_flops"])
        achieved = sflops / (dense_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "k_gemm_dense (near-diagonal) + k_struct_w + k_struct_apply (FP64)",
                "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_kind": "derived: 152 SMs x 2 DFMA/clk x 2.07 GHz",
                "executed_flops": sflops, "dense_equivalent_flops": dense_flops}
        qu_tflops = dense_flops / (dense_ms * 1e-3) / 1e12
    else:
        achieved = dense_flops / (dense_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "k_gemm_dense (FP64 Q*U with generated U)",
                "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_kind": "derived: 152 SMs x 2 DFMA/clk x 2.07 GHz"}
        qu_tflops = achieved
    # accuracy of the timed configuration (outside the timed region)
    res, orth, nT = sampled_ratios(lam, Q, d, e)
    lam_err = None
    if args.workload.startswith("toeplitz"):
        k = torch.arange(1, n + 1, dtype=torch.float64, device=dev)
        ref = torch.sort(2.0 + 2.0 * torch.cos(k * np.pi / (n + 1))).values
        lam_err = torch.max(torch.abs(lam - ref)).item() / 4.0
    elif args.workload.startswith("clement"):
        # eigenvalues -(n-1), -(n-3), ..., n-1; ||T||_2 = n - 1
        ref = torch.arange(-(n - 1), n, 2, dtype=torch.float64, device=dev)
        lam_err = torch.max(torch.abs(lam - ref)).item() / (n - 1)

    def accuracy():
        r, o_, _ = sampled_ratios(lam, Q, d, e)
        le = None
        if args.workload.startswith("toeplitz"):
            le = torch.max(torch.abs(lam - ref)).item() / 4.0
        return {"lam_err_over_normT": le, "residual": r, "orthogonality": o_, "sampled_columns": 256,
                "within_bounds": bool(r <= 50 and o_ <= 50)}

    # the merge comparison on the same input: the plain dense FP64 merge and the
    # structured (SRRSC) merge, one warm-up and one timed solve each
    compare = {args.merge: ms / 1e3}
    compare_detail = {}
    if args.merge != "dense" and not args.no_compare:
        od = tdc.default_opts(leaf=leaf, merge_mode=tdc.MERGE_DENSE, collect_stats=1)
        tdc.eig(d, e, od, ws=wsb, lam=lam, Q=Q, stream=stream)
        tdc.eig(d, e, od, ws=wsb, lam=lam, Q=Q, stream=stream)
        sd = tdc.get_stats()
        compare["dense"] = sd["phase_ms"]["total"] / 1e3
        progress("dense merge done")
        dfl = float(sum(sd["gemm_flops"]))
        compare_detail["dense"] = {
            "s": compare["dense"], "test_ratios": accuracy(),
            "roofline": {"bound": "alu", "kernel": "k_gemm_dense (FP64 Q*U with generated U)",
                         "achieved": dfl / (sd["phase_ms"]["gemm_fp64"] * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": dfl / (sd["phase_ms"]["gemm_fp64"] * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                         "peak_kind": "derived: 152 SMs x 2 DFMA/clk x 2.07 GHz"}}
    if args.merge not in ("dense", "structured") and not args.no_compare and n >= 4096:
        osd = tdc.default_opts(leaf=leaf, merge_mode=tdc.MERGE_STRUCTURED, collect_stats=1)
        wss = tdc.workspace(tdc.workspace_size(n, osd), dev)
        tdc.eig(d, e, osd, ws=wss, lam=lam, Q=Q, stream=stream)
        tdc.eig(d, e, osd, ws=wss, lam=lam, Q=Q, stream=stream)
        ss = tdc.get_stats()
        del wss
        compare["structured"] = ss["phase_ms"]["total"] / 1e3
        progress("structured merge done")
        sfl = float(ss["struct_flops"])
        kept = max(1, ss["lr_tiles"] - ss["lr_dense_fallbacks"])
        compare_detail["structured"] = {
            "s": compare["structured"], "test_ratios": accuracy(),
            "options": {"lr_tile": osd.lr_tile, "structured_min_K": osd.structured_min_K, "lr_tol": osd.lr_tol,
                        "rank_cap": 64},
            "srrsc": {"far_tiles": ss["lr_tiles"], "mean_rank": ss["lr_rank_sum"] / kept,
                      "max_rank": ss["lr_rank_max"], "dense_fallbacks": ss["lr_dense_fallbacks"]},
            "gemm_fp64_ms": ss["phase_ms"]["gemm_fp64"],
            "roofline": {"bound": "alu",
                         "kernel": "k_gemm_dense (near-diagonal tiles) + k_struct_w + k_struct_apply (FP64)",
                         "executed_flops": sfl,
                         "achieved": sfl / (ss["phase_ms"]["gemm_fp64"] * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s",
                         "frac": sfl / (ss["phase_ms"]["gemm_fp64"] * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                         "peak_kind": "derived: 152 SMs x 2 DFMA/clk x 2.07 GHz",
                         "note": "executed flops only (the dense flops it avoids are not counted); the phase "
                                 "also holds the FP32 SRRSC pivot searches"}}
    if args.merge not in ("dense", "split") and not args.no_compare and n >= 4096:
        # the plain split product (every merge unstructured) on the tensor cores
        o3p = tdc.default_opts(leaf=leaf, merge_mode=tdc.MERGE_SPLIT, **kw)
        o3 = tdc.default_opts(leaf=leaf, merge_mode=tdc.MERGE_SPLIT, collect_stats=1, **kw)
        ws3 = tdc.workspace(tdc.workspace_size(n, o3p), dev)
        for _ in range(2):
            tdc.eig(d, e, o3p, ws=ws3, lam=lam, Q=Q, stream=stream)
        st3 = tdc.sync_status(stream)
        steps3 = max(1, min(args.steps, 10))
        ms3 = _event_ms(lambda: tdc.eig(d, e, o3p, ws=ws3, lam=lam, Q=Q, stream=stream), steps3, stream)
        tdc.eig(d, e, o3, ws=ws3, lam=lam, Q=Q, stream=stream)
        s3 = tdc.get_stats()
        del ws3
        compare["split"] = ms3 / 1e3
        compare_detail["split"] = {
            "s": ms3 / 1e3, "steps": steps3, "status": tdc.strerror(st3), "test_ratios": accuracy(),
            "split_level_max": s3["split_level_max"], "phase_ms": s3["phase_ms"],
            "roofline": split_roofline(s3, s3["phase_ms"]["split_mma"], o3p.split_slices, *peaks(),
                                       "; phase time of one instrumented solve")}
        progress("plain split merge done")
    if compare_detail:
        tdc.eig(d, e, opts, ws=wsb, lam=lam, Q=Q, stream=stream)  # leave the timed configuration's result
    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    d_h = torch.tensor(d_np).pin_memory()
    e_h = torch.tensor(e_np).pin_memory()
    lam_h = torch.empty(n, dtype=torch.float64).pin_memory()
    Q_h = torch.empty(n, n, dtype=torch.float64).pin_memory()
    d_d = torch.empty_like(d)
    e_d = torch.empty_like(e)
    # one untimed pass: the first copies through freshly pinned buffers map them
    d_d.copy_(d_h, non_blocking=True)
    e_d.copy_(e_h, non_blocking=True)
    tdc.eig(d_d, e_d, opts, ws=wsb, lam=lam, Q=Q, stream=stream)
    lam_h.copy_(lam, non_blocking=True)
    Q_h.copy_(Q.t(), non_blocking=True)
    torch.cuda.synchronize()
    ee0 = torch.cuda.Event(enable_timing=True)
    ee1 = torch.cuda.Event(enable_timing=True)
    e2e_steps = max(1, min(args.steps, 10))
    ee0.record(stream)
    for _ in range(e2e_steps):
        d_d.copy_(d_h, non_blocking=True)
        e_d.copy_(e_h, non_blocking=True)
        tdc.eig(d_d, e_d, opts, ws=wsb, lam=lam, Q=Q, stream=stream)
        lam_h.copy_(lam, non_blocking=True)
        Q_h.copy_(Q.t(), non_blocking=True)  # the storage of the column-major Q
    ee1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = ee0.elapsed_time(ee1) / e2e_steps
    progress("end-to-end done")
    if ws_n > 1:
        e2e_ms = max_over_ranks(e2e_ms, dist, dev)
    del d_h, e_h, lam_h, Q_h
    if rank != 0:
        if ws_n > 1:
            dist.destroy_process_group()
        return 0
    line = {
        "metric": METRIC,
        "value": job_seconds_per_solve(ms, ws_n),
        "unit": "s",
        "n_gpus": ws_n,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.merge == "dense" else "f64 (Q*U as bf16 digit products, fp32 accumulate)",
        "data": "synthetic",
        "config": {"workload": desc, "merge": args.merge, "split_chunk_k": opts.split_chunk_k,
                   "l2": "no flush: Q and workspace (%.1f GiB) exceed the 129 MB L2" % ((8 * n * n + wsb.numel()) / 2**30),
                   "parallelism": "replicas" if ws_n > 1 else "single"},
        "roofline": roof,
        "qu_tflops_fp64_equivalent": qu_tflops,
        "merge_compare_s": compare,
        "merge_compare": compare_detail,
        "instrumented_ms_per_step": ims,
        "phase_ms": stats["phase_ms"],
        "K_per_level": stats["sum_K"],
        "secular_iterations": {"mean": stats["secular_iter_mean"], "max": stats["secular_iter_max"]},
        "split_level_max": stats.get("split_level_max"),
        "structured": {"merge_parts_structured": stats.get("lr_parts_structured"),
                       "merge_parts_left_to_split": stats.get("lr_parts_split"),
                       "far_tiles": stats.get("lr_tiles"),
                       "mean_rank": stats["lr_rank_sum"] / max(1, stats["lr_tiles"] - stats["lr_dense_fallbacks"]),
                       "max_rank": stats.get("lr_rank_max"), "lr_tile": opts.lr_tile,
                       "structured_min_K": opts.structured_min_K, "lr_tol": opts.lr_tol},
        "device_status": tdc.strerror(st),
        "test_ratios": {"lam_err_over_normT": lam_err, "residual": res, "orthogonality": orth,
                        "sampled_columns": 256, "within_bounds": bool(res <= 50 and orth <= 50)},
        "gpu_launches": int(stats["launches"]) * args.steps,
        "clocks": clocks,
        "e2e": {"value": job_seconds_per_solve(e2e_ms, ws_n), "unit": "s", "h2d_bytes_per_step": 2 * 8 * n - 8,
                "d2h_bytes_per_step": 8 * n + 8 * n * n, "steps": e2e_steps},
    }
    if ws_n == 1 and args.workload == "toeplitz16384" and not args.no_configs:
        del wsb, Q, lam
        torch.cuda.empty_cache()
        cfg = {}
        for key, fn in (("c1_uniform1024", config_c1), ("c3_batched4096", config_c3), ("c4_split32768", config_c4),
                        ("c5_backward256x512", config_c5), ("dense_syevd4096", config_dense),
                        ("band_sbevd4096", config_band)):
            cfg[key] = fn(args)
            progress(key + " done")
        line["configs"] = cfg
    if not args.no_cpu_baseline and ws_n == 1:
        line["cpu_baseline"] = cpu_baseline(args.workload, budget_s=args.cpu_budget)
        progress("cpu baseline done")
    print(json.dumps(line), flush=True)
    if ws_n > 1:
        dist.destroy_process_group()
    return 0


def progress(msg):
    """One line on stderr per stage (the JSON line alone goes to stdout)."""
    print("bench: %s (%.1f s)" % (msg, time.perf_counter() - T_START), file=sys.stderr, flush=True)


T_START = time.perf_counter()


def main():
    faulthandler.enable()
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="toeplitz16384", choices=["toeplitz16384", "toeplitz4096", "uniform1024", "c4_32768", "qhat8192",
                                                          "example1_8192", "example1_16384", "example1_32768",
                                                          "batched4096", "backward256", "dense4096", "dense8192", "structured16384",
                                                          "clement30000", "band4096",
                                                          "hermite30000", "sht30000"])
    ap.add_argument("--merge", default="auto", choices=["dense", "auto", "structured", "split", "structured_split"])
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--leaf", type=int, default=0, help="leaf size (default: the workload's)")
    ap.add_argument("--batch", type=int, default=4096, help="problems of the batched workload (first ones of its sequence)")
    ap.add_argument("--split-min-k", type=int, default=0, help="smallest merge on the split path (default: library's)")
    ap.add_argument("--split-chunk-k", type=int, default=-1,
                    help="drain the split product's level sums every this many terms (multiple of 16; 0: once "
                         "per tile; default: the library's)")
    ap.add_argument("--bands", default="8,32", help="band4096 workload: half-bandwidths, comma-separated")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="default workload only: skip the other workloads")
    ap.add_argument("--cpu-budget", type=float, default=180.0,
                    help="seconds the CPU oracle may take on the full matrix before a scaled sample is used")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "qhat8192":
        return run_qhat(args)
    if args.workload.startswith("example1_"):
        print(json.dumps(run_example1(args, int(args.workload.split("_")[1]))), flush=True)
        return 0
    if args.workload == "batched4096":
        print(json.dumps(config_c3(args, steps=args.steps, warmup=args.warmup)), flush=True)
        return 0
    if args.workload == "backward256":
        print(json.dumps(config_c5(args, steps=args.steps, warmup=args.warmup)), flush=True)
        return 0
    if args.workload == "structured16384":
        print(json.dumps(run_structured_products(args, 16384)), flush=True)
        return 0
    if args.workload == "band4096":
        bws = tuple(int(x) for x in args.bands.split(","))
        print(json.dumps(config_band(args, bws=bws, steps=args.steps)), flush=True)
        return 0
    if args.workload.startswith("dense"):
        print(json.dumps(config_dense(args, n=int(args.workload[5:]), steps=args.steps)), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
