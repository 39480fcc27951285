"""Autotuner for the runtime knobs of the solver: leaf size and the size above which
merges run on the split (tensor-core) path.

Candidates are timed with CUDA events on a representative input (a sample of the
batch, or the matrix itself), best of a few repetitions after a warm-up, and the
winner is cached in a JSON file keyed by (workload kind, size bucket, merge mode)
so that later calls skip the search.  Only the library's own entry points run.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import torch

from . import tdc

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "tdc_autotune.json")
LEAVES = (8, 16, 32, 48, 64)
SPLIT_MIN_K = (64, 128, 256, 512)


def _bucket(n: int) -> int:
    return 1 << max(0, int(np.ceil(np.log2(max(int(n), 1)))))


def _load(path):
    try:
        return json.load(open(path))
    except Exception:
        return {}


def _save(path, cache):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".%d.tmp" % os.getpid()
    json.dump(cache, open(tmp, "w"), indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time(fn, reps=3):
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune_batched(sizes, d: torch.Tensor, e: torch.Tensor, off_de, merge_mode=tdc.MERGE_AUTO,
                 sample: int = 256, cache_path: str | None = DEFAULT_CACHE, seed: int = 0, verbose=False):
    """Options for tdc_eig_batched on problems of the given sizes (d, e on the device,
    problem b at off_de[b]).  Tunes on `sample` problems drawn from the batch."""
    sizes = np.asarray(sizes, dtype=np.int64)
    key = "batched:%d:%d:%d" % (_bucket(int(sizes.max())), _bucket(len(sizes)), merge_mode)
    cache = _load(cache_path) if cache_path else {}
    if key in cache:
        c = cache[key]
        return tdc.default_opts(leaf=c["leaf"], merge_mode=merge_mode, split_min_K=c["split_min_K"])
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(len(sizes), min(sample, len(sizes)), replace=False))
    ss = sizes[pick]
    offs = np.zeros(len(ss) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(ss)
    qoffs = np.zeros(len(ss) + 1, dtype=np.int64)
    qoffs[1:] = np.cumsum(ss * ss)
    dev = d.device
    ds = torch.cat([d[int(off_de[b]):int(off_de[b]) + int(sizes[b])] for b in pick])
    es = torch.zeros_like(ds)
    for k, b in enumerate(pick):
        nb = int(sizes[b])
        es[int(offs[k]):int(offs[k]) + nb - 1] = e[int(off_de[b]):int(off_de[b]) + nb - 1]
    lam = torch.empty(int(offs[-1]), dtype=torch.float64, device=dev)
    Q = torch.empty(int(qoffs[-1]), dtype=torch.float64, device=dev)
    results = []
    for leaf in LEAVES:
        for smk in SPLIT_MIN_K if merge_mode in (tdc.MERGE_AUTO, tdc.MERGE_SPLIT) else (256,):
            o = tdc.default_opts(leaf=leaf, merge_mode=merge_mode, split_min_K=smk)
            ws = tdc.workspace(tdc.batched_workspace_size(ss, o), dev)
            t = _time(lambda: tdc.eig_batched(ss, ds, es, offs[:-1], qoffs[:-1], lam, Q, o, ws=ws))
            results.append((t, leaf, smk))
            del ws
    results.sort()
    t, leaf, smk = results[0]
    if verbose:
        print("autotune", key, "best leaf %d split_min_K %d: %.3f ms" % (leaf, smk, t))
    if cache_path:
        cache[key] = {"leaf": leaf, "split_min_K": smk, "ms_sample": t, "candidates": len(results)}
        _save(cache_path, cache)
    return tdc.default_opts(leaf=leaf, merge_mode=merge_mode, split_min_K=smk)


def tune_single(d: torch.Tensor, e: torch.Tensor, merge_mode=tdc.MERGE_AUTO, leaves=LEAVES, split_min_k=SPLIT_MIN_K,
                cache_path: str | None = DEFAULT_CACHE, verbose=False):
    """Options for tdc_eig on the tridiagonal (d, e) (device FP64): every (leaf,
    split_min_K) candidate timed on the matrix itself.  Cached under the order, the
    merge mode and a digest of the entries."""
    n = int(d.numel())
    h = hashlib.sha1(d.detach().cpu().numpy().tobytes() + e.detach().cpu().numpy().tobytes()).hexdigest()[:16]
    key = "single:%d:%d:%s" % (n, merge_mode, h)
    cache = _load(cache_path) if cache_path else {}
    if key in cache:
        c = cache[key]
        return tdc.default_opts(leaf=c["leaf"], merge_mode=merge_mode, split_min_K=c["split_min_K"])
    smks = split_min_k if merge_mode in (tdc.MERGE_AUTO, tdc.MERGE_SPLIT) else (128,)
    cands = [tdc.default_opts(leaf=lf, merge_mode=merge_mode, split_min_K=sk) for lf in leaves for sk in smks]
    ws = tdc.workspace(max(tdc.workspace_size(n, o) for o in cands), d.device)
    lam = torch.empty(n, dtype=torch.float64, device=d.device)
    Q = torch.empty(n, n, dtype=torch.float64, device=d.device).t()
    results = []
    for o in cands:
        t = _time(lambda: tdc.eig(d, e, o, ws=ws, lam=lam, Q=Q), reps=2)
        results.append((t, o.leaf, o.split_min_K))
    del ws, Q
    results.sort()
    t, leaf, smk = results[0]
    if verbose:
        print("autotune", key, "best leaf %d split_min_K %d: %.3f ms" % (leaf, smk, t))
    if cache_path:
        cache[key] = {"leaf": leaf, "split_min_K": smk, "ms": t, "candidates": len(results)}
        _save(cache_path, cache)
    return tdc.default_opts(leaf=leaf, merge_mode=merge_mode, split_min_K=smk)
