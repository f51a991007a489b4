"""Autotuner of the degree-bin and segment thresholds (sclap_set_tuning).

The thresholds only route rows (by their number of entries) and contested
target segments (by their number of proposals) between kernel paths that
compute the same selection and arbitration, so every setting gives the same
partition; they change the speed.  For one device and one workload graph the
tuner times candidate settings with CUDA events, either on the level-0 SCLaP
sweeps (the clustering and refinement rounds) or on one whole multilevel
partition, checks that all candidates return the same labels or partition,
keeps the fastest, applies it and caches it as JSON keyed by the device name
and a signature of the graph and the run parameters.
"""
from __future__ import annotations

import hashlib
import json
import os

import torch

from . import get_tuning, set_tuning, set_validation, sclap_cluster, sclap_refine

# (small_max, med_max, mid_max, seg_smem); the first is the built-in default
CANDIDATES = [
    (32, 256, 2048, 6144),
    (16, 256, 2048, 6144),
    (8, 256, 2048, 6144),
    (32, 128, 2048, 6144),
    (32, 256, 1024, 6144),
    (32, 256, 4096, 6144),
    (16, 256, 4096, 6144),
    (32, 256, 2048, 2048),
    (16, 128, 1024, 4096),
]

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build",
                             "tuning.json")


def signature(g: dict, k: int, eps: float, cluster_rounds: int, refine_rounds: int,
              subrounds: int, ml_params: dict | None = None) -> str:
    """Graph size, degree profile and run parameters, hashed."""
    deg = (g["xadj"][1:] - g["xadj"][:-1]).to(torch.int64)
    hist = torch.bincount(torch.clamp(torch.log2(deg.clamp(min=1).double()).to(torch.int64),
                                      max=40), minlength=41)
    key = (int(g["vwgt"].numel()), int(g["adjncy"].numel()), hist.cpu().tolist(), k, eps,
           cluster_rounds, refine_rounds, subrounds,
           sorted(ml_params.items()) if ml_params else None)
    return hashlib.sha256(repr(key).encode()).hexdigest()[:16]


def _device_name() -> str:
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _sweeps(g, k, eps, cluster_rounds, refine_rounds, subrounds, seed, p0):
    n = g["vwgt"].numel()
    U = max(int(g["vwgt"].max()), int(g["vwgt"].sum()) // (10 * k))
    lab, _ = sclap_cluster(g, U, cluster_rounds, subrounds, seed)
    part = sclap_refine(g, k, eps, refine_rounds, subrounds, seed, p0)[0]
    return lab, part


def _multilevel(g, ml_params):
    from . import partition_multilevel
    return (partition_multilevel(g, ml_params)[0],)


def autotune(g: dict, k: int, eps: float = 0.03, cluster_rounds: int = 3,
             refine_rounds: int = 6, subrounds: int = 4, seed: int = 1, candidates=None,
             reps: int = 2, cache: str | None = DEFAULT_CACHE,
             ml_params: dict | None = None) -> dict:
    """Times every candidate, applies the fastest and returns {"best", "ms",
    "identical", "signature", "device"}; with `cache`, stores the result.
    The timed work is the level-0 sweeps, or with `ml_params` one multilevel
    partition of g with those parameters (the whole call a user makes)."""
    from . import inputs as I
    candidates = list(candidates or CANDIDATES)
    dev = g["xadj"].device
    n = g["vwgt"].numel()
    p0 = I.rand_below(seed, 7, torch.arange(n, device=dev), k).to(torch.int32)
    old_val = set_validation(False)
    start = get_tuning()
    times, ref, identical = {}, None, True
    try:
        for cand in candidates:
            set_tuning(*cand)
            out = (_multilevel(g, ml_params) if ml_params else
                   _sweeps(g, k, eps, cluster_rounds, refine_rounds, subrounds, seed, p0))
            if ref is None:
                ref = out
            else:
                identical &= all(torch.equal(a, b) for a, b in zip(ref, out))
            torch.cuda.synchronize(dev)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record()
            for _ in range(reps):
                if ml_params:
                    _multilevel(g, ml_params)
                else:
                    _sweeps(g, k, eps, cluster_rounds, refine_rounds, subrounds, seed, p0)
            ev1.record()
            torch.cuda.synchronize(dev)
            times[cand] = ev0.elapsed_time(ev1) / reps
    finally:
        set_validation(old_val)
    best = min(times, key=times.get)
    if identical:
        set_tuning(*best)
    else:  # never expected: keep the previous setting and report it
        set_tuning(**start)
    res = {"best": dict(zip(("small_max", "med_max", "mid_max", "seg_smem"), best)),
           "ms": {"/".join(map(str, c)): round(t, 3) for c, t in times.items()},
           "identical": identical, "device": _device_name(),
           "signature": signature(g, k, eps, cluster_rounds, refine_rounds, subrounds, ml_params),
           "workload": "multilevel" if ml_params else "level-0 sweeps"}
    if cache and identical:
        data = {}
        if os.path.exists(cache):
            try:
                with open(cache) as f:
                    data = json.load(f)
            except (OSError, ValueError):
                data = {}
        data[f"{res['device']}|{res['signature']}"] = res
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tmp = cache + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1)
        os.replace(tmp, cache)
    return res


def load_or_tune(g: dict, k: int, eps: float = 0.03, cluster_rounds: int = 3,
                 refine_rounds: int = 6, subrounds: int = 4, seed: int = 1,
                 cache: str = DEFAULT_CACHE, ml_params: dict | None = None) -> dict:
    """Applies the cached setting for this device and graph, or tunes (and
    caches) one.  Returns the entry with "cached" set accordingly."""
    sig = signature(g, k, eps, cluster_rounds, refine_rounds, subrounds, ml_params)
    key = f"{_device_name()}|{sig}"
    if os.path.exists(cache):
        try:
            with open(cache) as f:
                entry = json.load(f).get(key)
        except (OSError, ValueError):
            entry = None
        if entry and entry.get("identical"):
            set_tuning(**entry["best"])
            return dict(entry, cached=True)
    return dict(autotune(g, k, eps, cluster_rounds, refine_rounds, subrounds, seed,
                         cache=cache, ml_params=ml_params), cached=False)
