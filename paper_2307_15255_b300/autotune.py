"""Autotuner for a transfer: launch shapes, and filter size and blocking.

The scan kernel's best shape depends on the data: how large the incoming
filters turn out to be (they are sized on the device from survivor
counts), whether they fit the shared-memory budget, and how much L1 is
left for the filters that do not.  The tuner times the session's whole
transfer, replayed from a CUDA graph, under each candidate (threads per
CTA, shared-memory filter budget) and keeps the fastest.  Results are
cached in a JSON file keyed by the workload's shape (row counts, key
dtypes, join graph, filter parameters), so a later session on the same
shape reuses them without timing.

:func:`tune_filter` picks the filter parameters themselves -- bits per key
(the filter's size for a given survivor count), block bits (256 or 512)
and k -- by timing the same transfer under each candidate.  Unlike a launch
shape these change the filters and so the survivors (a smaller filter lets
more non-matching keys through, which the later visits then carry), so the
result is a configuration to create sessions with, not a setting applied
to an existing one; the transfer with it is checked like any other
configuration.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

import torch

from . import pt as _pt

DEFAULT_CANDIDATES: Tuple[Tuple[int, int, int], ...] = (
    (256, 40 * 1024, 0), (256, 24 * 1024, 0), (256, 64 * 1024, 0), (256, 0, 0),
    (128, 40 * 1024, 0), (128, 64 * 1024, 0),
)


def default_cache_path() -> str:
    return os.environ.get("PT_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "pt_autotune.json"))


def signature(session) -> str:
    """A stable key for the session's workload shape."""
    desc = {"n_rows": session.n_rows, "dtypes": session.col_dtypes,
            "edges": [[e[0], list(e[1]), e[2], list(e[3])] + list(e[4:]) for e in session.edges],
            "cfg": [session.bits_per_key, session.k, session.block_bits],
            "device": torch.cuda.get_device_name()}
    return hashlib.sha256(json.dumps(desc, sort_keys=True).encode()).hexdigest()[:24]


def _time_graph(session, warmup: int, runs: int) -> float:
    s = session.stream
    for _ in range(warmup):
        session.run()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(runs):
        session.run()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / runs


def tune(session, candidates: Optional[Iterable[Tuple[int, int, int]]] = None, warmup: int = 3, runs: int = 20,
         cache_path: Optional[str] = None, use_cache: bool = True) -> Dict[str, object]:
    """Pick the fastest launch shape for ``session`` and leave it applied.

    Returns {"launch": (threads, smem, ctas_per_sm), "ms": best time,
    "trials": [(launch, ms), ...], "cached": bool}.
    """
    path = cache_path or default_cache_path()
    key = signature(session)
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        launch = tuple(cache[key]["launch"])
        _pt.pt_set_launch(session.ctx, *launch)
        return {"launch": launch, "ms": cache[key]["ms"], "trials": [], "cached": True}

    _pt.pt_set_graph_mode(session.ctx, True)
    trials = []
    for launch in (candidates or DEFAULT_CANDIDATES):
        _pt.pt_set_launch(session.ctx, *launch)
        trials.append((tuple(launch), _time_graph(session, warmup, runs)))
    best = min(trials, key=lambda t: t[1])
    _pt.pt_set_launch(session.ctx, *best[0])
    _pt.pt_set_graph_mode(session.ctx, False)
    if use_cache:
        cache[key] = {"launch": list(best[0]), "ms": best[1]}
        try:
            os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
            with open(path + ".tmp", "w") as f:
                json.dump(cache, f, indent=1)
            os.replace(path + ".tmp", path)
        except OSError:
            pass
    return {"launch": best[0], "ms": best[1], "trials": trials, "cached": False}


# (bits per key, block bits, k)
FILTER_CANDIDATES: Tuple[Tuple[int, int, int], ...] = (
    (16, 256, 4), (12, 256, 4), (8, 256, 4), (16, 512, 4), (10, 512, 4), (16, 256, 5),
)


def tune_filter(tables, edges, seed: int = 0, candidates: Optional[Iterable[Tuple[int, int, int]]] = None,
                stream=None, launch_candidates: Optional[Sequence[Tuple[int, int, int]]] = None,
                first_probe: Optional[bool] = None, warmup: int = 2, runs: int = 5) -> Dict[str, object]:
    """Time the transfer of ``tables`` / ``edges`` (as for
    :class:`~paper_2307_15255_b300.session.TransferSession`) under each
    filter configuration (bits per key, block bits, k) and return the
    fastest: {"bits_per_key", "block_bits", "k", "launch", "ms", "trials"}.
    With ``launch_candidates``, each configuration also gets its best
    launch shape (:func:`tune`).  Each trial records the survivors left
    after both passes, summed over the tables."""
    from .session import TransferSession
    trials: List[Dict[str, object]] = []
    for bpk, block_bits, k in (candidates or FILTER_CANDIDATES):
        with TransferSession(tables, edges, bpk, k, block_bits, seed, stream=stream,
                             first_probe=first_probe) as s:
            launch = None
            if launch_candidates:
                launch = tune(s, launch_candidates, warmup=warmup, runs=runs, use_cache=False)["launch"]
            _pt.pt_set_graph_mode(s.ctx, True)
            ms = _time_graph(s, warmup, runs)
            survivors = sum(_pt.pt_get_survivors(s.ctx, v, None) for v in range(len(s.n_rows)))
            trials.append({"bits_per_key": bpk, "block_bits": block_bits, "k": k,
                           "launch": None if launch is None else list(launch), "ms": ms,
                           "survivors": survivors})
    best = min(trials, key=lambda t: t["ms"])
    return {"bits_per_key": best["bits_per_key"], "block_bits": best["block_bits"], "k": best["k"],
            "launch": best["launch"], "ms": best["ms"], "trials": trials}
