"""Oracle solves of every colony of a named workload in a pool of spawned processes (test
infrastructure). Each worker builds the workload once and then solves the colonies it is handed. Only a
SHA-256 digest of each final pheromone table comes back, not the table itself. Spawned workers inherit
no CUDA state, so the pool may start before or after the first GPU call."""
from __future__ import annotations

import hashlib
import multiprocessing as mp
import os

import numpy as np

_WL = None
_ONET = None


def _make(name):
    from paper_2010_14244_gb300 import workloads as W

    return {"grid64": W.grid64, "geo100k": W.geo100k, "city_batch": W.city_batch}[name]()


def _init(name):
    global _WL, _ONET
    _WL = _make(name)
    _ONET = {}


def _solve(item):
    """item: a colony index, or (graph, colony) for a list of workloads such as city_batch."""
    from oracle import oracle as orc

    g, qi = item if isinstance(item, tuple) else (None, item)
    wl = _WL if g is None else _WL[g]
    if g not in _ONET:
        _ONET[g] = orc.Net.from_workload(wl)
    o = orc.solve(_ONET[g], orc.Params(), wl.queries[qi], want_tau=True)
    o["tau_sha256"] = tau_digest(o.pop("tau"))
    return item, o


def tau_digest(tau) -> str:
    return hashlib.sha256(np.ascontiguousarray(tau, np.uint64).tobytes()).hexdigest()


def start(name: str, indices, processes: int | None = None):
    """Start solving colonies `indices` of workload `name` (for city_batch: (graph, colony) pairs);
    returns (pool, pending). pending.get() gives [(index, oracle result)] in the order of `indices`."""
    indices = list(indices)
    n = processes or max(1, min(len(indices), os.cpu_count() or 1))
    pool = mp.get_context("spawn").Pool(n, initializer=_init, initargs=(name,))
    return pool, pool.map_async(_solve, indices, chunksize=max(1, len(indices) // (4 * n)))


def check(gres, o, pheromone=None):
    """One colony: the GPU result (and its pheromone table, if given) equal to the oracle's."""
    assert gres["status"] == o["status"], (gres["status"], o["status"])
    for k in ("travel_ms", "wait_ms", "ant_steps", "n_success", "route_len"):
        assert gres[k] == o[k], (k, gres[k], o[k])
    if o["status"] == 0:
        assert gres["best_iter"] == o["best_iter"] and gres["best_ant"] == o["best_ant"]
        np.testing.assert_array_equal(gres["route"], o["route"])
    if pheromone is not None:
        assert tau_digest(pheromone) == o["tau_sha256"]
