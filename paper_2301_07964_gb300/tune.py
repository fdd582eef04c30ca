"""Measured choice of q, the number of sweeps grouped per generate/apply iteration of stage 2
(Section "Blocked stage two"; 1 <= q <= r).

The paper fixes q for its CPUs. On a GPU the best q depends on the update mode and on n: a
larger q means fewer groups, so fewer delayed-update launches and fewer passes over A, B, Q
and Z, but a longer wavefront lag inside each chase launch. So q is measured:
- each candidate runs the public stage-2 call on the caller's device, on a seeded synthetic
  r-HT pencil of the same n, timed with CUDA events on the calling stream;
- the fastest wins; ties within 1 % go to the larger q, which launches fewer groups;
- the choice is cached per device name, n, r and mode.

Only the public entry point is called; nothing here computes any part of the reduction.
"""
from __future__ import annotations

import json
import os
from typing import Callable, Dict, Iterable, Optional

from . import binding as b


def candidates(r: int) -> list:
    """The q values tried: quarters of r (at least 1) and r itself."""
    return sorted({max(1, r // 4), max(1, r // 2), max(1, (3 * r) // 4), r})


def measure(run: Callable[[int], float], qs: Iterable[int], reps: int = 2, warmup: int = 1) -> Dict[int, float]:
    """run(q) returns the milliseconds of one call; each q keeps its fastest of `reps` timed
    calls after `warmup` untimed ones."""
    times = {}
    for q in qs:
        for _ in range(warmup):
            run(q)
        times[q] = min(run(q) for _ in range(reps))
    return times


def choose(times: Dict[int, float], tie: float = 0.01) -> int:
    """The fastest q; among those within `tie` of the fastest, the largest."""
    best = min(times.values())
    return max(q for q, t in times.items() if t <= best * (1.0 + tie))


def default_cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "hts_tune.json")


def _key(device_name: str, n: int, r: int, mode: int) -> str:
    return "%s|n=%d|r=%d|mode=%d" % (device_name, n, r, mode)


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(path: str, key: str, q: int, times: Dict[int, float]) -> None:
    data = load_cache(path)
    data[key] = {"q": int(q), "ms": {str(k): float(v) for k, v in sorted(times.items())}}
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tuned_q(red, n: int, r: int, mode: int = b.HTS_GEMM_EMU_BF16, seed: int = 0,
            cache_path: Optional[str] = None, reps: int = 2, retune: bool = False) -> int:
    """The measured q for stage 2 of an n x n pencil with r subdiagonals in `mode` on the
    device of the Reducer `red` (cached; `retune` measures again)."""
    import torch

    from .device import colmajor_empty, to_device
    from .inputs import random_rht_pencil

    path = cache_path or default_cache_path()
    key = _key(torch.cuda.get_device_name(red.device), n, r, mode)
    if not retune:
        hit = load_cache(path).get(key)
        if hit and isinstance(hit.get("q"), int) and 1 <= hit["q"] <= r:
            return hit["q"]
    A, B = random_rht_pencil(n, r, seed)
    A0, B0 = to_device(A), to_device(B)
    dA, dB, dQ, dZ = colmajor_empty(n), colmajor_empty(n), colmajor_empty(n), colmajor_empty(n)
    stream = torch.cuda.current_stream()

    def run(q: int) -> float:
        dA.copy_(A0)
        dB.copy_(B0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        red.stage2(dA, dB, r, dQ, dZ, compq=b.HTS_COMP_INIT, compz=b.HTS_COMP_INIT, q=q, mode=mode,
                   stream=stream)
        e1.record(stream)
        e1.synchronize()
        st, info = red.sync_status(stream)
        if st != b.HTS_OK:
            raise b.HTSError(st, "stage 2 while tuning q=%d (info %s)" % (q, info))
        return e0.elapsed_time(e1)

    times = measure(run, candidates(r), reps=reps)
    q = choose(times)
    store_cache(path, key, q, times)
    return q
