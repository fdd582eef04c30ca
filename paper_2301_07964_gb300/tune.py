"""Measured launch parameters: q, the number of sweeps grouped per generate/apply iteration
of stage 2 (Section "Blocked stage two"; 1 <= q <= r), the tile shape of the emulated delayed
updates, stage 1's p (the p r x p r blocks of Alg. 1) and the batched launch's shape (p and
persistent blocks per SM).

The paper fixes such parameters for its CPUs. On a GPU the best values depend on the update
mode and on n: a larger q means fewer groups, so fewer delayed-update launches and fewer
passes over A, B, Q and Z, but a longer wavefront lag inside each chase launch; smaller update
tiles shorten the chain of windows the next chase waits for but run more tiles. So they are
measured:
- each candidate runs the public call on the caller's device, on a seeded synthetic input of
  the same size, timed with CUDA events on the calling stream;
- several parameters are searched one at a time (coordinate search: each in turn over its
  candidates with the others held at their current best);
- the fastest wins; ties within 1 % go to the value that launches less work (the larger q,
  the library's default tile and p, the full persistent grid);
- the choice is cached per device name and workload.

Only the public entry points are called; nothing here computes any part of the reduction.
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


def choose(times: Dict, tie: float = 0.01, prefer=max):
    """The fastest key; among those within `tie` of the fastest, prefer(...) of them (the
    largest by default)."""
    best = min(times.values())
    return prefer(k for k, t in times.items() if t <= best * (1.0 + tie))


def tile_candidates(r: int, mode: int) -> list:
    """Update tile heights tried: the tensor-core kernel's 64 lines and the warp-level kernel's
    32 where the emulated look-ahead path takes either (r = 16), else the library's choice."""
    return [32, 64] if (mode == b.HTS_GEMM_EMU_BF16 and r == 16) else [0]


def p_candidates(r: int, limit: int) -> list:
    """Block counts p tried for stage 1 (limit 128) or the batched kernel (limit 64): 2, 4 and
    8 where p r fits the limit."""
    return [p for p in (2, 4, 8) if p * r <= limit]


def batch_shape_candidates() -> list:
    """Persistent blocks per SM tried for the batched launch (0: as many as fit)."""
    return [0, 1, 2]


def default_then_largest(values):
    """Tie preference for p: 0 (the library's per-pencil default) first, else the largest."""
    values = list(values)
    return 0 if 0 in values else max(values)


def coordinate_search(run: Callable[[dict], float], start: dict, axes: list, reps: int = 2,
                      warmup: int = 1, tie: float = 0.01):
    """Minimise run(config) one parameter at a time.  axes: (name, candidates, prefer) in the
    order searched; start: the configuration the first axis is searched from.  Returns the best
    configuration and the times of every configuration run (keyed by a sorted tuple of items)."""
    best = dict(start)
    seen: Dict[tuple, float] = {}

    def timed(cfg: dict) -> float:
        key = tuple(sorted(cfg.items()))
        if key not in seen:
            seen[key] = measure(lambda _k: run(cfg), [key], reps=reps, warmup=warmup)[key]
        return seen[key]

    for name, cands, prefer in axes:
        times = {v: timed(dict(best, **{name: v})) for v in cands}
        best[name] = choose(times, tie, prefer)
    return best, seen


def _label(key: tuple) -> str:
    return ",".join("%s=%s" % kv for kv in key)


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


def store_cache(path: str, key: str, q, times: Dict) -> None:
    """Record a choice: q an int (the q of stage 2) or a dict of parameters; times keyed by
    the values or configurations measured."""
    data = load_cache(path)
    entry = dict(q) if isinstance(q, dict) else {"q": int(q)}
    entry["ms"] = {(_label(k) if isinstance(k, tuple) else str(k)): float(v) for k, v in sorted(times.items())}
    data[key] = entry
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _timer(red, stream, call, what: str) -> float:
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    call()
    e1.record(stream)
    e1.synchronize()
    st, info = red.sync_status(stream)
    if st != b.HTS_OK:
        raise b.HTSError(st, "%s (info %s)" % (what, info))
    return e0.elapsed_time(e1)


def tuned_stage2(red, n: int, r: int, mode: int = b.HTS_GEMM_EMU_BF16, seed: int = 0,
                 cache_path: Optional[str] = None, reps: int = 2, retune: bool = False) -> dict:
    """The measured {"q", "tile_m"} for stage 2 of an n x n pencil with r subdiagonals in
    `mode` on the device of the Reducer `red`: q first (library tile), then the tile at that q
    (cached; `retune` measures again).  "ms" holds the times per configuration."""
    import torch

    from .device import colmajor_empty, to_device
    from .inputs import random_rht_pencil

    path = cache_path or default_cache_path()
    key = _key(torch.cuda.get_device_name(red.device), n, r, mode)
    tiles = tile_candidates(r, mode)
    if not retune:
        hit = load_cache(path).get(key)
        if hit and isinstance(hit.get("q"), int) and 1 <= hit["q"] <= r and hit.get("tile_m", 0) in tiles + [0]:
            return {"q": hit["q"], "tile_m": hit.get("tile_m", 0), "ms": hit.get("ms", {})}
    A, B = random_rht_pencil(n, r, seed)
    A0, B0 = to_device(A), to_device(B)
    dA, dB, dQ, dZ = colmajor_empty(n), colmajor_empty(n), colmajor_empty(n), colmajor_empty(n)
    stream = torch.cuda.current_stream()

    def run(cfg: dict) -> float:
        dA.copy_(A0)
        dB.copy_(B0)
        return _timer(red, stream, lambda: red.stage2(dA, dB, r, dQ, dZ, compq=b.HTS_COMP_INIT,
                                                      compz=b.HTS_COMP_INIT, q=cfg["q"], mode=mode,
                                                      stream=stream, tile_m=cfg["tile_m"]),
                      "stage 2 while tuning %s" % cfg)

    best, seen = coordinate_search(run, {"q": r, "tile_m": 0},
                                   [("q", candidates(r), max), ("tile_m", tiles, max)], reps=reps)
    choice = {"q": int(best["q"]), "tile_m": int(best["tile_m"])}
    store_cache(path, key, choice, seen)
    return dict(choice, ms={_label(k): v for k, v in seen.items()})


def tuned_q(red, n: int, r: int, mode: int = b.HTS_GEMM_EMU_BF16, seed: int = 0,
            cache_path: Optional[str] = None, reps: int = 2, retune: bool = False) -> int:
    """The measured q for stage 2 of an n x n pencil with r subdiagonals in `mode` on the
    device of the Reducer `red` (the q of tuned_stage2)."""
    return tuned_stage2(red, n, r, mode, seed, cache_path, reps, retune)["q"]


def tuned_stage1_p(red, n: int, r: int, mode: int = b.HTS_GEMM_EMU_BF16, seed: int = 0,
                   cache_path: Optional[str] = None, reps: int = 1, retune: bool = False) -> int:
    """The measured p of stage 1 (Alg. 1) for the full reduction of a dense n x n pencil with
    r subdiagonals, timed through hts_reduce (stage 2 in `mode`, the same for every p)."""
    import torch

    from .device import colmajor_empty, to_device
    from .inputs import random_pencil

    path = cache_path or default_cache_path()
    key = "stage1|" + _key(torch.cuda.get_device_name(red.device), n, r, mode)
    cands = p_candidates(r, 128)
    if not retune:
        hit = load_cache(path).get(key)
        if hit and hit.get("p") in cands:
            return hit["p"]
    A, B = random_pencil(n, seed)
    A0, B0 = to_device(A), to_device(B)
    dA, dB, dQ, dZ = colmajor_empty(n), colmajor_empty(n), colmajor_empty(n), colmajor_empty(n)
    stream = torch.cuda.current_stream()

    def run(cfg: dict) -> float:
        dA.copy_(A0)
        dB.copy_(B0)
        return _timer(red, stream, lambda: red.reduce(dA, dB, r, dQ, dZ, compq=b.HTS_COMP_INIT,
                                                      compz=b.HTS_COMP_INIT, p=cfg["p"], mode=mode,
                                                      stream=stream),
                      "full reduction while tuning %s" % cfg)

    best, seen = coordinate_search(run, {"p": max(cands)}, [("p", cands, max)], reps=reps, warmup=0)
    store_cache(path, key, {"p": int(best["p"])}, seen)
    return int(best["p"])


def tuned_batch(red, ns: list, rs: list, seed: int = 0, cache_path: Optional[str] = None, reps: int = 2,
                retune: bool = False) -> dict:
    """The measured {"p", "tile_n"} (stage 1's p and the persistent blocks per SM) of the
    batched reduction of pencils of sizes ns with rs subdiagonals: blocks per SM first (the
    default p), then p (cached under the batch's sizes)."""
    import hashlib

    import torch

    from .device import colmajor_empty

    path = cache_path or default_cache_path()
    sig = hashlib.sha1(json.dumps([list(map(int, ns)), list(map(int, rs))]).encode()).hexdigest()[:16]
    key = "batch|%s|count=%d|%s" % (torch.cuda.get_device_name(red.device), len(ns), sig)
    pc = p_candidates(max(rs), 64) + [0]
    if not retune:
        hit = load_cache(path).get(key)
        if hit and hit.get("p") in pc and hit.get("tile_n") in batch_shape_candidates():
            return {"p": hit["p"], "tile_n": hit["tile_n"], "ms": hit.get("ms", {})}
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    A0 = [torch.randn(n, n, dtype=torch.float64, device="cuda", generator=gen).t() for n in ns]
    B0 = [torch.randn(n, n, dtype=torch.float64, device="cuda", generator=gen).t() for n in ns]
    dA = [colmajor_empty(n) for n in ns]
    dB = [colmajor_empty(n) for n in ns]
    dQ = [colmajor_empty(n) for n in ns]
    dZ = [colmajor_empty(n) for n in ns]
    nbytes = b.hts_workspace_size_batched(ns, rs)
    work = torch.empty(max(256, nbytes), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def run(cfg: dict) -> float:
        for x, y in zip(dA, A0):
            x.copy_(y)
        for x, y in zip(dB, B0):
            x.copy_(y)
        params = {"p": cfg["p"], "tile_n": cfg["tile_n"]}

        def call():
            st = b.hts_reduce_batched(red.ctx, ns, rs, dA, ns, dB, ns, b.HTS_COMP_INIT, dQ, ns, b.HTS_COMP_INIT, dZ,
                                      ns, b.HTS_GEMM_FP64, params, work, work.numel(), stream)
            if st != b.HTS_OK:
                raise b.HTSError(st, "batched reduction while tuning %s" % cfg)
        return _timer(red, stream, call, "batched reduction while tuning %s" % cfg)

    best, seen = coordinate_search(run, {"p": 0, "tile_n": 0},
                                   [("tile_n", batch_shape_candidates(), min), ("p", pc, default_then_largest)],
                                   reps=reps)
    choice = {"p": int(best["p"]), "tile_n": int(best["tile_n"])}
    store_cache(path, key, choice, seen)
    return dict(choice, ms={_label(k): v for k, v in seen.items()})
