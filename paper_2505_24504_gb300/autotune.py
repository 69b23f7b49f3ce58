"""Launch-shape autotuner with a persisted cache.

`jfnk_autotune` (C ABI) times the tile choices of one context on the device:
threads per block of the DG face kernel, elements per DG volume block, threads
per block of the FV cell kernels and the level size below which FV levels run
four lanes per cell.  This module keys the winners by GPU name,
order, grid, viscosity, preconditioner precision and mg key, stores them in a
JSON file and applies them to the options of new contexts of the same shape.
The cache file
is $JFNK_TUNE_CACHE when set, else tune_cache.json in $XDG_CACHE_HOME/jfnk
(default ~/.cache/jfnk), never inside the package.
"""
from __future__ import annotations

import json
import os
import threading

from . import jfnk

_LOCK = threading.Lock()


def _default_cache() -> str:
    env = os.environ.get("JFNK_TUNE_CACHE")
    if env:
        return env
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "jfnk", "tune_cache.json")


DEFAULT_CACHE = _default_cache()


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def key_of(grid, k, phys, opts) -> str:
    return "|".join([_gpu_name(), f"k{k}", f"{grid.nx}x{grid.nz}", f"p{grid.periodic_x}",
                     "visc" if phys.mu != 0.0 else "euler", f"prec{opts.precond_prec}",
                     opts.mg_key.decode() if isinstance(opts.mg_key, bytes) else str(opts.mg_key)])


def load(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def save(cache: dict, path: str = DEFAULT_CACHE) -> None:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(opts, entry) -> None:
    opts.tile_faces = int(entry["tile_faces"])
    opts.tile_volume = int(entry["tile_volume"])
    opts.tile_fv = int(entry["tile_fv"])
    opts.fv_split_cells = int(entry.get("fv_split_cells", 0))


def tuned_context(grid, k, phys, opts, U, reps: int = 3, path: str = DEFAULT_CACHE, seed: int = 5):
    """A context whose launch shapes come from the cache, tuning on a miss at
    state U (device tensor) with a seeded random direction."""
    import torch
    key = key_of(grid, k, phys, opts)
    with _LOCK:
        cache = load(path)
        entry = cache.get(key)
    if entry is not None:
        apply(opts, entry)
        return jfnk.Context(grid, k, phys, opts), dict(entry, cached=True)
    ctx = jfnk.Context(grid, k, phys, opts)
    g = torch.Generator(device="cuda").manual_seed(seed)
    y = torch.randn(ctx.N, dtype=torch.float64, device="cuda", generator=g)
    entry = ctx.jfnk_autotune(U, y, reps=reps)
    torch.cuda.synchronize()
    apply(ctx.opts, entry)
    with _LOCK:
        cache = load(path)
        cache[key] = entry
        save(cache, path)
    return ctx, dict(entry, cached=False)


SCHEDULES = ("mg111111V", "mg112211V", "mg122211V", "mg131211V", "mg132211V", "mg132210V", "mg133211V",
             "mg123311V", "mg222211V", "mg133311V", "mg122222V", "mg001111V", "mg112222V")
SIGMA_FV = (0.7, 0.85, 1.0, 1.15)
SIGMA_DG = (0.7, 0.8, 0.9, 1.0, 1.3)


def schedule_key(grid, k, phys, opts, dt) -> str:
    return "|".join([_gpu_name(), "schedule", f"k{k}", f"{grid.nx}x{grid.nz}", f"p{grid.periodic_x}",
                     "visc" if phys.mu != 0.0 else "euler", f"prec{opts.precond_prec}", f"dt{dt:.6g}"])


def _trial(grid, k, phys, opts, U, dt, scheme, path):
    """Device time of one implicit step (after one untimed step) on a copy of U; None on failure."""
    import torch
    ctx, _ = tuned_context(grid, k, phys, opts, U, path=path)
    Uc = U.clone()
    try:
        st0 = ctx.implicit_step(Uc, dt, scheme=scheme, raise_on_error=False)
        if st0.status != 0:
            return None
        s = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        st = ctx.implicit_step(Uc, dt, scheme=scheme, raise_on_error=False)
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1) if st.status == 0 else None
    finally:
        ctx.close()
        del Uc


def tuned_schedule_context(grid, k, phys, opts, U, dt, scheme, candidates=SCHEDULES, path: str = DEFAULT_CACHE):
    """A context with the fastest preconditioner schedule for this shape and time
    step: the mg key among `candidates` (pseudo-time factors 1), then sigma_fv and
    sigma_dg by coordinate search.  One timed implicit step per trial on a copy of
    U; launch shapes tuned per key; everything cached.  The converged answer does
    not depend on these choices (the Newton tolerance decides it)."""
    import copy
    skey = schedule_key(grid, k, phys, opts, dt)
    with _LOCK:
        entry = load(path).get(skey)
    cached = entry is not None
    if entry is None:
        trials = {}

        def run(key, sfv, sdg):
            o = copy.copy(opts)
            o.mg_key = key.encode()
            o.sigma_fv = sfv
            o.sigma_dg = sdg
            t = _trial(grid, k, phys, o, U, dt, scheme, path)
            trials[f"{key}/{sfv}/{sdg}"] = t
            return t if t is not None else float("inf")

        best_key = min(candidates, key=lambda kk: run(kk, 1.0, 1.0))
        best_fv = min(SIGMA_FV, key=lambda sv: trials.get(f"{best_key}/{sv}/1.0") or run(best_key, sv, 1.0))
        best_dg = min(SIGMA_DG, key=lambda sd: trials.get(f"{best_key}/{best_fv}/{sd}") or run(best_key, best_fv, sd))
        entry = {"mg_key": best_key, "sigma_fv": best_fv, "sigma_dg": best_dg,
                 "trial_ms": {kk: v for kk, v in trials.items() if v is not None}}
        with _LOCK:
            cache = load(path)
            cache[skey] = entry
            save(cache, path)
    o = copy.copy(opts)
    o.mg_key = entry["mg_key"].encode()
    o.sigma_fv = entry["sigma_fv"]
    o.sigma_dg = entry["sigma_dg"]
    ctx, tiles = tuned_context(grid, k, phys, o, U, path=path)
    return ctx, dict(tiles, mg_key=entry["mg_key"], sigma_fv=entry["sigma_fv"], sigma_dg=entry["sigma_dg"],
                     schedule_trials_ms=entry["trial_ms"], schedule_cached=cached)
