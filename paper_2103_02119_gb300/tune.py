"""Launch-shape tuning with a JSON cache (library plumbing; the paper has no
tuner).

The single-lattice step kernel takes a block width (32, 64, 128 or 256
threads, two cells each) and a number of row bands; the batch kernel takes a
block width and rows per band.  A tuner times candidate shapes on the GPU and
keeps the fastest; the result goes to a JSON cache keyed by (nx, ny,
precision, layout, mask) -- for a batch, by its multiset of lattice sizes --
so that a later run of the same size takes the shape without measuring.
The shape changes only the work split: every shape gives the same states,
bit for bit.

Cache file: $LBM_TUNE_CACHE, else ~/.cache/paper_2103_02119_gb300/tune.json.
"""
from __future__ import annotations

import hashlib
import json
import os
import tempfile

LAYOUT = "soa9-pull"     # nine planes [9][ny][pitch], two buffers, pull streaming
BLOCK_X = (32, 64, 128, 256)
CELLS_PER_THREAD = 2


def cache_path() -> str:
    p = os.environ.get("LBM_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_2103_02119_gb300", "tune.json")


def load_cache(path: str) -> dict:
    """The cache's entries; an absent or unreadable file is an empty cache."""
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, cache: dict) -> None:
    """Writes the whole cache atomically (a temporary file, then a rename)."""
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(os.path.abspath(path)), suffix=".tmp")
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def lattice_key(nx: int, ny: int, precision: int, masked: bool) -> str:
    return f"lattice:{nx}x{ny}:fp{precision}:{LAYOUT}:{'mask' if masked else 'nomask'}"


def batch_key(sizes, precision: int = 32) -> str:
    """Key of a batch: its lattice sizes as a multiset (order-free)."""
    s = sorted((int(nx), int(ny)) for nx, ny in sizes)
    h = hashlib.sha1(json.dumps(s).encode()).hexdigest()[:16]
    return f"batch:{len(s)}:fp{precision}:{LAYOUT}:{h}"


def lattice_candidates(nx: int, ny: int):
    """(block_x, bands) pairs: block widths whose segment is not much wider
    than the lattice, and the automatic band count (0) with a few fixed
    band heights."""
    bxs = [b for b in BLOCK_X if b * CELLS_PER_THREAD <= max(2 * nx, 64)] or [BLOCK_X[0]]
    bands = [0] + sorted({max(1, ny // r) for r in (4, 7, 14, 28, 56)})
    return [(b, n) for b in bxs for n in bands]


def choose(key: str, candidates, measure, path: str | None = None, force: bool = False):
    """The cached shape of `key`, or the candidate with the smallest
    measure(candidate) (milliseconds), which is then cached."""
    path = path or cache_path()
    cache = load_cache(path)
    if not force and key in cache:
        return tuple(cache[key]["shape"])
    times = {tuple(c): float(measure(tuple(c))) for c in candidates}
    best = min(times, key=times.get)
    cache = load_cache(path)          # another process may have written meanwhile
    cache[key] = {"shape": list(best), "ms_per_step": times[best], "candidates": len(times)}
    save_cache(path, cache)
    return best


def measure_lattice(wl, precision: int, shape, steps: int = 20, warmup: int = 3) -> float:
    """Milliseconds per step of the workload's lattice with launch shape
    (block_x, bands), from a seeded developed state, timed with CUDA events."""
    import torch

    from . import workloads as W
    from .lbm import Lattice, lbm_set_small_path
    r, u, v = W.smooth_random_fields(wl.nx, wl.ny, 1, u_amp=0.02, rho_amp=2e-3)
    stream = torch.cuda.current_stream()
    lat = Lattice.from_workload(wl.with_(rho=r, ux=u, uy=v), precision=precision, stream=stream,
                                block_x=shape[0], bands=shape[1])
    try:
        if wl.nx * wl.ny <= 4096:
            lbm_set_small_path(lat.h, False)     # the row-band kernel's shape is tuned
        lat.step(warmup)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            lat.step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps
    finally:
        lat.close()


def tune_lattice(wl, precision: int = 32, path: str | None = None, force: bool = False,
                 steps: int = 20):
    """(block_x, bands) for the workload's lattice size, from the cache or
    measured."""
    key = lattice_key(wl.nx, wl.ny, precision, wl.mask is not None)
    return choose(key, lattice_candidates(wl.nx, wl.ny),
                  lambda s: measure_lattice(wl, precision, s, steps=steps), path, force)


def tuned_lattice(wl, precision: int = 32, stream=None, path: str | None = None, **kw):
    """A Lattice of the workload with the tuned launch shape."""
    from .lbm import Lattice
    bx, nb = tune_lattice(wl, precision, path)
    return Lattice.from_workload(wl, precision=precision, stream=stream, block_x=bx, bands=nb,
                                 **kw)


def tune_batch(batch, workloads, path: str | None = None, force: bool = False,
               trial_steps: int = 20):
    """Sets the batch's (block_x, rows per band) from the cache, or from the
    library's own sweep (lbm_batch_tune), which is then cached."""
    key = batch_key([(w.nx, w.ny) for w in workloads])
    path = path or cache_path()
    cache = load_cache(path)
    if not force and key in cache:
        shape = tuple(cache[key]["shape"])
        batch.set_shape(*shape)
        return shape
    shape = tuple(int(v) for v in batch.tune(trial_steps))
    cache = load_cache(path)
    cache[key] = {"shape": list(shape), "trial_steps": trial_steps}
    save_cache(path, cache)
    return shape
