"""Autotune cache: the sweep counts (nu1, nu2), inner V-cycles per
refinement step, refinement-pass tile (ir_zchunk) and staged half-sweep
planes per CTA (sweep_zchunk) that mg_autotune picked for a problem
signature, stored as
JSON keyed by device name and problem signature so that later runs on the
same device and problem class skip the search."""
import json
import os

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "gb300_mg_autotune.json")


def signature(device, shape, has_eps, has_mask, precision, tol):
    nz, ny, nx = shape
    return (f"{device}|{nx}x{ny}x{nz}|eps={int(bool(has_eps))}|mask={int(bool(has_mask))}"
            f"|prec={int(precision)}|tol={tol:.0e}")


def load(path):
    try:
        with open(path) as fh:
            data = json.load(fh)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store(path, key, entry):
    data = load(path)
    data[key] = entry
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tuned(solver, rho, S, kappa, tol=1e-10, has_eps=False, has_mask=False, precision=1,
          cache_path=DEFAULT_CACHE, device=None):
    """Install tuned options on `solver` (from the cache, else by running
    mg_autotune on this problem).  Returns (options dict, from_cache)."""
    if device is None:
        import torch

        device = torch.cuda.get_device_name()
    key = signature(device, solver.shape, has_eps, has_mask, precision, tol)
    entry = load(cache_path).get(key)
    if entry:
        solver.set_options(nu1=entry["nu1"], nu2=entry["nu2"], inner_cycles=entry["inner_cycles"],
                           ir_zchunk=entry.get("ir_zchunk", 0),
                           sweep_zchunk=entry.get("sweep_zchunk", 0))
        return entry, True
    opts, ms = solver.autotune(rho, S, kappa, tol)
    entry = dict(opts, ms=ms)
    store(cache_path, key, entry)
    return entry, False
