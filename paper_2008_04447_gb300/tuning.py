"""Persistent cache of the batched kernel's tuned tile policies.

A tuned policy (rq_tune_batched) is stored in a JSON file under a key that
names the device and the batch's class: precision and the powers of two
bounding the problem count and the largest m, n and k.  Batches of the same
class reuse the policy without timing again.  Host bookkeeping only; the
tuning itself is the library's.
"""
from __future__ import annotations

import json
import os
import tempfile

__all__ = ["batch_key", "lookup", "store"]


def _pow2(x: int) -> int:
    """Smallest power of two >= x (1 for x <= 1)."""
    x = int(x)
    return 1 if x <= 1 else 1 << (x - 1).bit_length()


def batch_key(problems, prec: int, device_name: str, sm_count: int) -> str:
    """Key of a batch [(A, Omega, b, p, k), ...]: device, SM count, precision,
    and the powers of two bounding the count and the largest m, n, k."""
    mm = max(int(t[0].shape[0]) for t in problems)
    mn = max(int(t[0].shape[1]) for t in problems)
    mk = max(int(t[4]) for t in problems)
    return (f"{device_name}/sm{int(sm_count)}/prec{int(prec)}/count{_pow2(len(problems))}"
            f"/m{_pow2(mm)}/n{_pow2(mn)}/k{_pow2(mk)}")


def _read(path: str) -> dict:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def lookup(path: str, key: str):
    """The entry {"tiles": [m, n], "ms": t} stored under key, or None (also for
    a missing or unreadable file, or a malformed entry)."""
    e = _read(path).get(key)
    if not isinstance(e, dict):
        return None
    t = e.get("tiles")
    if not (isinstance(t, list) and len(t) == 2 and all(type(v) is int and v >= 0 for v in t)):
        return None
    return {"tiles": t, "ms": e.get("ms")}


def store(path: str, key: str, tiles, ms) -> None:
    """Adds or replaces key's entry; the file is replaced atomically, so a
    reader sees the old or the new contents, never a partial write.  Two
    processes storing at once each read, add and replace: the later replace
    wins and the other's new entry is lost (it is tuned again next time)."""
    d = _read(path)
    d[key] = {"tiles": [int(tiles[0]), int(tiles[1])], "ms": None if ms is None else float(ms)}
    folder = os.path.dirname(os.path.abspath(path))
    os.makedirs(folder, exist_ok=True)
    fd, tmp = tempfile.mkstemp(prefix=".tiles", dir=folder)
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.remove(tmp)
        raise
