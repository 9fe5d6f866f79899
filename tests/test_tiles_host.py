"""Host logic of the batched kernel's tile autotuner (no GPU).

rq_tiles_search is driven by synthetic cost functions through its callback:
it must find the minimum of a separable landscape from any start, measure
each policy once, stay put when no candidate beats the incumbent by the 1 %
margin, stop after `passes`, and pass errors and bad times back as statuses.
The policy calls reject a missing handle before touching the device.  The
JSON cache of tuned policies keys a batch by its class, survives unreadable
files, and lets Handle.tune_batched skip the timing on a hit.
"""
import ctypes

import pytest

from paper_2008_04447_gb300 import _lib

STEPS = _lib.RQ_TILE_STEPS


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2008_04447_gb300 import build
    build.build()
    return _lib.load()


def l1_bowl(m0, n0):
    """1 + |i - i0| + |j - j0| over the step indices: every move toward the
    minimum gains at least 1/11 of the cost, well above the margin."""
    def f(t):
        return 1.0 + abs(STEPS.index(t[0]) - STEPS.index(m0)) + abs(STEPS.index(t[1]) - STEPS.index(n0))
    return f


def recorded(f):
    calls = []

    def g(t):
        calls.append(t)
        return f(t)
    return g, calls


def test_search_finds_the_minimum_from_the_default_start():
    for m0 in STEPS:
        for n0 in STEPS:
            g, calls = recorded(l1_bowl(m0, n0))
            rc, best, ms = _lib.rq_tiles_search(g, passes=3)
            assert rc == 0 and best == (m0, n0) and ms == 1.0
            assert calls[0] == (32, 32)
            assert len(calls) == len(set(calls))          # each policy measured once
            # pass 1: the start and 5 + 5 candidates; pass 2 only re-sweeps m
            # at the new n (the n sweep at m0 is remembered), then stops
            assert len(calls) == 11 + (5 if n0 != 32 else 0)


def test_search_from_a_given_start_and_a_one_pass_limit():
    g, calls = recorded(l1_bowl(128, 0))
    rc, best, _ = _lib.rq_tiles_search(g, start=(0, 256), passes=1)
    assert rc == 0 and best == (128, 0) and calls[0] == (0, 256) and len(calls) == 11
    g, calls = recorded(l1_bowl(128, 0))
    rc, best, ms = _lib.rq_tiles_search(g, start=(16, 16), passes=0)
    assert rc == 0 and best == (16, 16) and calls == [(16, 16)] and ms == l1_bowl(128, 0)((16, 16))


def test_a_start_outside_the_steps_is_kept_or_left():
    def f(t):
        return 2.0 if t == (48, 32) else 3.0
    rc, best, ms = _lib.rq_tiles_search(f, start=(48, 32))
    assert rc == 0 and best == (48, 32) and ms == 2.0


def test_noise_below_the_margin_does_not_move_it():
    # every other policy is 0.5 % faster than the start: not enough
    def f(t):
        return 1.0 if t == (32, 32) else 0.995
    g, calls = recorded(f)
    rc, best, ms = _lib.rq_tiles_search(g, passes=4)
    assert rc == 0 and best == (32, 32) and ms == 1.0 and len(calls) == 11

    # 2 % faster moves it
    def f2(t):
        return 0.98 if t == (64, 32) else 1.0
    rc, best, ms = _lib.rq_tiles_search(f2)
    assert rc == 0 and best == (64, 32) and ms == 0.98


def test_never_worse_than_the_start_on_a_coupled_landscape():
    # not separable: coordinate descent may stop at a local minimum, but it
    # only ever moves downhill
    def f(t):
        i, j = STEPS.index(t[0]), STEPS.index(t[1])
        return 1.0 + ((i - j) % 6) * 0.3 + (i == 5 and j == 5) * (-0.9)
    rc, best, ms = _lib.rq_tiles_search(f, passes=5)
    assert rc == 0 and ms <= f((32, 32)) and ms == f(best)


def test_measure_errors_and_bad_times_end_the_search():
    def boom(t):
        raise ZeroDivisionError("measure failed")
    with pytest.raises(ZeroDivisionError):
        _lib.rq_tiles_search(boom)
    for bad in (float("nan"), float("inf"), -1.0):
        g, calls = recorded(lambda t, bad=bad: bad if t == (0, 32) else 1.0)
        rc, _, _ = _lib.rq_tiles_search(g)
        assert rc == -1 and calls[-1] == (0, 32)


def test_argument_checks(lib):
    best = _lib.rq_batch_tiles()
    ok = _lib.rq_tiles_measure(lambda u, t, ms: 0)
    assert lib.rq_tiles_search(_lib.rq_tiles_measure(), None, None, 1, ctypes.byref(best), None) == -1
    assert lib.rq_tiles_search(ok, None, ctypes.byref(_lib.rq_batch_tiles(-1, 0)), 1, ctypes.byref(best), None) == -3
    assert lib.rq_tiles_search(ok, None, None, -1, ctypes.byref(best), None) == -4
    assert lib.rq_tiles_search(ok, None, None, 1, None, None) == -5
    assert _lib.rq_set_batch_tiles(None, 32, 32) == _lib.RQ_EHANDLE
    assert _lib.rq_get_batch_tiles(None)[0] == _lib.RQ_EHANDLE
    assert lib.rq_tune_batched(None, 2, 0, None, 1, 1, 1, 1, 0, 1, 1, None, None, None) == _lib.RQ_EHANDLE


def test_batch_key_names_the_class_of_a_batch():
    import torch
    from paper_2008_04447_gb300 import tuning
    probs = [(torch.zeros(300, 200), None, 16, 8, 40), (torch.zeros(64, 64), None, 8, 8, 8)]
    k1 = tuning.batch_key(probs, 2, "GB300", 152)
    assert k1 == "GB300/sm152/prec2/count2/m512/n256/k64"
    assert tuning.batch_key([(torch.zeros(257, 129), None, 16, 8, 33)] * 2, 2, "GB300", 152) == k1
    assert tuning.batch_key(probs, 1, "GB300", 152) != k1
    assert tuning.batch_key(probs * 2, 2, "GB300", 152) != k1
    assert tuning.batch_key(probs, 2, "GB300", 148) != k1


def test_cache_round_trip_and_unreadable_files(tmp_path):
    import json
    import os
    from paper_2008_04447_gb300 import tuning
    path = str(tmp_path / "tiles.json")
    assert tuning.lookup(path, "k") is None
    tuning.store(path, "k", (64, 16), 1.5)
    assert tuning.lookup(path, "k") == {"tiles": [64, 16], "ms": 1.5}
    tuning.store(path, "k2", (0, 256), None)
    assert tuning.lookup(path, "k")["tiles"] == [64, 16] and tuning.lookup(path, "k2")["ms"] is None
    with open(path, "w") as f:
        f.write("{not json")
    assert tuning.lookup(path, "k") is None
    tuning.store(path, "k", (32, 32), 2.0)          # an unreadable file is replaced
    assert tuning.lookup(path, "k")["tiles"] == [32, 32]
    with open(path, "w") as f:
        json.dump({"k": {"tiles": [-1, 3]}, "j": [1, 2], "b": {"tiles": [True, 3]}}, f)
    assert tuning.lookup(path, "k") is None and tuning.lookup(path, "j") is None and tuning.lookup(path, "b") is None
    assert not [f for f in os.listdir(tmp_path) if f.startswith(".tiles")]   # no temporary left behind


def test_tune_batched_fills_then_uses_the_cache(tmp_path, monkeypatch):
    import paper_2008_04447_gb300 as P
    calls = []
    h = object.__new__(P.Handle)
    h.h = None
    monkeypatch.setattr(P.Handle, "_batch", staticmethod(lambda problems, outputs, svd: ("outs", "info", "d",
                                                                                        (1, 1, 1, 1, 0))))
    monkeypatch.setattr(P._lib, "rq_tune_batched", lambda *a: (calls.append("tune"), (0, (64, 16), 1.25))[1])
    monkeypatch.setattr(P._lib, "rq_set_batch_tiles", lambda hh, m, n: (calls.append(("set", m, n)), 0)[1])
    monkeypatch.setattr(P, "rq_tuxv_batched", lambda *a: (calls.append("run"), 0)[1])
    cache = str(tmp_path / "tiles.json")
    assert h.tune_batched([("A",)], cache=cache, key="K") == ((64, 16), 1.25, "outs", "info")
    assert calls == ["tune"]
    calls.clear()
    tiles, ms, outs, info = h.tune_batched([("A",)], cache=cache, key="K")
    assert (tiles, ms, outs, info) == ((64, 16), 1.25, "outs", "info")
    assert calls == [("set", 64, 16), "run"]                      # no timing on a hit
