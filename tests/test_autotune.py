"""Host logic of the batch autotuner: cache keys, size classes, the coordinate
descent over the launch knobs (driven by a fake clock) and the JSON cache.
The GPU test tunes a small real batch and checks that the states are left
untouched and that a second call is served from the cache."""
import json

import numpy as np
import pytest

from paper_1909_06412_gb300 import autotune as at


def test_signature_ignores_problem_order_and_keys_precision_and_device():
    a = at.signature([(64, 64), (16, 16, 16)], 0, "GB300")
    b = at.signature([(16, 16, 16), (64, 64)], 0, "GB300")
    assert a == b
    assert a != at.signature([(64, 64), (16, 16, 16)], 1, "GB300")
    assert a != at.signature([(64, 64), (16, 16, 16)], 0, "other")
    assert a != at.signature([(64, 64), (16, 16, 18)], 0, "GB300")


def test_size_classes():
    assert at.size_class(16 ** 3) == 0
    assert at.size_class(8192) == 0
    assert at.size_class(8193) == 1
    assert at.size_class(256 * 256) == 1
    assert at.size_class(256 * 256 + 1) == 2


def test_coordinate_descent_finds_the_separable_optimum():
    # time = cluster cost + per-class tile cost + per-class radix cost
    opt = {"cluster": 4, "tile": [16384, 0, 65536], "radix": [4, 8, 0]}

    def measure(s):
        if s["cluster"] == 8:
            return None  # rejected setting
        t = 1.0 + 0.2 * abs(np.log2(max(s["cluster"], 2) / opt["cluster"]))
        for c in range(3):
            t += 0.1 * (s["tile"][c] != opt["tile"][c]) + 0.05 * (s["radix"][c] != opt["radix"][c])
        return t

    best, t, trials = at.coordinate_descent(measure, {0, 1, 2})
    assert best["cluster"] == 4 and best["tile"][:3] == opt["tile"] and best["radix"][:3] == opt["radix"]
    assert t == pytest.approx(1.0)
    assert any(tt is None for _, tt in trials)


def test_coordinate_descent_keeps_defaults_below_the_gain_threshold():
    best, t, _ = at.coordinate_descent(lambda s: 1.0 - 0.01 * (s["cluster"] == 1), {1}, min_gain=0.03)
    assert best == at.default_settings()


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "sub" / "cache.json")
    assert at.load_cache(p) == {}
    at.store_cache(p, "k1", {"settings": at.default_settings(), "seconds_per_step": 1e-3})
    at.store_cache(p, "k2", {"settings": {"cluster": 4, "tile": [0] * 3, "radix": [0] * 3}})
    d = json.load(open(p))
    assert set(d) == {"k1", "k2"} and d["k2"]["settings"]["cluster"] == 4
    tb, rm = at.expand(d["k2"]["settings"], [0, 2, 1])
    assert tb == [0, 0, 0] and rm == [0, 0, 0]


@pytest.mark.gpu
def test_tune_small_batch_restores_states_and_caches(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1909_06412_gb300 as mg

    shapes = [((32, 24), (0.5, 0.6)), ((16, 16, 16), (0.5, 0.5, 0.5)), ((64, 64), (0.3, 0.3)),
              ((24, 18, 16), (0.5, 0.6, 0.6))]
    props = []
    for N, dq in shapes:
        g = mg.Propagator(N, dq, precision=mg.MG_FP32_MIXED)
        D = len(N)
        g.set_potential(mg.MG_POT_HARMONIC, list(np.eye(D).ravel()) + [0.0] * D)
        g.set_separable([("gauss", 0.3, 0.1, 1.0)] * D, [0.3] * D, [0.1] * D)
        props.append(g)
    before = [p.psi.clone() for p in props]
    cache = str(tmp_path / "tune.json")
    s, tb, rm, entry = at.tune_batch(props, 4, 0.05, "suzuki4", trial_steps=2, cache_path=cache)
    for p, b in zip(props, before):
        assert torch.equal(p.psi, b)
    assert entry["trials"] >= 5 and entry["seconds_per_step"] <= entry["default_seconds_per_step"]
    s2, tb2, rm2, entry2 = at.tune_batch(props, 4, 0.05, "suzuki4", trial_steps=2, cache_path=cache)
    assert s2 == s and tb2 == tb and entry2 == entry
    b = mg.Batch(props, cluster=s["cluster"], tile_bytes=tb, radix_max=rm)
    b.propagate(4, 0.05, "suzuki4")
    b.sync()
