"""Latency ABR and throughput EMA (Sec. 4.3 and Sec. 5.3, "ABR Controller" and
"Throughput Monitoring") and the serving trace generator.

The controller's rules are checked on hand-built throughput sequences whose
outcome follows from the rules directly: the hold counter, the dead band
between t_target and t_margin, the reset of a counter by a request that does
not ask for the switch, and the immediate downgrade while panning."""
import math

import numpy as np
import pytest

import synth
from paper_2605_08699_b300.abr import LatencyABR, ThroughputEMA, assign_levels, ladder_sizes

SIZES = [100e3, 200e3, 400e3, 800e3]   # bytes per level


def test_ema_closed_form_over_last_five():
    e = ThroughputEMA(alpha=0.3, history=5)
    xs = [10.0, 20.0, 30.0, 40.0, 50.0, 60.0, 70.0]
    for x in xs:
        e.add(x)
    w = xs[-5:]
    # oldest sample weighted (1 - a)^4, sample k (k >= 1) weighted a (1 - a)^(4 - k)
    want = 0.7 ** 4 * w[0] + sum(0.3 * 0.7 ** (4 - k) * w[k] for k in range(1, 5))
    assert math.isclose(e.value(), want, rel_tol=1e-12)


def test_ema_single_and_empty():
    e = ThroughputEMA()
    assert e.value() is None
    e.add_download(1000.0, 0.5)
    assert e.value() == 2000.0
    with pytest.raises(ValueError):
        e.add(0.0)


def test_upgrade_needs_hold_consecutive_requests():
    a = LatencyABR(SIZES, level=0)
    r = SIZES[1] / 0.1   # level 1 predicted exactly at t_target: allowed (<=)
    assert a.update(r) == 0
    assert a.update(r) == 0
    assert a.update(r) == 1   # third consecutive request
    # level 2 needs twice the rate: at r it is predicted 0.2 s > target, level 1 at 0.1 s <= margin
    for _ in range(10):
        assert a.update(r) == 1   # dead band: no upgrade, no downgrade


def test_upgrade_counter_resets():
    a = LatencyABR(SIZES, level=0)
    fast, slow = SIZES[1] / 0.05, SIZES[1] / 0.12   # slow: level 1 above target but level 0 below margin
    a.update(fast)
    a.update(fast)
    a.update(slow)          # breaks the run
    assert a.update(fast) == 0
    assert a.update(fast) == 0
    assert a.update(fast) == 1


def test_downgrade_after_hold_and_dead_band():
    a = LatencyABR(SIZES, level=3)
    r_band = SIZES[3] / 0.125      # 0.125 s: between target and margin -> hold level 3
    for _ in range(5):
        assert a.update(r_band) == 3
    r_bad = SIZES[3] / 0.2         # over margin
    assert a.update(r_bad) == 3
    assert a.update(r_bad) == 3
    assert a.update(r_bad) == 2


def test_panning_bypasses_hold_for_downgrade_only():
    a = LatencyABR(SIZES, level=3)
    assert a.update(SIZES[3] / 0.2, panning=True) == 2
    b = LatencyABR(SIZES, level=0)
    assert b.update(SIZES[1] / 0.05, panning=True) == 0   # upgrades still wait


def test_invalid_configs():
    with pytest.raises(ValueError):
        LatencyABR(SIZES, t_target=0.2, t_margin=0.15)
    with pytest.raises(ValueError):
        LatencyABR([2.0, 1.0])
    with pytest.raises(ValueError):
        LatencyABR(SIZES, level=4)


def test_constant_bandwidth_converges_to_highest_fitting_level():
    levels = synth.ABR_LEVELS
    sizes = ladder_sizes(levels)
    for mbit in [5.0, 22.4, 60.0, 100.0]:
        r = mbit * 1e6 / 8
        a = LatencyABR(sizes, level=0)
        for _ in range(40):
            lvl = a.update(r)
        fits = [l for l in range(len(sizes)) if sizes[l] / r <= 0.1]
        assert lvl == (max(fits) if fits else 0)


def test_table1_ladder_under_typical_bandwidth():
    # Table 1's largest profile (1280x720, up to 300 KB) takes > 100 ms below 3 MB/s
    sizes = [hi * 1000.0 for (_, _, _, _, _, hi) in sorted(synth.TABLE1_LADDER, key=lambda r: r[1])]
    a = LatencyABR(sizes, level=0)
    for _ in range(20):
        lvl = a.update(2.8e6)
    assert lvl == 2


def test_serving_trace_statistics_and_determinism():
    tr = synth.serving_trace(seconds=4.0, n_clients=16)
    tr2 = synth.serving_trace(seconds=4.0, n_clients=16)
    assert np.array_equal(tr.t, tr2.t) and np.array_equal(tr.client, tr2.client)
    assert np.all(np.diff(tr.t) >= 0) and tr.t[0] >= 0 and tr.t[-1] < 4.0
    assert np.all((tr.rates_hz >= 60) & (tr.rates_hz <= 90))
    counts = np.bincount(tr.client, minlength=16)
    # Poisson counts: mean rate*T, sd sqrt(rate*T) (~17); allow 5 sd
    assert np.all(np.abs(counts - tr.rates_hz * 4.0) < 5 * np.sqrt(tr.rates_hz * 4.0))
    assert np.array_equal(tr.scene, tr.client % 4)
    mbit = tr.bw * 8 / 1e6
    assert mbit.min() >= 5.0 - 1e-9 and mbit.max() <= 100.0 + 1e-9
    # one bandwidth per client and second
    for c in range(16):
        for s in range(4):
            m = (tr.client == c) & (np.floor(tr.t) == s)
            if m.any():
                assert np.unique(tr.bw[m]).size == 1


def test_assign_levels_is_deterministic_and_per_client():
    tr = synth.serving_trace(seconds=2.0, n_clients=8)
    a = assign_levels(tr.client, tr.bw, synth.ABR_LEVELS)
    b = assign_levels(tr.client, tr.bw, synth.ABR_LEVELS)
    assert np.array_equal(a, b)
    assert a.min() >= 0 and a.max() < len(synth.ABR_LEVELS)
    # a client's level moves by at most one step per request
    for c in range(8):
        lv = a[tr.client == c]
        assert np.all(np.abs(np.diff(lv)) <= 1)
