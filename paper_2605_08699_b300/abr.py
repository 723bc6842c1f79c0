"""Receiver-driven resolution control of the serving loop (Sec. 4.3 "ABR
Controller" for the design, Sec. 5.3 "Throughput Monitoring" and "ABR
Controller" for the implementation).

``ThroughputEMA`` is the client's throughput monitor: one sample per
finished request, S_i / dt_i (bytes over download seconds), smoothed by an
exponential moving average over the last ``history`` samples (defaults 5 and
alpha = 0.3).

``LatencyABR`` is the "Latency" controller over a ladder of levels (index 0 =
lowest resolution), each with an expected frame size S_l in bytes.  The
predicted completion time of level l at throughput r (bytes/s) is
T_l = S_l / r (the paper writes S_l / (r * 1024) with r in KiB/s: the same
quantity).  One level up when T_{l+1} <= t_target, one level down when
T_l > t_margin, each only after ``hold`` consecutive requests asked for it;
a downgrade during rapid panning is taken at once.  t_target < t_margin
leaves a dead band in which the level holds.

``assign_levels`` runs one controller per client over a request trace, so the
resolution of every request is fixed before any rendering happens and two
serving arms replaying the same trace render the same frames.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

#: expected compressed frame size per pixel (bytes); Table 1's sizes span
#: about 0.09-0.26 B/px, this is the value the serving trace uses
BYTES_PER_PIXEL = 0.2


class ThroughputEMA:
    """EMA of the last ``history`` throughput samples, oldest first."""

    def __init__(self, alpha: float = 0.3, history: int = 5):
        if not (0.0 < alpha <= 1.0) or history < 1:
            raise ValueError("alpha in (0, 1], history >= 1")
        self.alpha = alpha
        self.history = history
        self.samples: list[float] = []

    def add(self, bytes_per_s: float) -> None:
        if not (bytes_per_s > 0.0) or not math.isfinite(bytes_per_s):
            raise ValueError("throughput sample must be positive and finite")
        self.samples.append(float(bytes_per_s))
        if len(self.samples) > self.history:
            self.samples.pop(0)

    def add_download(self, size_bytes: float, seconds: float) -> None:
        self.add(size_bytes / seconds)

    def value(self) -> float | None:
        if not self.samples:
            return None
        e = self.samples[0]
        for x in self.samples[1:]:
            e = self.alpha * x + (1.0 - self.alpha) * e
        return e


@dataclass
class LatencyABR:
    sizes_bytes: list[float]
    t_target: float = 0.100
    t_margin: float = 0.150
    hold: int = 3
    level: int = 0
    _up: int = field(default=0, repr=False)
    _down: int = field(default=0, repr=False)

    def __post_init__(self):
        if not self.sizes_bytes or any(not (s > 0) for s in self.sizes_bytes):
            raise ValueError("sizes must be positive")
        if any(b < a for a, b in zip(self.sizes_bytes, self.sizes_bytes[1:])):
            raise ValueError("ladder sizes must not decrease with the level")
        if not (self.t_target < self.t_margin):
            raise ValueError("t_target must be below t_margin (dead band)")
        if self.hold < 1 or not (0 <= self.level < len(self.sizes_bytes)):
            raise ValueError("hold >= 1 and a valid start level")

    def predicted_time(self, level: int, r_bytes_per_s: float) -> float:
        return self.sizes_bytes[level] / r_bytes_per_s

    def update(self, r_bytes_per_s: float | None, panning: bool = False) -> int:
        """Level for the next request, given the current throughput estimate."""
        if r_bytes_per_s is None:
            return self.level
        top = len(self.sizes_bytes) - 1
        up = self.level < top and self.predicted_time(self.level + 1, r_bytes_per_s) <= self.t_target
        down = self.level > 0 and self.predicted_time(self.level, r_bytes_per_s) > self.t_margin
        if down and panning:
            self.level -= 1
            self._up = self._down = 0
            return self.level
        self._up = self._up + 1 if up else 0
        self._down = self._down + 1 if down else 0
        if self._up >= self.hold:
            self.level += 1
            self._up = self._down = 0
        elif self._down >= self.hold:
            self.level -= 1
            self._up = self._down = 0
        return self.level


def ladder_sizes(levels, bytes_per_pixel: float = BYTES_PER_PIXEL) -> list[float]:
    return [bytes_per_pixel * w * h for (w, h) in levels]


def assign_levels(client: np.ndarray, bw: np.ndarray, levels, pan: np.ndarray | None = None,
                  start_level: int | None = None, **abr_kw) -> np.ndarray:
    """Level of every request of a trace (requests in arrival order).

    Each client's controller decides from the EMA of its earlier requests'
    download throughput; the request itself then downloads at the client's
    bandwidth ``bw`` (bytes/s), which becomes the next sample.  ``pan`` marks
    requests made during rapid panning."""
    sizes = ladder_sizes(levels)
    start = len(levels) // 2 if start_level is None else start_level
    abrs: dict[int, LatencyABR] = {}
    emas: dict[int, ThroughputEMA] = {}
    out = np.empty(len(client), np.int32)
    for i, c in enumerate(np.asarray(client).tolist()):
        a = abrs.get(c)
        if a is None:
            a = abrs[c] = LatencyABR(sizes, level=start, **abr_kw)
            emas[c] = ThroughputEMA()
        lvl = a.update(emas[c].value(), bool(pan[i]) if pan is not None else False)
        out[i] = lvl
        emas[c].add_download(sizes[lvl], sizes[lvl] / float(bw[i]))
    return out
