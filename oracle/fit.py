"""Growth-rate fit of the transverse field energy (oracle side; test infrastructure only).

The paper reports "maximum numerical instability growth rates" of the field energy (Fig. 2 and
Fig. 4 captions) without stating how they were fitted. Reading used here and, independently
re-implemented, by the CUDA library's host code:

* L(t) = log10 W_perp(t) over samples with W_perp > 0;
* noise floor = median of L over the first tenth of those samples (at least 3);
* saturation = max L;
* window = from the first sample with L >= floor + 2 to the first later sample with
  L >= saturation - 1 (inclusive); it is used when it holds at least 5 samples;
* otherwise the sliding window of max(5, n // 5) consecutive samples with the largest slope, searched
  only after the first tenth (the start-up from E = B = 0 is not instability growth);
* Gamma = (1/2) d ln W_perp / dt from an FP64 least-squares line over the window, i.e. the growth
  rate of the field amplitude.
"""
from __future__ import annotations

import numpy as np


def _slope(t: np.ndarray, y: np.ndarray) -> float:
    tm = t.mean()
    ym = y.mean()
    return float(((t - tm) * (y - ym)).sum() / ((t - tm) ** 2).sum())


def growth_rate(t, w):
    """Return (Gamma, i0, i1): amplitude growth rate and the inclusive sample window used."""
    t = np.asarray(t, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    keep = w > 0
    t, w = t[keep], w[keep]
    n = len(w)
    if n < 5:
        raise ValueError("need at least 5 positive samples")
    lg = np.log10(w)
    head = max(3, n // 10)
    floor = float(np.median(lg[:head]))
    sat = float(lg.max())
    lo, hi = floor + 2.0, sat - 1.0
    i0 = int(np.argmax(lg >= lo)) if (lg >= lo).any() else n
    i1 = i0
    while i1 < n - 1 and lg[i1] < hi:
        i1 += 1
    if hi > lo and i1 - i0 + 1 >= 5:
        return 0.5 * _slope(t[i0:i1 + 1], np.log(w[i0:i1 + 1])), i0, i1
    m = max(5, n // 5)
    best, bi = -np.inf, 0
    for s in range(min(head, n - m), n - m + 1):
        sl = _slope(t[s:s + m], np.log(w[s:s + m]))
        if sl > best:
            best, bi = sl, s
    return 0.5 * best, bi, bi + m - 1
