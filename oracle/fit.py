"""Growth-rate fit of the transverse field energy (oracle side; test infrastructure only).

The paper's Fig. 2 and Fig. 4 captions give the largest growth rates of the instability, taken from
the field energy, without stating how they were fitted. Reading used here and, independently
re-implemented, by the CUDA library's host code:

* sample times finite and strictly increasing (an error otherwise);
* L(t) = log10 W_perp(t) over the samples with finite W_perp > 0 (the others are skipped; the
  window's indices i0, i1 refer to the caller's arrays);
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
    """Return (Gamma, i0, i1): amplitude growth rate and the inclusive sample window used, as indices
    into t and w."""
    t = np.asarray(t, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    if not np.isfinite(t).all() or (np.diff(t) <= 0).any():
        raise ValueError("the sample times must be finite and strictly increasing")
    keep = (w > 0) & np.isfinite(w)
    src = np.nonzero(keep)[0]  # index of each kept sample in the caller's arrays
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
        return 0.5 * _slope(t[i0:i1 + 1], np.log(w[i0:i1 + 1])), int(src[i0]), int(src[i1])
    m = max(5, n // 5)
    best, bi = -np.inf, 0
    for s in range(min(head, n - m), n - m + 1):
        sl = _slope(t[s:s + m], np.log(w[s:s + m]))
        if sl > best:
            best, bi = sl, s
    return 0.5 * best, int(src[bi]), int(src[bi + m - 1])
