"""Importance weights, effective sample size and evidence per event (oracle; test
infrastructure).

Sec. 6 checks the network's posteriors against runs that use the standard GW
likelihood.  The plain way to turn samples theta_s ~ q (a proposal: the prior, or
a trained flow) into posterior samples is importance sampling with that likelihood:

    ln w_s = ln L(theta_s) + ln pi(theta_s) - ln q(theta_s),

normalised within each event e (samples event_offsets[e] <= s < event_offsets[e+1]):

    weight_s     = w_s / sum_{s in e} w_s,
    ess_e        = (sum w)^2 / sum w^2            (Kish's effective sample size),
    efficiency_e = ess_e / S_e,
    ln Z_e       = ln( (1/S_e) sum w_s )          (the importance-sampling evidence).

``log_ratio`` is ln pi - ln q (None for the prior as proposal: zero).  Readings:
an event without samples has ess = efficiency = 0 and ln Z = -inf; a sample with
ln w = -inf has weight 0; an event whose every ln w is -inf has all weights 0,
ess = efficiency = 0 and ln Z = -inf.

Written as the definitions, one event at a time, with the largest ln w factored
out of the sums so that exp does not overflow (exp(ln w - m) <= 1).
"""
import math
import numpy as np


def importance_weights(lnl, event_offsets, log_ratio=None):
    """Returns (weights [S], ess [E], efficiency [E], ln_evidence [E]), all float64."""
    lnl = np.asarray(lnl, dtype=np.float64)
    offs = np.asarray(event_offsets, dtype=np.int64)
    lnw = lnl if log_ratio is None else lnl + np.asarray(log_ratio, dtype=np.float64)
    E = len(offs) - 1
    weights = np.zeros(len(lnw))
    ess = np.zeros(E)
    eff = np.zeros(E)
    lnz = np.full(E, -np.inf)
    for e in range(E):
        a, b = int(offs[e]), int(offs[e + 1])
        n = b - a
        if n == 0:
            continue
        seg = lnw[a:b]
        m = np.max(seg)
        if m == -np.inf:
            continue
        w = np.exp(seg - m)
        s1 = np.sum(w)
        s2 = np.sum(w * w)
        weights[a:b] = w / s1
        ess[e] = s1 * s1 / s2
        eff[e] = ess[e] / n
        lnz[e] = m + math.log(s1) - math.log(n)
    return weights, ess, eff, lnz
