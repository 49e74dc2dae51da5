"""Oracle for the Risky Gate (Sec. II-B and Sec. V-D), plain numpy in fp64.

TEST INFRASTRUCTURE ONLY: used by the tests and the benchmark's CPU baseline,
never by the library.

What the paper fixes:
  * the CPU cost model is alpha*N*log N or alpha*N*K (Sec. II-B); the fitted
    full-sort form is T_cpu(N) = a*N*log2(N) + b (Sec. V-D);
  * key-only transfer is T_tx(N) = c*N + d (Sec. V-D), here in bytes so that a
    wider row costs more (Sec. II-B, transfer bytes B);
  * C_gpu = Transfer + Kernel + Post-processing (Sec. II-B), post-processing
    being result return plus late materialization (Sec. V-D);
  * offload only when C_cpu - C_gpu exceeds a threshold, the gate margin in ms
    (Sec. II-B, Sec. IV "gate margin");
  * the break-even N* solves T_cpu(N*) = T_tx(N*) + T_gpu(N*) (Sec. V-D).

Readings where it is open (kept identical in the library's contract):
  * fits are least squares y = slope*x + intercept on the given points, in
    the centred closed form of the normal equations, either ordinary or
    weighted by 1/y^2 (relative error: measured times span decades of N, and
    unweighted the largest sizes decide the small-N costs the gate exists
    for);
  * Top-K fits both CPU forms, x = N*log2(N) and x = N*K, and keeps the one
    with the smaller residual sum of squares (N*log2 N on a tie); or, on
    request (CPU_MAX), keeps both and estimates the larger of the two;
  * probe CPU cost uses x = N*M, M the expected candidates per probe;
  * kernel time is linear in N (e*N + f), post-processing linear in the
    number of returned rows (g*out + h);
  * "exceeds" is strict: offload iff C_cpu - C_gpu > margin;
  * N* is the smallest integer N in [1, 2^34] with C_cpu(N) - C_gpu(N) >
    margin, by bisection; 1 if that already holds at N = 1, 0 ("none") if it
    does not hold at 2^34.
  * the CPU engine may change regime at a known size (a host engine that goes
    parallel above some N): then the CPU cost is fitted on its own over the
    samples below that size and over those at or above it, each estimate
    uses its size's regime, and N* is searched in the lower regime first,
    then in the upper one from its first size on (the gain is taken to grow
    with N within each regime, not across the step between them).
"""
from __future__ import annotations

import math

import numpy as np

TOPK, PROBE = 0, 1
CPU_NLOGN, CPU_NK, CPU_NM, CPU_MAX = 0, 1, 2, 3
N_STAR_HI = 1 << 34


ORDINARY, RELATIVE = 0, 1


def weights(y, weighting):
    """Least-squares weights: 1 (ordinary) or 1 / y^2 (relative error; a
    non-positive y gets the weight of the smallest positive y)."""
    y = np.asarray(y, dtype=np.float64)
    if weighting == ORDINARY:
        return np.ones_like(y)
    pos = y[y > 0.0]
    floor = pos.min() if pos.shape[0] else 1.0
    return 1.0 / np.square(np.where(y > 0.0, y, floor))


def ols(x, y, weighting=ORDINARY):
    """(Weighted) least-squares slope and intercept of y = slope*x + intercept,
    from the centred normal equations."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    w = weights(y, weighting)
    sw = w.sum()
    xm = float(np.sum(w * x) / sw)
    ym = float(np.sum(w * y) / sw)
    sxx = float(np.sum(w * (x - xm) * (x - xm)))
    sxy = float(np.sum(w * (x - xm) * (y - ym)))
    slope = sxy / sxx if sxx > 0.0 else 0.0
    return slope, float(ym - slope * xm)


def rss(x, y, slope, intercept, weighting=ORDINARY):
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    r = y - (slope * x + intercept)
    return float(np.sum(weights(y, weighting) * r * r))


def cpu_x(form, n, k_or_m):
    n = float(n)
    if form == CPU_NLOGN:
        return n * math.log2(n) if n > 0 else 0.0
    return n * float(k_or_m)


class Model:
    """Cost model.  With split_n > 0, (a, b, a2, b2) is the CPU fit for
    N < split_n and (a_hi, b_hi, a2_hi, b2_hi) the fit for N >= split_n."""

    def __init__(self, op, cpu_form, a, b, c, d, e, f, g, h, margin_ms, a2=0.0, b2=0.0, split_n=0.0,
                 a_hi=0.0, b_hi=0.0, a2_hi=0.0, b2_hi=0.0):
        self.op, self.cpu_form = op, cpu_form
        self.a2, self.b2 = a2, b2
        self.a, self.b, self.c, self.d = a, b, c, d
        self.e, self.f, self.g, self.h = e, f, g, h
        self.margin_ms = margin_ms
        self.split_n = split_n
        self.a_hi, self.b_hi, self.a2_hi, self.b2_hi = a_hi, b_hi, a2_hi, b2_hi


def _cpu_fits(op, n, k_or_m, t_cpu, wt):
    """CPU fits of one regime: {form: (slope, intercept)} and {form: rss}."""
    forms = (CPU_NLOGN, CPU_NK) if op == TOPK else (CPU_NM,)
    xs = {f: [cpu_x(f, ni, ki) for ni, ki in zip(n, k_or_m)] for f in forms}
    fits = {f: ols(xs[f], t_cpu, wt) for f in forms}
    return fits, {f: rss(xs[f], t_cpu, *fits[f], wt) for f in forms}


def calibrate(op, n, k_or_m, tx_bytes, out_rows, t_cpu, t_tx, t_ker, t_post, margin_ms=0.0,
              weighting=ORDINARY, topk_cpu=0, cpu_split_n=0.0):
    """Fit every cost term from measured samples (all times in ms); with
    cpu_split_n > 0 the CPU cost is fitted separately on the samples with
    N < cpu_split_n and on the others."""
    wt = weighting
    n, k_or_m, t_cpu = (np.asarray(v, dtype=np.float64) for v in (n, k_or_m, t_cpu))
    if cpu_split_n > 0.0:
        below = n < cpu_split_n
        parts = [below, ~below]
    else:
        parts = [np.ones(n.shape[0], dtype=bool)]
    regimes = [_cpu_fits(op, n[p], k_or_m[p], t_cpu[p], wt) for p in parts]
    if op == TOPK:
        r_nlogn = sum(r[CPU_NLOGN] for _, r in regimes)
        r_nk = sum(r[CPU_NK] for _, r in regimes)
        form = CPU_NLOGN if r_nlogn <= r_nk else CPU_NK
        if topk_cpu == CPU_MAX:
            form = CPU_MAX
    else:
        form = CPU_NM

    def coef(fits):
        if form == CPU_MAX:
            return fits[CPU_NLOGN] + fits[CPU_NK]
        return fits[form] + (0.0, 0.0)

    a, b, a2, b2 = coef(regimes[0][0])
    a_hi = b_hi = a2_hi = b2_hi = 0.0
    if cpu_split_n > 0.0:
        a_hi, b_hi, a2_hi, b2_hi = coef(regimes[1][0])
    c, d = ols(tx_bytes, t_tx, wt)
    e, f = ols(n, t_ker, wt)
    g, h = ols(out_rows, t_post, wt)
    return Model(op, form, a, b, c, d, e, f, g, h, margin_ms, a2, b2, float(cpu_split_n), a_hi, b_hi, a2_hi, b2_hi)


def costs(m: Model, n, k_or_m, tx_bytes, out_rows):
    if m.split_n > 0.0 and float(n) >= m.split_n:
        a, b, a2, b2 = m.a_hi, m.b_hi, m.a2_hi, m.b2_hi
    else:
        a, b, a2, b2 = m.a, m.b, m.a2, m.b2
    if m.cpu_form == CPU_MAX:
        c_cpu = max(a * cpu_x(CPU_NLOGN, n, k_or_m) + b, a2 * cpu_x(CPU_NK, n, k_or_m) + b2)
    else:
        c_cpu = a * cpu_x(m.cpu_form, n, k_or_m) + b
    c_tx = m.c * float(tx_bytes) + m.d
    c_ker = m.e * float(n) + m.f
    c_post = m.g * float(out_rows) + m.h
    return c_cpu, c_tx, c_ker, c_post


def decide(m: Model, n, k_or_m, tx_bytes, out_rows):
    c_cpu, c_tx, c_ker, c_post = costs(m, n, k_or_m, tx_bytes, out_rows)
    return (c_cpu - (c_tx + c_ker + c_post)) > m.margin_ms


def gain(m: Model, n, k_or_m, bytes_per_row, out_per_row, out_fixed):
    """C_cpu - C_gpu - margin at size n, with transfer bytes and returned rows
    growing with n as the query describes."""
    out = out_fixed if out_fixed is not None else out_per_row * n
    if m.op == TOPK and out_fixed is not None:
        out = min(out_fixed, n)
    c_cpu, c_tx, c_ker, c_post = costs(m, n, k_or_m, bytes_per_row * n, out)
    return c_cpu - (c_tx + c_ker + c_post) - m.margin_ms


def _first_positive(g, lo, hi):
    """Bisection for the smallest n in (lo, hi] with g(n) > 0, given
    g(lo) <= 0 < g(hi)."""
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if g(mid) > 0.0:
            hi = mid
        else:
            lo = mid
    return hi


def n_star(m: Model, k_or_m, bytes_per_row, out_per_row=0.0, out_fixed=None):
    g = lambda nn: gain(m, nn, k_or_m, bytes_per_row, out_per_row, out_fixed)
    if g(1) > 0.0:
        return 1
    start = 1
    if m.split_n > 1.0:
        s = min(int(math.ceil(m.split_n)), N_STAR_HI)      # first size of the upper regime
        if s >= 2 and g(s - 1) > 0.0:
            return _first_positive(g, 1, s - 1)
        if s >= N_STAR_HI:
            return N_STAR_HI if g(N_STAR_HI) > 0.0 else 0
        if g(s) > 0.0:
            return s
        start = s
    if not g(N_STAR_HI) > 0.0:
        return 0
    return _first_positive(g, start, N_STAR_HI)
