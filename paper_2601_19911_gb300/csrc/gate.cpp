// Risky Gate (Sec. II-B) with measured constants fitted by least squares and
// the break-even N* (Sec. V-D).  Pure host arithmetic in fp64.  The CPU cost
// may be fitted per regime of the host engine (below and above a size where
// it changes strategy, e.g. goes parallel).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "olap.h"

namespace {

constexpr uint64_t N_STAR_HI = 1ull << 34;

// Weight of a sample: 1 (ordinary) or 1 / y^2 (relative error); a
// non-positive y takes the weight of the smallest positive y.
struct Weights {
    int mode;
    double floor;
    double operator()(double y) const {
        if (mode == OLAP_FIT_ORDINARY) return 1.0;
        const double v = y > 0.0 ? y : floor;
        return 1.0 / (v * v);
    }
};

Weights make_weights(const double* y, uint64_t n, int mode) {
    double fl = 0.0;
    for (uint64_t i = 0; i < n; ++i)
        if (y[i] > 0.0 && (fl == 0.0 || y[i] < fl)) fl = y[i];
    return Weights{mode, fl > 0.0 ? fl : 1.0};
}

// (Weighted) least squares y = slope * x + intercept, centred normal equations.
void ols(const double* x, const double* y, uint64_t n, int mode, double* slope, double* intercept) {
    const Weights w = make_weights(y, n, mode);
    double sw = 0.0, xm = 0.0, ym = 0.0;
    for (uint64_t i = 0; i < n; ++i) {
        const double wi = w(y[i]);
        sw += wi;
        xm += wi * x[i];
        ym += wi * y[i];
    }
    xm /= sw;
    ym /= sw;
    double sxx = 0.0, sxy = 0.0;
    for (uint64_t i = 0; i < n; ++i) {
        const double wi = w(y[i]);
        sxx += wi * (x[i] - xm) * (x[i] - xm);
        sxy += wi * (x[i] - xm) * (y[i] - ym);
    }
    *slope = sxx > 0.0 ? sxy / sxx : 0.0;
    *intercept = ym - *slope * xm;
}

double rss(const double* x, const double* y, uint64_t n, int mode, double slope, double intercept) {
    const Weights w = make_weights(y, n, mode);
    double r = 0.0;
    for (uint64_t i = 0; i < n; ++i) {
        const double e = y[i] - (slope * x[i] + intercept);
        r += w(y[i]) * e * e;
    }
    return r;
}

double cpu_x(olap_cpu_form form, double n, double k_or_m) {
    if (form == OLAP_CPU_NLOGN) return n > 0.0 ? n * std::log2(n) : 0.0;
    return n * k_or_m;
}

struct Costs {
    double cpu, tx, ker, post;
};

Costs costs(const olap_gate_model& m, double n, double k_or_m, double tx_bytes, double out_rows) {
    Costs c;
    // the CPU fit of the host engine's regime at this size
    const bool hi = m.split_n > 0.0 && n >= m.split_n;
    const double a = hi ? m.a_hi : m.a, b = hi ? m.b_hi : m.b;
    const double a2 = hi ? m.a2_hi : m.a2, b2 = hi ? m.b2_hi : m.b2;
    if (m.cpu_form == OLAP_CPU_MAX)
        c.cpu = std::max(a * cpu_x(OLAP_CPU_NLOGN, n, k_or_m) + b, a2 * cpu_x(OLAP_CPU_NK, n, k_or_m) + b2);
    else
        c.cpu = a * cpu_x(m.cpu_form, n, k_or_m) + b;
    c.tx = m.c * tx_bytes + m.d;
    c.ker = m.e * n + m.f;
    c.post = m.g * out_rows + m.h;
    return c;
}

// C_cpu - C_gpu - margin at size n for the query's shape.
double gain(const olap_gate_model& m, const olap_gate_query& q, uint64_t n) {
    const double nd = static_cast<double>(n);
    double out;
    if (m.op == OLAP_OP_TOPK) out = q.k_or_m < nd ? q.k_or_m : nd;
    else out = q.out_per_row * nd;
    const Costs c = costs(m, nd, q.k_or_m, q.bytes_per_row * nd, out);
    return c.cpu - (c.tx + c.ker + c.post) - m.margin_ms;
}

// Smallest n in (lo, hi] with a positive gain, given gain(lo) <= 0 < gain(hi)
// and a gain that grows with n in between.
uint64_t bisect(const olap_gate_model& m, const olap_gate_query& q, uint64_t lo, uint64_t hi) {
    while (hi - lo > 1) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (gain(m, q, mid) > 0.0) hi = mid;
        else lo = mid;
    }
    return hi;
}

// N*: the smallest n in [1, 2^34] whose gain exceeds the margin, on a gain
// that grows with n within each CPU regime.  With two regimes the lower one
// is searched first, then the upper one from its first size on.
uint64_t n_star(const olap_gate_model& m, const olap_gate_query& q) {
    if (gain(m, q, 1) > 0.0) return 1;
    uint64_t from = 1;
    if (m.split_n > 1.0) {
        const double sc = std::ceil(m.split_n);
        const uint64_t s = sc >= static_cast<double>(N_STAR_HI) ? N_STAR_HI : static_cast<uint64_t>(sc);
        if (s >= 2 && gain(m, q, s - 1) > 0.0) return bisect(m, q, 1, s - 1);
        if (s >= N_STAR_HI) return gain(m, q, N_STAR_HI) > 0.0 ? N_STAR_HI : 0;
        if (gain(m, q, s) > 0.0) return s;
        from = s;
    }
    if (!(gain(m, q, N_STAR_HI) > 0.0)) return 0;
    return bisect(m, q, from, N_STAR_HI);
}

// Fit the CPU model of one regime (the samples in idx) in both Top-K forms or
// in the probe form; residuals are added to *r1 (N log N or N*M) and *r2 (N*K).
struct CpuFit {
    double a1, b1, a2, b2;
};

bool fit_cpu(const olap_gate_samples* s, const uint64_t* idx, uint64_t cnt, CpuFit* f, double* r1, double* r2) {
    if (cnt < 2) return false;
    double* x = new double[cnt];
    double* y = new double[cnt];
    for (uint64_t i = 0; i < cnt; ++i) y[i] = s->t_cpu_ms[idx[i]];
    const olap_cpu_form f1 = s->op == OLAP_OP_TOPK ? OLAP_CPU_NLOGN : OLAP_CPU_NM;
    for (uint64_t i = 0; i < cnt; ++i) x[i] = cpu_x(f1, s->n[idx[i]], s->k_or_m[idx[i]]);
    bool distinct = false;
    for (uint64_t i = 1; i < cnt; ++i) distinct = distinct || x[i] != x[0];
    ols(x, y, cnt, s->weighting, &f->a1, &f->b1);
    *r1 += rss(x, y, cnt, s->weighting, f->a1, f->b1);
    f->a2 = f->b2 = 0.0;
    if (s->op == OLAP_OP_TOPK) {
        for (uint64_t i = 0; i < cnt; ++i) x[i] = cpu_x(OLAP_CPU_NK, s->n[idx[i]], s->k_or_m[idx[i]]);
        ols(x, y, cnt, s->weighting, &f->a2, &f->b2);
        *r2 += rss(x, y, cnt, s->weighting, f->a2, f->b2);
    }
    delete[] x;
    delete[] y;
    return distinct;
}

}  // namespace

extern "C" {

olap_status olap_gate_calibrate(const olap_gate_samples* s, double margin_ms, olap_gate_model* out) {
    if (!s || !out || s->count < 2 || !s->n || !s->k_or_m || !s->tx_bytes || !s->out_rows || !s->t_cpu_ms ||
        !s->t_tx_ms || !s->t_ker_ms || !s->t_post_ms)
        return OLAP_E_INVALID;
    if (s->op != OLAP_OP_TOPK && s->op != OLAP_OP_PROBE) return OLAP_E_INVALID;
    if (s->weighting != OLAP_FIT_ORDINARY && s->weighting != OLAP_FIT_RELATIVE) return OLAP_E_INVALID;
    if (s->topk_cpu != 0 && s->topk_cpu != OLAP_CPU_MAX) return OLAP_E_INVALID;
    if (!(s->cpu_split_n >= 0.0)) return OLAP_E_INVALID;
    const uint64_t n = s->count;
    olap_gate_model m;
    std::memset(&m, 0, sizeof(m));
    m.op = s->op;
    m.margin_ms = margin_ms;
    // the samples of each CPU regime (one regime when there is no split)
    uint64_t* lo = new uint64_t[n];
    uint64_t* hi = new uint64_t[n];
    uint64_t nlo = 0, nhi = 0;
    for (uint64_t i = 0; i < n; ++i) {
        if (s->cpu_split_n > 0.0 && s->n[i] >= s->cpu_split_n) hi[nhi++] = i;
        else lo[nlo++] = i;
    }
    CpuFit fl{}, fh{};
    double r1 = 0.0, r2 = 0.0;
    bool ok = fit_cpu(s, lo, nlo, &fl, &r1, &r2);
    if (ok && s->cpu_split_n > 0.0) ok = fit_cpu(s, hi, nhi, &fh, &r1, &r2);
    delete[] lo;
    delete[] hi;
    if (!ok && s->cpu_split_n > 0.0) return OLAP_E_INVALID;
    if (s->op == OLAP_OP_TOPK) {
        m.rss_nlogn = r1;
        m.rss_nk = r2;
        m.cpu_form = s->topk_cpu == OLAP_CPU_MAX ? OLAP_CPU_MAX : (r1 <= r2 ? OLAP_CPU_NLOGN : OLAP_CPU_NK);
    } else {
        m.cpu_form = OLAP_CPU_NM;
    }
    // a, b hold the chosen form (N*log2 N for the two-form maximum, whose
    // N*K fit goes to a2, b2); likewise for the upper regime
    const bool nk = m.cpu_form == OLAP_CPU_NK;
    m.a = nk ? fl.a2 : fl.a1;
    m.b = nk ? fl.b2 : fl.b1;
    if (m.cpu_form == OLAP_CPU_MAX) {
        m.a2 = fl.a2;
        m.b2 = fl.b2;
    }
    if (s->cpu_split_n > 0.0) {
        m.split_n = s->cpu_split_n;
        m.a_hi = nk ? fh.a2 : fh.a1;
        m.b_hi = nk ? fh.b2 : fh.b1;
        if (m.cpu_form == OLAP_CPU_MAX) {
            m.a2_hi = fh.a2;
            m.b2_hi = fh.b2;
        }
    }
    ols(s->tx_bytes, s->t_tx_ms, n, s->weighting, &m.c, &m.d);
    ols(s->n, s->t_ker_ms, n, s->weighting, &m.e, &m.f);
    ols(s->out_rows, s->t_post_ms, n, s->weighting, &m.g, &m.h);
    *out = m;
    return OLAP_OK;
}

olap_status olap_gate_estimate(const olap_gate_model* m, const olap_gate_query* q, olap_gate_decision* out) {
    if (!m || !q || !out) return OLAP_E_INVALID;
    if (q->op != m->op) return OLAP_E_INVALID;
    const Costs c = costs(*m, static_cast<double>(q->n), q->k_or_m, q->tx_bytes, q->out_rows);
    out->c_cpu = c.cpu;
    out->c_tx = c.tx;
    out->c_ker = c.ker;
    out->c_post = c.post;
    out->c_gpu = c.tx + c.ker + c.post;
    out->gain_ms = c.cpu - out->c_gpu;
    out->margin_ms = m->margin_ms;
    out->offload = out->gain_ms > m->margin_ms ? 1 : 0;
    out->n_star = n_star(*m, *q);
    return OLAP_OK;
}

}  // extern "C"
