// Risky Gate (Sec. II-B) with measured constants fitted by least squares and
// the break-even N* (Sec. V-D).  Pure host arithmetic in fp64.
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
    if (m.cpu_form == OLAP_CPU_MAX)
        c.cpu = std::max(m.a * cpu_x(OLAP_CPU_NLOGN, n, k_or_m) + m.b, m.a2 * cpu_x(OLAP_CPU_NK, n, k_or_m) + m.b2);
    else
        c.cpu = m.a * cpu_x(m.cpu_form, n, k_or_m) + m.b;
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

uint64_t n_star(const olap_gate_model& m, const olap_gate_query& q) {
    if (gain(m, q, 1) > 0.0) return 1;
    if (!(gain(m, q, N_STAR_HI) > 0.0)) return 0;
    uint64_t lo = 1, hi = N_STAR_HI;
    while (hi - lo > 1) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (gain(m, q, mid) > 0.0) hi = mid;
        else lo = mid;
    }
    return hi;
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
    const uint64_t n = s->count;
    olap_gate_model m;
    std::memset(&m, 0, sizeof(m));
    m.op = s->op;
    m.margin_ms = margin_ms;
    double* x = new double[n];
    if (s->op == OLAP_OP_TOPK) {
        double a1, b1, a2, b2;
        for (uint64_t i = 0; i < n; ++i) x[i] = cpu_x(OLAP_CPU_NLOGN, s->n[i], s->k_or_m[i]);
        ols(x, s->t_cpu_ms, n, s->weighting, &a1, &b1);
        m.rss_nlogn = rss(x, s->t_cpu_ms, n, s->weighting, a1, b1);
        for (uint64_t i = 0; i < n; ++i) x[i] = cpu_x(OLAP_CPU_NK, s->n[i], s->k_or_m[i]);
        ols(x, s->t_cpu_ms, n, s->weighting, &a2, &b2);
        m.rss_nk = rss(x, s->t_cpu_ms, n, s->weighting, a2, b2);
        if (s->topk_cpu == OLAP_CPU_MAX) {
            m.cpu_form = OLAP_CPU_MAX;
            m.a = a1;
            m.b = b1;
            m.a2 = a2;
            m.b2 = b2;
        } else if (m.rss_nlogn <= m.rss_nk) {
            m.cpu_form = OLAP_CPU_NLOGN;
            m.a = a1;
            m.b = b1;
        } else {
            m.cpu_form = OLAP_CPU_NK;
            m.a = a2;
            m.b = b2;
        }
    } else {
        m.cpu_form = OLAP_CPU_NM;
        for (uint64_t i = 0; i < n; ++i) x[i] = cpu_x(OLAP_CPU_NM, s->n[i], s->k_or_m[i]);
        ols(x, s->t_cpu_ms, n, s->weighting, &m.a, &m.b);
    }
    delete[] x;
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
