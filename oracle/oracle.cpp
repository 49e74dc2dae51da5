// Plain, slow CPU oracle for the key-only OLAP primitives.
//
// TEST INFRASTRUCTURE ONLY.  This file is compiled into a separate shared
// library that only the test-suite, the smoke check and the benchmark's
// CPU-baseline leg load.  It shares no code, header, table or constant with
// the CUDA library, and the CUDA library never calls it.
//
// Each function is the plain definition of what the offloaded primitive
// returns, written for obviousness, not speed:
//   * Top-K (Sec. III-A, "LIMIT-based Top-K selection ... returning pointers
//     of the Top-K results"; Sec. V-B, ORDER BY value DESC LIMIT 100): build
//     the (key, row-id) pairs, stable-sort them by key in the requested order
//     with row-id ascending as the tie-break, keep the first min(k, n).
//   * Top-K over a two-column key (ORDER BY c0, c1 LIMIT K): the same with
//     the rows compared column by column, each in its own order.
//   * Join probe (Sec. III-B, "key-only hash table ... pointer return"; Sec.
//     II-C, "returns ... a set of matched pointers"): every (probe row-id,
//     build row-id) pair whose keys are equal, as a sorted multiset.
//
// Readings of points the paper leaves open (ties for ASC, K > N, float order)
// follow the library's documented contract: row-id ascending breaks ties in
// both orders; the output has min(k, n) entries; float32 and float64 keys
// (the paper's key column is a double, Sec. V-A) are ordered by IEEE 754-2019
// totalOrder (Sec. 5.10), implemented below from its case definition rather
// than from any bit trick; integer keys by their value (signed or unsigned).
// Key types: 0 int64, 1 float32, 2 float64, 3 uint64, 4 int32, 5 uint32.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace {

// IEEE 754-2019 Sec. 5.10 totalOrder(x, y) restricted to "x strictly below y",
// binary32.  The cases, in the standard's order:
//   * x < y numerically (neither NaN)               -> below
//   * x == y: -0 is below +0; equal non-zero values have equal encodings
//   * a NaN with the sign bit set is below every non-NaN; one with the sign
//     bit clear is above every non-NaN
//   * two NaNs: a negative one is below a positive one; for positive NaNs the
//     smaller (quiet bit, payload) field, read as an integer, is below; for
//     negative NaNs the larger one is below
// The same case list for any binary format: F is float or double, B its bit
// pattern type, FRAC the mask of its trailing significand (quiet bit and
// payload) field.
template <typename F, typename B, B FRAC>
bool total_below(B xb, B yb) {
    F x, y;
    std::memcpy(&x, &xb, sizeof(F));
    std::memcpy(&y, &yb, sizeof(F));
    const bool xn = std::isnan(x), yn = std::isnan(y);
    const bool xs = std::signbit(x), ys = std::signbit(y);
    if (xn && yn) {
        if (xs != ys) return xs;
        const B xf = xb & FRAC, yf = yb & FRAC;
        return xs ? (xf > yf) : (xf < yf);
    }
    if (xn) return xs;       // -NaN below all non-NaN, +NaN above all
    if (yn) return !ys;      // x below +NaN, above -NaN
    if (x < y) return true;
    if (x > y) return false;
    if (x == F(0)) return xs && !ys;   // -0 below +0
    return false;
}

bool f32_total_below(uint32_t xb, uint32_t yb) { return total_below<float, uint32_t, 0x007FFFFFu>(xb, yb); }
bool f64_total_below(uint64_t xb, uint64_t yb) {
    return total_below<double, uint64_t, 0x000FFFFFFFFFFFFFull>(xb, yb);
}

int key_width(int key_type) { return (key_type == 1 || key_type == 4 || key_type == 5) ? 4 : 8; }

struct Row {
    uint64_t key;     // raw key bits (4-byte keys in the low half)
    uint32_t rowid;
};

struct Less {
    int key_type;     // see the file header
    int order;        // 0 = ascending, 1 = descending
    bool key_below(uint64_t a, uint64_t b) const {
        switch (key_type) {
            case 0: return static_cast<int64_t>(a) < static_cast<int64_t>(b);
            case 1: return f32_total_below(static_cast<uint32_t>(a), static_cast<uint32_t>(b));
            case 2: return f64_total_below(a, b);
            case 3: return a < b;
            case 4:
                return static_cast<int32_t>(static_cast<uint32_t>(a)) < static_cast<int32_t>(static_cast<uint32_t>(b));
            default: return static_cast<uint32_t>(a) < static_cast<uint32_t>(b);
        }
    }
    bool operator()(const Row& a, const Row& b) const {
        const bool ab = order == 0 ? key_below(a.key, b.key) : key_below(b.key, a.key);
        if (ab) return true;
        const bool ba = order == 0 ? key_below(b.key, a.key) : key_below(a.key, b.key);
        if (ba) return false;
        return a.rowid < b.rowid;
    }
};

// Two-column key (ORDER BY c0, c1): the rows in lexicographic order of
// (c0 in its order, c1 in its order), then row-id ascending.
struct Row2 {
    uint64_t k0, k1;  // raw key bits of each column
    uint32_t rowid;
};

struct Less2 {
    Less c0, c1;      // each column's own comparator (its rowid tie-break unused)
    bool operator()(const Row2& a, const Row2& b) const {
        const bool a0 = c0.order == 0 ? c0.key_below(a.k0, b.k0) : c0.key_below(b.k0, a.k0);
        if (a0) return true;
        const bool b0 = c0.order == 0 ? c0.key_below(b.k0, a.k0) : c0.key_below(a.k0, b.k0);
        if (b0) return false;
        const bool a1 = c1.order == 0 ? c1.key_below(a.k1, b.k1) : c1.key_below(b.k1, a.k1);
        if (a1) return true;
        const bool b1 = c1.order == 0 ? c1.key_below(b.k1, a.k1) : c1.key_below(a.k1, b.k1);
        if (b1) return false;
        return a.rowid < b.rowid;
    }
};

uint64_t read_key(const void* keys, int key_type, uint64_t i) {
    if (key_width(key_type) == 8) {
        uint64_t v;
        std::memcpy(&v, static_cast<const uint64_t*>(keys) + i, 8);
        return v;
    }
    uint32_t v;
    std::memcpy(&v, static_cast<const uint32_t*>(keys) + i, 4);
    return v;
}

void write_key(void* out, int key_type, uint64_t i, uint64_t v) {
    if (key_width(key_type) == 8) {
        std::memcpy(static_cast<uint64_t*>(out) + i, &v, 8);
    } else {
        const uint32_t w = static_cast<uint32_t>(v);
        std::memcpy(static_cast<uint32_t*>(out) + i, &w, 4);
    }
}

}  // namespace

extern "C" {

// Top-K over a two-column key: the first min(k, n) rows of the stable sort by
// (c0 in order0, c1 in order1, row-id ascending); each output column receives
// its own key bits.  Any key types.  Returns the count.
uint64_t oracle_topk_pair(int type0, const void* keys0, int order0, int type1, const void* keys1, int order1,
                          const uint32_t* rowids, uint64_t n, uint64_t k, void* out0, void* out1,
                          uint32_t* out_rowids) {
    std::vector<Row2> rows(n);
    for (uint64_t i = 0; i < n; ++i) {
        rows[i].k0 = read_key(keys0, type0, i);
        rows[i].k1 = read_key(keys1, type1, i);
        rows[i].rowid = rowids ? rowids[i] : static_cast<uint32_t>(i);
    }
    std::stable_sort(rows.begin(), rows.end(), Less2{Less{type0, order0}, Less{type1, order1}});
    const uint64_t cnt = std::min(k, n);
    for (uint64_t i = 0; i < cnt; ++i) {
        write_key(out0, type0, i, rows[i].k0);
        write_key(out1, type1, i, rows[i].k1);
        out_rowids[i] = rows[i].rowid;
    }
    return cnt;
}


// Top-K: out_keys (same element type as keys) and out_rowids receive the
// first min(k, n) rows of the ordering; returns that count.  rowids == NULL
// means row-id = index (index must fit in 32 bits).
uint64_t oracle_topk(int key_type, const void* keys, const uint32_t* rowids, uint64_t n,
                     uint64_t k, int order, void* out_keys, uint32_t* out_rowids) {
    std::vector<Row> rows(n);
    const int w = key_width(key_type);
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t kb;
        if (w == 8) {
            std::memcpy(&kb, static_cast<const uint64_t*>(keys) + i, 8);
        } else {
            uint32_t v;
            std::memcpy(&v, static_cast<const uint32_t*>(keys) + i, 4);
            kb = v;
        }
        rows[i].key = kb;
        rows[i].rowid = rowids ? rowids[i] : static_cast<uint32_t>(i);
    }
    std::stable_sort(rows.begin(), rows.end(), Less{key_type, order});
    const uint64_t cnt = std::min(k, n);
    for (uint64_t i = 0; i < cnt; ++i) {
        if (w == 8) {
            std::memcpy(static_cast<uint64_t*>(out_keys) + i, &rows[i].key, 8);
        } else {
            const uint32_t v = static_cast<uint32_t>(rows[i].key);
            std::memcpy(static_cast<uint32_t*>(out_keys) + i, &v, 4);
        }
        out_rowids[i] = rows[i].rowid;
    }
    return cnt;
}

// Full ascending sort of (key, row-id) (the ORDER BY foil of Sec. V-B); the
// same ordering as oracle_topk with k = n.
void oracle_sort(int key_type, const void* keys, const uint32_t* rowids, uint64_t n, int order,
                 void* out_keys, uint32_t* out_rowids) {
    oracle_topk(key_type, keys, rowids, n, n, order, out_keys, out_rowids);
}

// Join: all pairs (probe row-id, build row-id) with equal int64 keys, packed
// as (probe << 32 | build) and sorted ascending.  Steps: sort a copy of the
// build rows by key; for every probe row in index order take the equal range
// and emit one pair per build row in it; sort the packed pairs.  The result
// buffer is malloc'd; *out receives it (free with oracle_free) and the
// return value is the number of pairs.
uint64_t oracle_join(const int64_t* bkeys, const uint32_t* brow, uint64_t nb,
                     const int64_t* pkeys, const uint32_t* prow, uint64_t np, uint64_t** out) {
    std::vector<std::pair<int64_t, uint32_t>> build(nb);
    for (uint64_t i = 0; i < nb; ++i)
        build[i] = {bkeys[i], brow ? brow[i] : static_cast<uint32_t>(i)};
    std::sort(build.begin(), build.end(),
              [](const std::pair<int64_t, uint32_t>& a, const std::pair<int64_t, uint32_t>& b) {
                  return a.first < b.first;
              });
    std::vector<uint64_t> pairs;
    for (uint64_t p = 0; p < np; ++p) {
        const int64_t key = pkeys[p];
        auto lo = std::lower_bound(build.begin(), build.end(), key,
                                   [](const std::pair<int64_t, uint32_t>& e, int64_t v) { return e.first < v; });
        const uint64_t pr = prow ? prow[p] : static_cast<uint32_t>(p);
        for (auto it = lo; it != build.end() && it->first == key; ++it)
            pairs.push_back((pr << 32) | it->second);
    }
    std::sort(pairs.begin(), pairs.end());
    uint64_t* buf = static_cast<uint64_t*>(std::malloc(std::max<size_t>(1, pairs.size()) * 8));
    if (!pairs.empty()) std::memcpy(buf, pairs.data(), pairs.size() * 8);
    *out = buf;
    return pairs.size();
}

// Nested-loop join for tiny inputs: the same definition with no sort and no
// search, one comparison per (probe, build) pair.
uint64_t oracle_join_nested(const int64_t* bkeys, const uint32_t* brow, uint64_t nb,
                            const int64_t* pkeys, const uint32_t* prow, uint64_t np, uint64_t** out) {
    std::vector<uint64_t> pairs;
    for (uint64_t p = 0; p < np; ++p)
        for (uint64_t b = 0; b < nb; ++b)
            if (pkeys[p] == bkeys[b]) {
                const uint64_t pr = prow ? prow[p] : static_cast<uint32_t>(p);
                const uint64_t br = brow ? brow[b] : static_cast<uint32_t>(b);
                pairs.push_back((pr << 32) | br);
            }
    std::sort(pairs.begin(), pairs.end());
    uint64_t* buf = static_cast<uint64_t*>(std::malloc(std::max<size_t>(1, pairs.size()) * 8));
    if (!pairs.empty()) std::memcpy(buf, pairs.data(), pairs.size() * 8);
    *out = buf;
    return pairs.size();
}

void oracle_free(void* p) { std::free(p); }

// Exposed so a test can check the comparator alone against IEEE's listed
// ordering of special values.
int oracle_f32_total_below(uint32_t x, uint32_t y) { return f32_total_below(x, y) ? 1 : 0; }
int oracle_f64_total_below(uint64_t x, uint64_t y) { return f64_total_below(x, y) ? 1 : 0; }

}  // extern "C"
