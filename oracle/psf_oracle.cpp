// psf_oracle.cpp -- CPU oracle for the progressive spatio-temporal filtering hot path.
//
// TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and the
// benchmark's CPU-baseline leg may load this library.  It shares no code, header,
// table or constant generator with the CUDA library: everything below is written
// out again from the paper's definitions.  Inputs come from the seeded generator
// module or from the tests themselves, never from the CUDA path.
//
// It is deliberately plain and slow: a std::map keyed by the full quantised cell
// tuple, one vertex at a time, FP64 blend and FP64 control variate.
//
// Passages followed (Pantaleoni, "Online path sampling control with progressive
// spatio-temporal filtering"):
//   * cell keys: Section "Basis functions and data structures: spatio-directional
//     hashing" -- basis functions are a grid over position times a grid over the
//     outgoing direction omega_o (the normal bin is an optional extra key field);
//   * accumulation: eq. (5) (c_h = sum of b_h * w) and eq. (6) (weighted sum of the
//     vertex values), in the order of Alg. 1 (increment_counters / update_approx);
//   * blend: Section "Temporal averaging", eq. (10) and eq. (11), with the global
//     counter reset described after eq. (11);
//   * query: Section "Control variates", equation CVEstimator, restated in the
//     estimator-value form out = L - beta * (t * C_next) + beta * C_self;
//   * biased query: Section "Biased estimation", equation BiasedEstimator,
//     out = gamma * (L - t * C_next) + C_self;
//   * progressive update values: Section "Progressive solver", eq. (9), Alg. 1 and 2;
//   * hierarchy levels: Section "Progressive hierarchical solver" (cells 2^l times wider at
//     level l; the level a vertex reads follows its path depth -- a reading, the paper's
//     footprint heuristic is only cited).
//
// Precision: the decisions that produce integers (cell indices, direction bins,
// fixed-point codes) are taken in FP32 with one correctly rounded IEEE operation
// per step, in the order written below, because the kernel takes them in FP32.
// This file must be compiled with -ffp-contract=off and without -ffast-math.
// Everything downstream of the integer sums (blend, query) is FP64.
//
// Parity status: every function is pinned by the CPU test suite (brute force,
// sum invariants, constant field, blend closed form, control-variate mean,
// hand-derived keys, octahedral decode/encode round trip).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

namespace {

constexpr uint32_t ST_TABLE_FULL = 1u;  // not produced by the oracle (unbounded map)
constexpr uint32_t ST_RANGE = 2u;
constexpr uint32_t ST_SUM_RANGE = 8u;  // an iteration received enough vertices that a sum may wrap

struct Config {
    uint32_t pos_bits_q;
    uint32_t dir_bits_d;
    uint32_t use_normal;
    uint32_t frac_bits;
    uint32_t blend_mode;  // 0: eq. (11) square-root hybrid; 1: constant alpha = alpha_min
    uint32_t cv_max_depth;
    double alpha_min;
    double beta;
    uint32_t levels;      // hierarchy levels (Section "Progressive hierarchical solver"); 0 or 1 = flat
    uint32_t pad;
};

// (level, normal bin, direction bin u, direction bin v, cell x, cell y, cell z);
// cell indices are stored biased by 2^15 so that they are non-negative.
using CellKey = std::tuple<uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t>;

struct Cell {
    int64_t sum[3] = {0, 0, 0};  // this iteration: sum of round(w * L_c * 2^F)
    int64_t c_new = 0;           // this iteration: sum of round(w * 2^F)   (eq. 5)
    int64_t c_old = 0;           // all earlier iterations (eq. 10-11)
    double L[3] = {0.0, 0.0, 0.0};  // the approximant L~_{o,h}
};

struct Oracle {
    Config cfg;
    std::map<CellKey, Cell> cells;
    uint64_t dropped = 0;       // vertices rejected by the range rule
    uint64_t zero_weight = 0;   // vertices whose weight rounds to zero in fixed point
    uint64_t iter_vertices = 0; // vertices handed to the inserts since the last update
};

bool finite3(const float* a) { return std::isfinite(a[0]) && std::isfinite(a[1]) && std::isfinite(a[2]); }

// floor(p * 2^q) for one coordinate; false when outside the 16-bit biased range.
bool cell_index(float p, uint32_t q, uint32_t* biased) {
    double t = std::floor(static_cast<double>(p) * std::ldexp(1.0, static_cast<int>(q)));
    if (t < -32768.0 || t > 32767.0) return false;
    *biased = static_cast<uint32_t>(static_cast<int64_t>(t) + 32768);
    return true;
}

// Dominant axis of the normal (ties prefer x, then y) and its sign: 2*axis + (negative).
uint32_t normal_bin(float nx, float ny, float nz) {
    float ax = std::fabs(nx), ay = std::fabs(ny), az = std::fabs(nz);
    if (ax >= ay && ax >= az) return nx >= 0.0f ? 0u : 1u;
    if (ay >= az) return ny >= 0.0f ? 2u : 3u;
    return nz >= 0.0f ? 4u : 5u;
}

// Octahedral map of a direction onto [-1,1]^2 followed by a 2^d x 2^d grid.
// Upper hemisphere (z >= 0): (u, v) = (x, y) / (|x| + |y| + |z|).
// Lower hemisphere: the triangles are folded outwards,
//   (u, v) <- ((1 - |v|) * sgn(u), (1 - |u|) * sgn(v)), with sgn(0) = +1.
// Bin = floor((u + 1) * 2^(d-1)), clamped to [0, 2^d - 1].
bool direction_bins(float wx, float wy, float wz, uint32_t d, uint32_t* bu, uint32_t* bv) {
    float ax = std::fabs(wx), ay = std::fabs(wy), az = std::fabs(wz);
    float s = ax + ay;
    s = s + az;
    if (!(s > 0.0f) || !std::isfinite(s)) return false;
    float u = wx / s;
    float v = wy / s;
    if (wz < 0.0f) {
        float su = (u >= 0.0f) ? 1.0f : -1.0f;
        float sv = (v >= 0.0f) ? 1.0f : -1.0f;
        float fu = 1.0f - std::fabs(v);
        float fv = 1.0f - std::fabs(u);
        u = fu * su;
        v = fv * sv;
    }
    const float half = std::ldexp(1.0f, static_cast<int>(d) - 1);
    const int top = (1 << d) - 1;
    float gu = u + 1.0f;
    float gv = v + 1.0f;
    gu = gu * half;
    gv = gv * half;
    int iu = static_cast<int>(std::floor(gu));
    int iv = static_cast<int>(std::floor(gv));
    *bu = static_cast<uint32_t>(std::min(std::max(iu, 0), top));
    *bv = static_cast<uint32_t>(std::min(std::max(iv, 0), top));
    return true;
}

// The basis function b_h a vertex lands on at hierarchy level `level` (a single cell: b_h is
// an indicator).  Level l uses cells 2^l times wider: index floor(p * 2^(q - l)); a vertex
// has a cell at every level exactly when it has one at level 0.
bool vertex_cell(const Config& c, const float* v, CellKey* key, uint32_t level = 0) {
    const float* p = v;
    const float* n = v + 4;
    const float* d = v + 8;
    if (!finite3(p) || !finite3(n) || !finite3(d)) return false;
    uint32_t bx, by, bz;
    if (!cell_index(p[0], c.pos_bits_q, &bx) || !cell_index(p[1], c.pos_bits_q, &by) ||
        !cell_index(p[2], c.pos_bits_q, &bz))
        return false;
    if (level > 0) {
        const int q = static_cast<int>(c.pos_bits_q) - static_cast<int>(level);
        auto coarse = [q](float x) {
            return static_cast<uint32_t>(static_cast<int64_t>(std::floor(static_cast<double>(x) * std::ldexp(1.0, q))) + 32768);
        };
        bx = coarse(p[0]);
        by = coarse(p[1]);
        bz = coarse(p[2]);
    }
    uint32_t nb = c.use_normal ? normal_bin(n[0], n[1], n[2]) : 0u;
    uint32_t bu, bv;
    // omega_o = -d (Alg. 1: the outgoing direction is the reversed incoming ray)
    if (!direction_bins(-d[0], -d[1], -d[2], c.dir_bits_d, &bu, &bv)) return false;
    *key = CellKey(level, nb, bu, bv, bx, by, bz);
    return true;
}

uint32_t level_count(const Config& c) { return c.levels == 0 ? 1u : c.levels; }

// The level a vertex at path depth j reads (Section "Progressive hierarchical solver": the
// level follows the path's footprint).  Reading: the footprint widens with every bounce, so
// vertex j reads level min(j, levels - 1); a flat table reads level 0.
uint32_t read_level(const Config& c, int64_t j) {
    const int64_t top = static_cast<int64_t>(level_count(c)) - 1;
    return static_cast<uint32_t>(j < top ? j : top);
}

uint64_t pack_key(const Config& c, const CellKey& k) {
    uint64_t level = std::get<0>(k), nb = std::get<1>(k), bu = std::get<2>(k), bv = std::get<3>(k);
    uint64_t bx = std::get<4>(k), by = std::get<5>(k), bz = std::get<6>(k);
    uint64_t dbin = (bu << c.dir_bits_d) | bv;
    return (level << 61) | (nb << 58) | (dbin << 48) | (bx << 32) | (by << 16) | bz;
}

// Fixed-point sums add modulo 2^64 (two's complement), as 64-bit integer adders do: the
// result is defined even where a sum leaves the int64 range.
int64_t wrap_add(int64_t a, int64_t b) {
    return static_cast<int64_t>(static_cast<uint64_t>(a) + static_cast<uint64_t>(b));
}

// The sum-range rule: every accepted vertex adds codes of magnitude at most 2^(15+F)
// (|fl32(w L_c)| <= 2^15 and w <= 2^15) to a cell, so the sums are exact while fewer than
// 2^(48-F) vertices are inserted between two updates; `extra_bits` tightens the count for a
// payload with larger codes.  Returns ST_SUM_RANGE once the iteration's count reaches it.
uint32_t count_vertices(uint64_t* iter_vertices, uint64_t n, uint32_t frac_bits, uint32_t extra_bits) {
    *iter_vertices += n;
    return *iter_vertices >= (uint64_t{1} << (48u - frac_bits - extra_bits)) ? ST_SUM_RANGE : 0u;
}

int64_t sat_add(int64_t a, int64_t b) {
    // both operands are non-negative counters
    if (a > INT64_MAX - b) return INT64_MAX;
    return a + b;
}

}  // namespace

extern "C" {

typedef struct {
    uint32_t pos_bits_q;
    uint32_t dir_bits_d;
    uint32_t use_normal;
    uint32_t frac_bits;
    uint32_t blend_mode;
    uint32_t cv_max_depth;
    double alpha_min;
    double beta;
    uint32_t levels;
    uint32_t pad;
} oracle_config;

typedef struct {
    uint64_t key;
    int64_t sum[3];
    int64_t c_new;
    int64_t c_old;
    double L[3];
} oracle_record;

void* oracle_create(const oracle_config* cfg) {
    if (!cfg || cfg->dir_bits_d > 5 || cfg->pos_bits_q > 20 || cfg->frac_bits < 8 || cfg->frac_bits > 32 ||
        cfg->levels > 4)
        return nullptr;
    Oracle* o = new Oracle();
    std::memcpy(&o->cfg, cfg, sizeof(Config));
    return o;
}

void oracle_destroy(void* h) { delete static_cast<Oracle*>(h); }

// Packed key of one 16-float vertex record; returns 1 if the vertex has a cell.
int oracle_key(const oracle_config* cfg, const float* v, uint64_t* key) {
    Config c;
    std::memcpy(&c, cfg, sizeof(Config));
    CellKey k;
    if (!vertex_cell(c, v, &k)) return 0;
    *key = pack_key(c, k);
    return 1;
}

// As oracle_key, for the vertex's cell at hierarchy level `level` (< 4).
int oracle_key_at(const oracle_config* cfg, const float* v, uint32_t level, uint64_t* key) {
    Config c;
    std::memcpy(&c, cfg, sizeof(Config));
    CellKey k;
    if (level > 3 || !vertex_cell(c, v, &k, level)) return 0;
    *key = pack_key(c, k);
    return 1;
}

// Scatter n vertices (eq. 5 and 6 accumulated in fixed point).  Returns status bits.
uint32_t oracle_insert(void* h, const float* verts, uint64_t n) {
    Oracle* o = static_cast<Oracle*>(h);
    const Config& c = o->cfg;
    const double scale = std::ldexp(1.0, static_cast<int>(c.frac_bits));
    uint32_t status = 0;
    for (uint64_t i = 0; i < n; ++i) {
        const float* v = verts + 16 * i;
        CellKey key;
        bool ok = vertex_cell(c, v, &key);
        const float w = v[3];
        ok = ok && (w >= 0.0f) && (w <= 32768.0f);
        float prod[3] = {0.0f, 0.0f, 0.0f};
        for (int ch = 0; ch < 3 && ok; ++ch) {
            prod[ch] = w * v[12 + ch];  // one FP32 rounding of w * L_c
            ok = std::isfinite(prod[ch]) && std::fabs(prod[ch]) <= 32768.0f;
        }
        if (!ok) {
            status |= ST_RANGE;
            o->dropped++;
            continue;
        }
        const int64_t cw = std::llrint(static_cast<double>(w) * scale);
        if (cw == 0) {
            o->zero_weight++;
            continue;
        }
        for (uint32_t l = 0; l < level_count(c); ++l) {  // every level's cell receives the vertex
            vertex_cell(c, v, &key, l);
            Cell& cell = o->cells[key];
            for (int ch = 0; ch < 3; ++ch)
                cell.sum[ch] = wrap_add(cell.sum[ch], std::llrint(static_cast<double>(prod[ch]) * scale));
            cell.c_new = wrap_add(cell.c_new, cw);
        }
    }
    return status | count_vertices(&o->iter_vertices, n, c.frac_bits, 0u);
}

// Progressive update values (Section "Progressive solver", eq. (9); Alg. 1 and Alg. 2):
// the value scattered for vertex j comes from the current approximant L~old at the next
// vertex of its path instead of from the path's own tail.  The record's v3.xyz is read as
// the emitted radiance L_e of the vertex; t_j is its throughput to vertex j + 1.
//   field 0, L~_o     (Alg. 1): value_j = L_e,j + t_j * L~old(x_{j+1})     (last vertex: L_e,j)
//   field 1, L~_{o\e} (Alg. 2): value_j = t_j * (L_e,j+1 + L~old(x_{j+1}))  (last vertex: 0;
//                               the optional next-event-estimation term is not modelled)
// L~old is read before anything of this call is scattered.  Each vertex is then scattered
// as oracle_insert does, with L = value_j (fixed point of w * value in FP64, saturated at
// |w * value| = 2^15; the range rule is applied to the vertex's own record).
uint32_t oracle_insert_progressive(void* h, const float* verts, uint32_t P, uint32_t D, uint32_t field) {
    Oracle* o = static_cast<Oracle*>(h);
    const Config& c = o->cfg;
    const double scale = std::ldexp(1.0, static_cast<int>(c.frac_bits));
    const uint64_t n = static_cast<uint64_t>(P) * D;
    std::vector<double> value(3 * n, 0.0);
    for (uint64_t p = 0; p < P; ++p) {
        double C_next[3] = {0.0, 0.0, 0.0}, Le_next[3] = {0.0, 0.0, 0.0};
        for (int64_t j = static_cast<int64_t>(D) - 1; j >= 0; --j) {
            const uint64_t idx = static_cast<uint64_t>(j) * P + p;
            const float* v = verts + 16 * idx;
            const double t[3] = {v[7], v[11], v[15]};
            double C[3] = {0.0, 0.0, 0.0};
            CellKey key;
            if (vertex_cell(c, v, &key, read_level(c, j))) {
                auto it = o->cells.find(key);
                if (it != o->cells.end())
                    for (int ch = 0; ch < 3; ++ch) C[ch] = it->second.L[ch];
            }
            for (int ch = 0; ch < 3; ++ch) {
                const double Le = v[12 + ch];
                value[3 * idx + ch] = field == 0 ? Le + t[ch] * C_next[ch] : t[ch] * (Le_next[ch] + C_next[ch]);
                C_next[ch] = C[ch];
                Le_next[ch] = Le;
            }
        }
    }
    // A vertex is dropped when its own record fails the range rule (with its L_e as the value:
    // |fl32(w L_e,c)| <= 2^15, finite throughput) or its computed value is NaN; otherwise the
    // product w * value saturates at +-2^15, so the FP64 value here and the FP32 value of a
    // kernel take the same decision even at the bound.
    uint32_t status = 0;
    for (uint64_t i = 0; i < n; ++i) {
        const float* v = verts + 16 * i;
        CellKey key;
        bool ok = vertex_cell(c, v, &key);
        const double w = v[3];
        ok = ok && (w >= 0.0) && (w <= 32768.0);
        for (int ch = 0; ch < 3 && ok; ++ch) {
            const float own = v[3] * v[12 + ch];  // one FP32 rounding, as oracle_insert
            ok = std::isfinite(own) && std::fabs(own) <= 32768.0f && std::isfinite(v[ch == 0 ? 7 : ch == 1 ? 11 : 15]);
        }
        double prod[3] = {0.0, 0.0, 0.0};
        for (int ch = 0; ch < 3 && ok; ++ch) {
            prod[ch] = w * value[3 * i + ch];
            ok = !std::isnan(prod[ch]);
            prod[ch] = std::min(std::max(prod[ch], -32768.0), 32768.0);
        }
        if (!ok) {
            status |= ST_RANGE;
            o->dropped++;
            continue;
        }
        const int64_t cw = std::llrint(w * scale);
        if (cw == 0) {
            o->zero_weight++;
            continue;
        }
        for (uint32_t l = 0; l < level_count(c); ++l) {
            vertex_cell(c, v, &key, l);
            Cell& cell = o->cells[key];
            for (int ch = 0; ch < 3; ++ch) cell.sum[ch] = wrap_add(cell.sum[ch], std::llrint(prod[ch] * scale));
            cell.c_new = wrap_add(cell.c_new, cw);
        }
    }
    return status | count_vertices(&o->iter_vertices, n, c.frac_bits, 0u);
}

// End-of-iteration temporal blend, eq. (10)-(11), for every cell touched this iteration.
uint32_t oracle_update(void* h) {
    Oracle* o = static_cast<Oracle*>(h);
    const Config& c = o->cfg;
    for (auto& kv : o->cells) {
        Cell& cell = kv.second;
        if (cell.c_new == 0) continue;  // not touched this iteration: left as it is
        if (cell.c_new < 0) {  // the counter wrapped (ST_SUM_RANGE): this iteration's sums are dropped
            for (int ch = 0; ch < 3; ++ch) cell.sum[ch] = 0;
            cell.c_new = 0;
            continue;
        }
        const double cn = static_cast<double>(cell.c_new);
        const double co = static_cast<double>(cell.c_old);
        double alpha;
        if (c.blend_mode == 0)
            alpha = std::max(std::sqrt(cn / (co + cn)), c.alpha_min);
        else
            alpha = c.alpha_min;
        for (int ch = 0; ch < 3; ++ch) {
            const double mean = static_cast<double>(cell.sum[ch]) / cn;
            cell.L[ch] = (1.0 - alpha) * cell.L[ch] + alpha * mean;
            cell.sum[ch] = 0;
        }
        cell.c_old = sat_add(cell.c_old, cell.c_new);
        cell.c_new = 0;
    }
    o->iter_vertices = 0;
    return 0;
}

// Global counter reset (the text after eq. (11)): c_old := 0 everywhere, approximant kept.
void oracle_reset(void* h) {
    Oracle* o = static_cast<Oracle*>(h);
    for (auto& kv : o->cells) kv.second.c_old = 0;
}

// Control-variate query (Section "Control variates", equation CVEstimator) for P paths of
// depth D in depth-major order; out receives D*P*3 doubles in the same order.
// For vertex j of a path, C_j is the approximant of the cell the vertex lands on (0 when the
// cell is absent) and t_j the RGB throughput to vertex j+1:
//   out_j = L_j - beta * t_j * C_{j+1} + beta * C_j   for j < min(D - 1, cv_max_depth),
//   out_j = L_j                                        otherwise.
void oracle_query_cv(void* h, const float* verts, uint32_t P, uint32_t D, double* out) {
    Oracle* o = static_cast<Oracle*>(h);
    const Config& c = o->cfg;
    for (uint64_t p = 0; p < P; ++p) {
        double C_next[3] = {0.0, 0.0, 0.0};
        for (int64_t j = static_cast<int64_t>(D) - 1; j >= 0; --j) {
            const uint64_t idx = static_cast<uint64_t>(j) * P + p;
            const float* v = verts + 16 * idx;
            double C[3] = {0.0, 0.0, 0.0};
            CellKey key;
            if (vertex_cell(c, v, &key, read_level(c, j))) {
                auto it = o->cells.find(key);
                if (it != o->cells.end())
                    for (int ch = 0; ch < 3; ++ch) C[ch] = it->second.L[ch];
            }
            const double t[3] = {v[7], v[11], v[15]};
            const bool cv = (j + 1 < static_cast<int64_t>(D)) && (static_cast<uint64_t>(j) < c.cv_max_depth);
            for (int ch = 0; ch < 3; ++ch) {
                const double L = v[12 + ch];
                out[3 * idx + ch] = cv ? (L - c.beta * (t[ch] * C_next[ch]) + c.beta * C[ch]) : L;
            }
            for (int ch = 0; ch < 3; ++ch) C_next[ch] = C[ch];
        }
    }
}

// Biased predictor-corrector estimator (Section "Biased estimation", equation
// BiasedEstimator: the control-variate estimator at beta = 1 with the corrector scaled by
// gamma).  For vertex j of a path with j_begin <= j < j_end and a successor:
//   out_j = gamma * (L_j - t_j * C_{j+1}) + C_j
// and out_j = L_j for every other vertex.  gamma = 0 at j = 1 alone is the paper's PSTF-B.
void oracle_query_biased(void* h, const float* verts, uint32_t P, uint32_t D, double gamma, uint32_t j_begin,
                         uint32_t j_end, double* out) {
    Oracle* o = static_cast<Oracle*>(h);
    const Config& c = o->cfg;
    for (uint64_t p = 0; p < P; ++p) {
        double C_next[3] = {0.0, 0.0, 0.0};
        for (int64_t j = static_cast<int64_t>(D) - 1; j >= 0; --j) {
            const uint64_t idx = static_cast<uint64_t>(j) * P + p;
            const float* v = verts + 16 * idx;
            double C[3] = {0.0, 0.0, 0.0};
            CellKey key;
            if (vertex_cell(c, v, &key, read_level(c, j))) {
                auto it = o->cells.find(key);
                if (it != o->cells.end())
                    for (int ch = 0; ch < 3; ++ch) C[ch] = it->second.L[ch];
            }
            const double t[3] = {v[7], v[11], v[15]};
            const bool on = (j + 1 < static_cast<int64_t>(D)) && (static_cast<uint64_t>(j) >= j_begin) &&
                            (static_cast<uint64_t>(j) < j_end);
            for (int ch = 0; ch < 3; ++ch) {
                const double L = v[12 + ch];
                out[3 * idx + ch] = on ? (gamma * (L - t[ch] * C_next[ch]) + C[ch]) : L;
            }
            for (int ch = 0; ch < 3; ++ch) C_next[ch] = C[ch];
        }
    }
}

// The approximant of each vertex's cell (0 when absent), as the query reads it: C_out
// receives n*3 doubles.  Used by tests to form the norm-wise error bound of the query.
void oracle_lookup(void* h, const float* verts, uint64_t n, double* C_out) {
    Oracle* o = static_cast<Oracle*>(h);
    for (uint64_t i = 0; i < n; ++i) {
        double* C = C_out + 3 * i;
        C[0] = C[1] = C[2] = 0.0;
        CellKey key;
        if (!vertex_cell(o->cfg, verts + 16 * i, &key)) continue;
        auto it = o->cells.find(key);
        if (it != o->cells.end())
            for (int ch = 0; ch < 3; ++ch) C[ch] = it->second.L[ch];
    }
}

// As oracle_lookup for P paths of depth D (depth-major): vertex j reads its cell at the level
// min(j, levels - 1), as the queries do.
void oracle_lookup_paths(void* h, const float* verts, uint32_t P, uint32_t D, double* C_out) {
    Oracle* o = static_cast<Oracle*>(h);
    for (uint64_t j = 0; j < D; ++j)
        for (uint64_t p = 0; p < P; ++p) {
            const uint64_t i = j * P + p;
            double* C = C_out + 3 * i;
            C[0] = C[1] = C[2] = 0.0;
            CellKey key;
            if (!vertex_cell(o->cfg, verts + 16 * i, &key, read_level(o->cfg, static_cast<int64_t>(j)))) continue;
            auto it = o->cells.find(key);
            if (it != o->cells.end())
                for (int ch = 0; ch < 3; ++ch) C[ch] = it->second.L[ch];
        }
}

uint64_t oracle_size(void* h) { return static_cast<Oracle*>(h)->cells.size(); }

void oracle_counters(void* h, uint64_t* dropped, uint64_t* zero_weight) {
    Oracle* o = static_cast<Oracle*>(h);
    *dropped = o->dropped;
    *zero_weight = o->zero_weight;
}

// All cells in ascending packed-key order; returns the number written (at most cap).
uint64_t oracle_export(void* h, oracle_record* out, uint64_t cap) {
    Oracle* o = static_cast<Oracle*>(h);
    uint64_t i = 0;
    for (const auto& kv : o->cells) {
        if (i >= cap) break;
        oracle_record& r = out[i++];
        r.key = pack_key(o->cfg, kv.first);
        for (int ch = 0; ch < 3; ++ch) {
            r.sum[ch] = kv.second.sum[ch];
            r.L[ch] = kv.second.L[ch];
        }
        r.c_new = kv.second.c_new;
        r.c_old = kv.second.c_old;
    }
    return i;
}

// Import cells (for setting up query cases directly): records with the same meaning as export.
// The packed key is unpacked with this file's own layout.
void oracle_import(void* h, const oracle_record* recs, uint64_t n) {
    Oracle* o = static_cast<Oracle*>(h);
    const uint32_t d = o->cfg.dir_bits_d;
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t k = recs[i].key;
        const uint32_t dbin = static_cast<uint32_t>((k >> 48) & 0x3FFu);
        CellKey key(static_cast<uint32_t>((k >> 61) & 3u), static_cast<uint32_t>((k >> 58) & 7u),
                    dbin >> d, dbin & ((1u << d) - 1u), static_cast<uint32_t>((k >> 32) & 0xFFFFu),
                    static_cast<uint32_t>((k >> 16) & 0xFFFFu), static_cast<uint32_t>(k & 0xFFFFu));
        Cell& cell = o->cells[key];
        for (int ch = 0; ch < 3; ++ch) {
            cell.sum[ch] = recs[i].sum[ch];
            cell.L[ch] = recs[i].L[ch];
        }
        cell.c_new = recs[i].c_new;
        cell.c_old = recs[i].c_old;
    }
}


// ------------------------------------------------------------------------------------
// YCoCg two-band spherical-harmonics payload (Section "Basis functions and data
// structures: spatio-directional hashing", last paragraph: luminance in two SH bands over
// the normal, chroma kept per cell, so that each cell's basis spans normal variation).
//
// Reading (the paper names the representation, not its estimator):
//   * colour: Y = R/4 + G/2 + B/4, Co = R/2 - B/2, Cg = G/2 - R/4 - B/4 (Malvar and
//     Sullivan's YCoCg), inverse R = Y + Co - Cg, G = Y + Cg, B = Y - Co - Cg;
//   * per cell and iteration, luminance over the normal n is fitted by weighted least
//     squares on the two SH bands, whose span is {1, n_x, n_y, n_z}: Y(n) ~ a + g . n
//     (a = c00 Y00, g = sqrt(3 / 4 pi) (c11, c1-1, c10)), minimising
//        sum_i w_i (Y_i - a - g . n_i)^2 + ridge * W * |g|^2,   W = sum_i w_i,
//     whose band-0 part alone is eq. (6)'s weighted mean; chroma is the weighted mean;
//   * in centred form: M = W sum w n n^T - (sum w n)(sum w n)^T and
//     r = W sum w Y n - (sum w Y)(sum w n) are formed exactly from the integer sums
//     (128-bit), then (M + ridge W^2 I) g = r and a = (sum w Y - g . sum w n) / W;
//     if the regularised matrix is not positive definite band 1 is 0 for that iteration;
//   * eq. (10)-(11) blend the six coefficients (a, g_x, g_y, g_z, Co, Cg) with the
//     cell's alpha; the approximant at a vertex is the cell's fit evaluated at the vertex's
//     own normal, turned back into RGB.
// Fixed-point codes, in FP32 with one rounding per step in this order (the kernel takes
// the same decisions): p_c = w L_c; wY = (p_r/4 + p_g/2) + p_b/4; wCo = p_r/2 - p_b/2;
// wCg = (p_g/2 - p_r/4) - p_b/4; m_k = w n_k; Yn_k = wY n_k; nn_jk = m_j n_k; each
// rounded to nearest even at 2^F.  Range rule: that of the RGB payload plus |n_k| <= 1 + 2^-10
// (unit normals).
// ------------------------------------------------------------------------------------

namespace {

constexpr int SH_SUMS = 16;  // Y, Co, Cg, c_new, n(3), Y n(3), n n(xx, xy, xz, yy, yz, zz)

struct ShCell {
    int64_t s[SH_SUMS] = {};
    int64_t c_old = 0;
    double coef[6] = {0, 0, 0, 0, 0, 0};  // a, g_x, g_y, g_z, Co, Cg
};

struct ShOracle {
    Config cfg;
    double ridge;
    std::map<CellKey, ShCell> cells;
    uint64_t dropped = 0;
    uint64_t zero_weight = 0;
    uint64_t iter_vertices = 0;
};

// The cell fit's RGB at normal n.
void sh_rgb(const double coef[6], const float* n, double out[3]) {
    const double Y = coef[0] + coef[1] * n[0] + coef[2] * n[1] + coef[3] * n[2];
    out[0] = Y + coef[4] - coef[5];
    out[1] = Y + coef[5];
    out[2] = Y - coef[4] - coef[5];
}

// 3x3 determinant by cofactors.
double det3(const double m[3][3]) {
    return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
           m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
}

// eq. (11) for the SH payload's cells: the same rule as the RGB blend.
double sh_alpha(const Config& c, int64_t c_new, int64_t c_old) {
    const double cn = static_cast<double>(c_new);
    const double total = static_cast<double>(c_old) + cn;
    return c.blend_mode == 0 ? std::max(std::sqrt(cn / total), c.alpha_min) : c.alpha_min;
}

// This iteration's fit of one touched cell (the reading above), in FP64.
void sh_fit(const ShCell& c, double ridge, double out[6]) {
    using i128 = __int128;
    const int64_t W = c.s[3];
    const int64_t* sn = c.s + 4;
    const int64_t* sYn = c.s + 7;
    const int64_t* snn = c.s + 10;
    const int idx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    double m[3][3], r[3];
    const double Wd = static_cast<double>(W);
    for (int j = 0; j < 3; ++j) {
        for (int k = 0; k < 3; ++k) {
            const i128 mjk = static_cast<i128>(W) * snn[idx[j][k]] - static_cast<i128>(sn[j]) * sn[k];
            m[j][k] = static_cast<double>(mjk);
        }
        m[j][j] += ridge * Wd * Wd;
        r[j] = static_cast<double>(static_cast<i128>(W) * sYn[j] - static_cast<i128>(c.s[0]) * sn[j]);
    }
    // positive definite: the leading principal minors are positive (Sylvester's criterion)
    const double d1 = m[0][0], d2 = m[0][0] * m[1][1] - m[0][1] * m[1][0], d3 = det3(m);
    double g[3] = {0.0, 0.0, 0.0};
    if (d1 > 0.0 && d2 > 0.0 && d3 > 0.0) {
        for (int col = 0; col < 3; ++col) {  // Cramer's rule
            double mc[3][3];
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) mc[j][k] = (k == col) ? r[j] : m[j][k];
            g[col] = det3(mc) / d3;
        }
    }
    out[0] = (static_cast<double>(c.s[0]) - (g[0] * sn[0] + g[1] * sn[1] + g[2] * sn[2])) / Wd;
    out[1] = g[0];
    out[2] = g[1];
    out[3] = g[2];
    out[4] = static_cast<double>(c.s[1]) / Wd;
    out[5] = static_cast<double>(c.s[2]) / Wd;
}

}  // namespace

typedef struct {
    uint64_t key;
    int64_t sum[16];  // Y, Co, Cg, c_new, n(3), Y n(3), n n(6) -- this iteration's fixed-point sums
    int64_t c_old;
    double coef[6];   // a, g_x, g_y, g_z, Co, Cg
} oracle_sh_record;

void* oracle_sh_create(const oracle_config* cfg, double ridge) {
    if (!cfg || cfg->dir_bits_d > 5 || cfg->pos_bits_q > 20 || cfg->frac_bits < 8 || cfg->frac_bits > 32 ||
        cfg->levels > 1 || !(ridge >= 0.0))
        return nullptr;
    ShOracle* o = new ShOracle();
    std::memcpy(&o->cfg, cfg, sizeof(Config));
    o->ridge = ridge;
    return o;
}

void oracle_sh_destroy(void* h) { delete static_cast<ShOracle*>(h); }

uint32_t oracle_sh_insert(void* h, const float* verts, uint64_t n) {
    ShOracle* o = static_cast<ShOracle*>(h);
    const Config& c = o->cfg;
    const double scale = std::ldexp(1.0, static_cast<int>(c.frac_bits));
    auto fx = [scale](float x) { return std::llrint(static_cast<double>(x) * scale); };
    uint32_t status = 0;
    for (uint64_t i = 0; i < n; ++i) {
        const float* v = verts + 16 * i;
        const float* nr = v + 4;
        CellKey key;
        bool ok = vertex_cell(c, v, &key);
        const float w = v[3];
        ok = ok && (w >= 0.0f) && (w <= 32768.0f);
        for (int k = 0; k < 3 && ok; ++k) ok = std::fabs(nr[k]) <= 1.0009765625f;
        float p[3] = {0.0f, 0.0f, 0.0f};
        for (int ch = 0; ch < 3 && ok; ++ch) {
            p[ch] = w * v[12 + ch];
            ok = std::isfinite(p[ch]) && std::fabs(p[ch]) <= 32768.0f;
        }
        if (!ok) {
            status |= ST_RANGE;
            o->dropped++;
            continue;
        }
        const int64_t cw = fx(w);
        if (cw == 0) {
            o->zero_weight++;
            continue;
        }
        float wY = 0.25f * p[0] + 0.5f * p[1];
        wY = wY + 0.25f * p[2];
        const float wCo = 0.5f * p[0] - 0.5f * p[2];
        float wCg = 0.5f * p[1] - 0.25f * p[0];
        wCg = wCg - 0.25f * p[2];
        const float m[3] = {w * nr[0], w * nr[1], w * nr[2]};
        const int64_t code[SH_SUMS] = {fx(wY), fx(wCo), fx(wCg), cw,
                                       fx(m[0]), fx(m[1]), fx(m[2]),
                                       fx(wY * nr[0]), fx(wY * nr[1]), fx(wY * nr[2]),
                                       fx(m[0] * nr[0]), fx(m[0] * nr[1]), fx(m[0] * nr[2]),
                                       fx(m[1] * nr[1]), fx(m[1] * nr[2]), fx(m[2] * nr[2])};
        ShCell& cell = o->cells[key];
        for (int k = 0; k < SH_SUMS; ++k) cell.s[k] = wrap_add(cell.s[k], code[k]);
    }
    // the normal moments reach 2^15 (1 + 2^-10)^2 per vertex: one bit fewer vertices
    return status | count_vertices(&o->iter_vertices, n, c.frac_bits, 1u);
}

// eq. (10)-(11) on the six coefficients of every touched cell.
uint32_t oracle_sh_update(void* h) {
    ShOracle* o = static_cast<ShOracle*>(h);
    const Config& c = o->cfg;
    for (auto& kv : o->cells) {
        ShCell& cell = kv.second;
        if (cell.s[3] == 0) continue;
        if (cell.s[3] < 0) {  // the counter wrapped (ST_SUM_RANGE): this iteration's sums are dropped
            for (int k = 0; k < SH_SUMS; ++k) cell.s[k] = 0;
            continue;
        }
        const double alpha = sh_alpha(c, cell.s[3], cell.c_old);
        double fit[6];
        sh_fit(cell, o->ridge, fit);
        for (int k = 0; k < 6; ++k) cell.coef[k] = (1.0 - alpha) * cell.coef[k] + alpha * fit[k];
        cell.c_old = sat_add(cell.c_old, cell.s[3]);
        for (int k = 0; k < SH_SUMS; ++k) cell.s[k] = 0;
    }
    o->iter_vertices = 0;
    return 0;
}

void oracle_sh_reset(void* h) {
    for (auto& kv : static_cast<ShOracle*>(h)->cells) kv.second.c_old = 0;
}

// RGB approximant of each vertex's cell at the vertex's own normal (0 when absent).
void oracle_sh_lookup(void* h, const float* verts, uint64_t n, double* C_out) {
    ShOracle* o = static_cast<ShOracle*>(h);
    for (uint64_t i = 0; i < n; ++i) {
        double* C = C_out + 3 * i;
        C[0] = C[1] = C[2] = 0.0;
        CellKey key;
        if (!vertex_cell(o->cfg, verts + 16 * i, &key)) continue;
        auto it = o->cells.find(key);
        if (it != o->cells.end()) sh_rgb(it->second.coef, verts + 16 * i + 4, C);
    }
}

// The control variate of oracle_query_cv with C_j the SH payload's RGB at vertex j's normal.
void oracle_sh_query_cv(void* h, const float* verts, uint32_t P, uint32_t D, double* out) {
    ShOracle* o = static_cast<ShOracle*>(h);
    const Config& c = o->cfg;
    std::vector<double> C(3 * static_cast<size_t>(P) * D);
    oracle_sh_lookup(h, verts, static_cast<uint64_t>(P) * D, C.data());
    for (uint64_t p = 0; p < P; ++p)
        for (uint64_t j = 0; j < D; ++j) {
            const uint64_t idx = j * P + p;
            const float* v = verts + 16 * idx;
            const double t[3] = {v[7], v[11], v[15]};
            const bool cv = j + 1 < D && j < c.cv_max_depth;
            for (int ch = 0; ch < 3; ++ch) {
                const double L = v[12 + ch];
                out[3 * idx + ch] = cv ? (L - c.beta * (t[ch] * C[3 * (idx + P) + ch]) + c.beta * C[3 * idx + ch]) : L;
            }
        }
}

uint64_t oracle_sh_size(void* h) { return static_cast<ShOracle*>(h)->cells.size(); }

void oracle_sh_counters(void* h, uint64_t* dropped, uint64_t* zero_weight) {
    ShOracle* o = static_cast<ShOracle*>(h);
    *dropped = o->dropped;
    *zero_weight = o->zero_weight;
}

uint64_t oracle_sh_export(void* h, oracle_sh_record* out, uint64_t cap) {
    ShOracle* o = static_cast<ShOracle*>(h);
    uint64_t i = 0;
    for (const auto& kv : o->cells) {
        if (i >= cap) break;
        oracle_sh_record& r = out[i++];
        r.key = pack_key(o->cfg, kv.first);
        for (int k = 0; k < SH_SUMS; ++k) r.sum[k] = kv.second.s[k];
        r.c_old = kv.second.c_old;
        for (int k = 0; k < 6; ++k) r.coef[k] = kv.second.coef[k];
    }
    return i;
}

uint32_t oracle_status_range() { return ST_RANGE; }
uint32_t oracle_status_sum_range() { return ST_SUM_RANGE; }
uint32_t oracle_status_table_full() { return ST_TABLE_FULL; }

}  // extern "C"
