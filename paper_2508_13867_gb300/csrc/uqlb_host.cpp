// Host side of libuqlb: the UQ manager (sampling, quadrature, gPC basis), the ensemble
// planner (arena layout, tile order, obstacle masks), CUDA-graph chunking of the time loop
// and the C ABI of include/uqlb.h.  arXiv 2508.13867: Sec. 4 (MC, gPC), Sec. 6 (class
// design), Sec. 7 and Algorithm 1 (workflow), Sec. 8.1 (user API of the cylinder example).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "uqlb_internal.h"

using namespace uqlb;

namespace {

thread_local std::string g_last_error;

struct GraphEntry {
    std::vector<unsigned char> key;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

constexpr int kMaxDim = 8;
constexpr int kMaxGraphs = 32;  // a batch run as groups takes one graph per group

}  // namespace

// Launch shape the autotuner picked for a batch shape (0: default).
struct TuneChoice {
    int rows = 0, npt = 0;              // tile geometry
    int bps = 0, stage = 0, smem_kb = 0;  // three-step strips
};

struct uqlb_ctx {
    int device = 0;
    std::string err;
    int dim = 0;
    std::vector<uqlb_dist> dists;
    int method = UQLB_METHOD_NONE;
    int64_t S = 0;
    std::vector<double> z, xi, a;
    int order = 0, basis = 0, K = 0;
    std::vector<int32_t> alpha;
    std::vector<double> W;
    std::vector<double> w_block;  // host staging of the W columns of a sample block (uqlb_project_block)
    // Sum-factorized projection of a tensor Gauss-Legendre grid (n = 0: not available): one stage per
    // input dimension, the last first; stage m has groups[m] groups of jprev[m] partial indices in and
    // jout[m] out, its admission table at idx_off[m] in `tables` (after G, the (order + 1) x n matrix of
    // the 1-D factors); stages before the last write rows_out[m] rows into buffer A (odd stages) or B.
    struct SumFactorPlan {
        int n = 0, p1 = 0;
        std::vector<int64_t> groups, rows_out;
        std::vector<int> jprev, jout;
        std::vector<size_t> idx_off;  // byte offsets into tables
        std::vector<unsigned char> tables;
        int64_t rows_a = 0, rows_b = 0;
    } sf;
    cudaStream_t capture_stream = nullptr;
    cudaStream_t side_stream = nullptr;           // CHANNEL groups of a grouped batch (high priority)
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    std::vector<GraphEntry> graphs;
    cudaEvent_t loop_begin = nullptr, loop_end = nullptr;
    bool loop_timed = false;
    int64_t loop_steps = 0, run_launches = 0;
    struct Tuned {
        int storage, mixed;
        int64_t n, nodes;
        TuneChoice choice;
    };
    std::vector<Tuned> tuned;
    std::vector<uqlb_tune_candidate> tune_report;  // candidates of the last autotune (largest group)
    int tune_chosen = -1;
    int last_rows = 0, last_npt = 0, last_scheme = 0;
    int last_projection = 0;  // the contraction of the last uqlb_project: 0 dense, 1 sum-factorized
    int cluster_blocks = 0, cluster_cols = 0;  // geometry of the last cluster launch
    int64_t counter_host[2] = {0, 0};  // source of the step-counter upload (step, first step of the run)
    int32_t* bar_err = nullptr;  // device error word of the last run
};

namespace {

int set_err(uqlb_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g_last_error = buf;
    return code;
}

int cuda_fail(uqlb_ctx* c, cudaError_t e, const char* what) {
    return set_err(c, UQLB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Whether UQLB_SCHEME_AUTO takes three steps per launch on the row strips where the width allows it
// (measured faster on GB300 for every storage format: 625 x 256^2 ensemble, GLUPS three- / two-step
// strips: FP32 203 / 177, FP16 174 / 161, BF16 183 / 172, FX16 171 / 160).
constexpr bool kAutoThreeStep = true;
constexpr bool kAutoCluster = true;

// Whether a batch run as groups runs its CHANNEL groups on a second stream beside the periodic
// groups (1), or every group one after another on the caller's stream (0).  Measured on the uneven
// batch (256 TGV samples of three widths and 64 channel samples, BF16): 0.739 against 0.814 s; the
// side stream's priority and the launch order of the cluster group changed it by under 0.2 %.
#ifndef UQLB_GROUPS_CONCURRENT
#define UQLB_GROUPS_CONCURRENT 1
#endif

// Whether a batch can run on the cluster scheme: CHANNEL samples with the halfway obstacle and the
// face inlet/outlet, FP32 or 16-bit storage, graph mode, the largest width and height held by a
// cluster.
bool cluster_eligible(const uqlb_sample* smp, int64_t n, int storage, int mode) {
    if (n < 1 || storage == UQLB_F64 || mode != UQLB_MODE_GRAPH) return false;
    int mx = 0, my = 0;
    for (int64_t s = 0; s < n; ++s) {
        if (smp[s].kind != UQLB_CASE_CHANNEL || smp[s].obstacle_bc != UQLB_OBSTACLE_HALFWAY ||
            smp[s].inout_bc != UQLB_INOUT_FACE)
            return false;
        mx = std::max(mx, smp[s].nx);
        my = std::max(my, smp[s].ny);
    }
    return cluster_fits(storage, mx, my);
}

int storage_bytes(int storage) {
    switch (storage) {
        case UQLB_F64: return 8;
        case UQLB_F32: return 4;
        case UQLB_F16:
        case UQLB_BF16:
        case UQLB_FX16: return 2;
        default: return 0;
    }
}

// Quanta of the 16-bit fixed-point storage for one sample: d_c = margin B_c / 32767, B_c a bound on
// |g_i| of velocity class c (rest, axis, diagonal) over the run.  With drho <= R, every |c_i . u| <= U
// and every velocity-gradient component <= G, the shifted equilibrium
// g_i^eq = w_i (drho + rho (3 c_i.u + 4.5 (c_i.u)^2 - 1.5 u.u)) and the first-order non-equilibrium
// part -3 tau w_i rho Q_i : grad u (Q_i = c_i c_i - I/3; |Q_i : grad u| <= G on the axes, 2 G on the
// diagonals, 0 at rest for a divergence-free flow) give
//   |g_0| <= w_0 (R + (1 + R) 1.5 U^2),  |g_i| <= w_i (R + (1 + R)(3 U + 6 U^2 + 3 tau q_i G)), q_i = 1, 2.
//   TGV: U = |u0| + |amp2| + |amp3| (each mode keeps |u| + |v| <= its amplitude, and the decaying
//     flow never exceeds its start), G = k (|u0| + 2 |amp2| + 3 |amp3|), k = 2 pi / min(nx, ny),
//     R = 1.5 U^2 (|p| <= u0^2 / 2); margin 1.5.
//   TGV_PERTURBED (Sec. 8.3): U = |u0| + S / 4 with S = |zeta_00| + ... + |zeta_11|,
//     G = k (2 |u0| + 1.5 S), R = 1.5 U^2, margin 1.5.
//   Either Taylor-Green kind on a lattice with nx != ny: the initial field is not divergence-free
//     there (k differs along x and y), its acoustic waves carry |drho| up to ~1.7 U (measured in an
//     FP64 emulation at aspect ratios 2 to 32), so R = 2 sqrt(3) U (the acoustic density of a
//     velocity jump U is sqrt(3) U, doubled).
//   CHANNEL (Sec. 8.1): U = 4 |u0| (u0 the mean inflow; |u_x| + |u_y| peaks near 2.8 u0 around the
//     obstacle and in the start-up), G = U / 2 (the shear at the staircase obstacle), and R = 6 |u0|
//     (start-up pressure waves reach |drho| near 2 u0 with the ramp; an impulsive start gives about
//     sqrt(3) times the inflow peak, doubled on reflection); margin 1.
// A value beyond the range saturates and the run reports the sample unstable.
void fx16_quanta(const uqlb_sample& s, double d[3]) {
    double U, G, R, margin;
    const double k = 2.0 * M_PI / std::max(1, std::min(s.nx, s.ny));
    if (s.kind == UQLB_CASE_CHANNEL) {
        U = 4.0 * std::fabs(s.u0);
        G = 0.5 * U;
        R = 6.0 * std::fabs(s.u0);
        margin = 1.0;
    } else if (s.kind == UQLB_CASE_TGV_PERTURBED) {
        const double S = std::fabs(s.pert[0]) + std::fabs(s.pert[1]) + std::fabs(s.pert[2]) + std::fabs(s.pert[3]);
        U = std::fabs(s.u0) + 0.25 * S;
        G = k * (2.0 * std::fabs(s.u0) + 1.5 * S);
        R = 1.5 * U * U;
        margin = 1.5;
    } else {
        U = std::fabs(s.u0) + std::fabs(s.amp2) + std::fabs(s.amp3);
        G = k * (std::fabs(s.u0) + 2.0 * std::fabs(s.amp2) + 3.0 * std::fabs(s.amp3));
        R = 1.5 * U * U;
        margin = 1.5;
    }
    if (s.kind != UQLB_CASE_CHANNEL && s.nx != s.ny) R = std::max(R, 2.0 * std::sqrt(3.0) * U);
    U = std::max(U, 1e-6);
    const double tau = 3.0 * std::max(s.nu, 0.0) + 0.5;
    const double rho = 1.0 + R;
    const double b[3] = {4.0 / 9.0 * (R + rho * 1.5 * U * U),
                         1.0 / 9.0 * (R + rho * (3.0 * U + 6.0 * U * U + 3.0 * tau * G)),
                         1.0 / 36.0 * (R + rho * (3.0 * U + 6.0 * U * U + 6.0 * tau * G))};
    for (int c = 0; c < 3; ++c) d[c] = (double)(float)(margin * b[c] / 32767.0);
}

// ---------------------------------------------------------------------------------------
// Quadrature, random numbers and the Legendre chaos (Sec. 4, Sec. 6.1-6.3)
// ---------------------------------------------------------------------------------------

// P_n(x) and P_n'(x) by the three-term recurrence.
void legendre_eval(int n, double x, double* p_out, double* dp_out) {
    double pm1 = 1.0, p = x;
    if (n == 0) {
        *p_out = 1.0;
        *dp_out = 0.0;
        return;
    }
    for (int k = 2; k <= n; ++k) {
        const double pk = ((2.0 * k - 1.0) * x * p - (k - 1.0) * pm1) / k;
        pm1 = p;
        p = pk;
    }
    *p_out = p;
    *dp_out = n * (x * p - pm1) / (x * x - 1.0);
}

void gauss_legendre_rule(int n, double* x, double* w) {
    for (int j = 0; j < n; ++j) {
        double r = std::cos(M_PI * (j + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p, dp;
            legendre_eval(n, r, &p, &dp);
            const double step = p / dp;
            r -= step;
            if (std::fabs(step) < 1e-16) break;
        }
        double p, dp;
        legendre_eval(n, r, &p, &dp);
        x[n - 1 - j] = r;  // the initial guesses run from the largest root down
        w[n - 1 - j] = 2.0 / ((1.0 - r * r) * dp * dp);
    }
}

// Clenshaw-Curtis rule with m nodes cos(pi j / (m - 1)), returned ascending; weights from the
// cosine-sum formula (weights sum to 2).
void clenshaw_curtis_rule(int m, std::vector<double>& x, std::vector<double>& w) {
    x.assign(m, 0.0);
    w.assign(m, 0.0);
    if (m == 1) {
        w[0] = 2.0;
        return;
    }
    const int n = m - 1;
    for (int j = 0; j < m; ++j) {
        const double th = M_PI * j / n;
        double s = 0.0;
        for (int k = 1; k <= n / 2; ++k) s += (2 * k == n ? 1.0 : 2.0) / (4.0 * k * k - 1.0) * std::cos(2.0 * k * th);
        const double c = (j == 0 || j == n) ? 1.0 : 2.0;
        // ascending order: node j of the cosine ordering is position n - j
        x[n - j] = std::cos(th);
        w[n - j] = c / n * (1.0 - s);
    }
}

int cc_size(int level) { return level == 1 ? 1 : (1 << (level - 1)) + 1; }

// Smolyak combination over nested Clenshaw-Curtis rules: sum over 1 <= i_j, q - d + 1 <= |i| <= q
// (q = d + level) of (-1)^(q - |i|) C(d - 1, q - |i|) times the tensor rule; nested nodes merge
// on their index in the finest one-dimensional grid.
void smolyak_cc_grid(int d, int level, std::vector<double>& xi, std::vector<double>& a) {
    const int q = d + level;
    const int finest = cc_size(level + 1);
    std::map<std::vector<int>, double> acc;
    std::vector<int> idx(d, 1);
    std::vector<std::vector<double>> rx(level + 2), rw(level + 2);
    for (int l = 1; l <= level + 1; ++l) clenshaw_curtis_rule(cc_size(l), rx[l], rw[l]);
    auto binom = [](int n, int k) {
        double c = 1.0;
        for (int i = 1; i <= k; ++i) c = c * (n - k + i) / i;
        return c;
    };
    while (true) {
        int s = 0;
        for (int v : idx) s += v;
        if (s >= q - d + 1 && s <= q) {
            const double coef = ((q - s) % 2 ? -1.0 : 1.0) * binom(d - 1, q - s);
            std::vector<int> pos(d, 0), key(d, 0);
            while (true) {
                double w = coef;
                for (int k = 0; k < d; ++k) {
                    const int m = cc_size(idx[k]);
                    key[k] = m == 1 ? (finest - 1) / 2 : pos[k] * ((finest - 1) / (m - 1));
                    w *= 0.5 * rw[idx[k]][pos[k]];
                }
                acc[key] += w;
                int k = d - 1;
                while (k >= 0 && ++pos[k] == cc_size(idx[k])) pos[k--] = 0;
                if (k < 0) break;
            }
        }
        int k = d - 1;
        while (k >= 0 && ++idx[k] > level + 1) idx[k--] = 1;
        if (k < 0) break;
    }
    std::vector<double> xf, wf;
    clenshaw_curtis_rule(finest, xf, wf);
    xi.clear();
    a.clear();
    for (auto& kv : acc) {  // std::map iterates keys in lexicographic order
        for (int k = 0; k < d; ++k) xi.push_back(xf[kv.first[k]]);
        a.push_back(kv.second);
    }
}

double radical_inverse(uint64_t i, int base) {
    double f = 1.0, r = 0.0;
    while (i > 0) {
        f /= base;
        r += f * (double)(i % base);
        i /= base;
    }
    return r;
}

void philox10(const uint32_t in[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = in[0], c1 = in[1], c2 = in[2], c3 = in[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t m0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t m1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(m1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(m0 >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)m1;
        c3 = (uint32_t)m0;
        c0 = n0;
        c2 = n2;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

// Orthonormal Legendre values phi_0..phi_p at xi: sqrt(2n+1) P_n(xi).
void phi_values(int p, double xi, double* out) {
    double pm1 = 1.0, pn = xi;
    out[0] = 1.0;
    if (p >= 1) out[1] = std::sqrt(3.0) * xi;
    for (int n = 2; n <= p; ++n) {
        const double pk = ((2.0 * n - 1.0) * xi * pn - (n - 1.0) * pm1) / n;
        pm1 = pn;
        pn = pk;
        out[n] = std::sqrt(2.0 * n + 1.0) * pn;
    }
}

void enumerate_indices(int dim, int order, int basis, std::vector<int32_t>& out) {
    std::vector<std::vector<int32_t>> all;
    std::vector<int32_t> cur(dim, 0);
    // odometer over [0, order]^dim, pruned by the total degree where that applies
    while (true) {
        int sum = 0;
        for (int d = 0; d < dim; ++d) sum += cur[d];
        if (basis == UQLB_BASIS_TENSOR || sum <= order) all.push_back(cur);
        int d = dim - 1;
        while (d >= 0) {
            if (++cur[d] <= order) {
                int s2 = 0;
                for (int e = 0; e <= d; ++e) s2 += cur[e];
                if (basis == UQLB_BASIS_TENSOR || s2 <= order) break;
            }
            cur[d] = 0;
            --d;
        }
        if (d < 0) break;
    }
    std::sort(all.begin(), all.end(), [](const std::vector<int32_t>& l, const std::vector<int32_t>& r) {
        int sl = 0, sr = 0;
        for (int v : l) sl += v;
        for (int v : r) sr += v;
        if (sl != sr) return sl < sr;
        return l > r;  // descending lexicographic within a degree
    });
    out.clear();
    for (auto& v : all) out.insert(out.end(), v.begin(), v.end());
}

int64_t count_indices(int dim, int order, int basis) {
    if (basis == UQLB_BASIS_TENSOR) {
        double n = std::pow((double)order + 1.0, dim);
        return n > 1e7 ? -1 : (int64_t)n;
    }
    // C(dim + order, order)
    double c = 1.0;
    for (int i = 1; i <= order; ++i) c = c * (dim + i) / i;
    return c > 1e7 ? -1 : (int64_t)std::llround(c);
}

// ---------------------------------------------------------------------------------------
// Batch planning: arena layout, table of samples ordered by descending steps, masks
// ---------------------------------------------------------------------------------------

bool sample_solid(const uqlb_sample& s, int x, int y) {
    if (s.kind != UQLB_CASE_CHANNEL || !(s.cyl_r > 0.0)) return false;
    const double dx = (x + 0.5) - s.cyl_cx, dy = (y + 0.5) - s.cyl_cy;
    return dx * dx + dy * dy < s.cyl_r * s.cyl_r;
}

struct BatchPlan {
    std::vector<SampleDev> table;
    std::vector<InitDev> init;
    std::vector<int32_t> steps_sorted;
    std::vector<int32_t> row_base;
    std::vector<uint32_t> masks;
    size_t off_arena = 0, off_arena2 = 0, off_sel = 0, off_rowbase = 0, off_bcpop = 0, off_samples = 0, off_init = 0, off_steps = 0, off_masks = 0, off_side = 0,
           off_partials = 0, off_counters = 0, off_done = 0, off_steps_run = 0, off_cd_prev = 0,
           off_step_counter = 0, off_flag = 0, off_streak = 0, off_sync = 0, total = 0;
    BatchGeometry geom{};
    int n_steady = 0;
    bool uniform_size = true;
};

int validate_sample(const uqlb_sample& s, int64_t idx, std::string& why) {
    char buf[256];
    if (s.kind != UQLB_CASE_TGV && s.kind != UQLB_CASE_CHANNEL && s.kind != UQLB_CASE_TGV_PERTURBED) {
        snprintf(buf, sizeof buf, "sample %lld: unknown kind %d", (long long)idx, s.kind);
    } else if (s.nx < 2 || s.ny < 2 || s.nx > 65536 || s.ny > 65536) {
        snprintf(buf, sizeof buf, "sample %lld: lattice %d x %d out of range", (long long)idx, s.nx, s.ny);
    } else if (s.steps < 0 || s.steps >= (1ll << 31) - 2048) {
        snprintf(buf, sizeof buf, "sample %lld: steps %lld out of range", (long long)idx, (long long)s.steps);
    } else if (!(s.nu > 0.0) || !std::isfinite(s.nu)) {
        snprintf(buf, sizeof buf, "sample %lld: viscosity must be positive", (long long)idx);
    } else if (!std::isfinite(s.u0) || !std::isfinite(s.amp2) || !std::isfinite(s.amp3)) {
        snprintf(buf, sizeof buf, "sample %lld: non-finite velocity parameter", (long long)idx);
    } else if (s.kind == UQLB_CASE_CHANNEL &&
               (!std::isfinite(s.cyl_cx) || !std::isfinite(s.cyl_cy) || !std::isfinite(s.cyl_r))) {
        snprintf(buf, sizeof buf, "sample %lld: non-finite obstacle geometry", (long long)idx);
    } else if (s.obstacle_bc != UQLB_OBSTACLE_HALFWAY && s.obstacle_bc != UQLB_OBSTACLE_BOUZIDI) {
        snprintf(buf, sizeof buf, "sample %lld: unknown obstacle scheme %d", (long long)idx, s.obstacle_bc);
    } else if (s.inout_bc != UQLB_INOUT_FACE && s.inout_bc != UQLB_INOUT_INTERPOLATED) {
        snprintf(buf, sizeof buf, "sample %lld: unknown inlet/outlet scheme %d", (long long)idx, s.inout_bc);
    } else if (s.kind == UQLB_CASE_CHANNEL && s.inout_bc == UQLB_INOUT_INTERPOLATED &&
               (s.nx < 6 || s.ny < 3 ||
                (s.cyl_r > 0.0 && (s.cyl_cx - s.cyl_r < 4.0 || s.cyl_cx + s.cyl_r > s.nx - 4.0)))) {
        snprintf(buf, sizeof buf,
                 "sample %lld: the interpolated inlet/outlet needs nx >= 6, ny >= 3 and the obstacle clear of "
                 "the three end columns",
                 (long long)idx);
    } else {
        return 0;
    }
    why = buf;
    return UQLB_ERR_ARG;
}

// ids: the caller's index of each sample (the output row), nullptr for 0..n-1.
int plan_batch(const uqlb_sample* smp, int64_t n, const uqlb_run_opts* o, BatchPlan& P, std::string& why,
               const TuneChoice& tuned = TuneChoice(), const int64_t* ids = nullptr) {
    if (n <= 0 || n > (1 << 24)) {
        why = "sample count out of range";
        return UQLB_ERR_ARG;
    }
    const int storage = o ? o->storage : UQLB_F32;
    const int eb = storage_bytes(storage);
    if (eb == 0) {
        why = "unknown storage format";
        return UQLB_ERR_ARG;
    }
    for (int64_t s = 0; s < n; ++s)
        if (int rc = validate_sample(smp[s], s, why)) return rc;
    bool mixed = false;
    for (int64_t s = 0; s < n; ++s) mixed = mixed || smp[s].kind == UQLB_CASE_CHANNEL;
    const int mode = o ? o->mode : UQLB_MODE_GRAPH;
    if (mode < UQLB_MODE_GRAPH || mode > UQLB_MODE_PERSISTENT_TEST_TIMEOUT) {
        why = "unknown execution mode";
        return UQLB_ERR_ARG;
    }
    const int scheme = o ? o->scheme : UQLB_SCHEME_AUTO;
    if (scheme < UQLB_SCHEME_AUTO || scheme > UQLB_SCHEME_CLUSTER || scheme == UQLB_SCHEME_GROUPED) {
        why = "unknown time-stepping scheme";
        return UQLB_ERR_ARG;
    }
    // auto: the two-step scheme where it measured faster (periodic FP32, FP16 and BF16 batches)
    // cluster runs: every sample a channel with the face inlet/outlet and the halfway obstacle, 16-bit
    // or FP32 storage, the largest sample's lattice held once in the shared memory of at most 16
    // blocks; under auto every channel batch that allows them (measured 2.2x the one-step kernel on
    // the 9-sample cylinder at 20 nodes per diameter)
    const bool cluster_ok = cluster_eligible(smp, n, storage, mode);
    const bool cluster = scheme == UQLB_SCHEME_CLUSTER || (scheme == UQLB_SCHEME_AUTO && kAutoCluster && cluster_ok);
    if (scheme == UQLB_SCHEME_CLUSTER && !cluster_ok) {
        why = "the cluster scheme runs CHANNEL samples with the halfway obstacle and the face inlet/outlet, "
              "FP32 or 16-bit storage, in UQLB_MODE_GRAPH, whose lattice fits the shared memory of 16 blocks";
        return UQLB_ERR_ARG;
    }
    const bool two = (scheme >= UQLB_SCHEME_TWO_STEP && scheme != UQLB_SCHEME_ONE_STEP && !cluster) ||
                     (scheme == UQLB_SCHEME_AUTO && !cluster && !mixed && mode == UQLB_MODE_GRAPH &&
                      storage != UQLB_F64);
    if (two && (mixed || mode != UQLB_MODE_GRAPH)) {
        why = "the two-step scheme runs periodic (TGV) batches in UQLB_MODE_GRAPH only";
        return UQLB_ERR_ARG;
    }
    // row strips wherever the batch allows them, unless tiles are asked for
    bool strip_ok = strip_supported(storage, smp[0].nx);
    for (int64_t s = 1; s < n && strip_ok; ++s) strip_ok = smp[s].nx == smp[0].nx;
    if (scheme == UQLB_SCHEME_TWO_STEP_STRIPS && !strip_ok) {
        why = "the row-strip kernel needs FP32, FP16 or BF16 storage and one sample width of at most 2048 (1600 with FP32)";
        return UQLB_ERR_ARG;
    }
    const bool strips = two && strip_ok && scheme != UQLB_SCHEME_TWO_STEP_TILES;
    // three steps per launch on the strips where asked for, or under auto where the width allows it
    const bool strip3_ok = strips && strip3_supported(storage, smp[0].nx);
    if (scheme == UQLB_SCHEME_THREE_STEP_STRIPS && !strip3_ok) {
        why = "the three-step row strips need FP32, FP16, BF16 or FX16 storage and one sample width of at most 1600 "
              "(1280 with FP32)";
        return UQLB_ERR_ARG;
    }
    const int spl = !two ? 1
                         : ((strip3_ok && (scheme == UQLB_SCHEME_THREE_STEP_STRIPS ||
                                           (scheme == UQLB_SCHEME_AUTO && kAutoThreeStep)))
                                ? 3
                                : 2);
    auto supported = [&](int r, int q) {
        return two ? geometry_supported2(storage, r, q) : geometry_supported(storage, mixed, r, q);
    };
    int tr = o ? o->tile_rows : 0, npt = o ? o->nodes_per_thread : 0;
    if (tr == 0 && npt == 0) {
        tr = tuned.rows;
        npt = tuned.npt;
        if (tr == 0 || !supported(tr, npt)) {
            if (two) {
                tr = 8;
                npt = storage == UQLB_F64 ? 1 : 4;
            } else {
                tr = (mixed || storage == UQLB_F64) ? 8 : 4;
                npt = (mixed || storage == UQLB_F64) ? 1 : 2;
            }
        }
    }
    if (!supported(tr, npt)) {
        char buf[160];
        snprintf(buf, sizeof buf, "tile geometry tile_rows=%d nodes_per_thread=%d is not compiled for this batch", tr, npt);
        why = buf;
        return UQLB_ERR_ARG;
    }

    std::vector<int64_t> order(n);
    for (int64_t s = 0; s < n; ++s) order[s] = s;
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t l, int64_t r) { return smp[l].steps > smp[r].steps; });

    const int row_align = 128 / eb;
    P.table.assign(n, SampleDev{});
    P.init.assign(n, InitDev{});
    P.steps_sorted.assign(n, 0);
    P.row_base.assign(n + 1, 0);
    P.masks.clear();
    int64_t f_off = 0, tiles = 0, side = 0;
    int max_steps = 0, any_channel = 0, any_bouzidi = 0, any_inout = 0, tiles0 = -1;
    int64_t bcnodes = 0;
    bool uniform_tiles = true;
    P.n_steady = 0;
    P.uniform_size = true;
    // Lattice regions and boundary buffers in the caller's order (the slot), so that they do not
    // move when the step counts, and with them the table order, change between a run and its
    // resumption.
    std::vector<int64_t> f_off_of(n), side_of(n, -1), bc_of(n, -1);
    for (int64_t k = 0; k < n; ++k) {
        const uqlb_sample& s = smp[k];
        const int64_t plane = (int64_t)align_up((size_t)s.nx, (size_t)row_align) * s.ny;
        if (9 * plane >= (1ll << 31)) {
            why = "a sample's nine population planes must hold fewer than 2^31 values";
            return UQLB_ERR_ARG;
        }
        f_off_of[k] = f_off;
        f_off += 9 * plane;
        if (s.kind == UQLB_CASE_CHANNEL) {
            side_of[k] = side;
            side += s.ny;
            if (s.inout_bc == UQLB_INOUT_INTERPOLATED) {
                bc_of[k] = bcnodes;
                bcnodes += 2 * (int64_t)s.ny;
            }
        }
    }
    for (int64_t j = 0; j < n; ++j) {
        const uqlb_sample& s = smp[order[j]];
        SampleDev& d = P.table[j];
        d.nx = s.nx;
        d.ny = s.ny;
        // one-step runs: population planes of ny rows (arena[i * plane + y * pitch + x]); the
        // multi-step kernels keep a row's nine populations together, row after row
        // (arena[(9 y + i) cols + x]), expressed in the same fields as plane = cols, pitch = 9 cols, so
        // that a row load or push is one block of 9 cols values
        const int32_t cols = (int32_t)align_up((size_t)s.nx, (size_t)row_align);
        d.pitch = two ? 9 * cols : cols;
        d.plane = two ? (int64_t)cols : (int64_t)cols * s.ny;
        d.f_off = f_off_of[order[j]];
        d.slot = (int32_t)order[j];
        d.kind = s.kind;
        d.steps = (int32_t)s.steps;
        d.sample_id = (int32_t)(ids ? ids[order[j]] : order[j]);
        d.tiles_x = (s.nx + 32 * npt - 1) / (32 * npt);
        d.tiles = d.tiles_x * ((s.ny + tr - 1) / tr);
        d.tile_base = (int32_t)tiles;
        tiles += d.tiles;
        P.row_base[j + 1] = (int32_t)std::min<int64_t>((int64_t)P.row_base[j] + s.ny, INT32_MAX);
        if (tiles0 < 0) tiles0 = d.tiles;
        if (d.tiles != tiles0) uniform_tiles = false;
        if (s.nx != smp[0].nx || s.ny != smp[0].ny) P.uniform_size = false;
        d.omega = 1.0 / (3.0 * s.nu + 0.5);
        d.u_ref_inv2 = (s.u_ref > 0.0) ? 2.0 / ((double)s.nx * (double)s.ny * s.u_ref * s.u_ref) : 0.0;
        d.mask_off = -1;
        d.side_off = -1;
        d.uin_max = 0.0;
        d.force_norm = 0.0;
        d.ramp_steps = 0.0;
        d.steady_tol = 0.0;
        if (s.kind == UQLB_CASE_CHANNEL) {
            any_channel = 1;
            d.uin_max = 1.5 * s.u0;
            d.ramp_steps = (double)std::max<int64_t>(s.ramp_steps, 0);
            d.steady_tol = s.steady_tol > 0.0 ? s.steady_tol : 0.0;
            d.steady_checks = s.steady_checks > 1 ? s.steady_checks : 1;
            if (d.steady_tol > 0.0) ++P.n_steady;
            d.side_off = (int32_t)side_of[order[j]];
            if (s.inout_bc == UQLB_INOUT_INTERPOLATED) {
                d.inout = 1;
                d.bc_off = (int32_t)bc_of[order[j]];
                any_inout = 1;
            }
            // the only nodes that can be solid or have a solid neighbour (empty box: no obstacle);
            // the Bouzidi links and the channel step's interior tiles rely on it
            InitDev& in = P.init[j];
            in.bbox[0] = in.bbox[2] = -1;
            in.bbox[1] = in.bbox[3] = -2;
            if (s.cyl_r > 0.0) {
                d.force_norm = (s.u0 != 0.0) ? 2.0 / (s.u0 * s.u0 * 2.0 * s.cyl_r) : 0.0;
                // a node with a solid neighbour lies within r + sqrt(2) of the centre
                auto lo = [](double v, int n) {
                    return (int)std::max(0.0, std::min((double)(n - 1), std::floor(v)));
                };
                in.bbox[0] = lo(s.cyl_cx - s.cyl_r - 2.0, s.nx);
                in.bbox[1] = lo(s.cyl_cx + s.cyl_r + 1.0, s.nx);
                in.bbox[2] = lo(s.cyl_cy - s.cyl_r - 2.0, s.ny);
                in.bbox[3] = lo(s.cyl_cy + s.cyl_r + 1.0, s.ny);
                if (s.obstacle_bc == UQLB_OBSTACLE_BOUZIDI) {
                    d.bouzidi = 1;
                    any_bouzidi = 1;
                    in.cyl_cx = s.cyl_cx;
                    in.cyl_cy = s.cyl_cy;
                    in.cyl_r = s.cyl_r;
                }
                d.mask_off = (int32_t)P.masks.size();
                P.masks.resize(P.masks.size() + (size_t)mask_words(d) * s.ny, 0u);
                uint32_t* m = P.masks.data() + d.mask_off;
                for (int y = 0; y < s.ny; ++y)
                    for (int x = 0; x < s.nx; ++x)
                        if (sample_solid(s, x, y)) m[(size_t)y * mask_words(d) + (x >> 5)] |= 1u << (x & 31);
            }
        }
        if (storage == UQLB_FX16) {
            double q[3];
            fx16_quanta(s, q);
            for (int c = 0; c < 3; ++c) {
                P.init[j].quanta[c] = (float)q[c];
                P.init[j].inv_quanta[c] = (float)(1.0 / q[c]);
            }
        }
        P.init[j].u0 = s.u0;
        P.init[j].amp2 = s.amp2;
        P.init[j].amp3 = s.amp3;
        for (int k = 0; k < 4; ++k) P.init[j].pert[k] = s.pert[k];
        P.steps_sorted[j] = (int32_t)s.steps;
        max_steps = std::max(max_steps, (int)s.steps);
    }
    if (tiles >= (1ll << 31)) {
        why = "too many tiles";
        return UQLB_ERR_ARG;
    }
    const int64_t total_rows = P.row_base[n];
    if (total_rows >= INT32_MAX) {
        why = "too many lattice rows";
        return UQLB_ERR_ARG;
    }
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + std::max<size_t>(bytes, 1), 256);
        return at;
    };
    P.off_arena = take((size_t)f_off * eb);
    P.off_arena2 = two ? take((size_t)f_off * eb) : 0;
    P.off_sel = two ? take(sizeof(int32_t) * n) : 0;
    P.off_samples = take(sizeof(SampleDev) * n);
    P.off_init = take(sizeof(InitDev) * n);
    P.off_steps = take(sizeof(int32_t) * n);
    P.off_rowbase = take(sizeof(int32_t) * (n + 1));
    P.off_masks = take(sizeof(uint32_t) * P.masks.size());
    P.off_side = take((size_t)side * 2 * 8);
    P.off_bcpop = take((size_t)bcnodes * 9 * sizeof(double));
    // per-tile sums (7 per tile); the row-strip kernels keep 2 or 3 per row at the first row of each piece.
    // Sized alike for both two-step kernels: the buffers behind it (done, steps_run, ...) carry a run
    // into its resumption, which may use the other kernel.
    P.off_partials = take((size_t)std::max<int64_t>(tiles * 7, two ? total_rows * 3 : 0) * sizeof(double));
    P.off_counters = take(sizeof(int32_t) * n);
    P.off_done = take(sizeof(int32_t) * n);
    P.off_steps_run = take(sizeof(int32_t) * n);
    P.off_cd_prev = take(sizeof(double) * n);
    P.off_step_counter = take(2 * sizeof(int64_t));
    P.off_flag = take(sizeof(int32_t));
    P.off_streak = take(sizeof(int32_t) * n);
    P.off_sync = take(64);  // barrier count, generation, error word, ticket counter
    P.total = off;

    BatchGeometry& g = P.geom;
    g.nsamples = n;
    g.total_tiles = tiles;
    g.total_rows = total_rows;
    g.tile_rows = tr;
    g.npt = npt;
    g.max_steps = max_steps;
    g.storage = storage;
    g.any_channel = any_channel;
    g.uniform_tiles = uniform_tiles ? tiles0 : 0;
    const int rounding = o ? o->rounding : UQLB_ROUND_AUTO;
    if (rounding < UQLB_ROUND_AUTO || rounding > UQLB_ROUND_STOCHASTIC) {
        why = "unknown rounding mode";
        return UQLB_ERR_ARG;
    }
    g.stochastic = (eb == 2 && rounding != UQLB_ROUND_NEAREST) ? 1 : 0;
    g.two_step = two ? 1 : 0;
    g.strips = strips ? 1 : 0;
    g.strip_nx = strips ? smp[0].nx : 0;
    g.spl = spl;
    g.cluster = cluster ? 1 : 0;
    g.cluster_nx = g.cluster_ny = 0;
    g.pad_ = 0;
    {
        // launch shape of the three-step strips: the caller's, else the tuned one, else the default
        const int sb = o ? o->strip_blocks_per_sm : 0, ss = o ? o->strip_stage : 0, sk = o ? o->strip_smem_kb : 0;
        bool kb_ok = sk == 0;
        for (int c : kSmemConfigsKB) kb_ok = kb_ok || (c > 0 && sk == c);
        if (sb < 0 || sb > 32 || ss < 0 || ss > 3 || !kb_ok) {
            why = "strip_blocks_per_sm must be 0..32, strip_stage 0..3 and strip_smem_kb 0 or a shared-memory "
                  "configuration (8, 16, 32, 64, 100, 132, 164, 196, 228)";
            return UQLB_ERR_ARG;
        }
        const bool s3 = strips && spl == 3;
        if (s3 && ss != 0 && !strip3_fixed_width(smp[0].nx)) {
            why = "strip_stage applies to the three-step strips at widths 64, 128, 256, 512 and 1024 only";
            return UQLB_ERR_ARG;
        }
        g.strip_bps = s3 ? (sb ? sb : tuned.bps) : 0;
        g.strip_stage = s3 && strip3_fixed_width(smp[0].nx) ? (ss ? ss : tuned.stage) : 0;
        g.strip_smem_kb = s3 ? (sk ? sk : tuned.smem_kb) : 0;
    }
    if (cluster)
        for (int64_t s = 0; s < n; ++s) {
            g.cluster_nx = std::max(g.cluster_nx, smp[s].nx);
            g.cluster_ny = std::max(g.cluster_ny, smp[s].ny);
        }
    g.test_withhold = mode == UQLB_MODE_PERSISTENT_TEST_TIMEOUT ? 1 : 0;
    g.any_bouzidi = any_bouzidi;
    g.any_inout = any_inout;
    if ((any_bouzidi || any_inout) && mode != UQLB_MODE_GRAPH) {
        why = "samples with the Bouzidi obstacle or the interpolated inlet/outlet run in UQLB_MODE_GRAPH only";
        return UQLB_ERR_ARG;
    }
    return 0;
}

BatchBuffers carve(const BatchPlan& P, void* ws) {
    char* b = static_cast<char*>(ws);
    BatchBuffers B{};
    B.arena = b + P.off_arena;
    B.arena2 = P.geom.two_step ? b + P.off_arena2 : nullptr;
    B.sel = P.geom.two_step ? reinterpret_cast<int32_t*>(b + P.off_sel) : nullptr;
    B.row_base = reinterpret_cast<int32_t*>(b + P.off_rowbase);
    B.samples = reinterpret_cast<SampleDev*>(b + P.off_samples);
    B.init = reinterpret_cast<InitDev*>(b + P.off_init);
    B.steps_sorted = reinterpret_cast<int32_t*>(b + P.off_steps);
    B.masks = reinterpret_cast<uint32_t*>(b + P.off_masks);
    B.side = reinterpret_cast<float*>(b + P.off_side);
    B.side_d = reinterpret_cast<double*>(b + P.off_side);
    B.bcpop = reinterpret_cast<double*>(b + P.off_bcpop);
    B.partials = reinterpret_cast<double*>(b + P.off_partials);
    B.counters = reinterpret_cast<int32_t*>(b + P.off_counters);
    B.done = reinterpret_cast<int32_t*>(b + P.off_done);
    B.steps_run = reinterpret_cast<int32_t*>(b + P.off_steps_run);
    B.cd_prev = reinterpret_cast<double*>(b + P.off_cd_prev);
    B.step_counter = reinterpret_cast<int64_t*>(b + P.off_step_counter);
    B.active_flag = reinterpret_cast<int32_t*>(b + P.off_flag);
    B.streak = reinterpret_cast<int32_t*>(b + P.off_streak);
    B.bar_count = reinterpret_cast<unsigned int*>(b + P.off_sync);
    B.bar_gen = reinterpret_cast<unsigned int*>(b + P.off_sync + 4);
    B.bar_err = reinterpret_cast<int32_t*>(b + P.off_sync + 8);
    B.tickets = reinterpret_cast<unsigned long long*>(b + P.off_sync + 16);
    return B;
}

template <typename T>
void key_put(std::vector<unsigned char>& k, const T& v) {
    const unsigned char* p = reinterpret_cast<const unsigned char*>(&v);
    k.insert(k.end(), p, p + sizeof(T));
}

// Captured chunk of `chunk` time steps plus the step-counter advance, cached per context.
int chunk_graph(uqlb_ctx* ctx, const BatchBuffers& B, const BatchGeometry& G, const RunOutputs& O, int chunk,
                int parity, cudaGraphExec_t* out) {
    std::vector<unsigned char> key;
    key_put(key, B);
    key_put(key, G);
    key_put(key, O);
    key_put(key, chunk);
    key_put(key, parity);
    for (auto& e : ctx->graphs) {
        if (e.key == key) {
            *out = e.exec;
            return 0;
        }
    }
    cudaError_t err;
    if (!ctx->capture_stream) {
        err = cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking);
        if (err != cudaSuccess) return cuda_fail(ctx, err, "cudaStreamCreateWithFlags");
    }
    err = cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess) return cuda_fail(ctx, err, "cudaStreamBeginCapture");
    cudaError_t lerr = cudaSuccess;
    if (G.two_step) {
        for (int dt = 0; dt < chunk && lerr == cudaSuccess; dt += G.spl)
            lerr = launch_step2(B, G, O, dt, ctx->capture_stream);
    } else {
        for (int dt = 0; dt < chunk && lerr == cudaSuccess; ++dt) {
            lerr = launch_step(B, G, O, dt, parity, ctx->capture_stream);
            if (lerr == cudaSuccess && G.any_inout) lerr = launch_inout(B, G, dt, ctx->capture_stream);
            if (lerr == cudaSuccess && G.any_bouzidi && O.qoi_every > 0)
                lerr = launch_bouzidi_force(B, G, O, dt, parity, ctx->capture_stream);
        }
    }
    if (lerr == cudaSuccess) lerr = launch_advance(B, chunk, ctx->capture_stream);
    cudaGraph_t graph = nullptr;
    err = cudaStreamEndCapture(ctx->capture_stream, &graph);
    if (lerr != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(ctx, lerr, "kernel launch during capture");
    }
    if (err != cudaSuccess) return cuda_fail(ctx, err, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    err = cudaGraphInstantiate(&exec, graph, 0);
    if (err != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_fail(ctx, err, "cudaGraphInstantiate");
    }
    if ((int)ctx->graphs.size() >= kMaxGraphs) {
        cudaGraphExecDestroy(ctx->graphs.front().exec);
        cudaGraphDestroy(ctx->graphs.front().graph);
        ctx->graphs.erase(ctx->graphs.begin());
    }
    GraphEntry e;
    e.key = std::move(key);
    e.graph = graph;
    e.exec = exec;
    ctx->graphs.push_back(std::move(e));
    *out = exec;
    return 0;
}

int check_ctx(uqlb_ctx* ctx) {
    if (!ctx) return set_err(nullptr, UQLB_ERR_ARG, "null context");
    const cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    return 0;
}

void build_ensemble(const uqlb_ctx* ctx, const uqlb_case* c, uqlb_sample* out) {
    for (int64_t s = 0; s < ctx->S; ++s) {
        uqlb_sample r = c->base;
        double zeta2 = NAN, zeta3 = NAN, pert[4] = {NAN, NAN, NAN, NAN};
        for (int d = 0; d < ctx->dim; ++d) {
            const double v = ctx->z[(size_t)s * ctx->dim + d];
            const int prm = c->param_of_dim[d];
            switch (prm) {
                case UQLB_PARAM_NU: r.nu = v; break;
                case UQLB_PARAM_U0: r.u0 = v; break;
                case UQLB_PARAM_ZETA2: zeta2 = v; break;
                case UQLB_PARAM_ZETA3: zeta3 = v; break;
                default:
                    if (prm >= UQLB_PARAM_PERT00 && prm <= UQLB_PARAM_PERT11) pert[prm - UQLB_PARAM_PERT00] = v;
                    break;
            }
        }
        if (!std::isnan(zeta2)) r.amp2 = zeta2 * r.u0;
        if (!std::isnan(zeta3)) r.amp3 = zeta3 * r.u0;
        for (int k = 0; k < 4; ++k)
            if (!std::isnan(pert[k])) r.pert[k] = pert[k] * r.u0;
        out[s] = r;
    }
}

int check_case(uqlb_ctx* ctx, const uqlb_case* c) {
    if (!c) return set_err(ctx, UQLB_ERR_ARG, "null case");
    if (ctx->S <= 0) return set_err(ctx, UQLB_ERR_STATE, "no sample set: call uqlb_init_mc or uqlb_init_gpc");
    for (int d = 0; d < ctx->dim; ++d)
        if (c->param_of_dim[d] < UQLB_PARAM_NU || c->param_of_dim[d] > UQLB_PARAM_PERT11)
            return set_err(ctx, UQLB_ERR_ARG, "param_of_dim[%d] = %d is not a known parameter", d, c->param_of_dim[d]);
    return 0;
}

const int kGeomRows[] = {2, 4, 8, 16};
const int kGeomNpt[] = {1, 2, 4};

// A batch of unlike samples under UQLB_SCHEME_AUTO (graph mode, FP32/FP16/BF16 storage) runs as
// groups of like samples, one after another, each on its own kernel and its own slice of the
// workspace: CHANNEL samples on the one-step scheme, periodic samples of each width the row-strip
// kernel takes on strips, wider periodic samples on two-step tiles.  Empty when the batch is one
// such group (it then runs as one batch, as before).
struct Group {
    std::vector<int64_t> idx;  // caller's indices, ascending
    int32_t scheme;
    std::vector<uqlb_sample> smp;
    uqlb_run_opts opts;
};
std::vector<Group> make_groups(const uqlb_sample* smp, int64_t n, const uqlb_run_opts* o) {
    std::vector<Group> out;
    if (!o || o->scheme != UQLB_SCHEME_AUTO || o->mode != UQLB_MODE_GRAPH || o->storage == UQLB_F64 || n < 2)
        return out;
    Group chan{{}, UQLB_SCHEME_ONE_STEP, {}, *o}, tiles{{}, UQLB_SCHEME_TWO_STEP_TILES, {}, *o};
    Group clus{{}, UQLB_SCHEME_CLUSTER, {}, *o};
    std::map<int, Group> strips;
    // channel samples: on clusters where the sample allows it (the group's largest width and height
    // must fit, so samples join in order of size while they do), else on the one-step kernel
    std::vector<int64_t> cand;
    for (int64_t s = 0; s < n; ++s)
        if (smp[s].kind == UQLB_CASE_CHANNEL && kAutoCluster && cluster_eligible(smp + s, 1, o->storage, o->mode))
            cand.push_back(s);
    std::stable_sort(cand.begin(), cand.end(), [&](int64_t a, int64_t b) {
        return (int64_t)smp[a].nx * smp[a].ny < (int64_t)smp[b].nx * smp[b].ny;
    });
    std::vector<char> on_cluster(n, 0);
    {
        int mx = 0, my = 0;
        for (int64_t s : cand) {
            const int nx2 = std::max(mx, smp[s].nx), ny2 = std::max(my, smp[s].ny);
            if (!cluster_fits(o->storage, nx2, ny2)) break;
            mx = nx2;
            my = ny2;
            on_cluster[s] = 1;
        }
    }
    for (int64_t s = 0; s < n; ++s) {
        if (on_cluster[s])
            clus.idx.push_back(s);
        else if (smp[s].kind == UQLB_CASE_CHANNEL)
            chan.idx.push_back(s);
        else if (strip_supported(o->storage, smp[s].nx)) {
            auto it = strips.find(smp[s].nx);
            const int32_t sch = kAutoThreeStep && strip3_supported(o->storage, smp[s].nx) ? UQLB_SCHEME_THREE_STEP_STRIPS
                                                                                         : UQLB_SCHEME_TWO_STEP_STRIPS;
            if (it == strips.end()) it = strips.emplace(smp[s].nx, Group{{}, sch, {}, *o}).first;
            it->second.idx.push_back(s);
        } else
            tiles.idx.push_back(s);
    }
    if (!clus.idx.empty()) out.push_back(std::move(clus));
    if (!chan.idx.empty()) out.push_back(std::move(chan));
    if (!tiles.idx.empty()) out.push_back(std::move(tiles));
    for (auto& kv : strips) out.push_back(std::move(kv.second));
    if (out.size() < 2) return {};
    for (auto& g : out) {
        for (int64_t s : g.idx) g.smp.push_back(smp[s]);
        g.opts.scheme = g.scheme;
    }
    return out;
}

// Workspace of a batch: the planned layout, and with both geometry fields 0 the largest layout of
// any compiled geometry (the autotuner may pick any of them later).  A batch run in groups takes
// the groups' workspaces one after another, each 256-byte aligned.
int batch_bytes_one(const uqlb_sample* samples, int64_t n, const uqlb_run_opts* opts, size_t* bytes, std::string& why);
int batch_bytes(const uqlb_sample* samples, int64_t n, const uqlb_run_opts* opts, size_t* bytes, std::string& why) {
    auto groups = make_groups(samples, n, opts);
    if (groups.empty()) return batch_bytes_one(samples, n, opts, bytes, why);
    size_t total = 0;
    for (auto& g : groups) {
        size_t b = 0;
        if (int rc = batch_bytes_one(g.smp.data(), (int64_t)g.smp.size(), &g.opts, &b, why)) return rc;
        total = align_up(total + b, 256);
    }
    *bytes = total;
    return 0;
}
int batch_bytes_one(const uqlb_sample* samples, int64_t n, const uqlb_run_opts* opts, size_t* bytes, std::string& why) {
    BatchPlan P;
    if (int rc = plan_batch(samples, n, opts, P, why)) return rc;
    size_t best = P.total;
    if (opts->tile_rows == 0 && opts->nodes_per_thread == 0) {
        for (int r : kGeomRows)
            for (int q : kGeomNpt) {
                uqlb_run_opts o = *opts;
                o.tile_rows = r;
                o.nodes_per_thread = q;
                BatchPlan Q;
                std::string ignore;
                if (plan_batch(samples, n, &o, Q, ignore) == 0) best = std::max(best, Q.total);
            }
    }
    *bytes = best;
    return 0;
}

// One planned batch: tables, init (or resume), the time loop, finalize.  own_timing: the loop
// records the context's loop events (a batch run in groups times all groups from outside).
int run_planned(uqlb_ctx* ctx, const BatchPlan& P, int64_t n, const uqlb_run_opts* opts, void* workspace_dev,
                void* fields_dev, int64_t fields_ld, double* qoi_dev, double* series_dev, double* series_cl_dev,
                int64_t series_ld, cudaStream_t s, bool own_timing) {
    const bool resume = opts->start_step > 0;
    // a chunk is a whole number of launches
    const int spl = std::max(P.geom.spl, 1);
    const int chunk = ((opts->chunk_steps > 0 ? opts->chunk_steps : 64) + spl - 1) / spl * spl;
    BatchBuffers B = carve(P, workspace_dev);
    char* ws = static_cast<char*>(workspace_dev);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(ws + P.off_samples, P.table.data(), sizeof(SampleDev) * n, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(ws + P.off_init, P.init.data(), sizeof(InitDev) * n, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(ws + P.off_steps, P.steps_sorted.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(ws + P.off_rowbase, P.row_base.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, s)) ||
        (!P.masks.empty() && (e = cudaMemcpyAsync(ws + P.off_masks, P.masks.data(), sizeof(uint32_t) * P.masks.size(),
                                                  cudaMemcpyHostToDevice, s))) ||
        (e = cudaMemsetAsync(B.active_flag, 0, sizeof(int32_t), s)) ||
        (e = cudaMemsetAsync(B.bar_count, 0, 64, s)) ||
        (!resume && (e = cudaMemsetAsync(ws + P.off_side, 0, P.off_partials - P.off_side, s))))
        return cuda_fail(ctx, e, "run_batch: table upload");
    // the device step counter starts at start_step (0 for a fresh run); ctx keeps the host copy alive
    ctx->counter_host[0] = ctx->counter_host[1] = opts->start_step;
    if ((e = cudaMemcpyAsync(B.step_counter, ctx->counter_host, 2 * sizeof(int64_t), cudaMemcpyHostToDevice, s)))
        return cuda_fail(ctx, e, "run_batch: step counter");

    RunOutputs O{};
    O.fields = fields_dev;
    O.fields_ld = fields_ld;
    O.fields_dtype = opts->fields_dtype;
    O.qoi = qoi_dev;
    O.series = series_dev;
    O.series_cl = series_cl_dev;
    O.series_ld = series_ld;
    O.qoi_every = opts->qoi_every;

    ctx->run_launches += 2;
    if (!resume) {
        if ((e = launch_init(B, P.geom, s)) != cudaSuccess) return cuda_fail(ctx, e, "run_batch: init launch");
    } else {
        if ((e = launch_resume(B, P.geom, s)) != cudaSuccess) return cuda_fail(ctx, e, "run_batch: resume launch");
    }
    ctx->bar_err = B.bar_err;
    if (P.geom.cluster) {
        // one launch runs every sample's whole time loop (each sample on one thread-block cluster)
        if (own_timing && (e = cudaEventRecord(ctx->loop_begin, s)) != cudaSuccess)
            return cuda_fail(ctx, e, "run_batch: event record");
        if ((e = launch_cluster(B, P.geom, O, s)) != cudaSuccess) return cuda_fail(ctx, e, "run_batch: cluster launch");
        ctx->run_launches += 1;
        last_cluster_choice(&ctx->cluster_blocks, &ctx->cluster_cols);
        if (own_timing) {
            if ((e = cudaEventRecord(ctx->loop_end, s)) != cudaSuccess) return cuda_fail(ctx, e, "run_batch: event record");
            ctx->loop_timed = true;
        }
    } else if (P.geom.max_steps > opts->start_step && opts->mode != UQLB_MODE_GRAPH) {
        // persistent: one cooperative launch per chunk, then the step counter advances
        const int pchunk = opts->chunk_steps > 0 ? chunk : 1024;
        const int64_t nchunks = (P.geom.max_steps - opts->start_step + pchunk - 1) / pchunk;
        const bool steady = P.n_steady > 0 && P.n_steady == (int)n;
        if (own_timing && (e = cudaEventRecord(ctx->loop_begin, s)) != cudaSuccess)
            return cuda_fail(ctx, e, "run_batch: event record");
        for (int64_t q = 0; q < nchunks; ++q) {
            if ((e = cudaMemsetAsync(B.tickets, 0, sizeof(unsigned long long), s)) ||
                (e = launch_persistent(B, P.geom, O, pchunk, s)) || (e = launch_advance(B, pchunk, s)))
                return cuda_fail(ctx, e, "run_batch: persistent launch");
            ctx->run_launches += 2;
            if (steady && q + 1 < nchunks) {
                int32_t ndone = 0;
                if ((e = cudaMemcpyAsync(&ndone, B.active_flag, sizeof ndone, cudaMemcpyDeviceToHost, s)) ||
                    (e = cudaStreamSynchronize(s)))
                    return cuda_fail(ctx, e, "run_batch: convergence check");
                if (ndone >= P.n_steady) break;
            }
        }
        if (own_timing) {
            if ((e = cudaEventRecord(ctx->loop_end, s)) != cudaSuccess) return cuda_fail(ctx, e, "run_batch: event record");
            ctx->loop_timed = true;
        }
    } else if (P.geom.max_steps > opts->start_step) {
        cudaGraphExec_t exec = nullptr;
        if (P.geom.two_step && (e = prepare_step2(P.geom)) != cudaSuccess) return cuda_fail(ctx, e, "run_batch: prepare");
        if (int rc = chunk_graph(ctx, B, P.geom, O, chunk, (int)(opts->start_step & 1), &exec)) return rc;
        const int64_t nchunks = (P.geom.max_steps - opts->start_step + chunk - 1) / chunk;
        const bool steady = P.n_steady > 0 && P.n_steady == (int)n;
        if (own_timing && (e = cudaEventRecord(ctx->loop_begin, s)) != cudaSuccess)
            return cuda_fail(ctx, e, "run_batch: event record");
        for (int64_t q = 0; q < nchunks; ++q) {
            if ((e = cudaGraphLaunch(exec, s)) != cudaSuccess) return cuda_fail(ctx, e, "run_batch: graph launch");
            ctx->run_launches += P.geom.two_step ? chunk / spl + 1
                                                 : chunk + 1 + ((P.geom.any_bouzidi && O.qoi_every > 0) ? chunk : 0) +
                                                       (P.geom.any_inout ? chunk : 0);
            if (steady && (q % 8) == 7 && q + 1 < nchunks) {
                int32_t ndone = 0;
                if ((e = cudaMemcpyAsync(&ndone, B.active_flag, sizeof ndone, cudaMemcpyDeviceToHost, s)) ||
                    (e = cudaStreamSynchronize(s)))
                    return cuda_fail(ctx, e, "run_batch: convergence check");
                if (ndone >= P.n_steady) break;
            }
        }
        if (own_timing) {
            if ((e = cudaEventRecord(ctx->loop_end, s)) != cudaSuccess) return cuda_fail(ctx, e, "run_batch: event record");
            ctx->loop_timed = true;
        }
    }
    if ((e = launch_finalize(B, P.geom, O, s)) != cudaSuccess) return cuda_fail(ctx, e, "run_batch: finalize launch");
    if (P.geom.two_step && (e = launch_commit(B, P.geom, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "run_batch: commit launch");
    return 0;
}


}  // namespace

namespace uqlb {

int ctx_projection_view(uqlb_ctx* ctx, const double** W, int* K, int64_t* S, int* device) {
    if (!ctx) return set_err(nullptr, UQLB_ERR_ARG, "null context");
    if (ctx->method != UQLB_METHOD_GPC) return set_err(ctx, UQLB_ERR_STATE, "call uqlb_init_gpc first");
    *W = ctx->W.data();
    *K = ctx->K;
    *S = ctx->S;
    *device = ctx->device;
    return 0;
}

int ctx_fail(uqlb_ctx* ctx, int code, const char* msg) { return set_err(ctx, code, "%s", msg); }

}  // namespace uqlb

// =========================================================================================
// C ABI
// =========================================================================================
extern "C" {

int uqlb_gauss_legendre(int n, double* x, double* w) {
    if (n < 1 || n > 64 || !x || !w) return set_err(nullptr, UQLB_ERR_ARG, "gauss_legendre: need 1 <= n <= 64");
    gauss_legendre_rule(n, x, w);
    return 0;
}

int uqlb_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    if (!ctr || !key || !out) return set_err(nullptr, UQLB_ERR_ARG, "philox: null pointer");
    philox10(ctr, key, out);
    return 0;
}

int uqlb_num_multi_indices(int dim, int order, int basis, int64_t* k) {
    if (dim < 1 || dim > kMaxDim || order < 0 || order > 64 || !k ||
        (basis != UQLB_BASIS_TOTAL && basis != UQLB_BASIS_TENSOR))
        return set_err(nullptr, UQLB_ERR_ARG, "num_multi_indices: bad arguments");
    const int64_t c = count_indices(dim, order, basis);
    if (c < 0) return set_err(nullptr, UQLB_ERR_ARG, "num_multi_indices: basis too large");
    *k = c;
    return 0;
}

int uqlb_multi_indices(int dim, int order, int basis, int32_t* alpha) {
    int64_t k = 0;
    if (int rc = uqlb_num_multi_indices(dim, order, basis, &k)) return rc;
    if (!alpha) return set_err(nullptr, UQLB_ERR_ARG, "multi_indices: null output");
    std::vector<int32_t> v;
    enumerate_indices(dim, order, basis, v);
    std::memcpy(alpha, v.data(), v.size() * sizeof(int32_t));
    return 0;
}

int uqlb_unit_converter(int n, double ma, double re, double* dx, double* dt, double* tau, double* u_lattice) {
    if (n < 2 || !(ma > 0.0) || !(re > 0.0)) return set_err(nullptr, UQLB_ERR_ARG, "unit_converter: need n >= 2, Ma > 0, Re > 0");
    const double h = 2.0 * M_PI / (n - 1);
    const double k = ma / std::sqrt(3.0) * h;
    if (dx) *dx = h;
    if (dt) *dt = k;
    if (tau) *tau = 3.0 * (1.0 / re) * k / (h * h) + 0.5;
    if (u_lattice) *u_lattice = k / h;
    return 0;
}

int uqlb_fx16_quanta(const uqlb_sample* s, double* quanta) {
    if (!s || !quanta) return set_err(nullptr, UQLB_ERR_ARG, "fx16_quanta: null argument");
    fx16_quanta(*s, quanta);
    return 0;
}

int uqlb_obstacle_mask(const uqlb_sample* s, uint8_t* mask) {
    if (!s || !mask || s->nx < 1 || s->ny < 1) return set_err(nullptr, UQLB_ERR_ARG, "obstacle_mask: bad arguments");
    for (int y = 0; y < s->ny; ++y)
        for (int x = 0; x < s->nx; ++x) mask[(size_t)y * s->nx + x] = sample_solid(*s, x, y) ? 1 : 0;
    return 0;
}

int uqlb_mean_host(const double* v, int64_t n, double* out) {
    if (!v || !out || n < 1) return set_err(nullptr, UQLB_ERR_ARG, "mean_host: need n >= 1");
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += v[i];
    *out = s / (double)n;
    return 0;
}

int uqlb_std_host(const double* v, int64_t n, int ddof, double* out) {
    if (!v || !out || n < 1 || ddof < 0 || n - ddof < 1) return set_err(nullptr, UQLB_ERR_ARG, "std_host: need n - ddof >= 1");
    double mu = 0.0;
    uqlb_mean_host(v, n, &mu);
    double ss = 0.0;
    for (int64_t i = 0; i < n; ++i) ss += (v[i] - mu) * (v[i] - mu);
    *out = std::sqrt(ss / (double)(n - ddof));
    return 0;
}

int uqlb_create(uqlb_ctx** out, int cuda_device) {
    if (!out) return set_err(nullptr, UQLB_ERR_ARG, "create: null output");
    *out = nullptr;
    if (cuda_device < 0) return set_err(nullptr, UQLB_ERR_ARG, "create: negative device");
    uqlb_ctx* c = new (std::nothrow) uqlb_ctx();
    if (!c) return set_err(nullptr, UQLB_ERR_OOM, "create: out of host memory");
    c->device = cuda_device;
    *out = c;
    return 0;
}

int uqlb_destroy(uqlb_ctx* ctx) {
    if (!ctx) return 0;
    cudaSetDevice(ctx->device);
    for (auto& e : ctx->graphs) {
        if (e.exec) cudaGraphExecDestroy(e.exec);
        if (e.graph) cudaGraphDestroy(e.graph);
    }
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
    if (ctx->loop_begin) cudaEventDestroy(ctx->loop_begin);
    if (ctx->loop_end) cudaEventDestroy(ctx->loop_end);
    delete ctx;
    return 0;
}

const char* uqlb_last_error(const uqlb_ctx* ctx) { return ctx ? ctx->err.c_str() : g_last_error.c_str(); }

int uqlb_set_inputs(uqlb_ctx* ctx, int dim, const uqlb_dist* d) {
    if (!ctx) return set_err(nullptr, UQLB_ERR_ARG, "null context");
    if (dim < 1 || dim > kMaxDim || !d) return set_err(ctx, UQLB_ERR_ARG, "set_inputs: need 1 <= dim <= %d", kMaxDim);
    for (int k = 0; k < dim; ++k) {
        if (d[k].kind != UQLB_DIST_UNIFORM) return set_err(ctx, UQLB_ERR_ARG, "set_inputs: input %d is not uniform", k);
        if (!(d[k].b > d[k].a) || !std::isfinite(d[k].a) || !std::isfinite(d[k].b))
            return set_err(ctx, UQLB_ERR_ARG, "set_inputs: input %d needs finite a < b", k);
    }
    ctx->dim = dim;
    ctx->dists.assign(d, d + dim);
    ctx->method = UQLB_METHOD_NONE;
    ctx->S = 0;
    ctx->K = 0;
    return 0;
}

int uqlb_init_mc(uqlb_ctx* ctx, int64_t n, uint64_t seed) {
    if (!ctx) return set_err(nullptr, UQLB_ERR_ARG, "null context");
    if (ctx->dim < 1) return set_err(ctx, UQLB_ERR_STATE, "init_mc: call uqlb_set_inputs first");
    if (n < 1 || n > (1 << 24)) return set_err(ctx, UQLB_ERR_ARG, "init_mc: need 1 <= n <= 2^24");
    const int d = ctx->dim;
    ctx->z.assign((size_t)n * d, 0.0);
    ctx->xi.assign((size_t)n * d, 0.0);
    ctx->a.assign((size_t)n, 1.0 / (double)n);
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t s = 0; s < n; ++s) {
        for (int k = 0; k < d; ++k) {
            const uint32_t ctr[4] = {(uint32_t)s, (uint32_t)((uint64_t)s >> 32), (uint32_t)k, 0u};
            uint32_t r[4];
            philox10(ctr, key, r);
            const uint64_t bits = ((uint64_t)r[1] << 32) | r[0];
            const double u = (double)(bits >> 11) * 0x1.0p-53;
            ctx->z[(size_t)s * d + k] = ctx->dists[k].a + (ctx->dists[k].b - ctx->dists[k].a) * u;
            ctx->xi[(size_t)s * d + k] = 2.0 * u - 1.0;
        }
    }
    ctx->S = n;
    ctx->method = UQLB_METHOD_MC;
    ctx->K = 0;
    ctx->W.clear();
    ctx->alpha.clear();
    return 0;
}

int uqlb_init_qmc(uqlb_ctx* ctx, int64_t n, int64_t skip) {
    static const int primes[kMaxDim] = {2, 3, 5, 7, 11, 13, 17, 19};
    if (!ctx) return set_err(nullptr, UQLB_ERR_ARG, "null context");
    if (ctx->dim < 1) return set_err(ctx, UQLB_ERR_STATE, "init_qmc: call uqlb_set_inputs first");
    if (n < 1 || n > (1 << 24) || skip < 0) return set_err(ctx, UQLB_ERR_ARG, "init_qmc: need 1 <= n <= 2^24, skip >= 0");
    const int d = ctx->dim;
    ctx->z.assign((size_t)n * d, 0.0);
    ctx->xi.assign((size_t)n * d, 0.0);
    ctx->a.assign((size_t)n, 1.0 / (double)n);
    for (int64_t s = 0; s < n; ++s)
        for (int k = 0; k < d; ++k) {
            const double u = radical_inverse((uint64_t)(s + skip), primes[k]);
            ctx->z[(size_t)s * d + k] = ctx->dists[k].a + (ctx->dists[k].b - ctx->dists[k].a) * u;
            ctx->xi[(size_t)s * d + k] = 2.0 * u - 1.0;
        }
    ctx->S = n;
    ctx->method = UQLB_METHOD_MC;
    ctx->K = 0;
    ctx->W.clear();
    ctx->alpha.clear();
    return 0;
}

// The stage plan of the sum-factorized projection on the tensor grid of n points per dimension
// (`sf` of the context; left empty where the grid or the multi-index set does not allow it).
// Partial multi-indices over the dimensions q .. d - 1 are built from the last dimension down: stage
// m admits degree a after the partial index j' when the total degree stays <= order (total-degree
// basis) or a <= order (tensor basis); the full indices of the last stage are mapped to the rows k of
// the context's basis.
void build_sum_factor_plan(uqlb_ctx* ctx, int n, const std::vector<double>& gx, const std::vector<double>& gw) {
    auto& P = ctx->sf;
    P = uqlb_ctx::SumFactorPlan{};
    const int d = ctx->dim, p1 = ctx->order + 1;
    if (n < 1 || n > kSfMaxPoints || d < 1 || ctx->order > kSfMaxDegree) return;
    std::map<std::vector<int32_t>, int> k_of;
    for (int k = 0; k < ctx->K; ++k)
        k_of[std::vector<int32_t>(ctx->alpha.begin() + (size_t)k * d, ctx->alpha.begin() + (size_t)(k + 1) * d)] = k;
    std::vector<std::vector<int32_t>> prev(1);  // J_0: the empty partial index
    std::vector<int32_t> idx;
    std::vector<size_t> idx_at;
    int64_t npre = 1;  // n^q for the stage's dimension q
    for (int q = 0; q + 1 < d; ++q) npre *= n;
    for (int m = 1; m <= d; ++m) {
        std::vector<std::vector<int32_t>> cur;
        idx_at.push_back(idx.size());
        for (auto& jp : prev) {
            int deg = 0;
            for (int v : jp) deg += v;
            for (int a = 0; a < p1; ++a) {
                const bool ok = ctx->basis == UQLB_BASIS_TENSOR ? true : a + deg <= ctx->order;
                if (!ok) {
                    idx.push_back(-1);
                    continue;
                }
                std::vector<int32_t> full{a};
                full.insert(full.end(), jp.begin(), jp.end());
                if (m == d) {
                    auto it = k_of.find(full);
                    if (it == k_of.end()) return;  // not the context's basis: no plan
                    idx.push_back(it->second);
                } else {
                    idx.push_back((int32_t)cur.size());
                }
                cur.push_back(full);
            }
        }
        P.groups.push_back(npre * (int64_t)prev.size());
        P.jprev.push_back((int)prev.size());
        P.jout.push_back(m == d ? ctx->K : (int)cur.size());
        P.rows_out.push_back(m == d ? ctx->K : npre * (int64_t)cur.size());
        if (m < d) (m % 2 == 1 ? P.rows_a : P.rows_b) = std::max(m % 2 == 1 ? P.rows_a : P.rows_b, P.rows_out.back());
        if (m == d && (int)cur.size() != ctx->K) {
            P = uqlb_ctx::SumFactorPlan{};
            return;
        }
        prev.swap(cur);
        if (m < d) npre /= n;
    }
    std::vector<double> phis(p1);
    const size_t gbytes = (size_t)p1 * n * sizeof(double);
    P.tables.resize(gbytes + idx.size() * sizeof(int32_t));
    double* G = reinterpret_cast<double*>(P.tables.data());
    for (int q = 0; q < n; ++q) {
        phi_values(ctx->order, gx[q], phis.data());
        for (int a = 0; a < p1; ++a) G[(size_t)a * n + q] = 0.5 * gw[q] * phis[a];
    }
    std::memcpy(P.tables.data() + gbytes, idx.data(), idx.size() * sizeof(int32_t));
    for (size_t at : idx_at) P.idx_off.push_back(gbytes + at * sizeof(int32_t));
    P.n = n;
    P.p1 = p1;
}

// Row stride (doubles) of the sum-factorization buffers, and their workspace for F fields.
int64_t sf_ld(int64_t F) { return (F + 31) / 32 * 32; }
size_t sf_workspace(const uqlb_ctx* ctx, int64_t F) {
    const auto& P = ctx->sf;
    return align_up(P.tables.size(), 256) + align_up((size_t)P.rows_a * sf_ld(F) * 8, 256) +
           align_up((size_t)P.rows_b * sf_ld(F) * 8, 256);
}
bool sf_available(const uqlb_ctx* ctx) { return ctx->method == UQLB_METHOD_GPC && ctx->sf.n > 0; }

int uqlb_init_gpc(uqlb_ctx* ctx, int order, int pts_per_dim, int basis, int quad) {
    if (!ctx) return set_err(nullptr, UQLB_ERR_ARG, "null context");
    ctx->sf = uqlb_ctx::SumFactorPlan{};
    if (ctx->dim < 1) return set_err(ctx, UQLB_ERR_STATE, "init_gpc: call uqlb_set_inputs first");
    if (quad != UQLB_QUAD_GAUSS_LEGENDRE_TENSOR && quad != UQLB_QUAD_CLENSHAW_CURTIS_SMOLYAK)
        return set_err(ctx, UQLB_ERR_ARG, "init_gpc: unknown quadrature");
    if (quad == UQLB_QUAD_GAUSS_LEGENDRE_TENSOR && (pts_per_dim < 1 || pts_per_dim > 64))
        return set_err(ctx, UQLB_ERR_ARG, "init_gpc: need 1 <= pts_per_dim <= 64");
    if (quad == UQLB_QUAD_CLENSHAW_CURTIS_SMOLYAK && (pts_per_dim < 0 || pts_per_dim > 6))
        return set_err(ctx, UQLB_ERR_ARG, "init_gpc: the Smolyak level must be 0..6");
    int64_t K = 0;
    if (uqlb_num_multi_indices(ctx->dim, order, basis, &K) != 0)
        return set_err(ctx, UQLB_ERR_ARG, "init_gpc: %s", g_last_error.c_str());
    const int d = ctx->dim;
    int64_t S = 0;
    std::vector<double> ref_xi, ref_a;
    std::vector<double> gx, gw;
    if (quad == UQLB_QUAD_GAUSS_LEGENDRE_TENSOR) {
        const double Sd = std::pow((double)pts_per_dim, d);
        if (Sd > (double)(1 << 24)) return set_err(ctx, UQLB_ERR_ARG, "init_gpc: tensor grid too large");
        S = (int64_t)std::llround(Sd);
        gx.assign(pts_per_dim, 0.0);
        gw.assign(pts_per_dim, 0.0);
        gauss_legendre_rule(pts_per_dim, gx.data(), gw.data());
        ref_xi.assign((size_t)S * d, 0.0);
        ref_a.assign((size_t)S, 0.0);
        std::vector<int> idx(d, 0);
        for (int64_t s = 0; s < S; ++s) {
            // lexicographic, last dimension fastest
            int64_t r = s;
            for (int k = d - 1; k >= 0; --k) {
                idx[k] = (int)(r % pts_per_dim);
                r /= pts_per_dim;
            }
            double w = 1.0;
            for (int k = 0; k < d; ++k) {
                ref_xi[(size_t)s * d + k] = gx[idx[k]];
                w *= 0.5 * gw[idx[k]];
            }
            ref_a[s] = w;
        }
    } else {
        smolyak_cc_grid(d, pts_per_dim, ref_xi, ref_a);
        S = (int64_t)ref_a.size();
    }
    if (K * S > (int64_t)1 << 28) return set_err(ctx, UQLB_ERR_ARG, "init_gpc: K x S too large");
    ctx->xi = ref_xi;
    ctx->a = ref_a;
    ctx->z.assign((size_t)S * d, 0.0);
    for (int64_t s = 0; s < S; ++s)
        for (int k = 0; k < d; ++k) {
            const double lo = ctx->dists[k].a, hi = ctx->dists[k].b;
            ctx->z[(size_t)s * d + k] = 0.5 * (lo + hi) + 0.5 * (hi - lo) * ctx->xi[(size_t)s * d + k];
        }
    enumerate_indices(d, order, basis, ctx->alpha);
    ctx->K = (int)K;
    ctx->W.assign((size_t)K * S, 0.0);
    std::vector<double> phis((size_t)(order + 1) * d);
    for (int64_t s = 0; s < S; ++s) {
        for (int k = 0; k < d; ++k) phi_values(order, ctx->xi[(size_t)s * d + k], phis.data() + (size_t)k * (order + 1));
        for (int64_t t = 0; t < K; ++t) {
            double v = ctx->a[s];
            for (int k = 0; k < d; ++k) v *= phis[(size_t)k * (order + 1) + ctx->alpha[(size_t)t * d + k]];
            ctx->W[(size_t)t * S + s] = v;
        }
    }
    ctx->S = S;
    ctx->order = order;
    ctx->basis = basis;
    ctx->method = UQLB_METHOD_GPC;
    if (quad == UQLB_QUAD_GAUSS_LEGENDRE_TENSOR) build_sum_factor_plan(ctx, pts_per_dim, gx, gw);
    return 0;
}

int uqlb_num_samples(const uqlb_ctx* ctx, int64_t* n) {
    if (!ctx || !n) return set_err(nullptr, UQLB_ERR_ARG, "num_samples: null pointer");
    *n = ctx->S;
    return 0;
}

int uqlb_num_terms(const uqlb_ctx* ctx, int* k) {
    if (!ctx || !k) return set_err(nullptr, UQLB_ERR_ARG, "num_terms: null pointer");
    *k = ctx->K;
    return 0;
}

int uqlb_get_samples(const uqlb_ctx* ctx, double* z, double* xi, double* a) {
    if (!ctx) return set_err(nullptr, UQLB_ERR_ARG, "null context");
    if (ctx->S <= 0) return set_err(const_cast<uqlb_ctx*>(ctx), UQLB_ERR_STATE, "get_samples: no sample set");
    if (z) std::memcpy(z, ctx->z.data(), ctx->z.size() * sizeof(double));
    if (xi) std::memcpy(xi, ctx->xi.data(), ctx->xi.size() * sizeof(double));
    if (a) std::memcpy(a, ctx->a.data(), ctx->a.size() * sizeof(double));
    return 0;
}

int uqlb_get_weight_matrix(const uqlb_ctx* ctx, double* w) {
    if (!ctx || !w) return set_err(nullptr, UQLB_ERR_ARG, "get_weight_matrix: null pointer");
    if (ctx->method != UQLB_METHOD_GPC) return set_err(const_cast<uqlb_ctx*>(ctx), UQLB_ERR_STATE, "get_weight_matrix: call uqlb_init_gpc first");
    std::memcpy(w, ctx->W.data(), ctx->W.size() * sizeof(double));
    return 0;
}

int uqlb_batch_workspace_bytes(const uqlb_sample* samples, int64_t n, const uqlb_run_opts* opts, size_t* bytes) {
    if (!samples || !bytes || !opts) return set_err(nullptr, UQLB_ERR_ARG, "batch_workspace_bytes: null pointer");
    std::string why;
    if (int rc = batch_bytes(samples, n, opts, bytes, why)) return set_err(nullptr, rc, "%s", why.c_str());
    return 0;
}

int uqlb_autotune(uqlb_ctx* ctx, const uqlb_sample* samples, int64_t n, const uqlb_run_opts* opts,
                  void* workspace_dev, size_t workspace_bytes, int trial_steps, int32_t* tile_rows,
                  int32_t* nodes_per_thread, int32_t* rows_tried, int32_t* npt_tried, double* ms_per_step,
                  int32_t* n_tried, void* stream) {
    if (int rc = check_ctx(ctx)) return rc;
    if (!samples || !opts || !workspace_dev) return set_err(ctx, UQLB_ERR_ARG, "autotune: null argument");
    if (trial_steps < 2 || (trial_steps & 1) || trial_steps > 4096)
        return set_err(ctx, UQLB_ERR_ARG, "autotune: trial_steps must be even, 2..4096");
    {
        // a batch that runs as groups: each group is tuned on its own (the run looks each up by its
        // shape); the outputs describe the group with the most node updates
        auto groups = make_groups(samples, n, opts);
        if (!groups.empty()) {
            size_t big = 0;
            double most = -1.0;
            for (size_t g = 0; g < groups.size(); ++g) {
                double w = 0.0;
                for (auto& x : groups[g].smp) w += (double)x.nx * x.ny * (double)x.steps;
                if (w > most) {
                    most = w;
                    big = g;
                }
            }
            // the largest group last, so that the context's report describes it
            for (size_t k = 0; k <= groups.size(); ++k) {
                if (k == big) continue;
                const size_t g = k == groups.size() ? big : k;
                const bool out = g == big;
                if (int rc = uqlb_autotune(ctx, groups[g].smp.data(), (int64_t)groups[g].smp.size(), &groups[g].opts,
                                           workspace_dev, workspace_bytes, trial_steps, out ? tile_rows : nullptr,
                                           out ? nodes_per_thread : nullptr, out ? rows_tried : nullptr,
                                           out ? npt_tried : nullptr, out ? ms_per_step : nullptr,
                                           out ? n_tried : nullptr, stream))
                    return rc;
            }
            return 0;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e;
    if ((e = cudaEventCreate(&e0)) || (e = cudaEventCreate(&e1))) return cuda_fail(ctx, e, "autotune: events");
    int rc = 0, best = -1, spl = 1;
    double best_ms = 1e300;
    int storage = opts->storage, mixed = 0;
    int64_t nodes = 0;
    std::vector<uqlb_tune_candidate> cands;
    for (int64_t k = 0; k < n; ++k) {
        mixed |= samples[k].kind == UQLB_CASE_CHANNEL;
        nodes += (int64_t)samples[k].nx * samples[k].ny;
    }
    {
        BatchPlan P0;
        std::string why;
        uqlb_run_opts o0 = *opts;
        o0.tile_rows = o0.nodes_per_thread = 0;
        o0.strip_blocks_per_sm = o0.strip_stage = o0.strip_smem_kb = 0;
        if ((rc = plan_batch(samples, n, &o0, P0, why))) {
            rc = set_err(ctx, rc, "autotune: %s", why.c_str());
            goto done;
        }
        const BatchGeometry& g0 = P0.geom;
        const bool two = g0.two_step != 0;
        spl = two ? std::max(g0.spl, 2) : 1;
        const int scheme = !two ? UQLB_SCHEME_ONE_STEP
                                : (g0.strips ? (g0.spl == 3 ? UQLB_SCHEME_THREE_STEP_STRIPS : UQLB_SCHEME_TWO_STEP_STRIPS)
                                             : UQLB_SCHEME_TWO_STEP_TILES);
        if (scheme == UQLB_SCHEME_THREE_STEP_STRIPS) {
            // staging option x blocks per SM (the most that fit and up to three fewer) x share (the
            // smallest holding the blocks, and the largest)
            const bool fixed = strip3_fixed_width(g0.strip_nx);
            for (int stage : {fixed ? 2 : 0, fixed ? 1 : -1, fixed ? 3 : -1}) {
                int max_b = 0, def_b = 0, def_kb = 0, per = 0;
                if (stage < 0 || !strip3_blocks(g0, stage, &max_b, &def_b, &def_kb, &per)) continue;
                for (int b = max_b; b >= std::max(1, max_b - 3); --b) {
                    const int fit = smem_config_for((size_t)b * per);
                    cands.push_back({scheme, g0.tile_rows, g0.npt, b, stage, fit, 0.0});
                    if (fit != 228) cands.push_back({scheme, g0.tile_rows, g0.npt, b, stage, 228, 0.0});
                }
            }
        } else {
            for (int r : kGeomRows)
                for (int q : kGeomNpt) {
                    if (two ? !geometry_supported2(storage, r, q) : !geometry_supported(storage, mixed != 0, r, q))
                        continue;
                    // the two-step row strips do not use the tile geometry (only the init and finalize do)
                    if (g0.strips && (r != g0.tile_rows || q != g0.npt)) continue;
                    cands.push_back({scheme, r, q, 0, 0, 0, 0.0});
                }
        }
    }
    for (size_t c = 0; c < cands.size(); ++c) {
        uqlb_tune_candidate& cd = cands[c];
        uqlb_run_opts o = *opts;
        o.tile_rows = cd.tile_rows;
        o.nodes_per_thread = cd.nodes_per_thread;
        o.strip_blocks_per_sm = cd.strip_blocks_per_sm;
        o.strip_stage = cd.strip_stage;
        o.strip_smem_kb = cd.strip_smem_kb;
        o.qoi_every = 0;
        BatchPlan P;
        std::string why;
        if ((rc = plan_batch(samples, n, &o, P, why))) {
            rc = set_err(ctx, rc, "autotune: %s", why.c_str());
            goto done;
        }
        if (workspace_bytes < P.total) {
            rc = set_err(ctx, UQLB_ERR_OOM, "autotune: workspace of %zu bytes, need %zu", workspace_bytes, P.total);
            goto done;
        }
        const bool two = P.geom.two_step != 0;
        BatchBuffers B = carve(P, workspace_dev);
        char* ws = static_cast<char*>(workspace_dev);
        RunOutputs O{};
        // every sample steps for the whole trial, whatever its own step count: one untimed launch
        // (it also takes the write-back of the initial state), then trial_steps timed steps
        const int warm = spl, total = warm + trial_steps;
        P.geom.max_steps = total;
        for (auto& d : P.table) d.steps = total;
        for (auto& v : P.steps_sorted) v = total;
        if ((e = cudaMemcpyAsync(ws + P.off_samples, P.table.data(), sizeof(SampleDev) * n, cudaMemcpyHostToDevice, s)) ||
            (e = cudaMemcpyAsync(ws + P.off_init, P.init.data(), sizeof(InitDev) * n, cudaMemcpyHostToDevice, s)) ||
            (e = cudaMemcpyAsync(ws + P.off_steps, P.steps_sorted.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s)) ||
            (e = cudaMemcpyAsync(ws + P.off_rowbase, P.row_base.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, s)) ||
            (!P.masks.empty() && (e = cudaMemcpyAsync(ws + P.off_masks, P.masks.data(), sizeof(uint32_t) * P.masks.size(),
                                                      cudaMemcpyHostToDevice, s))) ||
            (e = cudaMemsetAsync(ws + P.off_side, 0, P.off_partials - P.off_side, s))) {
            rc = cuda_fail(ctx, e, "autotune: upload");
            goto done;
        }
        if (two && (e = prepare_step2(P.geom)) != cudaSuccess) {
            rc = cuda_fail(ctx, e, "autotune: prepare");
            goto done;
        }
        double ms_best = 1e300;
        for (int pass = 0; pass < 3; ++pass) {
            if ((e = cudaMemsetAsync(B.step_counter, 0, 2 * sizeof(int64_t), s)) || (e = launch_init(B, P.geom, s))) {
                rc = cuda_fail(ctx, e, "autotune: init");
                goto done;
            }
            for (int dt = 0; dt < total; dt += spl)
                if ((dt == warm && (e = cudaEventRecord(e0, s))) ||
                    (e = two ? launch_step2(B, P.geom, O, dt, s) : launch_step(B, P.geom, O, dt, 0, s))) {
                    rc = cuda_fail(ctx, e, "autotune: step launch");
                    goto done;
                }
            float f = 0.0f;
            if ((e = cudaEventRecord(e1, s)) || (e = cudaEventSynchronize(e1)) || (e = cudaEventElapsedTime(&f, e0, e1))) {
                rc = cuda_fail(ctx, e, "autotune: timing");
                goto done;
            }
            ms_best = std::min(ms_best, (double)f / trial_steps);
        }
        cd.ms_per_step = ms_best;
        if (c < 16) {
            if (rows_tried) rows_tried[c] = cd.tile_rows;
            if (npt_tried) npt_tried[c] = cd.nodes_per_thread;
            if (ms_per_step) ms_per_step[c] = ms_best;
        }
        if (ms_best < best_ms) {
            best_ms = ms_best;
            best = (int)c;
        }
    }
    if (best >= 0) {
        const uqlb_tune_candidate& w = cands[best];
        TuneChoice tc;
        tc.rows = w.tile_rows;
        tc.npt = w.nodes_per_thread;
        tc.bps = w.strip_blocks_per_sm;
        tc.stage = w.strip_stage;
        tc.smem_kb = w.strip_smem_kb;
        bool found = false;
        for (auto& t : ctx->tuned)
            if (t.storage == storage && t.mixed == mixed && t.n == n && t.nodes == nodes) {
                t.choice = tc;
                found = true;
            }
        if (!found) ctx->tuned.push_back({storage, mixed, n, nodes, tc});
        if (tile_rows) *tile_rows = w.tile_rows;
        if (nodes_per_thread) *nodes_per_thread = w.nodes_per_thread;
    }
    ctx->tune_report = cands;
    ctx->tune_chosen = best;
    if (n_tried) *n_tried = (int32_t)std::min<size_t>(cands.size(), 16);
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int uqlb_autotune_report(const uqlb_ctx* ctx, uqlb_tune_candidate* out, int32_t cap, int32_t* n, int32_t* chosen) {
    if (!ctx) return set_err(nullptr, UQLB_ERR_ARG, "null context");
    if (cap < 0 || (cap > 0 && !out)) return set_err(nullptr, UQLB_ERR_ARG, "autotune_report: bad output array");
    const size_t m = std::min<size_t>(ctx->tune_report.size(), (size_t)cap);
    for (size_t k = 0; k < m; ++k) out[k] = ctx->tune_report[k];
    if (n) *n = (int32_t)ctx->tune_report.size();
    if (chosen) *chosen = ctx->tune_chosen;
    return 0;
}

int uqlb_run_batch(uqlb_ctx* ctx, const uqlb_sample* samples, int64_t n, const uqlb_run_opts* opts,
                   void* workspace_dev, size_t workspace_bytes, void* fields_dev, int64_t fields_ld,
                   double* qoi_dev, double* series_dev, double* series_cl_dev, int64_t series_ld, void* stream) {
    if (int rc = check_ctx(ctx)) return rc;
    if (!samples || !opts || !workspace_dev) return set_err(ctx, UQLB_ERR_ARG, "run_batch: null argument");
    if (reinterpret_cast<uintptr_t>(workspace_dev) % 256 != 0) return set_err(ctx, UQLB_ERR_ARG, "run_batch: workspace must be 256-byte aligned");
    // the geometry the autotuner picked for a batch of this shape, if any
    auto tuned_for = [&](const uqlb_sample* smp, int64_t m) {
        int mixed = 0;
        int64_t nodes = 0;
        for (int64_t k = 0; k < m; ++k) {
            mixed |= smp[k].kind == UQLB_CASE_CHANNEL;
            nodes += (int64_t)smp[k].nx * smp[k].ny;
        }
        TuneChoice tc;
        for (auto& t : ctx->tuned)
            if (t.storage == opts->storage && t.mixed == mixed && t.n == m && t.nodes == nodes) tc = t.choice;
        return tc;
    };
    // plans: one, or one per group of like samples
    std::string why;
    auto groups = make_groups(samples, n, opts);
    std::vector<BatchPlan> plans(groups.empty() ? 1 : groups.size());
    std::vector<size_t> offs(plans.size(), 0);
    size_t need = 0;
    for (size_t g = 0; g < plans.size(); ++g) {
        const uqlb_sample* smp = groups.empty() ? samples : groups[g].smp.data();
        const int64_t m = groups.empty() ? n : (int64_t)groups[g].smp.size();
        const uqlb_run_opts* o = groups.empty() ? opts : &groups[g].opts;
        if (int rc = plan_batch(smp, m, o, plans[g], why, tuned_for(smp, m), groups.empty() ? nullptr : groups[g].idx.data()))
            return set_err(ctx, rc, "run_batch: %s", why.c_str());
        offs[g] = need;
        need = align_up(need + plans[g].total, 256);
    }
    if (groups.empty()) need = plans[0].total;
    if (workspace_bytes < need)
        return set_err(ctx, UQLB_ERR_OOM, "run_batch: workspace of %zu bytes, need %zu", workspace_bytes, need);
    int max_steps = 0, n_steady = 0;
    bool uniform_size = true;
    for (auto& P : plans) {
        max_steps = std::max(max_steps, P.geom.max_steps);
        n_steady += P.n_steady;
        uniform_size = uniform_size && P.uniform_size;
    }
    for (int64_t k = 1; k < n; ++k)
        if (samples[k].nx != samples[0].nx || samples[k].ny != samples[0].ny) uniform_size = false;
    const BatchPlan& P0 = plans[0];
    ctx->last_rows = P0.geom.tile_rows;
    ctx->last_npt = P0.geom.npt;
    ctx->last_scheme = !groups.empty() ? UQLB_SCHEME_GROUPED
                       : P0.geom.cluster ? UQLB_SCHEME_CLUSTER
                       : !P0.geom.two_step ? UQLB_SCHEME_ONE_STEP
                       : (P0.geom.strips ? (P0.geom.spl == 3 ? UQLB_SCHEME_THREE_STEP_STRIPS : UQLB_SCHEME_TWO_STEP_STRIPS)
                                         : UQLB_SCHEME_TWO_STEP_TILES);
    if (fields_dev) {
        if (!uniform_size) return set_err(ctx, UQLB_ERR_ARG, "run_batch: field output needs one lattice size");
        if (fields_ld < 2 * (int64_t)samples[0].nx * samples[0].ny + 1) return set_err(ctx, UQLB_ERR_ARG, "run_batch: fields_ld too small");
        if (opts->fields_dtype != UQLB_F64 && opts->fields_dtype != UQLB_F32)
            return set_err(ctx, UQLB_ERR_ARG, "run_batch: fields_dtype must be F64 or F32");
    }
    if (opts->qoi_every < 0) return set_err(ctx, UQLB_ERR_ARG, "run_batch: qoi_every must be >= 0");
    if (opts->start_step < 0 || opts->start_step > max_steps)
        return set_err(ctx, UQLB_ERR_ARG, "run_batch: start_step must be in [0, the largest step count]");
    if ((series_dev || series_cl_dev) && opts->qoi_every > 0) {
        const int64_t need_ld = max_steps / opts->qoi_every + 1;
        if (series_ld < need_ld) return set_err(ctx, UQLB_ERR_ARG, "run_batch: series_ld %lld < %lld", (long long)series_ld, (long long)need_ld);
    }
    const int chunk = opts->chunk_steps > 0 ? opts->chunk_steps : 64;
    if (chunk < 2 || chunk > 1024 || (chunk & 1)) return set_err(ctx, UQLB_ERR_ARG, "run_batch: chunk_steps must be even, 2..1024");
    if (n_steady > 0 && opts->qoi_every <= 0)
        return set_err(ctx, UQLB_ERR_ARG, "run_batch: a steady-state tolerance needs qoi_every > 0");

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (!ctx->loop_begin) {
        if ((e = cudaEventCreate(&ctx->loop_begin)) || (e = cudaEventCreate(&ctx->loop_end)))
            return cuda_fail(ctx, e, "run_batch: event create");
    }
    ctx->loop_timed = false;
    ctx->loop_steps = max_steps;
    ctx->run_launches = 0;
    if (groups.empty())
        return run_planned(ctx, P0, n, opts, workspace_dev, fields_dev, fields_ld, qoi_dev, series_dev, series_cl_dev,
                           series_ld, s, true);
    // The loop time spans all groups (their init and finalize included).  CHANNEL groups are bound by
    // latency (a cluster step, or one launch per step), the periodic groups by HBM and issue, so the
    // channel groups run on a second stream of the highest priority beside the periodic groups on the
    // caller's stream, and share the SMs with them; the caller's stream then waits for both.  Launch
    // order: the cluster group (one launch, the whole loop), the periodic groups, then the one-step
    // channel group, whose steady-state test synchronises its stream between graph launches after
    // every other group has been enqueued.
    auto is_channel = [&](size_t g) {
        return groups[g].scheme == UQLB_SCHEME_CLUSTER || groups[g].smp[0].kind == UQLB_CASE_CHANNEL;
    };
    bool any_channel = false, any_periodic = false;
    for (size_t g = 0; g < groups.size(); ++g) (is_channel(g) ? any_channel : any_periodic) = true;
    const bool fork = UQLB_GROUPS_CONCURRENT && any_channel && any_periodic;
    if (fork && !ctx->side_stream) {
        int least = 0, greatest = 0;
        if ((e = cudaDeviceGetStreamPriorityRange(&least, &greatest)) ||
            (e = cudaStreamCreateWithPriority(&ctx->side_stream, cudaStreamNonBlocking, greatest)) ||
            (e = cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming)) ||
            (e = cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming)))
            return cuda_fail(ctx, e, "run_batch: side stream");
    }
    const cudaStream_t cs = fork ? ctx->side_stream : s;
    if ((e = cudaEventRecord(ctx->loop_begin, s)) != cudaSuccess) return cuda_fail(ctx, e, "run_batch: event record");
    if (fork && ((e = cudaEventRecord(ctx->fork_ev, s)) || (e = cudaStreamWaitEvent(cs, ctx->fork_ev, 0))))
        return cuda_fail(ctx, e, "run_batch: fork");
    auto run_group = [&](size_t g, cudaStream_t st) {
        return run_planned(ctx, plans[g], (int64_t)groups[g].smp.size(), &groups[g].opts,
                           static_cast<char*>(workspace_dev) + offs[g], fields_dev, fields_ld, qoi_dev, series_dev,
                           series_cl_dev, series_ld, st, false);
    };
    for (int pass = 0; pass < 3; ++pass)
        for (size_t g = 0; g < groups.size(); ++g) {
            const int at = groups[g].scheme == UQLB_SCHEME_CLUSTER ? 0 : (is_channel(g) ? 2 : 1);
            if (at != pass) continue;
            if (int rc = run_group(g, is_channel(g) ? cs : s)) return rc;
        }
    if (fork && ((e = cudaEventRecord(ctx->join_ev, cs)) || (e = cudaStreamWaitEvent(s, ctx->join_ev, 0))))
        return cuda_fail(ctx, e, "run_batch: join");
    if ((e = cudaEventRecord(ctx->loop_end, s)) != cudaSuccess) return cuda_fail(ctx, e, "run_batch: event record");
    ctx->loop_timed = true;
    return 0;
}

int uqlb_last_run_geometry(const uqlb_ctx* ctx, int32_t* scheme, int32_t* tile_rows, int32_t* nodes_per_thread) {
    if (!ctx) return set_err(nullptr, UQLB_ERR_ARG, "null context");
    if (ctx->last_scheme == 0) return set_err(const_cast<uqlb_ctx*>(ctx), UQLB_ERR_STATE, "no run yet");
    if (scheme) *scheme = ctx->last_scheme;
    const bool cl = ctx->last_scheme == UQLB_SCHEME_CLUSTER;
    if (tile_rows) *tile_rows = cl ? ctx->cluster_blocks : ctx->last_rows;
    if (nodes_per_thread) *nodes_per_thread = cl ? ctx->cluster_cols : ctx->last_npt;
    return 0;
}

int uqlb_last_loop_time(uqlb_ctx* ctx, double* ms, int64_t* steps, int64_t* launches) {
    if (int rc = check_ctx(ctx)) return rc;
    if (steps) *steps = ctx->loop_steps;
    if (launches) *launches = ctx->run_launches;
    if (ms) {
        *ms = 0.0;
        if (ctx->loop_timed) {
            float f = 0.0f;
            cudaError_t e;
            if ((e = cudaEventSynchronize(ctx->loop_end)) || (e = cudaEventElapsedTime(&f, ctx->loop_begin, ctx->loop_end)))
                return cuda_fail(ctx, e, "last_loop_time");
            *ms = f;
        }
    }
    if (ctx->bar_err && ctx->loop_timed) {
        int32_t err = 0;
        cudaError_t e;
        if ((e = cudaEventSynchronize(ctx->loop_end)) || (e = cudaMemcpy(&err, ctx->bar_err, sizeof err, cudaMemcpyDeviceToHost)))
            return cuda_fail(ctx, e, "last_loop_time: status");
        if (err != 0) return set_err(ctx, UQLB_ERR_TIMEOUT, "last run: a bounded grid-barrier wait gave up");
    }
    return 0;
}

int uqlb_ensemble_samples(const uqlb_ctx* ctx, const uqlb_case* c, uqlb_sample* out) {
    if (!ctx || !c || !out) return set_err(nullptr, UQLB_ERR_ARG, "ensemble_samples: null pointer");
    if (int rc = check_case(const_cast<uqlb_ctx*>(ctx), c)) return rc;
    build_ensemble(ctx, c, out);
    return 0;
}

int uqlb_ensemble_workspace_bytes(const uqlb_ctx* ctx, const uqlb_case* c, const uqlb_run_opts* opts, size_t* bytes) {
    if (!ctx || !c || !bytes || !opts) return set_err(nullptr, UQLB_ERR_ARG, "ensemble_workspace_bytes: null pointer");
    if (int rc = check_case(const_cast<uqlb_ctx*>(ctx), c)) return rc;
    std::vector<uqlb_sample> smp(ctx->S);
    build_ensemble(ctx, c, smp.data());
    std::string why;
    if (int rc = batch_bytes(smp.data(), ctx->S, opts, bytes, why))
        return set_err(const_cast<uqlb_ctx*>(ctx), rc, "%s", why.c_str());
    return 0;
}

int uqlb_run_ensemble(uqlb_ctx* ctx, const uqlb_case* c, const uqlb_run_opts* opts, void* workspace_dev,
                      size_t workspace_bytes, void* fields_dev, int64_t fields_ld, double* qoi_dev,
                      double* series_dev, double* series_cl_dev, int64_t series_ld, void* stream) {
    if (!ctx) return set_err(nullptr, UQLB_ERR_ARG, "null context");
    if (int rc = check_case(ctx, c)) return rc;
    std::vector<uqlb_sample> smp(ctx->S);
    build_ensemble(ctx, c, smp.data());
    return uqlb_run_batch(ctx, smp.data(), ctx->S, opts, workspace_dev, workspace_bytes, fields_dev, fields_ld,
                          qoi_dev, series_dev, series_cl_dev, series_ld, stream);
}

int uqlb_plain_workspace_bytes(const uqlb_sample* samples, int64_t n, size_t* bytes) {
    if (!samples || !bytes || n < 1) return set_err(nullptr, UQLB_ERR_ARG, "plain_workspace_bytes: bad arguments");
    int64_t maxn = 0;
    std::string why;
    for (int64_t s = 0; s < n; ++s) {
        if (int rc = validate_sample(samples[s], s, why)) return set_err(nullptr, rc, "%s", why.c_str());
        maxn = std::max<int64_t>(maxn, (int64_t)samples[s].nx * samples[s].ny);
    }
    const int64_t blocks = (maxn + 255) / 256;
    *bytes = align_up((size_t)maxn * 9 * 8, 256) * 2 + align_up((size_t)maxn, 256) + align_up((size_t)blocks * 7 * 8, 256);
    return 0;
}

int uqlb_run_plain_f64(uqlb_ctx* ctx, const uqlb_sample* samples, int64_t n, int64_t qoi_every, void* workspace_dev,
                       size_t workspace_bytes, double* fields_dev, int64_t fields_ld, double* qoi_dev,
                       double* series_dev, int64_t series_ld, void* stream) {
    if (int rc = check_ctx(ctx)) return rc;
    size_t need = 0;
    if (int rc = uqlb_plain_workspace_bytes(samples, n, &need)) return set_err(ctx, rc, "run_plain_f64: %s", g_last_error.c_str());
    if (!workspace_dev || workspace_bytes < need)
        return set_err(ctx, UQLB_ERR_OOM, "run_plain_f64: workspace of %zu bytes, need %zu", workspace_bytes, need);
    if (qoi_every < 0) return set_err(ctx, UQLB_ERR_ARG, "run_plain_f64: qoi_every must be >= 0");
    for (int64_t s = 0; s < n; ++s)
        if (samples[s].kind == UQLB_CASE_CHANNEL &&
            ((samples[s].cyl_r > 0.0 && samples[s].obstacle_bc != UQLB_OBSTACLE_HALFWAY) ||
             samples[s].inout_bc != UQLB_INOUT_FACE))
            return set_err(ctx, UQLB_ERR_ARG,
                           "run_plain_f64: the plain path has halfway bounce-back and the face inlet/outlet only");
    int64_t maxn = 0;
    for (int64_t s = 0; s < n; ++s) maxn = std::max<int64_t>(maxn, (int64_t)samples[s].nx * samples[s].ny);
    if (fields_dev) {
        for (int64_t s = 0; s < n; ++s)
            if (samples[s].nx != samples[0].nx || samples[s].ny != samples[0].ny)
                return set_err(ctx, UQLB_ERR_ARG, "run_plain_f64: field output needs one lattice size");
        if (fields_ld < 2 * (int64_t)samples[0].nx * samples[0].ny + 1) return set_err(ctx, UQLB_ERR_ARG, "run_plain_f64: fields_ld too small");
    }
    char* ws = static_cast<char*>(workspace_dev);
    const size_t lat = align_up((size_t)maxn * 9 * 8, 256);
    double* fa = reinterpret_cast<double*>(ws);
    double* fb = reinterpret_cast<double*>(ws + lat);
    uint8_t* solid = reinterpret_cast<uint8_t*>(ws + 2 * lat);
    double* partials = reinterpret_cast<double*>(ws + 2 * lat + align_up((size_t)maxn, 256));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<uint8_t> mask;
    for (int64_t q = 0; q < n; ++q) {
        const uqlb_sample& sm = samples[q];
        PlainSample p{};
        p.nx = sm.nx;
        p.ny = sm.ny;
        p.kind = sm.kind;
        p.steps = (int32_t)sm.steps;
        p.omega = 1.0 / (3.0 * sm.nu + 0.5);
        p.u0 = sm.u0;
        p.amp2 = sm.amp2;
        p.amp3 = sm.amp3;
        p.u_ref_inv2 = sm.u_ref > 0.0 ? 2.0 / ((double)sm.nx * sm.ny * sm.u_ref * sm.u_ref) : 0.0;
        p.uin_max = 1.5 * sm.u0;
        p.force_norm = (sm.kind == UQLB_CASE_CHANNEL && sm.cyl_r > 0.0 && sm.u0 != 0.0) ? 2.0 / (sm.u0 * sm.u0 * 2.0 * sm.cyl_r) : 0.0;
        p.ramp_steps = (double)std::max<int64_t>(sm.ramp_steps, 0);
        p.cyl_cx = sm.cyl_cx;
        p.cyl_cy = sm.cyl_cy;
        p.cyl_r = sm.cyl_r;
        mask.assign((size_t)sm.nx * sm.ny, 0);
        for (int y = 0; y < sm.ny; ++y)
            for (int x = 0; x < sm.nx; ++x) mask[(size_t)y * sm.nx + x] = sample_solid(sm, x, y) ? 1 : 0;
        cudaError_t e = cudaMemcpyAsync(solid, mask.data(), mask.size(), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "run_plain_f64: mask upload");
        e = plain_run_sample(p, fa, fb, solid, partials, qoi_every, fields_dev ? fields_dev + q * fields_ld : nullptr,
                             qoi_dev ? qoi_dev + q * UQLB_QOI_COLS : nullptr,
                             series_dev ? series_dev + q * series_ld : nullptr, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "run_plain_f64: launch");
    }
    return 0;
}

int uqlb_w1_workspace_bytes(int bins, size_t* bytes) {
    if (bins < 1 || bins > (1 << 24) || !bytes) return set_err(nullptr, UQLB_ERR_ARG, "w1_workspace_bytes: need 1 <= bins <= 2^24");
    *bytes = align_up(256 + (size_t)2 * bins * sizeof(uint32_t), 256) + 256;
    return 0;
}

int uqlb_w1_speed(uqlb_ctx* ctx, const void* a_dev, int dtype_a, int64_t s_a, int64_t nodes_a, int64_t ld_a,
                  const void* b_dev, int dtype_b, int64_t s_b, int64_t nodes_b, int64_t ld_b, int bins,
                  void* workspace_dev, size_t workspace_bytes, double* out_host, double* bound_host,
                  int64_t* nonfinite_host, void* stream) {
    if (int rc = check_ctx(ctx)) return rc;
    size_t need = 0;
    if (int rc = uqlb_w1_workspace_bytes(bins, &need)) return set_err(ctx, rc, "w1_speed: %s", g_last_error.c_str());
    if (!a_dev || !b_dev || !workspace_dev || !out_host || s_a < 1 || s_b < 1 || nodes_a < 1 || nodes_b < 1 ||
        ld_a < 2 * nodes_a || ld_b < 2 * nodes_b)
        return set_err(ctx, UQLB_ERR_ARG, "w1_speed: bad arguments");
    if ((dtype_a != UQLB_F64 && dtype_a != UQLB_F32) || (dtype_b != UQLB_F64 && dtype_b != UQLB_F32))
        return set_err(ctx, UQLB_ERR_ARG, "w1_speed: dtype must be F64 or F32");
    if (workspace_bytes < need) return set_err(ctx, UQLB_ERR_OOM, "w1_speed: workspace of %zu bytes, need %zu", workspace_bytes, need);
    if ((double)s_a * nodes_a > 4.0e9 || (double)s_b * nodes_b > 4.0e9)
        return set_err(ctx, UQLB_ERR_ARG, "w1_speed: more than 4e9 values in one set");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* out_dev = reinterpret_cast<double*>(static_cast<char*>(workspace_dev) + need - 256);
    cudaError_t e = launch_w1_speed(a_dev, dtype_a, s_a, nodes_a, ld_a, b_dev, dtype_b, s_b, nodes_b, ld_b, bins,
                                    workspace_dev, out_dev, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "w1_speed: launch");
    double r[4] = {0.0, 0.0, 0.0, 0.0};
    if ((e = cudaMemcpyAsync(r, out_dev, sizeof r, cudaMemcpyDeviceToHost, s)) || (e = cudaStreamSynchronize(s)))
        return cuda_fail(ctx, e, "w1_speed: copy back");
    *out_host = r[0];
    if (bound_host) *bound_host = r[1];
    if (nonfinite_host) {
        nonfinite_host[0] = (int64_t)r[2];
        nonfinite_host[1] = (int64_t)r[3];
    }
    return 0;
}

int uqlb_post_workspace_bytes(const uqlb_ctx* ctx, size_t* bytes) {
    if (!ctx || !bytes) return set_err(nullptr, UQLB_ERR_ARG, "post_workspace_bytes: null pointer");
    *bytes = align_up(std::max<size_t>(ctx->W.size(), 1) * sizeof(double), 256);
    return 0;
}

int uqlb_project_workspace_bytes(const uqlb_ctx* ctx, int64_t n_fields, size_t* bytes) {
    if (!ctx || !bytes || n_fields < 0) return set_err(nullptr, UQLB_ERR_ARG, "project_workspace_bytes: bad arguments");
    if (ctx->method != UQLB_METHOD_GPC)
        return set_err(const_cast<uqlb_ctx*>(ctx), UQLB_ERR_STATE, "project_workspace_bytes: call uqlb_init_gpc first");
    if (sf_available(ctx)) {
        *bytes = sf_workspace(ctx, n_fields);
        return 0;
    }
    return uqlb_post_workspace_bytes(ctx, bytes);
}

int uqlb_project(uqlb_ctx* ctx, const void* m_dev, int dtype, int64_t n_fields, int64_t m_ld, double* coeffs_dev,
                 void* workspace_dev, size_t workspace_bytes, void* stream) {
    if (int rc = check_ctx(ctx)) return rc;
    if (ctx->method != UQLB_METHOD_GPC) return set_err(ctx, UQLB_ERR_STATE, "project: call uqlb_init_gpc first");
    if (!m_dev || !coeffs_dev || !workspace_dev || n_fields < 0 || m_ld < n_fields)
        return set_err(ctx, UQLB_ERR_ARG, "project: bad arguments");
    if (dtype != UQLB_F64 && dtype != UQLB_F32) return set_err(ctx, UQLB_ERR_ARG, "project: dtype must be F64 or F32");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    ctx->last_projection = 0;
    if (sf_available(ctx) && workspace_bytes >= sf_workspace(ctx, n_fields) &&
        reinterpret_cast<uintptr_t>(workspace_dev) % 8 == 0) {
        // tensor grid: one contraction per input dimension (sf_stage_kernel), buffers A and B alternate
        const auto& P = ctx->sf;
        char* ws = static_cast<char*>(workspace_dev);
        const int64_t ld = sf_ld(n_fields);
        double* bufs[2] = {reinterpret_cast<double*>(ws + align_up(P.tables.size(), 256)), nullptr};
        bufs[1] = bufs[0] + align_up((size_t)P.rows_a * ld * 8, 256) / 8;
        if ((e = cudaMemcpyAsync(ws, P.tables.data(), P.tables.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return cuda_fail(ctx, e, "project: table upload");
        const double* G = reinterpret_cast<const double*>(ws);
        const void* in = m_dev;
        int in_dtype = dtype;
        int64_t in_ld = m_ld;
        const int nst = (int)P.groups.size();
        for (int m = 0; m < nst; ++m) {
            const bool last = m + 1 == nst;
            double* out = last ? coeffs_dev : bufs[m % 2];
            const int64_t out_ld = last ? n_fields : ld;
            e = launch_sf_stage(in, in_dtype, in_ld, out, out_ld, P.groups[m], P.jprev[m], P.jout[m], P.n, P.p1,
                                reinterpret_cast<const int*>(ws + P.idx_off[m]), G, n_fields, s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "project: stage launch");
            in = out;
            in_dtype = UQLB_F64;
            in_ld = out_ld;
        }
        ctx->last_projection = 1;
        return 0;
    }
    size_t need = 0;
    uqlb_post_workspace_bytes(ctx, &need);
    if (workspace_bytes < need) return set_err(ctx, UQLB_ERR_OOM, "project: workspace of %zu bytes, need %zu", workspace_bytes, need);
    e = cudaMemcpyAsync(workspace_dev, ctx->W.data(), ctx->W.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "project: W upload");
    e = launch_project(static_cast<const double*>(workspace_dev), ctx->K, (int)ctx->S, m_dev, dtype, n_fields, m_ld,
                       coeffs_dev, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "project: launch");
    return 0;
}

int uqlb_last_projection(const uqlb_ctx* ctx, int32_t* kind) {
    if (!ctx || !kind) return set_err(nullptr, UQLB_ERR_ARG, "last_projection: null pointer");
    *kind = ctx->last_projection;
    return 0;
}

int uqlb_get_weight_block(const uqlb_ctx* ctx, int64_t s0, int64_t count, double* w) {
    if (!ctx || !w) return set_err(nullptr, UQLB_ERR_ARG, "get_weight_block: null pointer");
    if (ctx->method != UQLB_METHOD_GPC)
        return set_err(const_cast<uqlb_ctx*>(ctx), UQLB_ERR_STATE, "get_weight_block: call uqlb_init_gpc first");
    if (s0 < 0 || count < 1 || s0 + count > ctx->S)
        return set_err(const_cast<uqlb_ctx*>(ctx), UQLB_ERR_ARG, "get_weight_block: block outside the sample set");
    for (int k = 0; k < ctx->K; ++k)
        std::memcpy(w + (size_t)k * count, ctx->W.data() + (size_t)k * ctx->S + s0, (size_t)count * sizeof(double));
    return 0;
}

int uqlb_project_block(uqlb_ctx* ctx, const void* m_dev, int dtype, int64_t n_fields, int64_t m_ld, int64_t s0,
                       int64_t count, double* coeffs_dev, void* workspace_dev, size_t workspace_bytes, void* stream) {
    if (int rc = check_ctx(ctx)) return rc;
    if (ctx->method != UQLB_METHOD_GPC) return set_err(ctx, UQLB_ERR_STATE, "project_block: call uqlb_init_gpc first");
    if (!m_dev || !coeffs_dev || !workspace_dev || n_fields < 0 || m_ld < n_fields)
        return set_err(ctx, UQLB_ERR_ARG, "project_block: bad arguments");
    if (s0 < 0 || count < 1 || s0 + count > ctx->S)
        return set_err(ctx, UQLB_ERR_ARG, "project_block: block [%lld, %lld) outside the %lld samples", (long long)s0,
                       (long long)(s0 + count), (long long)ctx->S);
    if (dtype != UQLB_F64 && dtype != UQLB_F32) return set_err(ctx, UQLB_ERR_ARG, "project_block: dtype must be F64 or F32");
    size_t need = 0;
    uqlb_post_workspace_bytes(ctx, &need);
    if (workspace_bytes < need)
        return set_err(ctx, UQLB_ERR_OOM, "project_block: workspace of %zu bytes, need %zu", workspace_bytes, need);
    // the block's columns of W, compacted to [K x count] (the kernel reads rows of stride count)
    ctx->w_block.resize((size_t)ctx->K * count);
    uqlb_get_weight_block(ctx, s0, count, ctx->w_block.data());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(workspace_dev, ctx->w_block.data(), ctx->w_block.size() * sizeof(double),
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "project_block: W upload");
    // the upload reads the host copy asynchronously: keep it until the copy is done
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(ctx, e, "project_block: W upload");
    e = launch_project(static_cast<const double*>(workspace_dev), ctx->K, (int)count, m_dev, dtype, n_fields, m_ld,
                       coeffs_dev, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "project_block: launch");
    return 0;
}

int uqlb_block_moments(uqlb_ctx* ctx, const void* m_dev, int dtype, int64_t n_rows, int64_t n_fields, int64_t m_ld,
                       double* mean_dev, double* m2_dev, void* stream) {
    if (int rc = check_ctx(ctx)) return rc;
    if (!m_dev || !mean_dev || !m2_dev || n_rows < 1 || n_fields < 0 || m_ld < n_fields)
        return set_err(ctx, UQLB_ERR_ARG, "block_moments: bad arguments");
    if (dtype != UQLB_F64 && dtype != UQLB_F32) return set_err(ctx, UQLB_ERR_ARG, "block_moments: dtype must be F64 or F32");
    cudaError_t e = launch_mc_stats(m_dev, dtype, n_rows, n_fields, m_ld, mean_dev, m2_dev, -1,
                                    static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "block_moments: launch");
    return 0;
}

int uqlb_stats(uqlb_ctx* ctx, const void* in_dev, int dtype, int64_t n_fields, int64_t m_ld, double* mean_dev,
               double* var_dev, int ddof, void* stream) {
    if (int rc = check_ctx(ctx)) return rc;
    if (!in_dev || n_fields < 0) return set_err(ctx, UQLB_ERR_ARG, "stats: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (ctx->method == UQLB_METHOD_GPC) {
        if (dtype != UQLB_F64) return set_err(ctx, UQLB_ERR_ARG, "stats: gPC coefficients are FP64");
        e = launch_gpc_stats(static_cast<const double*>(in_dev), ctx->K, n_fields, mean_dev, var_dev, s);
    } else if (ctx->method == UQLB_METHOD_MC) {
        if (dtype != UQLB_F64 && dtype != UQLB_F32) return set_err(ctx, UQLB_ERR_ARG, "stats: dtype must be F64 or F32");
        if (m_ld < n_fields || ddof < 0 || ctx->S - ddof < 1) return set_err(ctx, UQLB_ERR_ARG, "stats: bad m_ld or ddof");
        e = launch_mc_stats(in_dev, dtype, ctx->S, n_fields, m_ld, mean_dev, var_dev, ddof, s);
    } else {
        return set_err(ctx, UQLB_ERR_STATE, "stats: no sample set");
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stats: launch");
    return 0;
}

int uqlb_uq_workspace_bytes(const uqlb_ctx* ctx, const uqlb_case* c, const uqlb_run_opts* opts, size_t* bytes) {
    if (!ctx || !c || !opts || !bytes) return set_err(nullptr, UQLB_ERR_ARG, "uq_workspace_bytes: null pointer");
    size_t b = 0;
    if (int rc = uqlb_ensemble_workspace_bytes(ctx, c, opts, &b)) return rc;
    const int64_t F = 2 * (int64_t)c->base.nx * c->base.ny + 1;
    const size_t eb = opts->fields_dtype == UQLB_F64 ? 8 : 4;
    b = align_up(b, 256) + align_up((size_t)ctx->S * F * eb, 256);                 // fields M
    b += align_up((size_t)std::max(ctx->K, 1) * F * 8, 256);                        // coefficients
    b += 2 * align_up((size_t)F * 8, 256);                                          // mean, var
    size_t pb = 0;                                                                   // projection scratch
    if (ctx->method == UQLB_METHOD_GPC) uqlb_project_workspace_bytes(ctx, F, &pb);
    b += align_up(std::max<size_t>(pb, 8), 256);
    b += align_up((size_t)ctx->S * UQLB_QOI_COLS * 8, 256);                         // qoi
    *bytes = b;
    return 0;
}

int uqlb_run_uq_host(uqlb_ctx* ctx, const uqlb_case* c, const uqlb_run_opts* opts, void* workspace_dev,
                     size_t workspace_bytes, double* mean_host, double* var_host, double* coeffs_host,
                     double* qoi_host, void* stream) {
    if (int rc = check_ctx(ctx)) return rc;
    if (!c || !opts || !workspace_dev || !mean_host || !var_host) return set_err(ctx, UQLB_ERR_ARG, "run_uq_host: null argument");
    size_t need = 0;
    if (int rc = uqlb_uq_workspace_bytes(ctx, c, opts, &need)) return set_err(ctx, rc, "run_uq_host: %s", g_last_error.c_str());
    if (workspace_bytes < need) return set_err(ctx, UQLB_ERR_OOM, "run_uq_host: workspace of %zu bytes, need %zu", workspace_bytes, need);
    if (opts->fields_dtype != UQLB_F64 && opts->fields_dtype != UQLB_F32) return set_err(ctx, UQLB_ERR_ARG, "run_uq_host: fields_dtype");
    size_t run_b = 0;
    uqlb_ensemble_workspace_bytes(ctx, c, opts, &run_b);
    const int64_t F = 2 * (int64_t)c->base.nx * c->base.ny + 1;
    const size_t eb = opts->fields_dtype == UQLB_F64 ? 8 : 4;
    char* p = static_cast<char*>(workspace_dev);
    size_t off = align_up(run_b, 256);
    void* M = p + off;
    off += align_up((size_t)ctx->S * F * eb, 256);
    double* C = reinterpret_cast<double*>(p + off);
    off += align_up((size_t)std::max(ctx->K, 1) * F * 8, 256);
    double* mean = reinterpret_cast<double*>(p + off);
    off += align_up((size_t)F * 8, 256);
    double* var = reinterpret_cast<double*>(p + off);
    off += align_up((size_t)F * 8, 256);
    void* wbuf = p + off;
    size_t wb = 0;
    if (ctx->method == UQLB_METHOD_GPC) uqlb_project_workspace_bytes(ctx, F, &wb);
    off += align_up(std::max<size_t>(wb, 8), 256);
    double* qoi = reinterpret_cast<double*>(p + off);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (int rc = uqlb_run_ensemble(ctx, c, opts, workspace_dev, run_b, M, F, qoi, nullptr, nullptr, 0, stream)) return rc;
    if (ctx->method == UQLB_METHOD_GPC) {
        if (int rc = uqlb_project(ctx, M, opts->fields_dtype, F, F, C, wbuf, wb, stream)) return rc;
        if (int rc = uqlb_stats(ctx, C, UQLB_F64, F, F, mean, var, 0, stream)) return rc;
    } else {
        if (int rc = uqlb_stats(ctx, M, opts->fields_dtype, F, F, mean, var, 1, stream)) return rc;
    }
    cudaError_t e;
    if ((e = cudaMemcpyAsync(mean_host, mean, (size_t)F * 8, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(var_host, var, (size_t)F * 8, cudaMemcpyDeviceToHost, s)) ||
        (coeffs_host && ctx->method == UQLB_METHOD_GPC &&
         (e = cudaMemcpyAsync(coeffs_host, C, (size_t)ctx->K * F * 8, cudaMemcpyDeviceToHost, s))) ||
        (qoi_host && (e = cudaMemcpyAsync(qoi_host, qoi, (size_t)ctx->S * UQLB_QOI_COLS * 8, cudaMemcpyDeviceToHost, s))) ||
        (e = cudaStreamSynchronize(s)))
        return cuda_fail(ctx, e, "run_uq_host: copy back");
    return 0;
}

}  // extern "C"
