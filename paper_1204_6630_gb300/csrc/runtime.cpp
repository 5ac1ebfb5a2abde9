// Host runtime of the pair-counting library: contexts, device scratch slots,
// catalogs, bin thresholds, kernel shapes, launches and the estimator.
//
// Paper: Ponce et al., "Application of GPUs for the calculation of two point
// correlation functions in cosmology" (Section 1, Eq. 1: DD, DR, RR and the
// Landy-Szalay estimator; Section 3: dot product + arc-cosine per pair,
// partial histograms merged into one, one histogram per GPU).
//
// Compiled with -ffp-contract=off: every binary64 operation here is rounded
// exactly as written (threshold derivation and the estimator depend on it).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "handles.h"
#include "plan.h"
#include "tpcf.h"
#include "tpcf_internal.h"

using namespace tpcf;

std::atomic<int> tpcf::g_alloc_fail_countdown{-1};

cudaError_t tpcf::dev_malloc(void** p, size_t bytes) {
    int c = g_alloc_fail_countdown.load();
    if (c >= 0) {
        if (c == 0) { *p = nullptr; return cudaErrorMemoryAllocation; }
        g_alloc_fail_countdown.fetch_sub(1);
    }
    return cudaMalloc(p, bytes);
}

cudaError_t tpcf::dev_malloc_async(void** p, size_t bytes, cudaStream_t st) {
    int c = g_alloc_fail_countdown.load();
    if (c >= 0) {
        if (c == 0) { *p = nullptr; return cudaErrorMemoryAllocation; }
        g_alloc_fail_countdown.fetch_sub(1);
    }
    return cudaMallocAsync(p, bytes, st);
}

int tpcf_ctx::fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    std::lock_guard<std::mutex> g(err_mu);
    last_error = buf;
    return code;
}

// ====================================================================== misc
extern "C" const char* tpcf_strerror(int s) {
    switch (s) {
        case TPCF_OK: return "ok";
        case TPCF_EINVAL: return "invalid argument";
        case TPCF_ENOMEM: return "out of memory";
        case TPCF_EBUDGET: return "job exceeds the device-memory budget";
        case TPCF_ECUDA: return "CUDA error";
        case TPCF_EAGAIN: return "not finished";
        case TPCF_ETIMEOUT: return "bounded device wait timed out";
        case TPCF_EOVERFLOW: return "size limit exceeded";
        case TPCF_ECANCELED: return "cancelled";
        case TPCF_ENOTFOUND: return "unknown job";
        case TPCF_ESTATE: return "invalid state";
        default: return "unknown status";
    }
}

extern "C" const char* tpcf_last_error(const tpcf_ctx* ctx) {
    return ctx ? ctx->last_error.c_str() : "";
}

extern "C" void tpcf_config_default(tpcf_config* cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof *cfg);
    cfg->precision = TPCF_SCREEN_RECHECK;
    cfg->guard_band = kDefaultGuard;
    cfg->wait_timeout_us = kDefaultWaitUs;
}

extern "C" int tpcf_version(void) { return 100; }

extern "C" uint64_t tpcf_kernel_launches(const tpcf_ctx* ctx) { return ctx ? ctx->launches.load() : 0; }

// Test hook: make the n-th following device allocation fail (n = -1: never).
extern "C" void tpcf_debug_fail_alloc_after(int n) { g_alloc_fail_countdown.store(n); }

// ====================================================================== context
extern "C" int tpcf_create(tpcf_ctx** out, const tpcf_config* cfg_in) {
    if (!out) return TPCF_EINVAL;
    *out = nullptr;
    tpcf_config cfg;
    tpcf_config_default(&cfg);
    if (cfg_in) cfg = *cfg_in;
    if (cfg.guard_band == 0.0) cfg.guard_band = kDefaultGuard;
    if (cfg.wait_timeout_us == 0) cfg.wait_timeout_us = kDefaultWaitUs;
    if (!(cfg.guard_band >= kMinGuard && cfg.guard_band < 0.25)) return TPCF_EINVAL;
    if (cfg.precision != TPCF_SCREEN_RECHECK && cfg.precision != TPCF_PLAIN_FP64) return TPCF_EINVAL;
    if (cfg.shard_count > 1 && cfg.shard_index >= cfg.shard_count) return TPCF_EINVAL;
    if (cfg.server_workers < 0 || cfg.server_workers > 64) return TPCF_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg.device < 0 || cfg.device >= ndev)
        return TPCF_ECUDA;
    if (cudaSetDevice(cfg.device) != cudaSuccess) return TPCF_ECUDA;
    tpcf_ctx* ctx = new tpcf_ctx();
    ctx->cfg = cfg;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, cfg.device) != cudaSuccess) { delete ctx; return TPCF_ECUDA; }
    ctx->num_sms = prop.multiProcessorCount;
    ctx->smem_optin = prop.sharedMemPerBlockOptin;
    for (auto& s : ctx->slots) {
        if (dev_malloc((void**)&s.dev, kSlotWords * 8) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess) {
            tpcf_destroy(ctx);
            return TPCF_ENOMEM;
        }
    }
    *out = ctx;
    return TPCF_OK;
}

extern "C" int tpcf_destroy(tpcf_ctx* ctx) {
    if (!ctx) return TPCF_EINVAL;
    server_shutdown(ctx);
    cudaSetDevice(ctx->cfg.device);
    for (auto& s : ctx->slots) {
        if (s.ev) cudaEventSynchronize(s.ev);
        if (s.dev) cudaFree(s.dev);
        if (s.ev) cudaEventDestroy(s.ev);
    }
    delete ctx;
    return TPCF_OK;
}

// ====================================================================== thresholds
namespace {

int64_t dkey(double d) {
    int64_t b;
    memcpy(&b, &d, 8);
    return b >= 0 ? b : -(b & INT64_MAX);
}

double dfromkey(int64_t k) {
    uint64_t b = k >= 0 ? (uint64_t)k : ((uint64_t)(-k) | 0x8000000000000000ull);
    double d;
    memcpy(&d, &b, 8);
    return d;
}


// The oracle's predicate for one pair and one edge: theta >= t with
// theta = acos(clamp(d, -1, 1)) from the host C library.
bool angle_at_least(double d, double t) {
    double c = d > 1.0 ? 1.0 : (d < -1.0 ? -1.0 : d);
    return acos(c) >= t;
}

float round_down_f32(double x) {
    float f = (float)x;
    if ((double)f > x) f = nextafterf(f, -INFINITY);
    return f;
}

float round_up_f32(double x) {
    float f = (float)x;
    if ((double)f < x) f = nextafterf(f, INFINITY);
    return f;
}

// C = the largest double d with acos(clamp(d)) >= t, found by bisection over
// the ordered doubles of [-1, 1]; then the predicate is checked on a window of
// neighbouring doubles wide enough to cover 4 ulps of t on each side.
double derive_threshold(double t, int* verified) {
    if (t <= 0.0) { *verified = 1; return INFINITY; }
    int64_t lo = dkey(-1.0), hi = dkey(1.0);  // pred(lo) true (t <= pi), pred(hi) false (t > 0)
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if (angle_at_least(dfromkey(mid), t)) lo = mid; else hi = mid;
    }
    const double C = dfromkey(lo);
    const double ulp_t = nextafter(t, INFINITY) - t;
    const double ac = fabs(C);
    const double ulp_c = ac > 0 ? nextafter(ac, INFINITY) - ac : 4.9406564584124654e-324;
    const double need = 4.0 * ulp_t * fmax(sin(t), 4.0 * ulp_t) / ulp_c;
    const int64_t kMaxWin = (int64_t)1 << 22;
    int64_t win = (int64_t)fmin(2.0 * ceil(need) + 64.0, (double)kMaxWin);
    bool ok = need * 2.0 + 64.0 <= (double)kMaxWin;
    const int64_t kmin = dkey(-1.0), kmax = dkey(1.0);
    for (int64_t k = std::max(kmin, lo - win); k <= lo && ok; ++k)
        if (!angle_at_least(dfromkey(k), t)) ok = false;
    for (int64_t k = lo + 1; k <= std::min(kmax, lo + win) && ok; ++k)
        if (angle_at_least(dfromkey(k), t)) ok = false;
    *verified = ok ? 1 : 0;
    return C;
}

// 3-D variant: S = the smallest double s >= 0 with sqrt(s) >= r (host sqrt,
// correctly rounded, hence monotone), so that a pair's r >= r_k exactly when
// its binary64 d^2 >= S_k.  Found by bisection over the ordered doubles, then
// the predicate is checked to flip once in a window of 64 doubles each side.
double derive_sq_threshold(double r, int* verified) {
    if (r <= 0.0) { *verified = 1; return 0.0; }
    const double top = 1.7976931348623157e308;
    if (!(std::sqrt(top) >= r)) { *verified = 1; return INFINITY; }  // no finite d^2 reaches r
    int64_t lo = dkey(0.0), hi = dkey(top);  // pred(lo) false (r > 0), pred(hi) true
    while (hi - lo > 1) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (std::sqrt(dfromkey(mid)) >= r) hi = mid; else lo = mid;
    }
    bool ok = true;
    for (int64_t k = std::max(dkey(0.0), hi - 64); k < hi && ok; ++k)
        if (std::sqrt(dfromkey(k)) >= r) ok = false;
    for (int64_t k = hi; k <= std::min(dkey(top), hi + 64) && ok; ++k)
        if (!(std::sqrt(dfromkey(k)) >= r)) ok = false;
    *verified = ok ? 1 : 0;
    return dfromkey(hi);
}

// 3-D edges: finite, >= 0, strictly increasing, the last > 0 and at most 1e18
// (a pair whose FP32 square overflows, |a - b| > 1.8e19, is then certainly
// beyond the range).
bool edges3_valid(const double* e, int ne) {
    if (!e || ne < 2 || ne > TPCF_MAX_EDGES) return false;
    for (int k = 0; k < ne; ++k)
        if (!(e[k] >= 0.0 && e[k] <= 1e18)) return false;
    for (int k = 1; k < ne; ++k)
        if (!(e[k] > e[k - 1])) return false;
    return e[ne - 1] > 0.0;
}

// Error bound of the 3-D screen value z = fl32(|a' - b'|^2) (a' = fl32(a)
// per coordinate; dx = fl32(a'x - b'x); z = fl(fma(dz,dz, fma(dy,dy, dx*dx))))
// against d^2 (the binary64 d^2 of the definition) for points of norm <= M,
// at d^2 ~ Z:  |a' - a| <= u |a| moves a - b by at most 2uM, so
// | |a'-b'|^2 - |a-b|^2 | <= 4uM|a-b| + 4u^2M^2; the subtractions and the three
// roundings of the non-negative sum add a relative 5u; the binary64 d^2 is
// within 9e-16 relative of |a - b|^2.
double euclid_delta(double Z, double M) {
    const double u = kUnit, s = std::sqrt(Z * (1.0 + 1e-15)) * (1.0 + 1e-15);
    const double t = s + 2.01 * u * M;
    return (4.001 * u * M * s + 4.01 * u * u * M * M + 5.01 * u * t * t + 9e-16 * Z) * (1.0 + 1e-9);
}

bool edges_valid(const double* e, int ne) {
    if (!e || ne < 2 || ne > TPCF_MAX_EDGES) return false;
    for (int k = 0; k < ne; ++k)
        if (!(e[k] >= 0.0 && e[k] <= 3.141592653589793)) return false;
    for (int k = 1; k < ne; ++k)
        if (!(e[k] > e[k - 1])) return false;
    return true;
}

void derive_all(const double* edges, int ne, double g, std::vector<double>& C,
                std::vector<float>& lo, std::vector<float>& hi, std::vector<float>& c32,
                std::vector<int>& ver) {
    C.resize(ne); lo.resize(ne); hi.resize(ne); c32.resize(ne); ver.resize(ne);
    for (int k = 0; k < ne; ++k) {
        C[k] = derive_threshold(edges[k], &ver[k]);
        if (isinf(C[k])) {
            lo[k] = hi[k] = c32[k] = INFINITY;
        } else {
            lo[k] = round_down_f32(C[k] - g);
            hi[k] = round_up_f32(C[k] + g);
            c32[k] = (float)C[k];
        }
    }
}

// The counting kernel classifies a pair by its screen value
//   e = fma(az,bz, fma(ay,by, fma(ax,bx, -T))),  T = RD(C_B - 10u),
// whose distance from d - T (d the binary64 dot) is at most 8.0003u.  With
// D_k = C_k - T, the e-space bounds elo_k = RD(D_k - g), ehi_k = RU(D_k + g),
// g >= 9u, decide every edge outside [elo_k, ehi_k]: e < elo_k => d <= C_k,
// e > ehi_k => d > C_k.  ec_k = RN(D_k) gives the FP32-only statistic.
void derive_e_space(const std::vector<double>& C, float T, double g, std::vector<float>& elo,
                    std::vector<float>& ehi, std::vector<float>& ec) {
    const int ne = (int)C.size();
    elo.resize(ne); ehi.resize(ne); ec.resize(ne);
    for (int k = 0; k < ne; ++k) {
        if (isinf(C[k])) {
            elo[k] = ehi[k] = ec[k] = INFINITY;
        } else {
            const double D = C[k] - (double)T;
            elo[k] = round_down_f32(D - g);
            ehi[k] = round_up_f32(D + g);
            ec[k] = (float)D;
        }
    }
}

// Chord-space bounds for the refinement of unsettled pairs.  The kernel
// computes z = fl32(|a' - b'|^2) from the FP32 copies a', b' (differences,
// then fl(fma(dz,dz, fma(dy,dy, dx*dx)))).  With Z = 2 (1 - d) (d the binary64
// dot product) and | |v|^2 - 1 | <= eps for every point:
//   |z - Z| <= delta(Z) = 4u(1 + 1e-6) s + (5u + 10u^2)(s + 2.01u)^2 + 4.1u^2
//                         + 2 eps + 6.7e-16,   s = sqrt(Z + 2 eps + 7e-16):
// input rounding moves a - b by at most 2u(1 + eps) (so |a-b|^2 by 4u|a-b| +
// 4u^2), the subtractions and the three roundings of the non-negative sum
// give a relative 5u, |a - b|^2 = Z + eps_a + eps_b - 2 (D - d), and the
// binary64 dot d is within 3.4e-16 of the exact D.  Edge k is crossed
// (theta >= t_k) iff Z >= Z_k = 2 (1 - C_k); with g_k >= delta(Z_k),
// z >= zhi_k = RU(Z_k + g_k) proves Z >= Z_k (else z <= Z + delta(Z) <
// Z_k + g_k), and z < zlo_k = RD(Z_k - g_k) proves Z < Z_k (Z - delta(Z) is
// increasing for Z >= 1e-12; smaller Z_k get no lower bound).
// LUT over a squared separation z >= 0 with cells of constant ratio: the cell
// of z is clamp((bits(z) - b0) >> shift, 0, kLutCells - 1), b0 = bits of
// RD(zmin), shift the smallest with every z up to ztop inside the cells.  Cell
// c covers [cmin, cmax] (cell 0 also every smaller z, the last every larger)
// and stores P = #{m : cmin >= zhi_m} (edges every z of the cell crosses) and
// Q = #{m : cmax >= zlo_m} (edges some z may cross); P == Q settles the cell.
void build_zlut(const std::vector<float>& zlo, const std::vector<float>& zhi, double zmin_d, double ztop_d,
                int32_t* b0_out, int* shift_out, std::vector<uint32_t>& lut) {
    const int ne = (int)zlo.size();
    const float zmin = round_down_f32(zmin_d);
    int32_t b0;
    memcpy(&b0, &zmin, 4);
    const float ztop = round_up_f32(ztop_d);
    int32_t bt;
    memcpy(&bt, &ztop, 4);
    int shift = 0;
    while (((int64_t)(bt - b0) >> shift) + 1 >= kLutCells - 1) ++shift;
    lut.assign(kLutCells, 0);
    for (int c = 0; c < kLutCells; ++c) {
        const int64_t lo_bits = (int64_t)b0 + ((int64_t)c << shift);
        const int64_t hi_bits = (int64_t)b0 + ((int64_t)(c + 1) << shift) - 1;
        float cmin, cmax;
        const int32_t lb = (int32_t)std::min<int64_t>(lo_bits, 0x7f7fffff);
        const int32_t hb = (int32_t)std::min<int64_t>(hi_bits, 0x7f7fffff);
        memcpy(&cmin, &lb, 4);
        memcpy(&cmax, &hb, 4);
        if (c == 0) cmin = 0.0f;                   // also every z below zmin
        if (c == kLutCells - 1) cmax = INFINITY;   // and every z above
        uint32_t P = 0, Q = 0;
        for (int m = 0; m < ne; ++m) {
            P += (cmin >= zhi[m]);
            Q += (cmax >= zlo[m]);
        }
        lut[c] = P | (Q << 16);
    }
    *b0_out = b0;
    *shift_out = shift;
}

void derive_chord_space(const std::vector<double>& C, std::vector<float>& zlo, std::vector<float>& zhi) {
    const int ne = (int)C.size();
    const double u = kUnit, eps = kChordEpsRef;
    zlo.resize(ne); zhi.resize(ne);
    auto delta = [&](double Z) {
        const double sq = std::sqrt(Z + 2.0 * eps + 7e-16) * (1.0 + 1e-15);
        const double t = sq + 2.01 * u;
        return 4.0 * u * (1.0 + 1e-6) * sq + (5.0 * u + 10.0 * u * u) * t * t + 4.1 * u * u + 2.0 * eps + 6.7e-16;
    };
    for (int k = 0; k < ne; ++k) {
        if (std::isinf(C[k])) {  // t_k = 0: every pair crosses it
            zlo[k] = zhi[k] = -INFINITY;
            continue;
        }
        double Zd = 2.0 * (1.0 - C[k]), Zu = Zd;
        if (C[k] < 0.5) {  // 1 - C may round (it is exact by Sterbenz's lemma for C >= 1/2)
            Zd = std::nextafter(Zd, -INFINITY);
            Zu = std::nextafter(Zu, INFINITY);
        }
        const double g = delta(Zu) * (1.0 + 1e-9);
        zhi[k] = round_up_f32(Zu + g);
        zlo[k] = Zd < 1e-12 ? -1.0f : round_down_f32(Zd - g);
    }
}

// Exponent q of the LUT span: the smallest q with 2^q >= e_top, where e_top
// bounds every screen value: |d| <= (1 + 1e-6)^2 for validated points, plus
// the screen error and the offset margin.
int lut_span_exponent(double e_top) {
    int q = -30;
    while (std::ldexp(1.0, q) < e_top) ++q;
    return q;
}

// LUT over the screen value e.  The kernel computes
//   k = rne(sat(e * 2^-q) * 2^14)       (exact scaling by powers of two)
// so cell k holds every e in [(k - 1/2) w, (k + 1/2) w] with w = 2^(q - 14),
// cell 0 also every e <= 0 (saturation; also NaN) and the last cell every
// e >= 2^q.  Entry k stores P = #{m : e_max < elo_m} (edges certainly
// crossed by every e of the cell) and Q = #{m : e_min <= ehi_m} (edges
// possibly crossed); P == Q settles the histogram index of the whole cell.
void build_lut(const std::vector<float>& elo, const std::vector<float>& ehi, int q, std::vector<uint32_t>& lut) {
    const int ne = (int)elo.size();
    const double w = std::ldexp(1.0, q - kLutBits);
    lut.assign(kLutCells, 0);
    for (int k = 0; k < kLutCells; ++k) {
        const double e_min = k == 0 ? -INFINITY : (k - 0.5) * w;
        const double e_max = k == kLutCells - 1 ? INFINITY : (k + 0.5) * w;
        uint32_t P = 0, Q = 0;
        for (int m = 0; m < ne; ++m) {
            P += (e_max < (double)elo[m]);
            Q += (e_min <= (double)ehi[m]);
        }
        lut[k] = P | (Q << 16);
    }
}

}  // namespace

// Binary64 thresholds C_k for nedges valid edges into a caller array; no
// allocation (used by the no-allocation entry point).
bool tpcf::derive_cos_thresholds(const double* edges, int nedges, double* cos_thr) {
    if (!edges_valid(edges, nedges)) return false;
    for (int k = 0; k < nedges; ++k) {
        int ver;
        cos_thr[k] = derive_threshold(edges[k], &ver);
    }
    return true;
}

extern "C" int tpcf_bins_thresholds(const double* edges, int nedges, double guard, double* cos_thr,
                                    float* lo, float* hi, int* verified) {
    if (!edges_valid(edges, nedges)) return TPCF_EINVAL;
    if (guard == 0.0) guard = kDefaultGuard;
    if (!(guard >= kMinGuard && guard < 0.25)) return TPCF_EINVAL;
    std::vector<double> C;
    std::vector<float> l, h, c;
    std::vector<int> v;
    derive_all(edges, nedges, guard, C, l, h, c, v);
    for (int k = 0; k < nedges; ++k) {
        if (cos_thr) cos_thr[k] = C[k];
        if (lo) lo[k] = l[k];
        if (hi) hi[k] = h[k];
        if (verified) verified[k] = v[k];
    }
    return TPCF_OK;
}

int tpcf::bins_create_impl(tpcf_ctx* ctx, const double* edges, int nedges, cudaStream_t st,
                           bool stream_ordered, tpcf_bins** out) {
    if (!ctx || !out) return TPCF_EINVAL;
    *out = nullptr;
    if (!edges_valid(edges, nedges))
        return ctx->fail(TPCF_EINVAL, "edges: need 2..%d strictly increasing values in [0, pi]",
                         TPCF_MAX_EDGES);
    cudaSetDevice(ctx->cfg.device);
    tpcf_bins* b = new tpcf_bins();
    b->ctx = ctx;
    b->nedges = nedges;
    b->stream_ordered = stream_ordered;
    b->free_stream = st;
    b->edges.assign(edges, edges + nedges);
    derive_all(edges, nedges, ctx->cfg.guard_band, b->cos_thr, b->lo, b->hi, b->c32, b->verified);
    // Screen offset T: the fast test fma(az,bz, fma(ay,by, fma(ax,bx, -T))) has
    // error <= 8.0003u + 3u (|T| - 1)+ against d - T (2u input rounding, three
    // roundings of terms bounded by |T| + 1), below the guard band g >= 9u, so
    // a negative value means d < T + g <= C_B.  T = RD(C_B - g - u - w) sits
    // one LUT cell w below that bound so that LUT cell 0, which also receives
    // every e < 0, lies wholly beyond the last edge (e_max of cell 0 = w / 2 <
    // w <= elo_B = RD(C_B - T - g)) and settles as overflow.
    const double C_B = b->cos_thr[nedges - 1];
    const double g = ctx->cfg.guard_band;
    int q = lut_span_exponent(1.0 + 3e-6 - C_B + g + 2.0 * kUnit);
    float T = 0.f;
    for (;; ++q) {
        T = round_down_f32(C_B - g - kUnit - std::ldexp(1.0, q - kLutBits));
        if (std::ldexp(1.0, q) >= 1.0 + 3e-6 + 12.0 * kUnit - (double)T) break;
    }
    derive_e_space(b->cos_thr, T, ctx->cfg.guard_band, b->elo, b->ehi, b->ec);
    build_lut(b->elo, b->ehi, q, b->lut);
    derive_chord_space(b->cos_thr, b->zlo, b->zhi);
    // one device buffer: C (double), lo, hi, c32, zlo, zhi (float), lut (uint32), then the descriptor
    const size_t nd = (size_t)nedges * 8, nf = (size_t)nedges * 4, nl = b->lut.size() * 4;
    const size_t nf16 = (nf + 15) / 16 * 16;
    const size_t off_lo = (nd + 15) / 16 * 16, off_hi = off_lo + nf16, off_c32 = off_hi + nf16,
                 off_zlo = off_c32 + nf16, off_zhi = off_zlo + nf16, off_lut = off_zhi + nf16,
                 off_desc = (off_lut + nl + 255) / 256 * 256, total = off_desc + sizeof(BinsDev);
    auto cleanup = [&](int code) {
        bins_destroy_impl(b);
        return ctx->fail(code, "bins: device allocation or copy failed");
    };
    if ((stream_ordered ? dev_malloc_async(&b->dev_buf, total, st) : dev_malloc(&b->dev_buf, total)) != cudaSuccess)
        return cleanup(TPCF_ENOMEM);
    unsigned char* base = (unsigned char*)b->dev_buf;
    b->host.cos_thr = (const double*)base;
    b->host.lo = (const float*)(base + off_lo);
    b->host.hi = (const float*)(base + off_hi);
    b->host.cos32 = (const float*)(base + off_c32);
    b->host.lut = (const uint32_t*)(base + off_lut);
    b->host.zlo = (const float*)(base + off_zlo);
    b->host.zhi = (const float*)(base + off_zhi);
    b->host.nedges = nedges;
    b->host.lut_scale = (float)std::ldexp(1.0, -q);
    b->host.fast_t = T;
    b->host.cos_last = b->cos_thr[nedges - 1];
    b->dev_desc = (BinsDev*)(base + off_desc);
    b->staging.assign(total, 0);
    unsigned char* hs = b->staging.data();
    memcpy(hs, b->cos_thr.data(), nd);
    memcpy(hs + off_lo, b->elo.data(), nf);
    memcpy(hs + off_hi, b->ehi.data(), nf);
    memcpy(hs + off_c32, b->ec.data(), nf);
    memcpy(hs + off_zlo, b->zlo.data(), nf);
    memcpy(hs + off_zhi, b->zhi.data(), nf);
    memcpy(hs + off_lut, b->lut.data(), nl);
    memcpy(hs + off_desc, &b->host, sizeof(BinsDev));
    const cudaError_t e = stream_ordered
                              ? cudaMemcpyAsync(b->dev_buf, hs, total, cudaMemcpyHostToDevice, st)
                              : cudaMemcpy(b->dev_buf, hs, total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cleanup(TPCF_ECUDA);
    *out = b;
    return TPCF_OK;
}

int tpcf::bins_destroy_impl(tpcf_bins* b) {
    if (!b) return TPCF_EINVAL;
    cudaSetDevice(b->ctx->cfg.device);
    if (!b->sets.empty()) {
        cudaDeviceSynchronize();
        for (auto& kv : b->sets) cudaFree(kv.second.dev_buf);
    }
    if (b->dev_buf) {
        if (b->stream_ordered) {
            cudaFreeAsync(b->dev_buf, b->free_stream);
            cudaStreamSynchronize(b->free_stream);  // the staging image may back a pending copy
        } else {
            cudaDeviceSynchronize();
            cudaFree(b->dev_buf);
        }
    }
    delete b;
    return TPCF_OK;
}

// ---------------------------------------------------------------------- 3-D bins
// The device arrays of a 3-D bin set for points of norm <= M = 2^key: S_k, the
// z-space bounds zlo/zhi (z >= zhi_k proves d^2 >= S_k, z < zlo_k proves
// d^2 < S_k, both with g_k = euclid_delta(S_k)), the fast-test limit H (every
// pair with d^2 <= S_B has H - z' >= 0 for the fast loop's fl32 value z'),
// and a LUT over z cells uniform in the float bits of z (constant ratio).
static int euclid_set(tpcf_ctx* ctx, tpcf_bins* b, int key, const tpcf::BinsDev** host, tpcf::BinsDev** dev) {
    std::lock_guard<std::mutex> g(b->set_mu);
    auto it = b->sets.find(key);
    if (it == b->sets.end()) {
        const int ne = b->nedges;
        const double M = std::ldexp(1.0, key), u = kUnit;
        std::vector<float> zlo(ne), zhi(ne), s32(ne), zero(ne, 0.f);
        double min_pos = INFINITY;
        for (int k = 0; k < ne; ++k) {
            const double S = b->cos_thr[k];
            if (S == 0.0) {  // r_k = 0: every pair crosses it
                zlo[k] = zhi[k] = -INFINITY;
            } else if (std::isinf(S)) {
                zlo[k] = zhi[k] = INFINITY;
            } else {
                const double gk = euclid_delta(S, M);
                // past the FP32 range there is no upper bound: NaN makes z >= zhi
                // false for every z (an overflowed z = +inf proves nothing; the
                // pair goes to binary64)
                zhi[k] = S + gk <= 3.4028234663852886e38 ? round_up_f32(S + gk) : NAN;
                // z - delta(z) increases only once |a - b| is well above 2uM
                zlo[k] = S < 1e6 * (u * M) * (u * M) ? -1.0f : round_down_f32(S - gk);
                min_pos = std::min(min_pos, S);
            }
            s32[k] = (float)S;
        }
        const double SB = b->cos_thr[ne - 1];
        const double zmax = std::pow(std::sqrt(SB * (1.0 + 1e-15)) + 2.001 * u * M, 2) * (1.0 + 2.01 * u);
        // (at least 2^-100: then an in-range pair's fast-test value H - z', which
        // exceeds 3u H, is a positive normal float, never zero)
        const float H = round_up_f32(std::max(zmax * (1.0 + 6.1 * u) + 1e-300, 0x1p-100));
        // LUT: cells of constant ratio from zmin = min S / 64 up past 2 H
        int32_t b0;
        int shift;
        std::vector<uint32_t> lut;
        build_zlut(zlo, zhi, std::max(min_pos / 64.0, 1e-30), 2.0 * (double)H + 1e-30, &b0, &shift, lut);
        // one device buffer with the angular layout (lo/hi unused), then the descriptor
        const size_t nd = (size_t)ne * 8, nf = (size_t)ne * 4, nl = lut.size() * 4, nf16 = (nf + 15) / 16 * 16;
        const size_t off_lo = (nd + 15) / 16 * 16, off_hi = off_lo + nf16, off_c32 = off_hi + nf16,
                     off_zlo = off_c32 + nf16, off_zhi = off_zlo + nf16, off_lut = off_zhi + nf16,
                     off_desc = (off_lut + nl + 255) / 256 * 256, total = off_desc + sizeof(BinsDev);
        tpcf_bins::Set set;
        if (dev_malloc(&set.dev_buf, total) != cudaSuccess) return ctx->fail(TPCF_ENOMEM, "bins: allocation failed");
        unsigned char* base = (unsigned char*)set.dev_buf;
        memset(&set.host, 0, sizeof set.host);
        set.host.cos_thr = (const double*)base;
        set.host.lo = (const float*)(base + off_lo);
        set.host.hi = (const float*)(base + off_hi);
        set.host.cos32 = (const float*)(base + off_c32);
        set.host.zlo = (const float*)(base + off_zlo);
        set.host.zhi = (const float*)(base + off_zhi);
        set.host.lut = (const uint32_t*)(base + off_lut);
        set.host.nedges = ne;
        set.host.lut_scale = 0.f;
        set.host.fast_t = H;
        set.host.cos_last = SB;
        set.host.euclid = 1;
        set.host.zbits0 = b0;
        set.host.zshift = shift;
        set.dev_desc = (BinsDev*)(base + off_desc);
        std::vector<unsigned char> hs(total, 0);
        memcpy(hs.data(), b->cos_thr.data(), nd);
        memcpy(hs.data() + off_lo, zero.data(), nf);
        memcpy(hs.data() + off_hi, zero.data(), nf);
        memcpy(hs.data() + off_c32, s32.data(), nf);
        memcpy(hs.data() + off_zlo, zlo.data(), nf);
        memcpy(hs.data() + off_zhi, zhi.data(), nf);
        memcpy(hs.data() + off_lut, lut.data(), nl);
        memcpy(hs.data() + off_desc, &set.host, sizeof(BinsDev));
        if (cudaMemcpy(set.dev_buf, hs.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(set.dev_buf);
            return ctx->fail(TPCF_ECUDA, "bins: upload failed");
        }
        it = b->sets.emplace(key, set).first;
    }
    *host = &it->second.host;
    *dev = it->second.dev_desc;
    return TPCF_OK;
}

extern "C" int tpcf_bins_create_3d(tpcf_ctx* ctx, const double* edges, int nedges, tpcf_bins** out) {
    if (!ctx || !out) return TPCF_EINVAL;
    *out = nullptr;
    if (!edges3_valid(edges, nedges))
        return ctx->fail(TPCF_EINVAL, "edges: need 2..%d strictly increasing finite distances >= 0, the last > 0",
                         TPCF_MAX_EDGES);
    tpcf_bins* b = new tpcf_bins();
    b->ctx = ctx;
    b->nedges = nedges;
    b->euclid = true;
    b->edges.assign(edges, edges + nedges);
    b->cos_thr.resize(nedges);
    b->verified.resize(nedges);
    for (int k = 0; k < nedges; ++k) b->cos_thr[k] = derive_sq_threshold(edges[k], &b->verified[k]);
    *out = b;
    return TPCF_OK;
}

extern "C" int tpcf_bins_thresholds_3d(const double* edges, int nedges, double* sq_thr, int* verified) {
    if (!edges3_valid(edges, nedges)) return TPCF_EINVAL;
    for (int k = 0; k < nedges; ++k) {
        int v;
        const double S = derive_sq_threshold(edges[k], &v);
        if (sq_thr) sq_thr[k] = S;
        if (verified) verified[k] = v;
    }
    return TPCF_OK;
}

extern "C" int tpcf_bins_create(tpcf_ctx* ctx, const double* edges, int nedges, tpcf_bins** out) {
    return bins_create_impl(ctx, edges, nedges, nullptr, false, out);
}

extern "C" int tpcf_bins_destroy(tpcf_bins* b) { return bins_destroy_impl(b); }

// ====================================================================== catalogs
size_t tpcf::catalog_bytes(uint64_t n) {
    const uint64_t n_pad = ((n + kPad - 1) / kPad + 1) * kPad;
    return (size_t)n_pad * (sizeof(Point64) + sizeof(float4) + 3 * sizeof(float));
}

int tpcf::catalog_create_impl(tpcf_ctx* ctx, const double* xyz, uint64_t n, int where, const uint64_t* offsets,
                              int nseg, cudaStream_t st, bool stream_ordered, tpcf_catalog** out, bool euclid) {
    if (!ctx || !out) return TPCF_EINVAL;
    *out = nullptr;
    if (n > TPCF_MAX_POINTS) return ctx->fail(TPCF_EOVERFLOW, "catalog: %llu points > limit",
                                              (unsigned long long)n);
    if (n > 0 && !xyz) return ctx->fail(TPCF_EINVAL, "catalog: NULL coordinates");
    if (where != TPCF_HOST && where != TPCF_DEVICE) return ctx->fail(TPCF_EINVAL, "catalog: bad where");
    if (nseg < 0 || (nseg > 0 && !offsets)) return ctx->fail(TPCF_EINVAL, "catalog: bad segments");
    if (nseg > 0) {
        if (offsets[0] != 0 || offsets[nseg] != n)
            return ctx->fail(TPCF_EINVAL, "catalog: offsets must start at 0 and end at n");
        for (int s = 0; s < nseg; ++s)
            if (offsets[s + 1] < offsets[s]) return ctx->fail(TPCF_EINVAL, "catalog: offsets decrease");
        if (nseg > 65535) return ctx->fail(TPCF_EOVERFLOW, "catalog: too many segments");
    }
    cudaSetDevice(ctx->cfg.device);
    tpcf_catalog* c = new tpcf_catalog();
    c->ctx = ctx;
    c->n = n;
    c->euclid = euclid;
    c->stream_ordered = stream_ordered;
    c->free_stream = st;
    uint64_t n_layout = n;  // device positions in use (segments are aligned: gaps of zero vectors)
    if (nseg > 0) {
        c->offsets.assign(offsets, offsets + nseg + 1);
        c->seg_start.assign(nseg + 1, 0);
        for (int s = 0; s < nseg; ++s)
            c->seg_start[s + 1] = (c->seg_start[s] + (offsets[s + 1] - offsets[s]) + kSegAlign - 1) / kSegAlign * kSegAlign;
        n_layout = c->seg_start[nseg];
        if (n_layout > TPCF_MAX_POINTS) {
            catalog_destroy_impl(c);
            return ctx->fail(TPCF_EOVERFLOW, "catalog: aligned segments exceed the point limit");
        }
    }
    c->n_pad = (uint32_t)(((n_layout + kPad - 1) / kPad) * kPad);
    if (c->n_pad == 0) c->n_pad = kPad;
    // a segment's tiles and i-blocks may run up to one block past its last point
    if (nseg > 0) c->n_pad += kPad;
    const bool sort = !(ctx->cfg.flags & TPCF_F_NO_SORT);
    uint32_t n_pow2 = 2048;
    while (n_pow2 < n) n_pow2 <<= 1;

    void* tmp_in = nullptr;
    unsigned long long* keys = nullptr;
    uint32_t* vals = nullptr;
    uint32_t* seg = nullptr;
    uint32_t* seg_delta = nullptr;
    unsigned long long* err = nullptr;
    int rc = TPCF_OK;
    auto release = [&]() {
        if (tmp_in) cudaFreeAsync(tmp_in, st);
        if (keys) cudaFreeAsync(keys, st);
        if (vals) cudaFreeAsync(vals, st);
        if (seg) cudaFreeAsync(seg, st);
        if (seg_delta) cudaFreeAsync(seg_delta, st);
        if (err) cudaFreeAsync(err, st);
        cudaStreamSynchronize(st);
    };
    auto fail_with = [&](int code, const char* what) {
        release();
        catalog_destroy_impl(c);
        return ctx->fail(code, "catalog: %s", what);
    };
    auto alloc = [&](void** p, size_t bytes) {
        return stream_ordered ? dev_malloc_async(p, bytes, st) : dev_malloc(p, bytes);
    };
    if (alloc((void**)&c->d64, (size_t)c->n_pad * sizeof(Point64)) != cudaSuccess ||
        alloc((void**)&c->d32, (size_t)c->n_pad * sizeof(float4)) != cudaSuccess ||
        alloc((void**)&c->soa, (size_t)c->n_pad * 3 * sizeof(float)) != cudaSuccess ||
        alloc((void**)&c->caps, (size_t)(c->n_pad / kCapPoints) * sizeof(float4)) != cudaSuccess)
        return fail_with(TPCF_ENOMEM, "device allocation failed");
    const double* in = xyz;
    if (n > 0 && where == TPCF_HOST) {
        if (cudaMallocAsync(&tmp_in, n * 24, st) != cudaSuccess)
            return fail_with(TPCF_ENOMEM, "staging allocation failed");
        if (cudaMemcpyAsync(tmp_in, xyz, n * 24, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return fail_with(TPCF_ECUDA, "host-to-device copy failed");
        in = (const double*)tmp_in;
    }
    // err: error word, largest |v|^2 or | |v|^2 - 1 |, then the bounding box (3 min, 3 max keys)
    if (cudaMallocAsync((void**)&err, 64, st) != cudaSuccess ||
        cudaMallocAsync((void**)&keys, (size_t)n_pow2 * 8, st) != cudaSuccess ||
        cudaMallocAsync((void**)&vals, (size_t)n_pow2 * 4, st) != cudaSuccess)
        return fail_with(TPCF_ENOMEM, "scratch allocation failed");
    if (cudaMemsetAsync(err, 0, 64, st) != cudaSuccess || cudaMemsetAsync(err + 2, 0xff, 24, st) != cudaSuccess)
        return fail_with(TPCF_ECUDA, "memset failed");
    if (nseg > 0) {
        // segment of each input point, shift of each segment to its aligned start, and the
        // segment of each kSegAlign-point block of the device layout (blocks past the last
        // segment: the last segment; they hold only zero vectors)
        std::vector<uint32_t> hs(n), hd(nseg);
        for (int s = 0; s < nseg; ++s) {
            hd[s] = (uint32_t)(c->seg_start[s] - offsets[s]);
            for (uint64_t i = offsets[s]; i < offsets[s + 1]; ++i) hs[i] = (uint32_t)s;
        }
        const uint32_t nblk = c->n_pad / kSegAlign;
        std::vector<uint32_t> hb(nblk, (uint32_t)(nseg - 1));
        for (int s = 0; s < nseg; ++s)
            for (uint64_t b = c->seg_start[s] / kSegAlign; b < c->seg_start[s + 1] / kSegAlign; ++b) hb[b] = (uint32_t)s;
        if (alloc((void**)&c->seg_of_block, (size_t)nblk * 4) != cudaSuccess ||
            cudaMallocAsync((void**)&seg_delta, (size_t)nseg * 4, st) != cudaSuccess ||
            (n > 0 && cudaMallocAsync((void**)&seg, n * 4, st) != cudaSuccess))
            return fail_with(TPCF_ENOMEM, "segment allocation failed");
        if ((n > 0 && cudaMemcpyAsync(seg, hs.data(), n * 4, cudaMemcpyHostToDevice, st) != cudaSuccess) ||
            cudaMemcpyAsync(seg_delta, hd.data(), (size_t)nseg * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(c->seg_of_block, hb.data(), (size_t)nblk * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return fail_with(TPCF_ECUDA, "segment copy failed");
    }
    uint32_t nl = 0;
    cudaError_t e = launch_prepare(in, (uint32_t)n, seg, seg_delta, sort ? 1 : 0, euclid ? 1 : 0, err + 2, c->d64,
                                   c->d32, c->soa, c->caps, c->n_pad, keys, vals, n_pow2, err, err + 1, st, &nl);
    ctx->launches.fetch_add(nl);
    if (e != cudaSuccess) return fail_with(TPCF_ECUDA, cudaGetErrorString(e));
    unsigned long long hw[2] = {0, 0};
    if (cudaMemcpyAsync(hw, err, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail_with(TPCF_ECUDA, "preparation failed");
    const unsigned long long herr = hw[0];
    double word;
    memcpy(&word, &hw[1], 8);
    if (euclid) {
        c->eps_max = INFINITY;  // not unit vectors: no chord refinement of angular counts
        c->norm_max = std::sqrt(word * (1.0 + 1e-15)) * (1.0 + 1e-15);  // the device |v|^2 is within 3.4e-16 relative
    } else {
        c->eps_max = word + 4e-16;  // the device sum of squares is within 3.4e-16 of |v|^2
        c->norm_max = 1.0 + 1e-6;
    }
    if (herr & kErrBadPoint) {
        rc = TPCF_EINVAL;
        return fail_with(rc, euclid ? "a point is not finite"
                                    : "a point is not finite or not a unit vector (| |v| - 1 | > 1e-6)");
    }
    release();
    *out = c;
    return TPCF_OK;
}

extern "C" int tpcf_catalog_create_segmented(tpcf_ctx* ctx, const double* xyz, uint64_t n, int where,
                                             const uint64_t* offsets, int nseg, void* stream,
                                             tpcf_catalog** out) {
    return catalog_create_impl(ctx, xyz, n, where, offsets, nseg, (cudaStream_t)stream, false, out);
}

extern "C" int tpcf_catalog_create(tpcf_ctx* ctx, const double* xyz, uint64_t n, int where,
                                   void* stream, tpcf_catalog** out) {
    return catalog_create_impl(ctx, xyz, n, where, nullptr, 0, (cudaStream_t)stream, false, out);
}

extern "C" int tpcf_catalog_create_3d(tpcf_ctx* ctx, const double* xyz, uint64_t n, int where,
                                      const uint64_t* offsets, int nseg, void* stream, tpcf_catalog** out) {
    return catalog_create_impl(ctx, xyz, n, where, offsets, nseg, (cudaStream_t)stream, false, out, true);
}

int tpcf::catalog_destroy_impl(tpcf_catalog* c) {
    if (!c) return TPCF_EINVAL;
    cudaSetDevice(c->ctx->cfg.device);
    void* bufs[5] = {c->d64, c->d32, c->soa, c->seg_of_block, c->caps};
    if (c->stream_ordered) {
        for (void* p : bufs)
            if (p) cudaFreeAsync(p, c->free_stream);
    } else {
        cudaDeviceSynchronize();
        for (void* p : bufs)
            if (p) cudaFree(p);
    }
    delete c;
    return TPCF_OK;
}

extern "C" int tpcf_catalog_destroy(tpcf_catalog* c) { return catalog_destroy_impl(c); }

extern "C" uint64_t tpcf_catalog_size(const tpcf_catalog* c) { return c ? c->n : 0; }

// ====================================================================== shapes
namespace {

struct SubSpec {
    const tpcf_catalog* a;
    const tpcf_catalog* b;
    bool auto_mode;
    uint32_t na, nb;        // counts (segments: sub-ranges)
    uint32_t a_off, b_off;  // first point of the range in the catalog
    int nhist = 1;                      // histograms filled (row attribution: one per segment of A)
    const uint32_t* row_seg = nullptr;  // device segment table of A's kSegAlign blocks (row attribution)
    bool no_self = false;               // A == B over the full square except i == j
    const uint64_t* totals = nullptr;   // pair total of each histogram (nhist entries); NULL: all pairs
};

int kernel_mode(const tpcf_config& cfg, bool euclid) {
    if (cfg.precision == TPCF_PLAIN_FP64) return kModePlainFP64;
    return euclid ? kModeEuclidScreen : kModeScreenScalar;
}

// Shape for T threads x R i-points, j-tile J (0: default) and S stages per
// warp (0: default); false when it does not fit shared memory.  Every warp
// works on items of its own 32 R i-points x Jc = 4096 j-points, streamed in
// tiles of J j-points through a ring of S stages.
bool shape_for(tpcf_ctx* ctx, int mode, int nedges, int T, int R, int Jreq, int Sreq, Shape* sh) {
    if (!count_shape_supported(T, R)) return false;
    const int I = 32 * R;
    constexpr int kChunk = 4096;
    // two stages of 256 j-points by default (a warp's tile of 256 x 256 pairs takes
    // tens of microseconds, its copy from L2 about one: double buffering hides it);
    // the all-binary64 kernel stages 32-byte points in tiles of 128
    int J = Jreq ? Jreq : (mode == kModePlainFP64 ? 128 : 256);
    // (a tile is a whole number of the fast loop's mask chunks and of 128-point pruning groups)
    if ((int)kPad % J != 0 || J % 128 != 0 || kChunk % J != 0 || kChunk % I != 0) return false;
    int S = Sreq ? Sreq : 2;
    if (S < 2 || S > 16) return false;
    size_t smem = count_smem_bytes(mode, T, R, J, S, nedges);
    while (smem > ctx->smem_optin && J > 128 && Jreq == 0) {
        J /= 2;
        smem = count_smem_bytes(mode, T, R, J, S, nedges);
    }
    if (smem > ctx->smem_optin) return false;
    sh->threads = T;
    sh->ipt = R;
    sh->jtile = J;
    sh->stages = S;
    sh->smem = smem;
    sh->blocks = ctx->num_sms;  // one persistent block per SM
    sh->jchunk = kChunk;
    return true;
}

// Default shape: 512 x 8 for large problems, smaller i-blocks when the
// catalogs (or sub-ranges) are small or the per-thread histograms do not fit.
bool choose_shape(tpcf_ctx* ctx, int mode, int nedges, uint64_t total_pairs, uint64_t max_n, Shape* sh) {
    const tpcf_config& cfg = ctx->cfg;
    if (cfg.threads != 0 && cfg.ipt != 0)
        return shape_for(ctx, mode, nedges, cfg.threads, cfg.ipt, cfg.jtile, cfg.stages, sh);
    const double per_sm = (double)total_pairs / std::max(1, ctx->num_sms);
    if (per_sm >= 4e7 && max_n >= 8192) {
        if (shape_for(ctx, mode, nedges, 512, 8, cfg.jtile, cfg.stages, sh)) return true;
        if (shape_for(ctx, mode, nedges, 256, 8, cfg.jtile, cfg.stages, sh)) return true;
    }
    return shape_for(ctx, mode, nedges, 128, 8, cfg.jtile, cfg.stages, sh);
}

uint64_t full_pairs(const SubSpec& s) {
    if (s.auto_mode) return (uint64_t)s.na * (s.na ? s.na - 1 : 0) / 2;
    return (uint64_t)s.na * s.nb - (s.no_self ? (uint64_t)std::min(s.na, s.nb) : 0);
}

// Pairs of sub-problem `sp` inside the global item range [lo, hi).
uint64_t range_pairs(const SubProblem& sp, uint64_t lo, uint64_t hi, uint32_t I, uint32_t Jc,
                     uint32_t J) {
    uint64_t a = std::max(lo, sp.item_begin), b = std::min(hi, sp.item_begin + sp.n_items);
    uint64_t total = 0;
    for (uint64_t q = a; q < b; ++q) {
        const uint64_t local = walk_item(q - sp.item_begin, sp.n_items, sp.walk_mult);
        ItemGeom g = item_geom(local, sp.na, sp.nb, sp.n_iblk, sp.n_jchunk, sp.auto_mode != 0, I, Jc, J);
        if (g.t_first < g.t_end) total += item_pairs(g, sp.na, sp.nb, sp.auto_mode != 0, I, Jc);
    }
    return total;
}

// Fill the kernel's work description for `nsub` sub-problems with shape sh.
// subs_out receives the sub-problem records (placed inline or uploaded by the
// caller); acc is the accumulator array (stride acc_stride words per
// histogram); returns the number of items.
uint64_t build_work(tpcf_ctx* ctx, const SubSpec* specs, int nsub, const BinsDev* bins_dev, const Shape& sh,
                    unsigned long long* acc, size_t acc_stride, std::vector<SubProblem>& subs) {
    const uint32_t I = 32u * (uint32_t)sh.ipt, Jc = (uint32_t)sh.jchunk;
    subs.assign(nsub, SubProblem());
    uint64_t items = 0;
    size_t hist_base = 0;
    for (int s = 0; s < nsub; ++s) {
        const SubSpec& p = specs[s];
        SubProblem& sp = subs[s];
        memset(&sp, 0, sizeof sp);
        sp.a32 = p.a->d32 + p.a_off;
        sp.b32 = p.b->d32 + p.b_off;
        sp.b_soa = p.b->soa + p.b_off;
        sp.b_soa_stride = p.b->n_pad;
        sp.a64 = p.a->d64 + p.a_off;
        sp.b64 = p.b->d64 + p.b_off;
        sp.a_caps = p.a->caps + p.a_off / kCapPoints;  // sub-ranges start on kSegAlign boundaries
        sp.b_caps = p.b->caps + p.b_off / kCapPoints;
        sp.na = p.na;
        sp.nb = p.nb;
        sp.n_iblk = (p.na + I - 1) / I;
        sp.n_jchunk = (p.nb + Jc - 1) / Jc;
        sp.auto_mode = p.auto_mode ? 1u : 0u;
        sp.kratio = I / Jc;
        sp.item_begin = items;
        sp.n_items = (p.na == 0 || p.nb == 0) ? 0 : items_of(sp.n_iblk, sp.n_jchunk, p.auto_mode, I, Jc);
        sp.walk_mult = walk_multiplier(sp.n_items);
        sp.hist = acc + hist_base * acc_stride;
        sp.bins = bins_dev;
        sp.row_seg = p.row_seg ? p.row_seg + p.a_off / kSegAlign : nullptr;
        sp.row_stride = (uint32_t)acc_stride;
        sp.no_self = p.no_self ? 1u : 0u;
        hist_base += (size_t)p.nhist;
        items += sp.n_items;
    }
    (void)ctx;
    return items;
}

// The launch constants of a work description: shape, flags, bin scalars, the
// chord and index rules, spatial pruning (the sub-problems, statistics words
// and item range are set by the caller).
void fill_scalars(tpcf_ctx* ctx, const SubSpec* specs, int nsub, const BinsDev* bh, int mode, const Shape& shp,
                  bool force_idx, int ne, WorkDesc& wd) {
    wd.I = 32u * (uint32_t)shp.ipt;
    wd.J = (uint32_t)shp.jtile;
    wd.Jc = (uint32_t)shp.jchunk;
    wd.stages = (uint32_t)shp.stages;
    wd.flags = ctx->cfg.flags;
    wd.force_idx = force_idx ? 1u : 0u;
    wd.nedges_max = ne;
    wd.ne = ne;
    wd.euclid = bh->euclid ? 1u : 0u;
    wd.neg_fast_t = bh->euclid ? bh->fast_t : -bh->fast_t;  // 3-D: +H, angular: -T
    wd.lut_scale = bh->lut_scale;
    {
        const float t = -bh->fast_t;  // the fast loop's packed offset: -T (angles), -H (3-D)
        uint32_t b;
        memcpy(&b, &t, 4);
        wd.neg_fast_t2 = ((unsigned long long)b << 32) | b;
    }
    wd.cos_last = bh->cos_last;
    wd.zbits0 = bh->zbits0;
    wd.zshift = bh->zshift;
    // zero-vector padding has screen value e = -T: it can look in range only
    // when T <= 0 (3-D catalogs are padded with a far point instead); sub-ranges
    // of segmented catalogs are followed by real points
    wd.need_idx = (force_idx || (!bh->euclid && !(bh->fast_t > 0.f))) ? 1u : 0u;
    wd.chord_ok = bh->euclid ? 0u : 1u;
    for (int s2 = 0; s2 < nsub; ++s2)
        if (!(specs[s2].a->eps_max <= kChordEpsRef && specs[s2].b->eps_max <= kChordEpsRef)) wd.chord_ok = 0u;
    wd.wait_limit_ns = (uint64_t)ctx->cfg.wait_timeout_us * 1000ull;
    // Spatial pruning (screen kernels): a block whose spheres are at least
    // prune_thr apart (scaled space) holds only overflow pairs.  Angular: a
    // pair of points with | |v|^2 - 1 | <= eps at distance delta has exact
    // dot <= 1 + eps - delta^2 / 2, at most C_B - 1e-15 (so the binary64
    // dot, within 3.4e-16 of it, is <= C_B: overflow) once delta >=
    // sqrt(2 (1 + eps) - 2 (C_B - 1e-15)).  3-D: delta >= sqrt(S_B) (1 +
    // 1e-12) makes the binary64 d^2 (relative error < 1e-15) >= S_B.
    // the gap below which point groups may hold pairs in range: items with many
    // such groups (dense-cluster items, mostly slow-path pairs) are counted first
    wd.near_thr = bh->euclid ? (float)(std::sqrt(bh->cos_last) * kCapScale3d)
                             : (float)std::sqrt(std::max(0.0, 2.0 - 2.0 * bh->cos_last));
    wd.prune = 0u;
    wd.prune_thr = INFINITY;
    // (not with a counted overflow row: skipped blocks would have to be counted)
    if ((ctx->cfg.flags & TPCF_F_PRUNE) && !(ctx->cfg.flags & TPCF_F_CHECK_OVERFLOW) &&
        (mode == kModeScreenScalar || mode == kModeEuclidScreen)) {
        double thr;
        if (bh->euclid) {
            thr = std::sqrt(bh->cos_last) * (1.0 + 1e-12) * kCapScale3d;
        } else {
            double eps = 0.0;
            for (int s2 = 0; s2 < nsub; ++s2) eps = std::max(eps, std::max(specs[s2].a->eps_max, specs[s2].b->eps_max));
            thr = std::sqrt(std::max(0.0, 2.0 * (1.0 + eps) - 2.0 * (bh->cos_last - 1e-15)));
        }
        const float t32 = (float)thr;
        wd.prune_thr = (double)t32 >= thr ? t32 : std::nextafter(t32, INFINITY);
        wd.prune = std::isfinite(wd.prune_thr) ? 1u : 0u;
    }
}

int ilog2_u64(uint64_t v) { int k = 0; while (v > 1) { v >>= 1; ++k; } return k; }

// What run_counts leaves behind when it captures the counting sequence into a
// CUDA graph instead of running it.
struct GraphOut {
    cudaGraphExec_t exec = nullptr;
    void* buf = nullptr;                     // accumulators, sub-problems, totals (owned)
    unsigned long long* stat_w = nullptr;    // kStatWords statistics words inside buf
    uint32_t launches = 0;                   // kernels per graph launch
};

int run_counts(tpcf_ctx* ctx, const SubSpec* specs, int nsub, const tpcf_bins* bins,
               cudaStream_t st, unsigned long long* const* outs, int where, tpcf_stats* stats,
               bool force_idx = false, GraphOut* gout = nullptr) {
    if (where != TPCF_HOST && where != TPCF_DEVICE) return ctx->fail(TPCF_EINVAL, "bad where");
    const bool capture = gout != nullptr;
    if (capture && (where != TPCF_DEVICE || stats)) return ctx->fail(TPCF_EINVAL, "graph capture needs device outputs");
    if (where == TPCF_DEVICE && stats) return ctx->fail(TPCF_EINVAL, "stats need where = TPCF_HOST");
    if (!bins || bins->ctx != ctx) return ctx->fail(TPCF_EINVAL, "bins missing or from another context");
    if (nsub < 1) return ctx->fail(TPCF_EINVAL, "no histogram to count");
    // (the kernel's stage record holds a sub-problem index in 16 bits)
    if (nsub > 0xffff) return ctx->fail(TPCF_EINVAL, "more than 65535 sub-problems in one count");
    // histograms: sub-problem s fills nhist of them, from index hist_first[s]; outs has one per histogram
    int H = 0;
    bool any_rows = false;
    for (int s = 0; s < nsub; ++s) {
        if (!specs[s].a || !specs[s].b || specs[s].a->ctx != ctx || specs[s].b->ctx != ctx)
            return ctx->fail(TPCF_EINVAL, "catalog missing or from another context");
        if (specs[s].nhist < 1 || (specs[s].nhist > 1 && !specs[s].row_seg))
            return ctx->fail(TPCF_EINVAL, "bad histogram count");
        any_rows |= specs[s].row_seg != nullptr;
        H += specs[s].nhist;
    }
    for (int h = 0; h < H; ++h)
        if (!outs[h]) return ctx->fail(TPCF_EINVAL, "NULL histogram");
    if (any_rows && ctx->cfg.shard_count > 1)
        return ctx->fail(TPCF_EINVAL, "row-attributed counts are not split into shards");
    cudaSetDevice(ctx->cfg.device);
    const int ne = bins->nedges;
    // the device bin set: angular bins have one; 3-D bins one per bound 2^key on the points' norms
    const BinsDev* bh = &bins->host;
    const BinsDev* bdev = bins->dev_desc;
    if (bins->euclid) {
        double M = 0.0;
        for (int s = 0; s < nsub; ++s) {
            if (!specs[s].a->euclid || !specs[s].b->euclid)
                return ctx->fail(TPCF_EINVAL, "3-D bins count 3-D catalogs (tpcf_catalog_create_3d)");
            M = std::max(M, std::max(specs[s].a->norm_max, specs[s].b->norm_max));
        }
        int key = -64;
        while (std::ldexp(1.0, key) < M) ++key;
        BinsDev* dv = nullptr;
        const int rc = euclid_set(ctx, const_cast<tpcf_bins*>(bins), key, &bh, &dv);
        if (rc != TPCF_OK) return rc;
        bdev = dv;
    } else {
        for (int s = 0; s < nsub; ++s)
            if (specs[s].a->euclid || specs[s].b->euclid)
                return ctx->fail(TPCF_EINVAL, "angular bins count unit-vector catalogs");
    }
    int mode = kernel_mode(ctx->cfg, bins->euclid);
    uint64_t all_pairs = 0, max_n = 0;
    for (int s = 0; s < nsub; ++s) {
        all_pairs += full_pairs(specs[s]);
        max_n = std::max<uint64_t>(max_n, std::max(specs[s].na, specs[s].nb));
    }
    Shape sh;
    const bool fits = choose_shape(ctx, mode, ne, all_pairs, max_n, &sh);
    if (!fits)
        return ctx->fail(TPCF_EINVAL, "no kernel shape fits (threads=%d ipt=%d jtile=%d)",
                         ctx->cfg.threads, ctx->cfg.ipt, ctx->cfg.jtile);
    if (any_rows && 32u * (uint32_t)sh.ipt != kSegAlign)
        return ctx->fail(TPCF_EINVAL, "row-attributed counts need %u i-points per warp", kSegAlign);

    // ---- accumulators and statistics: a context slot for up to 3 histograms,
    // otherwise one stream-ordered allocation for this call (a plain allocation
    // owned by the graph when capturing)
    const bool use_slot = H <= 3 && !capture;
    tpcf_ctx::Slot* slot = nullptr;
    std::unique_lock<std::mutex> slot_lock;
    unsigned long long* acc = nullptr;
    unsigned long long* stat_w = nullptr;
    size_t acc_stride = 0;
    void* call_buf = nullptr;
    SubProblem* dev_subs = nullptr;
    unsigned long long* dev_totals = nullptr;
    const size_t sub_bytes = ((size_t)nsub * sizeof(SubProblem) + 255) / 256 * 256;
    const size_t tot_bytes = ((size_t)H * 8 + 255) / 256 * 256;
    size_t acc_words = 0;
    if (use_slot) {
        slot = &ctx->slots[ctx->slot_rr.fetch_add(1) % kSlots];
        slot_lock = std::unique_lock<std::mutex>(slot->mu);
        CUDA_TRY(ctx, cudaStreamWaitEvent(st, slot->ev, 0));
        acc = slot->dev;
        acc_stride = kHistStride;
        stat_w = slot->dev + kStatOff;
        acc_words = kSlotWords;
    } else {
        acc_stride = (size_t)ne + 1;
        acc_words = (size_t)H * acc_stride + kStatWords;
        const size_t bytes = acc_words * 8 + sub_bytes + tot_bytes;
        if ((capture ? dev_malloc(&call_buf, bytes) : cudaMallocAsync(&call_buf, bytes, st)) != cudaSuccess)
            return ctx->fail(TPCF_ENOMEM, "accumulator allocation failed (%zu bytes)", bytes);
        acc = (unsigned long long*)call_buf;
        stat_w = acc + (size_t)H * acc_stride;
        dev_subs = (SubProblem*)((char*)call_buf + acc_words * 8);
        dev_totals = (unsigned long long*)((char*)dev_subs + sub_bytes);
    }
    auto release = [&](int rc) {
        if (call_buf && capture) {
            cudaStreamSynchronize(st);
            cudaFree(call_buf);
        } else if (call_buf) {
            cudaFreeAsync(call_buf, st);
        }
        if (slot) cudaEventRecord(slot->ev, st);
        return rc;
    };

    WorkDesc wd;
    memset(&wd, 0, sizeof wd);
    std::vector<SubProblem> subs;
    auto setup = [&](const Shape& shp) -> int {
        const uint64_t items = build_work(ctx, specs, nsub, bdev, shp, acc, acc_stride, subs);
        if (items > 0xffff0000ull) return TPCF_EOVERFLOW;
        if (use_slot) {
            for (int s2 = 0; s2 < nsub; ++s2) wd.sub[s2] = subs[s2];
            wd.sub_dev = nullptr;
        } else {
            if (cudaMemcpyAsync(dev_subs, subs.data(), (size_t)nsub * sizeof(SubProblem),
                                cudaMemcpyHostToDevice, st) != cudaSuccess)
                return TPCF_ECUDA;
            wd.sub_dev = dev_subs;
        }
        wd.nsub = nsub;
        wd.item_lo = 0;
        wd.item_hi = items;
        if (ctx->cfg.shard_count > 1) {
            wd.item_lo = items * ctx->cfg.shard_index / ctx->cfg.shard_count;
            wd.item_hi = items * (ctx->cfg.shard_index + 1) / ctx->cfg.shard_count;
        }
        wd.stats = stat_w;
        wd.item_counter = stat_w + kStatNextItem;
        fill_scalars(ctx, specs, nsub, bh, mode, shp, force_idx, ne, wd);
        return TPCF_OK;
    };
    auto launch = [&](const Shape& shp) -> cudaError_t {
        if (wd.item_hi <= wd.item_lo) return cudaSuccess;
        Shape sl = shp;
        const uint64_t n_launch_items = wd.item_hi - wd.item_lo;
        if ((uint64_t)sl.blocks > n_launch_items) sl.blocks = (int)n_launch_items;
        if (!capture) {  // when capturing, set before the capture begins
            cudaError_t e = count_set_smem_limit(mode, shp.threads, shp.ipt, shp.smem);
            if (e != cudaSuccess) return e;
        }
        return launch_count(wd, sl, mode, ne, st);
    };

    // ---- optional autotuning: time every fitting shape on a bounded window of the
    // work (about 4 items per warp, the same window of the walk for every shape),
    // keep the one with the least time per pair
    if ((ctx->cfg.flags & TPCF_F_AUTOTUNE) && ctx->cfg.threads == 0 && ctx->cfg.jtile == 0) {
        const std::array<int, 5> key{mode, ne, nsub, ilog2_u64(all_pairs + 1), ilog2_u64(max_n + 1)};
        std::lock_guard<std::mutex> tl(ctx->tune_mu);
        auto it = ctx->tuned.find(key);
        if (it != ctx->tuned.end()) {
            sh = it->second;
        } else {
            const int cand_t[3] = {128, 256, 512};
            const int cand_j[3] = {128, 256, 512};
            double best = 1e300;
            Shape best_sh = sh;
            cudaEvent_t a0, a1;
            cudaEventCreate(&a0);
            cudaEventCreate(&a1);
            for (int ti = 0; ti < 3; ++ti) {
                for (int ji = 0; ji < 3; ++ji) {
                    Shape c;
                    if (!shape_for(ctx, mode, ne, cand_t[ti], 8, cand_j[ji], 0, &c)) continue;
                    if (setup(c) != TPCF_OK) continue;
                    const uint64_t window = (uint64_t)ctx->num_sms * (uint64_t)(c.threads / 32) * 4;
                    if (wd.item_hi - wd.item_lo > window) wd.item_hi = wd.item_lo + window;
                    uint64_t wpairs = 0;
                    for (int s2 = 0; s2 < nsub; ++s2)
                        wpairs += range_pairs(subs[s2], wd.item_lo, wd.item_hi, wd.I, wd.Jc, wd.J);
                    if (wpairs == 0) continue;
                    cudaMemsetAsync(acc, 0, acc_words * 8, st);
                    if (capture && count_set_smem_limit(mode, c.threads, c.ipt, c.smem) != cudaSuccess) continue;
                    cudaEventRecord(a0, st);
                    if (launch(c) != cudaSuccess) continue;
                    cudaEventRecord(a1, st);
                    float ms = 1e30f;
                    if (cudaEventSynchronize(a1) == cudaSuccess) cudaEventElapsedTime(&ms, a0, a1);
                    const double per_pair = (double)ms / (double)wpairs;
                    if (per_pair < best) { best = per_pair; best_sh = c; }
                }
            }
            cudaEventDestroy(a0);
            cudaEventDestroy(a1);
            sh = best_sh;
            ctx->tuned[key] = sh;
        }
    }

    {
        const int rc = setup(sh);
        if (rc != TPCF_OK) return release(ctx->fail(rc, "work description failed"));
    }
    // ---- per-histogram pair totals (the finalize step derives overflow from them)
    std::vector<unsigned long long> totals;
    totals.reserve(H);
    for (int s2 = 0; s2 < nsub; ++s2)
        for (int k = 0; k < specs[s2].nhist; ++k)
            totals.push_back(specs[s2].totals ? specs[s2].totals[k]
                             : ctx->cfg.shard_count > 1 ? range_pairs(subs[s2], wd.item_lo, wd.item_hi, wd.I, wd.Jc, wd.J)
                                                        : full_pairs(specs[s2]));
    if (!use_slot &&
        cudaMemcpyAsync(dev_totals, totals.data(), (size_t)H * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return release(ctx->fail(TPCF_ECUDA, "totals upload failed"));
    if (capture) {
        if (count_set_smem_limit(mode, sh.threads, sh.ipt, sh.smem) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess ||
            cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return release(ctx->fail(TPCF_ECUDA, "graph capture could not start"));
    }
    auto abort_capture = [&](int rc) {
        if (capture) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(st, &g);
            if (g) cudaGraphDestroy(g);
        }
        return release(rc);
    };
    if (cudaMemsetAsync(acc, 0, acc_words * 8, st) != cudaSuccess)
        return abort_capture(ctx->fail(TPCF_ECUDA, "memset failed"));
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (stats) {
        cudaEventCreate(&t0);
        cudaEventCreate(&t1);
        cudaEventRecord(t0, st);
    }
    uint32_t launches = 0;
    {
        const cudaError_t e = launch(sh);
        if (e != cudaSuccess)
            return abort_capture(ctx->fail(TPCF_ECUDA, "count launch failed: %s", cudaGetErrorString(e)));
        if (wd.item_hi > wd.item_lo) ++launches;
    }
    if (stats) cudaEventRecord(t1, st);

    // ---- finalize: overflow of each histogram = its pair total - sum of the other
    // entries, or (counted overflow) a check that the entries sum to the total
    // (2: the test hook that checks against the pair total plus one)
    const int count_over = (ctx->cfg.flags & TPCF_F_CHECK_OVERFLOW)
                               ? ((ctx->cfg.flags & TPCF_F_TEST_BAD_TOTAL) ? 2 : 1) : 0;
    if (use_slot) {
        for (int s2 = 0; s2 < H; ++s2) {
            unsigned long long* a = acc + (size_t)s2 * acc_stride;
            unsigned long long* dst = where == TPCF_DEVICE ? outs[s2] : a;
            if (launch_finalize(a, ne, dst, totals[s2], count_over, stat_w + kStatError, st) != cudaSuccess)
                return release(ctx->fail(TPCF_ECUDA, "finalize launch failed"));
            ++launches;
        }
    } else {
        // device outputs must be one contiguous array (outs[h] = outs[0] + h * (ne + 1))
        unsigned long long* dst = where == TPCF_DEVICE ? outs[0] : acc;
        if (launch_finalize_batch(acc, (int)acc_stride, ne, dst, ne + 1, dev_totals, H, count_over, stat_w + kStatError,
                                  st) !=
            cudaSuccess)
            return abort_capture(ctx->fail(TPCF_ECUDA, "finalize launch failed"));
        ++launches;
    }
    if (capture) {
        cudaGraph_t g = nullptr;
        if (cudaStreamEndCapture(st, &g) != cudaSuccess || !g)
            return release(ctx->fail(TPCF_ECUDA, "graph capture failed"));
        const cudaError_t e = cudaGraphInstantiate(&gout->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return release(ctx->fail(TPCF_ECUDA, "graph instantiation failed"));
        gout->buf = call_buf;
        gout->stat_w = stat_w;
        gout->launches = launches;
        return TPCF_OK;  // the graph owns call_buf
    }
    int rc = TPCF_OK;
    if (where == TPCF_HOST) {
        std::vector<unsigned long long> h(acc_words);
        if (cudaMemcpyAsync(h.data(), acc, acc_words * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return release(ctx->fail(TPCF_ECUDA, "result copy failed"));
        for (int s2 = 0; s2 < H; ++s2)
            memcpy(outs[s2], h.data() + (size_t)s2 * acc_stride, (size_t)(ne + 1) * 8);
        const unsigned long long* hs = h.data() + (stat_w - acc);
        const unsigned long long errw = hs[kStatError];
        if (stats) {
            memset(stats, 0, sizeof *stats);
            stats->pairs = hs[kStatPairs];
            stats->band_pairs = hs[kStatBand];
            stats->band_mismatch = hs[kStatMismatch];
            stats->device_error = (uint32_t)errw;
            stats->launches = launches;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, t0, t1);
            stats->kernel_ms = ms;
            stats->pruned_pairs = hs[kStatPruned];
        }
        if (errw & kErrWaitTimeout) rc = ctx->fail(TPCF_ETIMEOUT, "a bounded device wait timed out");
        else if (errw & kErrBadHist) rc = ctx->fail(TPCF_ECUDA, "histogram does not add up to its pair total");
        else if (errw) rc = ctx->fail(TPCF_ECUDA, "device error word 0x%llx", errw);
    }
    ctx->launches.fetch_add(launches);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    return release(rc);
}

}  // namespace

// ====================================================================== serving steps
// Shape of a serving step (the multi-job kernel exists for 512 x 8): j-tiles of
// 256 points, or 128 where the step's histograms need the shared memory;
// false when neither fits.
bool tpcf::serving_shape(tpcf_ctx* ctx, int nedges_max, Shape* sh) {
    return shape_for(ctx, kModeScreenScalar, nedges_max, 512, 8, 0, 2, sh);
}

// Work description of one served job for the serving-step kernel: the
// sub-problems RR, DR and DD of catalogs (d, r) with bins b, accumulating
// into three histograms of ne + 1 words at acc (in that order); also the
// job's item count and the three histograms' pair totals.
int tpcf::serving_job_desc(tpcf_ctx* ctx, const tpcf_catalog* d, const tpcf_catalog* r, const tpcf_bins* b,
                           const Shape& sh, unsigned long long* acc, WorkDesc* out, uint64_t* n_items,
                           uint64_t* totals) {
    if (b->euclid || d->euclid || r->euclid) return TPCF_EINVAL;
    SubSpec specs[3] = {{r, r, true, (uint32_t)r->n, (uint32_t)r->n, 0, 0},
                        {d, r, false, (uint32_t)d->n, (uint32_t)r->n, 0, 0},
                        {d, d, true, (uint32_t)d->n, (uint32_t)d->n, 0, 0}};
    std::vector<SubProblem> subs;
    const uint64_t items = build_work(ctx, specs, 3, b->dev_desc, sh, acc, (size_t)b->nedges + 1, subs);
    if (items > 0xffff0000ull) return TPCF_EOVERFLOW;
    WorkDesc wd;
    memset(&wd, 0, sizeof wd);
    for (int k = 0; k < 3; ++k) wd.sub[k] = subs[k];
    wd.sub_dev = nullptr;
    wd.nsub = 3;
    wd.item_lo = 0;
    wd.item_hi = items;
    fill_scalars(ctx, specs, 3, &b->host, kModeScreenScalar, sh, false, b->nedges, wd);
    *out = wd;
    *n_items = items;
    for (int k = 0; k < 3; ++k) totals[k] = full_pairs(specs[k]);
    return TPCF_OK;
}

// One serving step: slices (device, sorted by position) of `positions` work
// items in all, into the jobs' own accumulators; slice_ctr: one device counter
// per slice and stats: kStatWords device words, all zeroed by the caller.
int tpcf::serving_launch(tpcf_ctx* ctx, const Shape& sh, int nedges_max, const StepSlice* slices, int nslices,
                         unsigned long long* slice_ctr, uint32_t positions, unsigned long long* stats,
                         cudaStream_t st) {
    WorkDesc wd;
    memset(&wd, 0, sizeof wd);
    wd.stats = stats;
    wd.item_counter = stats + kStatNextItem;
    wd.slices = slices;
    wd.slice_ctr = slice_ctr;
    wd.nslices = nslices;
    wd.step_positions = positions;
    wd.I = 32u * (uint32_t)sh.ipt;
    wd.J = (uint32_t)sh.jtile;
    wd.Jc = (uint32_t)sh.jchunk;
    wd.stages = (uint32_t)sh.stages;
    wd.flags = ctx->cfg.flags;
    wd.nedges_max = nedges_max;
    wd.wait_limit_ns = (uint64_t)ctx->cfg.wait_timeout_us * 1000ull;
    Shape s2 = sh;  // (no more blocks than the step has items for their warps)
    const uint64_t warps = (uint64_t)sh.threads / 32;
    const uint64_t need = ((uint64_t)positions + warps - 1) / warps;
    if ((uint64_t)s2.blocks > need) s2.blocks = (int)std::max<uint64_t>(1, need);
    if (count_step_set_smem_limit(sh.smem) != cudaSuccess) return TPCF_ECUDA;
    if (launch_count_step(wd, s2, st) != cudaSuccess) return TPCF_ECUDA;
    ctx->launches.fetch_add(1);
    return TPCF_OK;
}

// One serving step that holds a single job (job: its work description from
// serving_job_desc): the one-job kernel, which reads the description from its
// parameter, over the items [q_begin, q_begin + n), drawing their order's
// positions from pos_lo on (the order laid out for draw_warps warps; 0: this
// launch's) until it ends or stats[kStatYield] is set; stats: kStatWords
// device words zeroed by the caller (its item counter included).
int tpcf::serving_launch_one(tpcf_ctx* ctx, const Shape& sh, const WorkDesc& job, uint32_t q_begin, uint32_t n,
                             uint64_t pos_lo, uint32_t draw_warps, unsigned long long* stats, cudaStream_t st) {
    WorkDesc wd = job;
    wd.item_lo = q_begin;
    wd.item_hi = (uint64_t)q_begin + n;
    wd.pos_lo = pos_lo;
    wd.draw_warps = draw_warps;
    wd.stats = stats;
    wd.item_counter = stats + kStatNextItem;
    wd.slices = nullptr;
    wd.slice_ctr = nullptr;
    wd.nslices = 0;
    Shape s2 = sh;
    const uint64_t warps = (uint64_t)sh.threads / 32;
    const uint64_t need = ((uint64_t)n + warps - 1) / warps;
    if ((uint64_t)s2.blocks > need) s2.blocks = (int)std::max<uint64_t>(1, need);
    if (count_preemptible_set_smem_limit(sh.smem) != cudaSuccess) return TPCF_ECUDA;
    if (launch_count_preemptible(wd, s2, st) != cudaSuccess) return TPCF_ECUDA;
    ctx->launches.fetch_add(1);
    return TPCF_OK;
}

uint64_t tpcf::serving_positions(uint64_t n, uint32_t warps) { return draw_positions(n, warps); }

// ====================================================================== counting ABI
extern "C" int tpcf_count_auto(tpcf_ctx* ctx, const tpcf_catalog* cat, const tpcf_bins* bins,
                               void* stream, uint64_t* hist, int where, tpcf_stats* st) {
    if (!ctx || !cat) return ctx ? ctx->fail(TPCF_EINVAL, "NULL catalog") : TPCF_EINVAL;
    SubSpec s{cat, cat, true, (uint32_t)cat->n, (uint32_t)cat->n, 0, 0};
    unsigned long long* outs[1] = {(unsigned long long*)hist};
    return run_counts(ctx, &s, 1, bins, (cudaStream_t)stream, outs, where, st);
}

extern "C" int tpcf_count_cross(tpcf_ctx* ctx, const tpcf_catalog* d, const tpcf_catalog* r,
                                const tpcf_bins* bins, void* stream, uint64_t* hist, int where,
                                tpcf_stats* st) {
    if (!ctx || !d || !r) return ctx ? ctx->fail(TPCF_EINVAL, "NULL catalog") : TPCF_EINVAL;
    SubSpec s{d, r, false, (uint32_t)d->n, (uint32_t)r->n, 0, 0};
    unsigned long long* outs[1] = {(unsigned long long*)hist};
    return run_counts(ctx, &s, 1, bins, (cudaStream_t)stream, outs, where, st);
}

extern "C" int tpcf_count_all(tpcf_ctx* ctx, const tpcf_catalog* d, const tpcf_catalog* r,
                              const tpcf_bins* bins, void* stream, uint64_t* dd, uint64_t* dr,
                              uint64_t* rr, int where, tpcf_stats* st) {
    if (!ctx || !d || !r) return ctx ? ctx->fail(TPCF_EINVAL, "NULL catalog") : TPCF_EINVAL;
    // Largest first (RR, DR, DD when nr >= nd) so the tail of the launch is the cheapest work.
    SubSpec s[3] = {{r, r, true, (uint32_t)r->n, (uint32_t)r->n, 0, 0},
                    {d, r, false, (uint32_t)d->n, (uint32_t)r->n, 0, 0},
                    {d, d, true, (uint32_t)d->n, (uint32_t)d->n, 0, 0}};
    unsigned long long* outs[3] = {(unsigned long long*)rr, (unsigned long long*)dr,
                                   (unsigned long long*)dd};
    return run_counts(ctx, s, 3, bins, (cudaStream_t)stream, outs, where, st);
}

extern "C" int tpcf_count_patches(tpcf_ctx* ctx, const tpcf_catalog* d, const tpcf_catalog* r,
                                  const tpcf_bins* bins, void* stream, uint64_t* hists, int where,
                                  tpcf_stats* st) {
    if (!ctx || !d || !r || !hists) return ctx ? ctx->fail(TPCF_EINVAL, "NULL argument") : TPCF_EINVAL;
    if (d->offsets.empty() || r->offsets.empty() || d->offsets.size() != r->offsets.size())
        return ctx->fail(TPCF_EINVAL, "patches: both catalogs must be segmented with the same count");
    const int np = (int)d->offsets.size() - 1;
    if (!bins) return ctx->fail(TPCF_EINVAL, "NULL bins");
    const size_t hs = (size_t)bins->nedges + 1;
    std::vector<SubSpec> specs(3 * (size_t)np);
    std::vector<unsigned long long*> outs(3 * (size_t)np);
    for (int p = 0; p < np; ++p) {
        const uint32_t d0 = (uint32_t)d->seg_start[p], dn = (uint32_t)(d->offsets[p + 1] - d->offsets[p]);
        const uint32_t r0 = (uint32_t)r->seg_start[p], rn = (uint32_t)(r->offsets[p + 1] - r->offsets[p]);
        specs[3 * p + 0] = SubSpec{d, d, true, dn, dn, d0, d0};
        specs[3 * p + 1] = SubSpec{d, r, false, dn, rn, d0, r0};
        specs[3 * p + 2] = SubSpec{r, r, true, rn, rn, r0, r0};
        for (int k = 0; k < 3; ++k) outs[3 * p + k] = (unsigned long long*)hists + (3 * (size_t)p + k) * hs;
    }
    return run_counts(ctx, specs.data(), 3 * np, bins, (cudaStream_t)stream, outs.data(), where, st, true);
}

// ====================================================================== leave-one-out jackknife
// One launch fills, for every segment p of the two segmented catalogs:
//   rows_DD[p] = ordered pairs (i, j), i != j, i in D_p, j in D     (full square, rows by D segment)
//   rows_RR[p] likewise over R;  rows_DR[p] = pairs (d in D_p, r in R);  rows_RD[p] = (r in R_p, d in D)
//   within_DD[p], within_DR[p], within_RR[p] (the per-patch counts of tpcf_count_patches).
// Pairs touching patch p: T_DD = rows_DD - within_DD (ordered rows count the pairs inside p twice),
// T_RR likewise, T_DR = rows_DR + rows_RD - within_DR.  Totals: DD = sum_p rows_DD / 2, RR alike,
// DR = sum_p rows_DR.  Leave-one-out: X_{-p} = X - T_X[p].
extern "C" int tpcf_jackknife(tpcf_ctx* ctx, const tpcf_catalog* d, const tpcf_catalog* r, const tpcf_bins* bins,
                              void* stream, int estimator, uint64_t* loo, double* w_loo, double* cov,
                              tpcf_stats* st) {
    if (!ctx) return TPCF_EINVAL;
    if (!d || !r || !bins || !loo) return ctx->fail(TPCF_EINVAL, "jackknife: NULL argument");
    if (d->offsets.empty() || r->offsets.empty() || d->offsets.size() != r->offsets.size())
        return ctx->fail(TPCF_EINVAL, "jackknife: both catalogs must be segmented with the same count");
    if (estimator != TPCF_LS_EXACT && estimator != TPCF_LS_PAPER)
        return ctx->fail(TPCF_EINVAL, "jackknife: unknown estimator");
    if (!bins->euclid && !(bins->host.fast_t > 0.f))
        return ctx->fail(TPCF_EINVAL, "jackknife: the histogram range must end below 90 degrees");
    const int P = (int)d->offsets.size() - 1;
    if (cov && P < 2) return ctx->fail(TPCF_EINVAL, "jackknife: the covariance needs at least 2 patches");
    const int ne = bins->nedges, hs = ne + 1, B = ne - 1;
    const uint64_t ND = d->n, NR = r->n;
    std::vector<uint64_t> tdd(P), trr(P), tdr(P), trd(P);
    for (int p = 0; p < P; ++p) {
        const uint64_t np_ = d->offsets[p + 1] - d->offsets[p], mp = r->offsets[p + 1] - r->offsets[p];
        tdd[p] = np_ * (ND ? ND - 1 : 0);
        trr[p] = mp * (NR ? NR - 1 : 0);
        tdr[p] = np_ * NR;
        trd[p] = mp * ND;
    }
    const uint32_t AD = (uint32_t)d->seg_start[P], AR = (uint32_t)r->seg_start[P];
    std::vector<SubSpec> specs;
    SubSpec s_dd{d, d, false, AD, AD, 0, 0, P, d->seg_of_block, true, tdd.data()};
    SubSpec s_rr{r, r, false, AR, AR, 0, 0, P, r->seg_of_block, true, trr.data()};
    SubSpec s_dr{d, r, false, AD, AR, 0, 0, P, d->seg_of_block, false, tdr.data()};
    SubSpec s_rd{r, d, false, AR, AD, 0, 0, P, r->seg_of_block, false, trd.data()};
    specs.push_back(s_rr);
    specs.push_back(s_dr);
    specs.push_back(s_rd);
    specs.push_back(s_dd);
    for (int p = 0; p < P; ++p) {
        const uint32_t d0 = (uint32_t)d->seg_start[p], dn = (uint32_t)(d->offsets[p + 1] - d->offsets[p]);
        const uint32_t r0 = (uint32_t)r->seg_start[p], rn = (uint32_t)(r->offsets[p + 1] - r->offsets[p]);
        specs.push_back(SubSpec{d, d, true, dn, dn, d0, d0});
        specs.push_back(SubSpec{d, r, false, dn, rn, d0, r0});
        specs.push_back(SubSpec{r, r, true, rn, rn, r0, r0});
    }
    // histogram order: rows_RR, rows_DR, rows_RD, rows_DD (P each), then (DD, DR, RR) per patch
    const int H = 7 * P;
    std::vector<uint64_t> h((size_t)H * hs);
    std::vector<unsigned long long*> outs(H);
    for (int k = 0; k < H; ++k) outs[k] = (unsigned long long*)h.data() + (size_t)k * hs;
    const int rc = run_counts(ctx, specs.data(), (int)specs.size(), bins, (cudaStream_t)stream, outs.data(), TPCF_HOST,
                              st, true);
    if (rc != TPCF_OK) return rc;
    auto rows_rr = [&](int p) { return h.data() + (size_t)(0 * P + p) * hs; };
    auto rows_dr = [&](int p) { return h.data() + (size_t)(1 * P + p) * hs; };
    auto rows_rd = [&](int p) { return h.data() + (size_t)(2 * P + p) * hs; };
    auto rows_dd = [&](int p) { return h.data() + (size_t)(3 * P + p) * hs; };
    auto within = [&](int p, int k) { return h.data() + (size_t)(4 * P + 3 * p + k) * hs; };
    std::vector<uint64_t> DD(hs, 0), DR(hs, 0), RR(hs, 0), DR2(hs, 0);
    for (int p = 0; p < P; ++p)
        for (int b = 0; b < hs; ++b) {
            DD[b] += rows_dd(p)[b];
            RR[b] += rows_rr(p)[b];
            DR[b] += rows_dr(p)[b];
            DR2[b] += rows_rd(p)[b];
        }
    for (int b = 0; b < hs; ++b) {
        if ((DD[b] & 1) || (RR[b] & 1) || DR[b] != DR2[b])
            return ctx->fail(TPCF_ECUDA, "jackknife: inconsistent row sums (bin %d)", b);
        DD[b] /= 2;
        RR[b] /= 2;
    }
    for (int p = 0; p < P; ++p) {
        uint64_t* o = loo + (size_t)3 * p * hs;
        uint64_t sdd = 0, sdr = 0, srr = 0;
        for (int b = 0; b < hs; ++b) {
            o[b] = DD[b] - (rows_dd(p)[b] - within(p, 0)[b]);
            o[hs + b] = DR[b] - (rows_dr(p)[b] + rows_rd(p)[b] - within(p, 1)[b]);
            o[2 * hs + b] = RR[b] - (rows_rr(p)[b] - within(p, 2)[b]);
            sdd += o[b];
            sdr += o[hs + b];
            srr += o[2 * hs + b];
        }
        const uint64_t nd = ND - (d->offsets[p + 1] - d->offsets[p]), nr = NR - (r->offsets[p + 1] - r->offsets[p]);
        if (sdd != nd * (nd ? nd - 1 : 0) / 2 || sdr != nd * nr || srr != nr * (nr ? nr - 1 : 0) / 2)
            return ctx->fail(TPCF_ECUDA, "jackknife: leave-one-out totals do not add up (patch %d)", p);
    }
    if (st) {
        uint64_t pairs = ND * (ND ? ND - 1 : 0) + NR * (NR ? NR - 1 : 0) + 2 * ND * NR;
        for (int p = 0; p < P; ++p) {
            const uint64_t np_ = d->offsets[p + 1] - d->offsets[p], mp = r->offsets[p + 1] - r->offsets[p];
            pairs += np_ * (np_ ? np_ - 1 : 0) / 2 + mp * (mp ? mp - 1 : 0) / 2 + np_ * mp;
        }
        st->pairs = pairs;  // the real pairs (the device figure includes the alignment padding)
    }
    if (!w_loo && !cov) return TPCF_OK;
    std::vector<double> w((size_t)P * (B > 0 ? B : 1), NAN);
    for (int p = 0; p < P; ++p) {
        const uint64_t nd = ND - (d->offsets[p + 1] - d->offsets[p]), nr = NR - (r->offsets[p + 1] - r->offsets[p]);
        const uint64_t* o = loo + (size_t)3 * p * hs;
        if (nd >= 2 && nr >= 2)
            tpcf_estimate(o + 1, o + hs + 1, o + 2 * hs + 1, B, nd, nr, estimator, w.data() + (size_t)p * B);
    }
    if (w_loo) memcpy(w_loo, w.data(), (size_t)P * B * sizeof(double));
    if (cov) {
        // C_ab = (P - 1) / P * sum_p (w_pa - mean_a)(w_pb - mean_b), sums in patch order
        std::vector<double> mean(B, 0.0);
        for (int a = 0; a < B; ++a) {
            double sum = 0.0;
            for (int p = 0; p < P; ++p) sum += w[(size_t)p * B + a];
            mean[a] = sum / (double)P;
        }
        const double f = (double)(P - 1) / (double)P;
        for (int a = 0; a < B; ++a)
            for (int b2 = 0; b2 < B; ++b2) {
                double sum = 0.0;
                for (int p = 0; p < P; ++p)
                    sum += (w[(size_t)p * B + a] - mean[a]) * (w[(size_t)p * B + b2] - mean[b2]);
                cov[(size_t)a * B + b2] = f * sum;
            }
    }
    return TPCF_OK;
}

// ====================================================================== captured counting graphs
struct tpcf_graph {
    tpcf_ctx* ctx = nullptr;
    GraphOut g;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaStream_t copy_st = nullptr;
    bool launched = false;
};

extern "C" int tpcf_graph_create(tpcf_ctx* ctx, int kind, const tpcf_catalog* d, const tpcf_catalog* r,
                                 const tpcf_bins* bins, uint64_t* out_dev, tpcf_graph** out) {
    if (!ctx || !out) return TPCF_EINVAL;
    *out = nullptr;
    if (!d || !bins || !out_dev || (kind != TPCF_GRAPH_AUTO && !r))
        return ctx->fail(TPCF_EINVAL, "graph: NULL argument");
    const size_t hs = (size_t)bins->nedges + 1;
    std::vector<SubSpec> specs;
    bool force_idx = false;
    switch (kind) {
        case TPCF_GRAPH_AUTO:
            specs.push_back(SubSpec{d, d, true, (uint32_t)d->n, (uint32_t)d->n, 0, 0});
            break;
        case TPCF_GRAPH_CROSS:
            specs.push_back(SubSpec{d, r, false, (uint32_t)d->n, (uint32_t)r->n, 0, 0});
            break;
        case TPCF_GRAPH_ALL:
            specs.push_back(SubSpec{d, d, true, (uint32_t)d->n, (uint32_t)d->n, 0, 0});
            specs.push_back(SubSpec{d, r, false, (uint32_t)d->n, (uint32_t)r->n, 0, 0});
            specs.push_back(SubSpec{r, r, true, (uint32_t)r->n, (uint32_t)r->n, 0, 0});
            break;
        case TPCF_GRAPH_PATCHES: {
            if (d->offsets.empty() || r->offsets.empty() || d->offsets.size() != r->offsets.size())
                return ctx->fail(TPCF_EINVAL, "graph: patches need two segmented catalogs with the same count");
            const int np = (int)d->offsets.size() - 1;
            for (int p = 0; p < np; ++p) {
                const uint32_t d0 = (uint32_t)d->seg_start[p], dn = (uint32_t)(d->offsets[p + 1] - d->offsets[p]);
                const uint32_t r0 = (uint32_t)r->seg_start[p], rn = (uint32_t)(r->offsets[p + 1] - r->offsets[p]);
                specs.push_back(SubSpec{d, d, true, dn, dn, d0, d0});
                specs.push_back(SubSpec{d, r, false, dn, rn, d0, r0});
                specs.push_back(SubSpec{r, r, true, rn, rn, r0, r0});
            }
            force_idx = true;
            break;
        }
        default:
            return ctx->fail(TPCF_EINVAL, "graph: unknown kind %d", kind);
    }
    std::vector<unsigned long long*> outs(specs.size());
    for (size_t k = 0; k < specs.size(); ++k) outs[k] = (unsigned long long*)out_dev + k * hs;
    tpcf_graph* gr = new (std::nothrow) tpcf_graph();
    if (!gr) return ctx->fail(TPCF_ENOMEM, "graph: host allocation failed");
    gr->ctx = ctx;
    cudaSetDevice(ctx->cfg.device);
    if (cudaStreamCreateWithFlags(&gr->copy_st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&gr->t0) != cudaSuccess || cudaEventCreate(&gr->t1) != cudaSuccess) {
        tpcf_graph_destroy(gr);
        return ctx->fail(TPCF_ECUDA, "graph: stream or event creation failed");
    }
    // captured on the graph's own stream (capture needs a stream other than the legacy default one)
    const int rc = run_counts(ctx, specs.data(), (int)specs.size(), bins, gr->copy_st, outs.data(), TPCF_DEVICE,
                              nullptr, force_idx, &gr->g);
    if (rc != TPCF_OK) {
        tpcf_graph_destroy(gr);
        return rc;
    }
    *out = gr;
    return TPCF_OK;
}

extern "C" int tpcf_graph_launch(tpcf_graph* g, void* stream) {
    if (!g || !g->g.exec) return TPCF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaSetDevice(g->ctx->cfg.device);
    if (cudaEventRecord(g->t0, st) != cudaSuccess || cudaGraphLaunch(g->g.exec, st) != cudaSuccess ||
        cudaEventRecord(g->t1, st) != cudaSuccess)
        return g->ctx->fail(TPCF_ECUDA, "graph launch failed");
    g->launched = true;
    g->ctx->launches.fetch_add(g->g.launches);
    return TPCF_OK;
}

extern "C" int tpcf_graph_stats(tpcf_graph* g, tpcf_stats* st) {
    if (!g || !g->g.exec) return TPCF_EINVAL;
    if (!g->launched) return g->ctx->fail(TPCF_ESTATE, "graph: not launched yet");
    tpcf_ctx* ctx = g->ctx;
    cudaSetDevice(ctx->cfg.device);
    unsigned long long h[kStatWords];
    if (cudaStreamWaitEvent(g->copy_st, g->t1, 0) != cudaSuccess ||
        cudaMemcpyAsync(h, g->g.stat_w, sizeof h, cudaMemcpyDeviceToHost, g->copy_st) != cudaSuccess ||
        cudaStreamSynchronize(g->copy_st) != cudaSuccess)
        return ctx->fail(TPCF_ECUDA, "graph: statistics copy failed");
    if (st) {
        memset(st, 0, sizeof *st);
        st->pairs = h[kStatPairs];
        st->band_pairs = h[kStatBand];
        st->band_mismatch = h[kStatMismatch];
        st->device_error = (uint32_t)h[kStatError];
        st->launches = g->g.launches;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, g->t0, g->t1);
        st->kernel_ms = ms;
        st->pruned_pairs = h[kStatPruned];
    }
    if (h[kStatError] & kErrWaitTimeout) return ctx->fail(TPCF_ETIMEOUT, "a bounded device wait timed out");
    if (h[kStatError]) return ctx->fail(TPCF_ECUDA, "device error word 0x%llx", h[kStatError]);
    return TPCF_OK;
}

extern "C" int tpcf_graph_destroy(tpcf_graph* g) {
    if (!g) return TPCF_EINVAL;
    if (g->ctx) cudaSetDevice(g->ctx->cfg.device);
    if (g->launched && g->t1) cudaEventSynchronize(g->t1);
    if (g->g.exec) cudaGraphExecDestroy(g->g.exec);
    if (g->g.buf) cudaFree(g->g.buf);
    if (g->t0) cudaEventDestroy(g->t0);
    if (g->t1) cudaEventDestroy(g->t1);
    if (g->copy_st) cudaStreamDestroy(g->copy_st);
    delete g;
    return TPCF_OK;
}

// ====================================================================== estimator
extern "C" int tpcf_estimate(const uint64_t* dd, const uint64_t* dr, const uint64_t* rr, int nbins,
                             uint64_t nd, uint64_t nr, int estimator, double* w) {
    if (!dd || !dr || !rr || !w || nbins < 1 || nd < 2 || nr < 2 || nd > 0xffffffffull ||
        nr > 0xffffffffull)
        return TPCF_EINVAL;
    if (estimator != TPCF_LS_EXACT && estimator != TPCF_LS_PAPER) return TPCF_EINVAL;
    // Denominators from exact integer pair counts (nd, nr < 2^32 keeps them exact in uint64).
    const double p_dd = (double)(nd * (nd - 1) / 2);
    const double p_rr = (double)(nr * (nr - 1) / 2);
    const double p_dr = (double)nd * (double)nr;
    const double q = (double)nr / (double)nd;
    for (int k = 0; k < nbins; ++k) {
        if (rr[k] == 0) { w[k] = NAN; continue; }
        if (estimator == TPCF_LS_EXACT) {
            const double n_dd = (double)dd[k] / p_dd;
            const double n_rr = (double)rr[k] / p_rr;
            const double n_dr = (double)dr[k] / p_dr;
            w[k] = ((n_dd - 2.0 * n_dr) + n_rr) / n_rr;
        } else {
            const double dd2 = 2.0 * (double)dd[k];
            const double rr2 = 2.0 * (double)rr[k];
            w[k] = (1.0 + (q * q) * (dd2 / rr2)) - ((2.0 * q) * ((double)dr[k] / rr2));
        }
    }
    return TPCF_OK;
}

extern "C" int tpcf_correlate(tpcf_ctx* ctx, const double* d_xyz, uint64_t nd, const double* r_xyz,
                              uint64_t nr, const double* edges, int nedges, int estimator,
                              void* stream, uint64_t* dd, uint64_t* dr, uint64_t* rr, double* w,
                              tpcf_stats* st) {
    if (!ctx) return TPCF_EINVAL;
    if (!edges_valid(edges, nedges)) return ctx->fail(TPCF_EINVAL, "bad edges");
    tpcf_catalog *cd = nullptr, *cr = nullptr;
    tpcf_bins* b = nullptr;
    std::vector<uint64_t> hdd(nedges + 1), hdr(nedges + 1), hrr(nedges + 1);
    int rc = tpcf_catalog_create(ctx, d_xyz, nd, TPCF_HOST, stream, &cd);
    if (rc == TPCF_OK) rc = tpcf_catalog_create(ctx, r_xyz, nr, TPCF_HOST, stream, &cr);
    if (rc == TPCF_OK) rc = tpcf_bins_create(ctx, edges, nedges, &b);
    if (rc == TPCF_OK)
        rc = tpcf_count_all(ctx, cd, cr, b, stream, hdd.data(), hdr.data(), hrr.data(), TPCF_HOST, st);
    if (rc == TPCF_OK && w)
        rc = tpcf_estimate(hdd.data() + 1, hdr.data() + 1, hrr.data() + 1, nedges - 1, nd, nr,
                           estimator, w);
    if (rc == TPCF_OK) {
        if (dd) memcpy(dd, hdd.data(), hdd.size() * 8);
        if (dr) memcpy(dr, hdr.data(), hdr.size() * 8);
        if (rr) memcpy(rr, hrr.data(), hrr.size() * 8);
    }
    if (b) tpcf_bins_destroy(b);
    if (cd) tpcf_catalog_destroy(cd);
    if (cr) tpcf_catalog_destroy(cr);
    return rc;
}

// ====================================================================== host-side self checks
// Enumerates the items and tiles of one histogram exactly as the kernel does
// and adds 1 to counts[i * nb + j] for every pair (i, j) an item counts.
// Returns the number of items; *pairs receives the item_pairs total.
extern "C" int64_t tpcf_plan_coverage(uint32_t na, uint32_t nb, int auto_mode, uint32_t I,
                                      uint32_t Jc, uint32_t J, uint32_t shard_index,
                                      uint32_t shard_count, uint32_t* counts, uint64_t* pairs) {
    if (I == 0 || J == 0 || Jc == 0 || Jc % J != 0 || (I % Jc != 0 && Jc % I != 0)) return -1;
    if (auto_mode && na != nb) return -1;
    if (shard_count > 1 && shard_index >= shard_count) return -1;
    if (na == 0 || nb == 0) { if (pairs) *pairs = 0; return 0; }
    const uint32_t n_iblk = (na + I - 1) / I, n_jchunk = (nb + Jc - 1) / Jc;
    const uint64_t items = items_of(n_iblk, n_jchunk, auto_mode != 0, I, Jc);
    // the same split as the counting launch: items [items*s/S, items*(s+1)/S)
    uint64_t q_lo = 0, q_hi = items;
    if (shard_count > 1) {
        q_lo = items * shard_index / shard_count;
        q_hi = items * (shard_index + 1) / shard_count;
    }
    uint64_t total = 0;
    const uint64_t mult = walk_multiplier(items);
    for (uint64_t q = q_lo; q < q_hi; ++q) {
        ItemGeom g = item_geom(walk_item(q, items, mult), na, nb, n_iblk, n_jchunk, auto_mode != 0, I, Jc, J);
        if (g.t_first >= g.t_end) continue;
        total += item_pairs(g, na, nb, auto_mode != 0, I, Jc);
        if (!counts) continue;
        for (uint32_t t = g.t_first; t < g.t_end; ++t) {
            const uint32_t jbase = g.j0 + t * J;
            const bool masked = auto_mode && (jbase < g.i0 + I);  // as in the kernel
            for (uint32_t ii = 0; ii < I; ++ii) {
                const uint32_t i = g.i0 + ii;
                if (i >= na) break;
                for (uint32_t jj = 0; jj < J; ++jj) {
                    const uint32_t j = jbase + jj;
                    if (j >= nb) break;
                    if (masked && !(j > i)) continue;
                    counts[(uint64_t)i * nb + j] += 1;
                }
            }
        }
    }
    if (pairs) *pairs = total;
    return (int64_t)(q_hi - q_lo);
}
