// Host-side support of libwdb: errors, launch counter, subband layout, Daubechies filters.
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "wdb_internal.h"

namespace wdb {

static thread_local std::string t_err;
static std::atomic<long long> g_launches{0};

wdb_status set_error(wdb_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return s;
}

wdb_status cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    return set_error(e == cudaErrorMemoryAllocation ? WDB_ENOMEM : WDB_ECUDA, "%s failed: %s (%s:%d)",
                     what, cudaGetErrorString(e), file, line);
}

void count_launch(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static int current_device_bit() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
    return dev;
}

bool done_on_device(const unsigned long long* mask) {
    const int d = current_device_bit();
    return d >= 0 && ((__atomic_load_n(mask, __ATOMIC_ACQUIRE) >> d) & 1ull);
}

void mark_on_device(unsigned long long* mask) {
    const int d = current_device_bit();
    if (d >= 0) __atomic_fetch_or(mask, 1ull << d, __ATOMIC_ACQ_REL);
}

long long launches(int reset) {
    long long v = reset ? g_launches.exchange(0) : g_launches.load();
    return v;
}

const char* last_error() { return t_err.c_str(); }

// ---------------------------------------------------------------------------------------
// Layout (Sec. 2: separable isotropic basis; planar order documented in wdb.h)
// ---------------------------------------------------------------------------------------
wdb_status make_layout(int n_rows, int n_cols, int J, Layout* out) {
    if (J < 1) return set_error(WDB_EINVAL, "levels must be >= 1 (got %d)", J);
    if (3 * J + 1 > kMaxS) return set_error(WDB_EUNSUPPORTED, "at most %d subbands", kMaxS);
    if (J > 12) return set_error(WDB_EUNSUPPORTED, "levels must be <= 12");
    if (n_rows <= 0 || n_cols <= 0) return set_error(WDB_EINVAL, "image sides must be positive");
    if ((n_rows % (1 << J)) || (n_cols % (1 << J)))
        return set_error(WDB_EINVAL, "image %dx%d not divisible by 2^%d", n_rows, n_cols, J);
    if ((long long)n_rows * n_cols > (1LL << 31) - 1)
        return set_error(WDB_EUNSUPPORTED, "images above 2^31 pixels are not supported");
    Layout L;
    L.n_rows = n_rows;
    L.n_cols = n_cols;
    L.J = J;
    L.S = 3 * J + 1;
    long long off = 0;
    int tab = 0;
    auto add = [&](int idx, int s) {
        SubbandDev& b = L.sb[idx];
        b.off = off;
        b.rows = n_rows >> s;
        b.cols = n_cols >> s;
        b.level = s;
        b.lgR = J - s;
        b.tab_off = tab;
        b.pad = 0;
        off += (long long)b.rows * b.cols;
        tab += 1 << (2 * (J - s));
    };
    add(0, J);
    int idx = 1;
    for (int s = J; s >= 1; --s)
        for (int e = 0; e < 3; ++e) add(idx++, s);
    L.N = off;
    L.tab_len = tab;
    *out = L;
    return WDB_OK;
}

Schedule make_schedule(const Layout& L) {
    Schedule s;
    s.vb_start.resize(L.S + 1);
    int v = 0;
    for (int b = 0; b < L.S; ++b) {
        s.vb_start[b] = v;
        long long n = (long long)L.sb[b].rows * L.sb[b].cols;
        v += (int)((n + kVB - 1) / kVB);
    }
    s.vb_start[L.S] = v;
    s.nvb = v;
    return s;
}

// ---------------------------------------------------------------------------------------
// Daubechies filters: spectral factorisation of
//   |m0(w)|^2 = cos^{2p}(w/2) P(sin^2(w/2)),  P(y) = sum_{k<p} C(p-1+k, k) y^k,
// keeping for every root of P the zero of H(Z) = sum_k h[k] Z^-k inside the unit circle
// (minimum phase), normalised to sum h = sqrt(2). Roots by Durand-Kerner with Newton
// polishing in long double.
// ---------------------------------------------------------------------------------------
using cld = std::complex<long double>;

static cld poly_eval(const std::vector<long double>& c_hi, cld x) {  // highest power first
    cld r = 0;
    for (long double c : c_hi) r = r * x + c;
    return r;
}

static cld poly_deriv_eval(const std::vector<long double>& c_hi, cld x) {
    int n = (int)c_hi.size() - 1;
    cld r = 0;
    for (int i = 0; i < n; ++i) r = r * x + c_hi[i] * (long double)(n - i);
    return r;
}

static std::vector<cld> poly_roots(const std::vector<long double>& c_hi) {
    int n = (int)c_hi.size() - 1;
    std::vector<cld> z(n);
    if (n <= 0) return z;
    std::vector<long double> mon(c_hi);
    for (auto& c : mon) c /= c_hi[0];
    cld seed(0.4L, 0.9L), p = 1;
    for (int i = 0; i < n; ++i) {
        p *= seed;
        z[i] = p;
    }
    for (int it = 0; it < 2000; ++it) {
        long double delta = 0;
        for (int i = 0; i < n; ++i) {
            cld den = 1;
            for (int j = 0; j < n; ++j)
                if (j != i) den *= (z[i] - z[j]);
            cld step = poly_eval(mon, z[i]) / den;
            z[i] -= step;
            delta = std::max(delta, std::abs(step));
        }
        if (delta < 1e-30L) break;
    }
    for (auto& r : z)
        for (int it = 0; it < 8; ++it) {
            cld d = poly_deriv_eval(mon, r);
            if (std::abs(d) == 0) break;
            r -= poly_eval(mon, r) / d;
        }
    return z;
}

static long double binom(int n, int k) {
    long double r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

static wdb_status daubechies(int p, Filters* f) {
    if (p < 1 || 2 * p > kMaxL) return set_error(WDB_EINVAL, "db%d not supported (db1..db10)", p);
    std::vector<long double> P_hi(p);
    for (int k = 0; k < p; ++k) P_hi[p - 1 - k] = binom(p - 1 + k, k);
    std::vector<cld> yr = poly_roots(P_hi);
    std::vector<cld> poly{cld(1)};
    auto mul = [&](cld a0, cld a1) {  // multiply by (a0 Z + a1)
        std::vector<cld> out(poly.size() + 1, cld(0));
        for (size_t i = 0; i < poly.size(); ++i) {
            out[i] += poly[i] * a0;
            out[i + 1] += poly[i] * a1;
        }
        poly.swap(out);
    };
    for (int i = 0; i < p; ++i) mul(1, 1);
    for (cld y : yr) {
        cld b = 2.0L - 4.0L * y;
        cld disc = std::sqrt(b * b - 4.0L);
        cld z1 = (b + disc) / 2.0L, z2 = (b - disc) / 2.0L;
        cld z = std::abs(z1) < 1.0L ? z1 : z2;
        mul(1, -z);
    }
    long double s = 0;
    for (auto& c : poly) s += c.real();
    long double scale = std::sqrt(2.0L) / s;
    f->L = 2 * p;
    for (int k = 0; k < kMaxL; ++k) f->h[k] = f->g[k] = 0.0;
    for (int k = 0; k < f->L; ++k) f->h[k] = (double)(poly[k].real() * scale);
    for (int k = 0; k < f->L; ++k) f->g[k] = ((k & 1) ? -1.0 : 1.0) * f->h[f->L - 1 - k];
    return WDB_OK;
}

// ---------------------------------------------------------------------------------------
// Symlets: the same |m0(w)|^2 as db<p>, but for every real root of P, and every complex-
// conjugate pair of roots, the zero of H(Z) may sit inside or outside the unit circle; the
// combination whose phase arg H(e^{iw}) is closest to a straight line (least squares over
// w_k = pi (k + 1/2) / 2048) is the least asymmetric filter. A filter and its time reverse
// tie (deviations within 1e-6 of each other); the one with the smaller energy centroid
// sum_k k h[k]^2 is kept.
// ---------------------------------------------------------------------------------------
// phase of prod_j (e^{iw} - z_j) summed factor by factor (each factor's phase is continuous
// in w: no zero lies on the unit circle but the zeros at -1, whose factor's phase is w/2 on
// [0, pi)), and its squared deviation from the least-squares line
static double phase_deviation(const std::vector<cld>& zeros) {
    constexpr int M = 2048;
    const long double pi = 3.141592653589793238462643383279502884L;
    std::vector<long double> ph(M, 0.0L), w(M);
    for (int k = 0; k < M; ++k) w[k] = pi * (k + 0.5L) / M;
    for (const cld& z : zeros) {
        long double prev = 0;
        for (int k = 0; k < M; ++k) {
            long double a = std::arg(std::polar(1.0L, w[k]) - z);
            if (k > 0) {
                while (a - prev > pi) a -= 2 * pi;
                while (a - prev < -pi) a += 2 * pi;
            }
            ph[k] += a;
            prev = a;
        }
    }
    long double sw = 0, sp = 0, sww = 0, swp = 0;
    for (int k = 0; k < M; ++k) {
        sw += w[k];
        sp += ph[k];
        sww += w[k] * w[k];
        swp += w[k] * ph[k];
    }
    const long double slope = (M * swp - sw * sp) / (M * sww - sw * sw);
    const long double icpt = (sp - slope * sw) / M;
    long double dev = 0;
    for (int k = 0; k < M; ++k) {
        const long double e = ph[k] - slope * w[k] - icpt;
        dev += e * e;
    }
    return (double)dev;
}

static wdb_status symlet(int p, Filters* f) {
    if (p < 1 || 2 * p > kMaxL) return set_error(WDB_EINVAL, "sym%d not supported (sym1..sym10)", p);
    std::vector<long double> P_hi(p);
    for (int k = 0; k < p; ++k) P_hi[p - 1 - k] = binom(p - 1 + k, k);
    std::vector<cld> yr = poly_roots(P_hi);
    struct Group {
        cld zin, zout;
        bool pair;
    };
    std::vector<Group> groups;
    for (cld y : yr) {
        const bool real = std::fabs(y.imag()) <= 1e-10L * std::max(1.0L, std::abs(y));
        if (!real && y.imag() < 0) continue;   // the conjugate's group holds it
        if (real) y = cld(y.real(), 0);
        cld b = 2.0L - 4.0L * y;
        cld disc = std::sqrt(b * b - 4.0L);
        cld z1 = (b + disc) / 2.0L, z2 = (b - disc) / 2.0L;
        if (std::abs(z1) < 1.0L) groups.push_back({z1, z2, !real});
        else groups.push_back({z2, z1, !real});
    }
    double best_dev = 0, best_cen = 0;
    std::vector<long double> best;
    for (unsigned mask = 0; mask < (1u << groups.size()); ++mask) {
        std::vector<cld> poly{cld(1)};
        auto mul = [&](cld a1) {   // multiply by (Z + a1)
            std::vector<cld> out(poly.size() + 1, cld(0));
            for (size_t i = 0; i < poly.size(); ++i) {
                out[i] += poly[i];
                out[i + 1] += poly[i] * a1;
            }
            poly.swap(out);
        };
        std::vector<cld> zeros(p, cld(-1));
        for (int i = 0; i < p; ++i) mul(1);
        for (size_t gi = 0; gi < groups.size(); ++gi) {
            const cld z = ((mask >> gi) & 1u) ? groups[gi].zout : groups[gi].zin;
            mul(-z);
            zeros.push_back(z);
            if (groups[gi].pair) {
                mul(-std::conj(z));
                zeros.push_back(std::conj(z));
            }
        }
        long double sum = 0;
        for (auto& c : poly) sum += c.real();
        std::vector<long double> h(poly.size());
        for (size_t k = 0; k < poly.size(); ++k) h[k] = poly[k].real() * std::sqrt(2.0L) / sum;
        const double dev = phase_deviation(zeros);
        long double cen = 0;
        for (size_t k = 0; k < h.size(); ++k) cen += (long double)k * h[k] * h[k];
        const bool better = best.empty() || dev < best_dev * (1 - 1e-6) ||
                            (std::fabs(dev - best_dev) <= 1e-6 * best_dev && (double)cen < best_cen);
        if (better) {
            best = h;
            best_dev = dev;
            best_cen = (double)cen;
        }
    }
    f->L = 2 * p;
    for (int k = 0; k < kMaxL; ++k) f->h[k] = f->g[k] = 0.0;
    for (int k = 0; k < f->L; ++k) f->h[k] = (double)best[k];
    for (int k = 0; k < f->L; ++k) f->g[k] = ((k & 1) ? -1.0 : 1.0) * f->h[f->L - 1 - k];
    return WDB_OK;
}

static wdb_status derive_filters(const char* name, Filters* out) {
    const bool db = std::strncmp(name, "db", 2) == 0, sym = std::strncmp(name, "sym", 3) == 0;
    if (!db && !sym) return set_error(WDB_EINVAL, "unknown wavelet '%s'", name);
    const char* num = name + (db ? 2 : 3);
    char* end = nullptr;
    long p = std::strtol(num, &end, 10);
    if (end == num || *end != '\0') return set_error(WDB_EINVAL, "unknown wavelet '%s'", name);
    return db ? daubechies((int)p, out) : symlet((int)p, out);
}

// The spectral factorisation runs once per wavelet name per process (the result depends on
// the name only); later calls copy the cached filters.
wdb_status wavelet_filters(const char* name, Filters* out) {
    if (!name) return set_error(WDB_EINVAL, "wavelet name is NULL");
    static std::mutex mu;
    static std::map<std::string, Filters> cache;
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(name);
        if (it != cache.end()) {
            *out = it->second;
            return WDB_OK;
        }
    }
    Filters f;
    WDB_TRY(derive_filters(name, &f));
    std::lock_guard<std::mutex> lock(mu);
    cache.emplace(name, f);
    *out = f;
    return WDB_OK;
}

}  // namespace wdb
