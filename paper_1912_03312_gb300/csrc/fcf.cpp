// Faber-Caratheodory-Fejer poles and weights of exp on i[-R1, R1] (Rittich &
// Speck, arXiv:1912.03312, Sec. 3.2, Algorithms 1 and 2), computed on the host
// in double-double arithmetic.
//
// Same mathematics as the paper's construction, different numerical route
// (each step is checked against an independent arbitrary-precision oracle):
//  * Faber coefficients: for eta(z) = (R1/2)(z - 1/z) (Eq. (9)),
//    exp(eta(z)) = sum_n J_n(R1) z^n (Bessel generating function), so the a_j
//    of Eq. (8) are J_j(R1), computed by Miller's backward recurrence.
//  * Theorem 1 / Algorithm 1: the Hankel matrix H_ij = a_{i+j} is real
//    symmetric; its (K+1)-st singular pair comes from a cyclic Jacobi
//    eigendecomposition (singular value |lambda|, v = eigenvector,
//    u = sign(lambda) v).
//  * Roots of q(z) = v_{L+1} + v_L z + ... + v_1 z^L by Aberth-Ehrlich
//    iteration (double, then polished in double-double); z_1..z_K = outer roots.
//  * Laurent coefficients d_0..d_{K-1} of q_out r~* (Algorithm 1) without an
//    FFT: with q = v_1 q_out q_in (q_in = inner roots),
//    q_out r~* = q_out h - (sigma_{K+1}/v_1) z^L p / q_in, and p / q_in is
//    expanded at infinity by exact polynomial long division.
//  * Weights (Algorithm 2): instead of the K x K system in the Faber
//    coefficients of 1/(w - sigma_k), the Faber generating function
//    eta'(t)/(eta(t) - w) = sum_j p_j(w) t^{-j-1} maps each partial fraction
//    rho_k/(z - z_k) of r^cf to rho_k eta'(z_k)/(w - eta(z_k)), so
//    sigma_k = eta(z_k) and beta_k = rho_k eta'(z_k), rho_k = Res_{z_k} r^cf.
//    (This solves the same linear system in closed form.)
#include <algorithm>
#include <cmath>
#include <complex>
#include <map>
#include <mutex>
#include <vector>

#include "dd.h"
#include "fcf.h"

namespace rexi {

namespace {

typedef std::complex<double> cd;

// J_j(R), j = 0..L, by Miller's backward recurrence normalised with
// J_0 + 2 sum_k J_{2k} = 1.  T is double or dd.
template <typename T>
std::vector<T> bessel_miller(int L, double R) {
    int N = std::max(L, (int)std::ceil(R)) + 80;
    if (N % 2) ++N;
    std::vector<T> j(N + 2, T(0.0));
    j[N + 1] = T(0.0);
    j[N] = T(1e-200);
    const T Rt = T(R);
    for (int k = N; k >= 1; --k) {
        j[k - 1] = (T(2.0 * k) / Rt) * j[k] - j[k + 1];
        if (std::fabs((double)j[k - 1]) > 1e200) {
            for (int i = k - 1; i <= N; ++i) j[i] = j[i] * T(1e-200);
        }
    }
    T s = j[0];
    for (int k = 2; k <= N; k += 2) s = s + T(2.0) * j[k];
    std::vector<T> out(L + 1);
    for (int i = 0; i <= L; ++i) out[i] = j[i] / s;
    return out;
}

// Smallest L >= ceil(R)+2 with |J_{L+1}(R)|, |J_{L+2}(R)| below 1e-34: the
// truncation of Sec. 3.2.1 at the double-double precision level.
int truncation_length(double R) {
    int L = (int)std::ceil(R) + 2;
    for (;;) {
        std::vector<double> J = bessel_miller<double>(L + 2, R);
        if (std::fabs(J[L + 1]) < 1e-34 && std::fabs(J[L + 2]) < 1e-34) return L;
        ++L;
    }
}

// Cyclic Jacobi eigendecomposition of a symmetric n x n matrix (row-major).
// On return A holds the eigenvalues on its diagonal; V (if non-null) the
// eigenvectors as columns.
template <typename T>
void jacobi_eig(std::vector<T>& A, int n, std::vector<T>* V, double rel_tol, int max_sweeps = 40) {
    if (V) {
        V->assign((size_t)n * n, T(0.0));
        for (int i = 0; i < n; ++i) (*V)[(size_t)i * n + i] = T(1.0);
    }
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int p = 0; p < n; ++p) {
            double d = (double)A[(size_t)p * n + p];
            diag += d * d;
            for (int q = p + 1; q < n; ++q) {
                double a = (double)A[(size_t)p * n + q];
                off += a * a;
            }
        }
        if (off <= rel_tol * rel_tol * diag) break;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                T apq = A[(size_t)p * n + q];
                double apq_d = std::fabs((double)apq);
                if (apq_d == 0.0) continue;
                T app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                if (apq_d < rel_tol * 1e-3 * std::sqrt(diag / n)) {
                    A[(size_t)p * n + q] = A[(size_t)q * n + p] = T(0.0);
                    continue;
                }
                T theta = (aqq - app) / (T(2.0) * apq);
                T th_abs = (double)theta < 0.0 ? -theta : theta;
                T t = T(1.0) / (th_abs + sqrt_t(T(1.0) + theta * theta));
                if ((double)theta < 0.0) t = -t;
                T c = T(1.0) / sqrt_t(T(1.0) + t * t);
                T s = t * c;
                for (int k = 0; k < n; ++k) {
                    if (k == p || k == q) continue;
                    T akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    T nkp = c * akp - s * akq;
                    T nkq = s * akp + c * akq;
                    A[(size_t)k * n + p] = A[(size_t)p * n + k] = nkp;
                    A[(size_t)k * n + q] = A[(size_t)q * n + k] = nkq;
                }
                A[(size_t)p * n + p] = app - t * apq;
                A[(size_t)q * n + q] = aqq + t * apq;
                A[(size_t)p * n + q] = A[(size_t)q * n + p] = T(0.0);
                if (V) {
                    for (int k = 0; k < n; ++k) {
                        T vkp = (*V)[(size_t)k * n + p], vkq = (*V)[(size_t)k * n + q];
                        (*V)[(size_t)k * n + p] = c * vkp - s * vkq;
                        (*V)[(size_t)k * n + q] = s * vkp + c * vkq;
                    }
                }
            }
        }
    }
}

// ---- polynomial helpers (coefficients lowest degree first) ---------------

// p(z)/p'(z) for a complex-double polynomial; evaluates the reversed
// polynomial when |z| > 1 to avoid overflow.
cd newton_ratio(const std::vector<cd>& c, cd z) {
    const int L = (int)c.size() - 1;
    if (std::abs(z) <= 1.0) {
        cd p = c[L], dp = 0.0;
        for (int i = L - 1; i >= 0; --i) { dp = dp * z + p; p = p * z + c[i]; }
        return p / dp;
    }
    cd w = 1.0 / z;
    cd p = c[0], dp = 0.0;                  // reversed: P~(w) = sum c_{L-k} w^k
    for (int i = 1; i <= L; ++i) { dp = dp * w + p; p = p * w + c[i]; }
    return z / ((double)L - w * dp / p);
}

cdd newton_ratio_dd(const std::vector<cdd>& c, cdd z) {
    const int L = (int)c.size() - 1;
    if ((double)cabs(z) <= 1.0) {
        cdd p = c[L], dp(0.0);
        for (int i = L - 1; i >= 0; --i) { dp = dp * z + p; p = p * z + c[i]; }
        return p / dp;
    }
    cdd w = cdd(1.0) / z;
    cdd p = c[0], dp(0.0);
    for (int i = 1; i <= L; ++i) { dp = dp * w + p; p = p * w + c[i]; }
    return z / (cdd(dd((double)L)) - w * dp / p);
}

// All roots of a polynomial with real double-double coefficients by the
// Aberth-Ehrlich simultaneous iteration.  Returns false if it fails to converge.
bool aberth_roots(const std::vector<dd>& coef, std::vector<cdd>* roots) {
    const int L = (int)coef.size() - 1;
    std::vector<cd> c(L + 1);
    std::vector<cdd> cq(L + 1);
    for (int i = 0; i <= L; ++i) { c[i] = cd((double)coef[i], 0.0); cq[i] = cdd(coef[i]); }
    // initial guesses on a circle of the geometric-mean root radius
    double r0 = std::pow(std::fabs((double)coef[0] / (double)coef[L]), 1.0 / L);
    if (!(r0 > 0.0) || !std::isfinite(r0)) r0 = 1.0;
    std::vector<cd> z(L);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < L; ++i) z[i] = std::polar(r0, 2.0 * pi * i / L + 0.4);
    // Double-precision phase: stop at convergence or once progress stalls at
    // the double rounding floor (clustered roots stall earlier).
    double best = 1e300;
    int since_best = 0;
    for (int it = 0; it < 1000; ++it) {
        double maxrel = 0.0;
        for (int i = 0; i < L; ++i) {
            cd ratio = newton_ratio(c, z[i]);
            cd sum = 0.0;
            for (int j = 0; j < L; ++j) if (j != i) sum += 1.0 / (z[i] - z[j]);
            cd w = ratio / (1.0 - ratio * sum);
            z[i] -= w;
            maxrel = std::max(maxrel, std::abs(w) / std::max(std::abs(z[i]), 1e-300));
        }
        if (!std::isfinite(maxrel)) return false;
        if (maxrel < 1e-8) break;
        if (maxrel < 0.5 * best) { best = maxrel; since_best = 0; } else if (++since_best > 40 && best < 1e-3) break;
    }
    // Double-double phase (Gauss-Seidel Aberth updates) to ~32 digits.
    std::vector<cdd> zq(L);
    for (int i = 0; i < L; ++i) zq[i] = cdd(dd(z[i].real()), dd(z[i].imag()));
    double maxrel = 1.0;
    for (int it = 0; it < 400 && maxrel >= 1e-30; ++it) {
        maxrel = 0.0;
        for (int i = 0; i < L; ++i) {
            cdd ratio = newton_ratio_dd(cq, zq[i]);
            cdd sum(0.0);
            for (int j = 0; j < L; ++j) if (j != i) sum += cdd(1.0) / (zq[i] - zq[j]);
            cdd w = ratio / (cdd(1.0) - ratio * sum);
            zq[i] -= w;
            maxrel = std::max(maxrel, (double)cabs(w) / std::max((double)cabs(zq[i]), 1e-300));
        }
        if (!std::isfinite(maxrel)) return false;
    }
    if (!(maxrel < 1e-18)) return false;                    // clustered roots stall near 1e-22
    *roots = zq;
    return true;
}

// prod (z - r_i), lowest degree first.
std::vector<cdd> poly_from_roots(const std::vector<cdd>& r) {
    std::vector<cdd> p(1, cdd(1.0));
    for (const cdd& ri : r) {
        std::vector<cdd> nx(p.size() + 1, cdd(0.0));
        for (size_t i = 0; i < p.size(); ++i) {
            nx[i + 1] += p[i];
            nx[i] -= ri * p[i];
        }
        p.swap(nx);
    }
    return p;
}

double hankel_sigma_double(int K, double R) {
    int L = truncation_length(R);
    std::vector<double> a = bessel_miller<double>(L, R);
    int n = L + 1;
    std::vector<double> H((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; i + j <= L; ++j) H[(size_t)i * n + j] = a[i + j];
    jacobi_eig<double>(H, n, nullptr, 1e-15);
    std::vector<double> s(n);
    for (int i = 0; i < n; ++i) s[i] = std::fabs(H[(size_t)i * n + i]);
    std::sort(s.begin(), s.end(), [](double x, double y) { return x > y; });
    return K < n ? s[K] : 0.0;
}

}  // namespace

double sqrt_t(double x) { return std::sqrt(x); }
dd sqrt_t(dd x) { return dsqrt(x); }

int fcf_construct(int K, double R1, FcfResult* out) {
    if (K < 1 || !(R1 > 0.0) || !std::isfinite(R1)) return -1;
    const int L = std::max(truncation_length(R1), K + 2);
    const int n = L + 1;
    std::vector<dd> a = bessel_miller<dd>(L, R1);

    // Theorem 1 / Algorithm 1: Hankel matrix and its (K+1)-st singular pair.
    std::vector<dd> H((size_t)n * n, dd(0.0)), Q;
    for (int i = 0; i < n; ++i)
        for (int j = 0; i + j <= L; ++j) H[(size_t)i * n + j] = a[i + j];
    jacobi_eig<dd>(H, n, &Q, 1e-33);
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int x, int y) {
        return std::fabs((double)H[(size_t)x * n + x]) > std::fabs((double)H[(size_t)y * n + y]);
    });
    if (K >= n) return -6;
    const int idx = order[K];
    const dd lam = H[(size_t)idx * n + idx];
    const dd s = dabs(lam);
    const double s1 = std::fabs((double)H[(size_t)order[0] * n + order[0]]);
    const double sK = std::fabs((double)H[(size_t)order[K - 1] * n + order[K - 1]]);
    if (std::fabs(sK - (double)s) <= 1e-28 * s1) return -6;   // non-unique CF approximant
    const double sgn = lam.hi >= 0.0 ? 1.0 : -1.0;
    std::vector<dd> v(n), u(n);
    for (int i = 0; i < n; ++i) { v[i] = Q[(size_t)i * n + idx]; u[i] = v[i] * dd(sgn); }
    // q(z) = v_{L+1} + v_L z + ... + v_1 z^L (lowest first); p(z) = sum u_{i+1} z^i.
    std::vector<dd> q(n);
    for (int i = 0; i < n; ++i) q[i] = v[L - i];

    std::vector<cdd> roots;
    if (!aberth_roots(q, &roots)) return -6;
    std::vector<cdd> outer, inner;
    for (const cdd& r : roots) {
        double m = (double)cabs(r);
        if (std::fabs(m - 1.0) < 1e-8) return -6;               // root on the unit circle
        (m > 1.0 ? outer : inner).push_back(r);
    }
    if ((int)outer.size() != K) return -6;
    std::sort(outer.begin(), outer.end(), [](const cdd& x, const cdd& y) {
        double ix = (double)x.im, iy = (double)y.im;
        return ix < iy || (ix == iy && (double)x.re < (double)y.re);
    });
    const std::vector<cdd> qout = poly_from_roots(outer);    // degree K, monic
    const std::vector<cdd> qin = poly_from_roots(inner);     // degree M = L - K, monic
    const int M = L - K;

    // Laurent coefficients of z^L p(z)/q_in(z) at infinity: e_i, i = K .. -L.
    std::vector<cdd> e(K + L + 1, cdd(0.0));                  // e[i + L]
    for (int i = K; i >= -L; --i) {
        cdd acc = (i + M >= 0 && i + M <= L) ? cdd(u[i + M]) : cdd(0.0);
        for (int l = 0; l < M; ++l) {
            int idx2 = i + M - l;
            if (idx2 <= K) acc -= qin[l] * e[idx2 + L];
        }
        e[i + L] = acc;
    }
    const dd scale = s / v[0];                                // sigma_{K+1} / v_1
    std::vector<cdd> d(K);
    for (int j = 0; j < K; ++j) {
        cdd acc(0.0);
        for (int l = 0; l <= std::min(j, K); ++l) acc += qout[l] * cdd(a[j - l]);
        acc -= e[j] * scale;                                   // e_{j-L} is stored at e[j]
        d[j] = acc;
    }

    // Algorithm 2 in closed form: sigma_k = eta(z_k), beta_k = Res r^cf * eta'(z_k).
    const dd half_R(0.5 * R1);
    out->sigma.resize(K);
    out->beta.resize(K);
    out->z.resize(K);
    double min_re = 1e300;
    for (int k = 0; k < K; ++k) {
        const cdd zk = outer[k];
        cdd Nk(0.0);
        for (int j = K - 1; j >= 0; --j) Nk = Nk * zk + d[j];
        cdd den(1.0);
        for (int l = 0; l < K; ++l) if (l != k) den *= (zk - outer[l]);
        const cdd rho = Nk / den;
        const cdd inv = cdd(1.0) / zk;
        const cdd eta = (zk - inv) * half_R;
        const cdd etap = (cdd(1.0) + inv * inv) * half_R;
        const cdd beta = rho * etap;
        out->sigma[k] = std::complex<double>((double)eta.re, (double)eta.im);
        out->beta[k] = std::complex<double>((double)beta.re, (double)beta.im);
        out->z[k] = std::complex<double>((double)zk.re, (double)zk.im);
        min_re = std::min(min_re, std::fabs((double)eta.re));
    }
    out->K = K;
    out->R1 = R1;
    out->L = L;
    out->sigma_K1 = (double)s;
    out->min_re_sigma = min_re;
    // amplification A = max_w sum |beta| / |w - sigma| over w in i[-R1, R1]
    double A = 0.0;
    const int S = 4001;
    for (int i = 0; i < S; ++i) {
        cd w(0.0, -R1 + 2.0 * R1 * i / (S - 1));
        double acc = 0.0;
        for (int k = 0; k < K; ++k) acc += std::abs(out->beta[k]) / std::abs(w - out->sigma[k]);
        A = std::max(A, acc);
    }
    out->amplification = A;
    if (min_re < 1.0) return -6;                               // spurious near-axis pole
    // Self-check of the construction: r(i w) must approximate e^{i w} on the
    // interval to about 2 sigma_{K+1} (Theorem 1) plus the FP64 evaluation floor
    // eps * A.  A construction whose cancellations exceeded double-double
    // precision (large K) fails here instead of returning wrong weights.
    double emax = 0.0;
    for (int i = 0; i < S; ++i) {
        const double w = -R1 + 2.0 * R1 * i / (S - 1);
        cd r = 0.0;
        for (int k = 0; k < K; ++k) r += out->beta[k] / (cd(0.0, w) - out->sigma[k]);
        emax = std::max(emax, std::abs(r - std::exp(cd(0.0, w))));
    }
    if (!(emax <= 10.0 * (2.0 * out->sigma_K1 + 4e-16 * A) + 1e-12)) return -6;
    for (int k = 0; k < K; ++k)
        if (!std::isfinite(out->beta[k].real()) || !std::isfinite(out->beta[k].imag())) return -6;
    return 0;
}

double fcf_default_R1(int K, double eps_target) {
    if (!(eps_target > 0.0)) eps_target = 1e-9;
    // 2 sigma_{K+1}(R) grows with R for fixed K: bracket and bisect.
    double lo = 0.5, hi = std::max(2.0, 1.2 * K);
    int guard = 0;
    while (2.0 * hankel_sigma_double(K, hi) <= eps_target && guard++ < 40) { lo = hi; hi *= 1.3; }
    guard = 0;
    while (2.0 * hankel_sigma_double(K, lo) > eps_target && guard++ < 40) lo *= 0.7;
    for (int it = 0; it < 30 && hi - lo > 1e-3; ++it) {
        double mid = 0.5 * (lo + hi);
        if (2.0 * hankel_sigma_double(K, mid) <= eps_target) lo = mid; else hi = mid;
    }
    return lo >= 2.0 ? std::floor(lo) : std::floor(lo * 10.0) / 10.0;
}

int fcf_cached(int K, double R1, FcfResult* out) {
    static std::mutex mu;
    static std::map<std::pair<int, double>, std::pair<int, FcfResult>> cache;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(std::make_pair(K, R1));
        if (it != cache.end()) { *out = it->second.second; return it->second.first; }
    }
    FcfResult r;
    int st = fcf_construct(K, R1, &r);
    std::lock_guard<std::mutex> lk(mu);
    cache[std::make_pair(K, R1)] = std::make_pair(st, r);
    *out = r;
    return st;
}

double fcf_default_R1_cached(int K, double eps_target) {
    static std::mutex mu;
    static std::map<std::pair<int, double>, double> cache;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(std::make_pair(K, eps_target));
        if (it != cache.end()) return it->second;
    }
    double R = fcf_default_R1(K, eps_target);
    std::lock_guard<std::mutex> lk(mu);
    cache[std::make_pair(K, eps_target)] = R;
    return R;
}

std::vector<double> bessel_j(int L, double R) {
    std::vector<dd> j = bessel_miller<dd>(L, R);
    std::vector<double> out(L + 1);
    for (int i = 0; i <= L; ++i) out[i] = (double)j[i];
    return out;
}

}  // namespace rexi
