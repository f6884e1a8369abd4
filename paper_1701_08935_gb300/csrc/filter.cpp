// Host construction of the Zolotarev-composite filter R_ab (the filter-construction steps of Algorithm 2).
//
//  * Moebius map T(x) = gamma (x - alpha)/(x - beta) with T(a-) = -1, T(a+) = 1,
//    T(b-) = l1, T(b+) = -l1 (eq. req).  l1 from cross-ratio invariance; alpha, beta,
//    gamma in closed form from the three conditions at a+, b-, b+.
//  * Theorem 1 (eq. ZoloFunc, eq. coef): c_j = l^2 sn^2(jK'/2r; l') / cn^2(jK'/2r; l').
//    Only j <= r is evaluated through the elliptic functions; the others follow from
//    the reflection sc(K' - u; l') = 1/(l sc(u; l')), i.e. c_j c_{2r-j} = l^2, which
//    keeps cn away from its zero at K'.  Elliptic functions: arithmetic-geometric mean
//    with the descending recurrence of Abramowitz & Stegun 16.4.  Accuracy of c_j
//    (against 40-digit references): <= 1e-12 relative for l >= 1e-4, <= 1e-11 for
//    l >= 1e-6, ~2e-10 at l = 5e-8 (the asin steps near u ~ K'/2 lose digits as l -> 0).
//  * M from the equioscillation (Theorem 1 and the remark after it): Z is smallest on
//    [l, 1] at x_1 = l and largest at x_2 = l / dn(K'/2r; l'), and min + max = 2.
//  * Proposition 1 weights a_j, written here as residues of Z/(Mx) at x^2 = -c_{2j-1}.
//  * Proposition 2 poles and weights of Zhat(T(x)); Corollary 1 for the outer shifts.
#include <cmath>
#include <cstring>
#include <algorithm>
#include "zolo_internal.h"

namespace zolo {

namespace {

// Jacobi sn, cn, dn for modulus k with complementary modulus kc = sqrt(1 - k^2)
// given separately (kc may be tiny when k ~ 1).  A&S 16.4 AGM.
void jacobi(double u, double k, double kc, double &sn, double &cn, double &dn, double &K) {
    double a[40], c[40];
    double aa = 1.0, bb = kc;
    a[0] = 1.0;
    c[0] = k;
    int n = 0;
    while (n < 38) {
        double an = 0.5 * (aa + bb);
        double bn = std::sqrt(aa * bb);
        double cn_ = 0.5 * (aa - bb);
        ++n;
        a[n] = an;
        c[n] = cn_;
        aa = an;
        bb = bn;
        if (std::fabs(cn_) <= 1e-17 * an) break;
    }
    K = M_PI / (2.0 * a[n]);
    double phi = std::ldexp(a[n] * u, n);
    for (int i = n; i >= 1; --i) {
        double s = c[i] * std::sin(phi) / a[i];
        s = std::max(-1.0, std::min(1.0, s));
        phi = 0.5 * (phi + std::asin(s));
    }
    sn = std::sin(phi);
    cn = std::cos(phi);
    dn = std::sqrt(cn * cn + kc * kc * sn * sn);
}

double complete_K(double k, double kc) {
    double sn, cn, dn, K;
    jacobi(0.0, k, kc, sn, cn, dn, K);
    return K;
}

double unscaled(const std::vector<double> &c, double x) {
    const int r = (int)(c.size() + 1) / 2;
    double v = x;
    const double x2 = x * x;
    for (int j = 1; j < r; ++j) v *= (x2 + c[2 * j - 1]);
    for (int j = 1; j <= r; ++j) v /= (x2 + c[2 * j - 2]);
    return v;
}

}  // namespace

double Zolo::operator()(double x) const { return M * unscaled(c, x); }

int zolo_build(int r, double ell, Zolo &z) {
    if (r < 1 || r > ZOLO_MAX_R * ZOLO_MAX_R * 4 || !(ell > 0.0 && ell < 1.0))
        return set_error(ZOLO_EINVAL, "Zolotarev order or parameter out of range");
    z.r = r;
    z.ell = ell;
    const double ellp = std::sqrt((1.0 - ell) * (1.0 + ell));     // modulus l'
    const double Kp = complete_K(ellp, ell);                      // K' = K(l')
    z.c.assign(2 * r - 1, 0.0);
    for (int j = 1; j <= r; ++j) {
        double sn, cn, dn, K;
        jacobi(j * Kp / (2.0 * r), ellp, ell, sn, cn, dn, K);
        double t = sn / cn;
        z.c[j - 1] = ell * ell * t * t;
    }
    for (int j = r + 1; j <= 2 * r - 1; ++j) z.c[j - 1] = ell * ell / z.c[2 * r - j - 1];
    z.c[r - 1] = ell;                                             // c_r = l exactly
    // extrema on [l, 1]: x_1 = l (minimum), x_2 = l / dn(K'/2r; l') (maximum)
    double sn, cn, dn, K;
    jacobi(Kp / (2.0 * r), ellp, ell, sn, cn, dn, K);
    const double x2 = ell / dn;
    const double fmin = unscaled(z.c, ell), fmax = unscaled(z.c, x2);
    z.M = 2.0 / (fmin + fmax);
    z.zmax = z.M * fmax;
    z.delta = (fmax - fmin) / (fmax + fmin);
    // Proposition 1 weights as residues: a_j = prod_{k<r}(c_2k - c_{2j-1}) / prod_{k!=j}(c_{2k-1} - c_{2j-1})
    z.a.assign(r, 0.0);
    for (int j = 1; j <= r; ++j) {
        const double cj = z.c[2 * j - 2];
        double num = 1.0, den = 1.0;
        for (int k = 1; k < r; ++k) num *= (z.c[2 * k - 1] - cj);
        for (int k = 1; k <= r; ++k)
            if (k != j) den *= (z.c[2 * k - 2] - cj);
        z.a[j - 1] = num / den;
    }
    return ZOLO_OK;
}

}  // namespace zolo

double zolo_filter_s::eval(double x) const {
    if (kind != ZOLO_FILTER_ZOLO) {
        // contour filters: sum over the conjugate point pairs of 2 Re(w_j / (x - sigma_j))
        double v = 0.0;
        for (int j = 0; j < info.r1; ++j) {
            const zolo::cplx w(info.w_hat[2 * j], info.w_hat[2 * j + 1]);
            const zolo::cplx sg(info.sigma_hat[2 * j], info.sigma_hat[2 * j + 1]);
            v += 2.0 * (w / (x - sg)).real();
        }
        return v;
    }
    // R_ab(x) = (Z_2r2(Zhat_2r1(T(x); l1); l2) + 1)/2;  T(beta) = inf maps to Zhat = 0
    double zi;
    if (x == beta) {
        zi = 0.0;
    } else {
        const double t = gamma * (x - alpha) / (x - beta);
        zi = inner(t) / inner.zmax;
    }
    return 0.5 * (outer(zi) + 1.0);
}

extern "C" {

int zolo_filter_build(const zolo_filter_spec *spec, zolo_filter *out) {
    using namespace zolo;
    clear_error();
    if (!spec || !out) return set_error(ZOLO_EINVAL, "null argument");
    *out = nullptr;
    const double am = spec->a_minus, ap = spec->a_plus, bm = spec->b_minus, bp = spec->b_plus;
    const bool am_inf = std::isinf(am) && am < 0;
    if (!(std::isfinite(ap) && std::isfinite(bm) && std::isfinite(bp) && (am_inf || std::isfinite(am))))
        return set_error(ZOLO_EINVAL, "gap ends must be finite (a- may be -inf)");
    if (!((am_inf || am < ap) && ap < bm && bm < bp))
        return set_error(ZOLO_EINVAL, "need a- < a+ < b- < b+");
    int r1 = spec->r1, r2 = spec->r2;
    const bool auto_r = (r1 <= 0 || r2 <= 0);
    if (r1 > ZOLO_MAX_R || r2 > ZOLO_MAX_R) return set_error(ZOLO_EINVAL, "r1, r2 must be <= ZOLO_MAX_R");
    if (auto_r && !(spec->eps > 0.0 && spec->eps < 0.5))
        return set_error(ZOLO_EINVAL, "automatic order needs 0 < eps < 0.5");

    auto *F = new zolo_filter_s();
    F->spec = *spec;
    // ---- eq. req: cross ratio (b- - a-)(b+ - a+)/((b- - a+)(b+ - a-)) = ((1+l1)/(1-l1))^2.
    // kcr - 1 = (a+ - a-)(b+ - b-)/((b- - a+)(b+ - a-)) exactly; with a- = -inf it is
    // (b+ - b-)/(b- - a+).
    const double gb = bp - bm, s = bm - ap;
    const double km1 = am_inf ? gb / s : (ap - am) * gb / (s * (bp - am));
    const double sq = std::sqrt(1.0 + km1);
    const double l1 = km1 / ((sq + 1.0) * (sq + 1.0));
    // T(x) = G - C/(x - beta) with G = gamma, C = gamma (alpha - beta).  The conditions at
    // b-, b+ and a+ give  gb (a+ - beta) = rho s (b+ - beta),  rho = 2 l1/(1 - l1).
    const double rho = 2.0 * l1 / (1.0 - l1);
    const double beta = (rho * s * bp - gb * ap) / (rho * s - gb);
    const double C = -2.0 * l1 * (bp - beta) * (bm - beta) / gb;
    const double G = l1 + C / (bm - beta);
    F->ell1 = l1;
    F->beta = beta;
    F->gamma = G;
    F->alpha = beta + C / G;

    auto build_pair = [&](int ri, int ro) -> int {
        int st = zolo_build(ri, F->ell1, F->inner);
        if (st) return st;
        F->ell2 = F->inner(F->ell1) / F->inner.zmax;              // l2 = Zhat(l1; l1)
        // an inner function exact to rounding gives l2 = 1; keep the outer one defined
        F->ell2 = std::min(F->ell2, 1.0 - 0x1p-50);
        st = zolo_build(ro, F->ell2, F->outer);
        if (st) return st;
        F->delta0 = 0.5 * F->outer.delta;                         // (1 - S(l1))/2
        return ZOLO_OK;
    };
    int st = ZOLO_OK;
    if (auto_r) {
        // Remark after Algorithm 2: the error (1 - S(l1; l1))/2 needs no matrix, so walk the
        // free order(s) upwards until it is <= eps
        const int fix1 = r1 > 0 ? r1 : 0, fix2 = r2 > 0 ? r2 : 0;
        int r = 1;
        for (; r <= ZOLO_MAX_R; ++r) {
            st = build_pair(fix1 ? fix1 : r, fix2 ? fix2 : r);
            if (st) break;
            if (F->delta0 <= spec->eps) break;
        }
        if (!st && r > ZOLO_MAX_R) st = set_error(ZOLO_EINVAL, "eps not reachable with orders <= ZOLO_MAX_R");
        r1 = fix1 ? fix1 : r;
        r2 = fix2 ? fix2 : r;
    } else {
        st = build_pair(r1, r2);
    }
    if (st) {
        delete F;
        return st;
    }
    // ---- info: Proposition 2 for Zhat (inner), Corollary 1 for the outer function
    zolo_filter_info &I = F->info;
    std::memset(&I, 0, sizeof(I));
    I.alpha = F->alpha;
    I.beta = F->beta;
    I.gamma = F->gamma;
    I.ell1 = F->ell1;
    I.ell2 = F->ell2;
    I.delta1 = F->inner.delta;
    I.delta0 = F->delta0;
    I.r1 = r1;
    I.r2 = r2;
    I.M_hat = F->inner.M / F->inner.zmax;
    double cst = 0.0;
    for (int j = 0; j < r1; ++j) {
        const double cj = F->inner.c[2 * j];
        const double aj = F->inner.a[j];
        I.a_hat[j] = aj;
        I.c_hat[j] = cj;
        cst += aj * F->gamma / (F->gamma * F->gamma + cj);
        const zolo::cplx isq(0.0, std::sqrt(cj));
        const zolo::cplx sig = (F->gamma * F->alpha + isq * F->beta) / (F->gamma + isq);
        const zolo::cplx w = I.M_hat * aj * (sig - F->beta) / (2.0 * (F->gamma + isq));
        I.sigma_hat[2 * j] = sig.real();
        I.sigma_hat[2 * j + 1] = sig.imag();
        I.w_hat[2 * j] = w.real();
        I.w_hat[2 * j + 1] = w.imag();
    }
    I.const_hat = I.M_hat * cst;
    I.M = F->outer.M;
    for (int j = 0; j < r2; ++j) {
        I.a[j] = F->outer.a[j];
        I.c[j] = F->outer.c[2 * j];
    }
    I.gap[0] = am;
    I.gap[1] = ap;
    I.gap[2] = bm;
    I.gap[3] = bp;
    I.kind = ZOLO_FILTER_ZOLO;
    *out = F;
    return ZOLO_OK;
}

int zolo_filter_table(const zolo_filter_spec *spec, int32_t rmax, double *delta0) {
    using namespace zolo;
    clear_error();
    if (!spec || !delta0 || rmax < 1 || rmax > ZOLO_MAX_R) return set_error(ZOLO_EINVAL, "bad argument");
    for (int r1 = 1; r1 <= rmax; ++r1)
        for (int r2 = 1; r2 <= rmax; ++r2) {
            zolo_filter_spec s = *spec;
            s.r1 = r1;
            s.r2 = r2;
            zolo_filter f = nullptr;
            const int st = zolo_filter_build(&s, &f);
            if (st) return st;
            delta0[(r1 - 1) * rmax + (r2 - 1)] = f->delta0;
            zolo_filter_destroy(f);
        }
    return ZOLO_OK;
}

int zolo_filter_build_contour(int32_t kind, double a, double b, int32_t npoles, zolo_filter *out) {
    using namespace zolo;
    clear_error();
    if (!out) return set_error(ZOLO_EINVAL, "null argument");
    *out = nullptr;
    if (kind != ZOLO_FILTER_CITZ && kind != ZOLO_FILTER_CIGQ) return set_error(ZOLO_EINVAL, "unknown contour filter kind");
    if (!(std::isfinite(a) && std::isfinite(b) && a < b)) return set_error(ZOLO_EINVAL, "need finite a < b");
    if (npoles < 2 || npoles % 2 || npoles > 2 * ZOLO_MAX_R)
        return set_error(ZOLO_EINVAL, "npoles must be even, 2 .. 2 ZOLO_MAX_R");
    const int h = npoles / 2;                          // points in the upper half plane
    const double c0 = 0.5 * (a + b), rho = 0.5 * (b - a);
    std::vector<double> theta(h), wq(h);
    if (kind == ZOLO_FILTER_CITZ) {
        // trapezoidal rule in the angle: z_j = c0 + rho e^{i theta_j}, theta_j = 2 pi (j - 1/2)/npoles;
        // the weight of (1/(2 pi i)) dz/(z - x) at z_j is rho e^{i theta_j} / npoles
        for (int j = 0; j < h; ++j) {
            theta[j] = 2.0 * M_PI * (j + 0.5) / npoles;
            wq[j] = 1.0 / npoles;
        }
    } else {
        // Gauss-Legendre on the upper half circle: theta = (pi/2)(1 + t), t the Legendre nodes of
        // degree h on [-1, 1] (Newton on the three-term recurrence), dtheta = (pi/2) dt, so the
        // weight at z_j is rho e^{i theta_j} omega_j / 4
        for (int i = 0; i < h; ++i) {
            double x = std::cos(M_PI * (i + 0.75) / (h + 0.5));
            double dp = 1.0;
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = x;
                for (int j = 2; j <= h; ++j) {
                    const double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
                    p0 = p1;
                    p1 = p2;
                }
                if (h == 1) { p1 = x; p0 = 1.0; }
                dp = h * (x * p1 - p0) / (x * x - 1.0);
                const double dx = p1 / dp;
                x -= dx;
                if (std::fabs(dx) <= 1e-16 * std::max(1.0, std::fabs(x))) break;
            }
            {   // derivative at the converged node
                double p0 = 1.0, p1 = x;
                for (int j = 2; j <= h; ++j) {
                    const double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
                    p0 = p1;
                    p1 = p2;
                }
                if (h == 1) { p1 = x; p0 = 1.0; }
                dp = h * (x * p1 - p0) / (x * x - 1.0);
            }
            theta[i] = 0.5 * M_PI * (1.0 + x);
            wq[i] = 2.0 / ((1.0 - x * x) * dp * dp) / 4.0;
        }
    }
    auto *F = new zolo_filter_s();
    std::memset(&F->spec, 0, sizeof(F->spec));
    F->kind = kind;
    zolo_filter_info &I = F->info;
    std::memset(&I, 0, sizeof(I));
    I.kind = kind;
    I.npoles = npoles;
    I.r1 = h;
    I.r2 = 0;
    I.gap[0] = I.gap[1] = a;
    I.gap[2] = I.gap[3] = b;
    for (int j = 0; j < h; ++j) {
        const cplx e(std::cos(theta[j]), std::sin(theta[j]));
        const cplx z = c0 + rho * e;
        const cplx cj = rho * e * wq[j];               // R(x) = sum_j c_j / (z_j - x) + conjugates
        I.sigma_hat[2 * j] = z.real();
        I.sigma_hat[2 * j + 1] = z.imag();
        I.w_hat[2 * j] = -cj.real();                   // w_j / (x - z_j) = c_j / (z_j - x)
        I.w_hat[2 * j + 1] = -cj.imag();
    }
    *out = F;
    return ZOLO_OK;
}

int zolo_filter_get_info(zolo_filter f, zolo_filter_info *out) {
    zolo::clear_error();
    if (!f || !out) return zolo::set_error(ZOLO_EINVAL, "null argument");
    *out = f->info;
    return ZOLO_OK;
}

int zolo_filter_eval(zolo_filter f, int64_t n, const double *x, double *out) {
    zolo::clear_error();
    if (!f || n < 0 || (n > 0 && (!x || !out))) return zolo::set_error(ZOLO_EINVAL, "bad argument");
    for (int64_t i = 0; i < n; ++i) out[i] = f->eval(x[i]);
    return ZOLO_OK;
}

void zolo_filter_destroy(zolo_filter f) { delete f; }

}  // extern "C"
