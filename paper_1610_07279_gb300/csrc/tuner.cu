// Tree-rebuild interval auto-tuning (Sec. 2.6, Eqs. 8-14; Appendix C).
//
// After a rebuild the walk time t_walk(i) of the i-th block step grows as the tree
// drifts away from the particles.  Three growth models are fitted to the measured
// times by least squares:
//   linear     t(i) = t1 + (i-1) dt                          (Eq. 9)
//   power law  t(i) = t1 r^(i-1)          (a line in log t)  (Appendix C)
//   parabolic  t(i) = t1 + (i-1) b + (i-1)^2 a               (Appendix C)
// and the one with the smallest reduced chi^2 (sigma_i = 1, nu = n - 2 or n - 3,
// Eq. 14) is kept.  The rebuild interval n minimises the mean time per step
// (t_make + sum_i t(i)) / n:
//   linear     n^2 = 2 t_make / dt                                   (Eq. 12)
//   power law  (n ln r - 1) r^n = (r - 1) t_make / t1 - 1             (Appendix C)
//   parabolic  n^2 = t_make / (b/2 + (4n - 3) a / 6)                  (Appendix C)
// A model whose minimum does not exist (dt <= 0, r <= 1, (2n - 1) a + b < 0) asks
// for no rebuild yet.  Host code only; the times come from the phase timers.
#include <math.h>
#include <string.h>

#include "gt_internal.cuh"

namespace {

// least squares of y against x for a polynomial of degree deg (1 or 2): coef[0..deg]
bool polyfit(const double *x, const double *y, int n, int deg, double *coef) {
    double A[3][4] = {};
    for (int i = 0; i < n; i++) {
        double p[3] = {1.0, x[i], x[i] * x[i]};
        for (int r = 0; r <= deg; r++) {
            for (int c = 0; c <= deg; c++) A[r][c] += p[r] * p[c];
            A[r][deg + 1] += p[r] * y[i];
        }
    }
    const int m = deg + 1;
    for (int c = 0; c < m; c++) {  // Gaussian elimination with partial pivoting
        int piv = c;
        for (int r = c + 1; r < m; r++)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (fabs(A[piv][c]) < 1e-300) return false;
        if (piv != c)
            for (int k = 0; k <= m; k++) {
                const double t = A[c][k];
                A[c][k] = A[piv][k];
                A[piv][k] = t;
            }
        for (int r = 0; r < m; r++) {
            if (r == c) continue;
            const double f = A[r][c] / A[c][c];
            for (int k = c; k <= m; k++) A[r][k] -= f * A[c][k];
        }
    }
    for (int c = 0; c < m; c++) coef[c] = A[c][m] / A[c][c];
    return true;
}

// bisection for a root of f on [lo, hi] where f changes sign
template <class F>
double bisect(F f, double lo, double hi) {
    double flo = f(lo);
    for (int it = 0; it < 200; it++) {
        const double mid = 0.5 * (lo + hi);
        const double fm = f(mid);
        if ((fm <= 0) == (flo <= 0)) {
            lo = mid;
            flo = fm;
        } else {
            hi = mid;
        }
    }
    return 0.5 * (lo + hi);
}

constexpr double N_CAP = 1e6;  // "never rebuild" is reported as this interval

}  // namespace

extern "C" int gt_rebuild_interval(const double *t_walk, int n, double t_make, int *model_out,
                                   double *n_opt_out, double *coef_out) {
    if (!t_walk || n < 3 || !(t_make >= 0.0) || !model_out || !n_opt_out) return GT_EINVAL;
    double x[4096], y[4096], ly[4096];
    if (n > 4096) n = 4096;
    bool logs = true;
    for (int i = 0; i < n; i++) {
        x[i] = (double)i;  // i - 1 for the i-th step
        y[i] = t_walk[i];
        if (!(t_walk[i] > 0.0)) logs = false;
        ly[i] = logs ? log(t_walk[i]) : 0.0;
    }
    double cl[2], cp[3], cw[2];
    double chi[3] = {INFINITY, INFINITY, INFINITY};
    if (polyfit(x, y, n, 1, cl)) {
        double s = 0;
        for (int i = 0; i < n; i++) s += pow(cl[0] + cl[1] * x[i] - y[i], 2);
        chi[0] = s / (n - 2);
    }
    if (logs && polyfit(x, ly, n, 1, cw)) {
        double s = 0;
        for (int i = 0; i < n; i++) s += pow(exp(cw[0]) * exp(cw[1] * x[i]) - y[i], 2);
        chi[1] = s / (n - 2);
    }
    if (n >= 4 && polyfit(x, y, n, 2, cp)) {
        double s = 0;
        for (int i = 0; i < n; i++) s += pow(cp[0] + cp[1] * x[i] + cp[2] * x[i] * x[i] - y[i], 2);
        chi[2] = s / (n - 3);
    }
    int best = 0;
    for (int k = 1; k < 3; k++)
        if (chi[k] < chi[best]) best = k;
    if (!isfinite(chi[best])) return GT_EINVAL;
    double nopt = N_CAP;
    if (best == 0) {  // linear: t1 = cl[0], dt = cl[1]
        const double dt = cl[1];
        if (dt > 0.0) nopt = sqrt(2.0 * t_make / dt);
        if (coef_out) { coef_out[0] = cl[0]; coef_out[1] = dt; coef_out[2] = 0.0; }
    } else if (best == 1) {  // power law: t1 = exp(cw[0]), r = exp(cw[1])
        const double t1 = exp(cw[0]), r = exp(cw[1]);
        if (r > 1.0) {
            const double rhs = (r - 1.0) * t_make / t1 - 1.0;
            auto f = [&](double m) { return (m * log(r) - 1.0) * pow(r, m) - rhs; };
            // f(0) = -1 - rhs; f grows without bound for m > 1/ln r
            double hi = 1.0;
            while (f(hi) < 0.0 && hi < N_CAP) hi *= 2.0;
            nopt = f(hi) >= 0.0 ? bisect(f, 0.0, hi) : N_CAP;
        }
        if (coef_out) { coef_out[0] = t1; coef_out[1] = r; coef_out[2] = 0.0; }
    } else {  // parabolic: t1 = cp[0], b = cp[1], a = cp[2]
        const double b = cp[1], a = cp[2];
        // d/dn (t_tot/n) = -t_make/n^2 + b/2 + (4n - 3) a / 6 = 0
        auto f = [&](double m) { return -t_make / (m * m) + 0.5 * b + (4.0 * m - 3.0) * a / 6.0; };
        double hi = 1.0;
        while (f(hi) < 0.0 && hi < N_CAP) hi *= 2.0;
        if (f(hi) >= 0.0) {
            const double m = bisect(f, 1e-9, hi);
            if ((2.0 * m - 1.0) * a + b >= 0.0) nopt = m;  // a minimum, not a maximum
        }
        if (coef_out) { coef_out[0] = cp[0]; coef_out[1] = b; coef_out[2] = a; }
    }
    *model_out = best;
    *n_opt_out = nopt;
    return GT_OK;
}

// ---- critical separation of groups (Sec. 2.4): Brent's method on line -----------
//
// Brent's minimisation keeps a bracket [a, b] around the minimum, the best point x
// found so far and the two previous best w, v.  Each step tries the vertex of the
// parabola through (x, w, v); it falls back to a golden-section step into the larger
// part of the bracket when the parabola is unusable (steps that do not shrink fast
// enough, or a vertex outside the bracket).  As an on-line search the state machine
// hands out one abscissa at a time (next) and takes its measured cost back (report).
void gt_brent_start(BrentSearch *b, double lo, double hi, double tol, double abs_tol) {
    constexpr double GOLD = 0.3819660112501051;  // (3 - sqrt 5) / 2
    b->a = lo < hi ? lo : hi;
    b->b = lo < hi ? hi : lo;
    b->x = b->w = b->v = b->a + GOLD * (b->b - b->a);
    b->fx = b->fw = b->fv = 0.0;
    b->d = b->e = 0.0;
    b->u = b->x;
    b->tol = tol;
    b->abs_tol = abs_tol;
    b->state = 0;
    b->evals = 0;
}

bool gt_brent_done(const BrentSearch *b) { return b->state == 2; }

double gt_brent_next(BrentSearch *b) {
    constexpr double GOLD = 0.3819660112501051;
    if (b->state == 0 || b->state == 2) return b->x;  // the first point, or the converged minimum
    const double m = 0.5 * (b->a + b->b);
    const double tol1 = b->tol * fabs(b->x) + b->abs_tol, tol2 = 2.0 * tol1;
    if (fabs(b->x - m) <= tol2 - 0.5 * (b->b - b->a)) {
        b->state = 2;
        return b->x;
    }
    bool golden = true;
    if (fabs(b->e) > tol1) {
        // vertex of the parabola through (x, fx), (w, fw), (v, fv): x + p/q
        const double r = (b->x - b->w) * (b->fx - b->fv);
        double q = (b->x - b->v) * (b->fx - b->fw);
        double p = (b->x - b->v) * q - (b->x - b->w) * r;
        q = 2.0 * (q - r);
        if (q > 0.0) p = -p;
        q = fabs(q);
        const double e_prev = b->e;
        b->e = b->d;
        if (fabs(p) < fabs(0.5 * q * e_prev) && p > q * (b->a - b->x) && p < q * (b->b - b->x)) {
            b->d = p / q;
            const double u = b->x + b->d;
            if (u - b->a < tol2 || b->b - u < tol2) b->d = m >= b->x ? tol1 : -tol1;
            golden = false;
        }
    }
    if (golden) {
        b->e = b->x >= m ? b->a - b->x : b->b - b->x;
        b->d = GOLD * b->e;
    }
    b->u = fabs(b->d) >= tol1 ? b->x + b->d : b->x + (b->d >= 0.0 ? tol1 : -tol1);
    return b->u;
}

void gt_brent_report(BrentSearch *b, double f) {
    b->evals++;
    if (b->state == 0) {
        b->fx = b->fw = b->fv = f;
        b->state = 1;
        return;
    }
    if (b->state == 2) return;
    const double u = b->u;
    if (f <= b->fx) {
        if (u >= b->x) b->a = b->x; else b->b = b->x;
        b->v = b->w; b->fv = b->fw;
        b->w = b->x; b->fw = b->fx;
        b->x = u; b->fx = f;
    } else {
        if (u < b->x) b->a = u; else b->b = u;
        if (f <= b->fw || b->w == b->x) {
            b->v = b->w; b->fv = b->fw;
            b->w = u; b->fw = f;
        } else if (f <= b->fv || b->v == b->x || b->v == b->w) {
            b->v = u; b->fv = f;
        }
    }
}

extern "C" int gt_brent_minimize(double (*f)(double, void *), void *ctx, double lo, double hi, double tol,
                                 int max_evals, double *x_min, double *f_min, int *evals) {
    if (!f || !x_min || !(hi > lo) || !(tol > 0.0) || max_evals < 1) return GT_EINVAL;
    BrentSearch b;
    gt_brent_start(&b, lo, hi, tol, 1e-12);
    while (!gt_brent_done(&b) && b.evals < max_evals) {
        const double x = gt_brent_next(&b);
        if (gt_brent_done(&b)) break;
        gt_brent_report(&b, f(x, ctx));
    }
    *x_min = b.x;
    if (f_min) *f_min = b.fx;
    if (evals) *evals = b.evals;
    return GT_OK;
}
