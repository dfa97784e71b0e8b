/*
 * Oracle special functions for the outer-region R-matrix hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, loads or
 * calls this file; only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg do, through oracle/_clib.py.
 *
 * What it computes (Section "Overview", Eq. radial with U = 0, Rydberg units):
 *   u'' + (eps + 2z/r - l(l+1)/r^2) u = 0 .
 * Open channels (eps = k^2 > 0): with rho = k r and eta = -z/k the equation is
 * the Coulomb wave equation, solved by the regular and irregular Coulomb
 * functions F_l(eta,rho), G_l(eta,rho) (Wronskian F'G - FG' = 1).
 * Closed channels (eps = -kappa^2 < 0): the solution that decays at infinity is
 * the Whittaker function W_{nu,l+1/2}(x), x = 2 kappa r, nu = z/kappa.
 * MQDT (Section "namelist stgf MQDT variables"): the energy-analytic regular
 * solution f, normalised at the origin as
 *   f -> (2 pi z)^{1/2} (2z)^l r^{l+1} / (2l+1)!   (r -> 0).
 *
 * Everything is evaluated in IEEE binary128 (_Float128, correctly rounded
 * basic operations on every gcc target) and rounded to double on output, so
 * that continued fractions whose double-precision evaluation loses digits
 * (r inside the centrifugal barrier, energies near threshold) still give
 * double results that are accurate to the last bit or two.
 *
 * Methods (each chosen to be plain and checkable, not fast):
 *  - F'/F from the continued fraction obtained from the three-term recurrence
 *    of F_l in l (minimal solution), evaluated bottom-up from a depth that is
 *    doubled until the value no longer changes. The sign of F_l is the product
 *    of the signs of the ratios F_{L+1}/F_L over the evaluated range, because
 *    F_L > 0 once rho lies deep inside the centrifugal barrier of L.
 *  - (G'+iF')/(G+iF) = p + iq from the continued fraction of the outgoing
 *    Coulomb function H+ at l = 0 (an attractive field puts r in no barrier
 *    there), bottom-up, doubled depth.
 *  - The Wronskian q (F_0^2 + G_0^2) = 1 then fixes |F_0|, and
 *    G_0 = (F_0' - pF_0)/q; G is carried up to l by its l-recurrence (it is
 *    the dominant solution upwards), and F_l = 1/(f_l G_l - G_l').
 *  - Whittaker log-derivative from W = e^{-x/2} x^{L+1} U(L+1-nu, 2L+2, x),
 *    U'(a,b,x) = -(a/x) [U(a,b,x) + (b-a-1) U(a+1,b,x)], with the ratio
 *    U(a+1,b,x)/U(a,b,x) taken from the recurrence of U(a+n,b,x) in n
 *    (minimal solution), bottom-up with doubled depth, at a low starting
 *    L and carried to l by the Coulomb ladder operator.
 *  - f by its Frobenius power series about r = 0.
 */
#include <math.h>
#include <stdint.h>

typedef _Float128 Q;

static const Q Q_PI = 3.14159265358979323846264338327950288419716939937510f128;

static Q qabs(Q x) { return x < 0 ? -x : x; }

static Q qsqrt(Q x)
{
    if (!(x > 0)) return 0;
    Q y = (Q)sqrt((double)x);
    y = (y + x / y) / 2;
    y = (y + x / y) / 2;
    y = (y + x / y) / 2;
    return y;
}

#define MAX_DEPTH (1 << 22)
#define CONV ((Q)1e-30)

/* ---- open channels -------------------------------------------------- */

/* v_L = F_{L+1}/F_L evaluated bottom-up from v_{l+M} = 0.
 * Returns f_l = F'_l/F_l and the sign of F_l. */
static void cf1_at_depth(int l, Q eta, Q rho, int M, Q *f, int *sgn)
{
    Q v = 0;
    int s = 1;
    for (int L = l + M - 1; L >= l; --L) {
        Q L1 = (Q)(L + 1), L2 = (Q)(L + 2);
        Q S1 = L1 / rho + eta / L1;
        Q S2 = L2 / rho + eta / L2;
        Q R1 = qsqrt(1 + (eta / L1) * (eta / L1));
        Q R2 = qsqrt(1 + (eta / L2) * (eta / L2));
        v = R1 / ((S1 + S2) - R2 * v);
        if (v < 0) s = -s;
    }
    Q L1 = (Q)(l + 1);
    Q S1 = L1 / rho + eta / L1;
    Q R1 = qsqrt(1 + (eta / L1) * (eta / L1));
    *f = S1 - R1 * v;
    *sgn = s;
}

/* H+'/H+ = p + i q, continued fraction with
 * a_m = (l+m+i eta)(m-1-l+i eta), b_m = 2(rho - eta + i m). */
static void cf2_at_depth(int l, Q eta, Q rho, int N, Q *p, Q *q)
{
    Q vr = 0, vi = 0;
    for (int m = N; m >= 1; --m) {
        Q ar = (Q)(l + m) * (Q)(m - 1 - l) - eta * eta;
        Q ai = eta * (Q)(2 * m - 1);
        Q br = 2 * (rho - eta) + vr;
        Q bi = (Q)(2 * m) + vi;
        Q d = br * br + bi * bi;
        Q nr = (ar * br + ai * bi) / d;
        Q ni = (ai * br - ar * bi) / d;
        vr = nr;
        vi = ni;
    }
    /* p + i q = i (1 - eta/rho) + (i/rho) v */
    *p = -vi / rho;
    *q = (1 - eta / rho) + vr / rho;
}

/* f_L = F_L'/F_L and sign(F_L) by CF1 at depths doubling from beyond the
 * turning region until three successive depths agree (so that a stretch
 * where the truncated fraction is insensitive to depth cannot pass for
 * convergence). Returns 1 if it does not settle within MAX_DEPTH. */
static int cf1_converged(int L, Q eta, Q rho, double rho_d, Q *f, int *sgn)
{
    Q f0, f1;
    int s0, s1, M = 64 + 2 * (int)rho_d, agree = 0;
    cf1_at_depth(L, eta, rho, M, &f0, &s0);
    while (agree < 2) {
        M *= 2;
        if (M > MAX_DEPTH) return 1;
        cf1_at_depth(L, eta, rho, M, &f1, &s1);
        agree = (qabs(f1 - f0) <= CONV * qabs(f1) && s0 == s1) ? agree + 1 : 0;
        f0 = f1;
        s0 = s1;
    }
    *f = f1;
    *sgn = s1;
    return 0;
}

/* out = {F, F', G, G'} (derivatives with respect to rho). Returns 0 on
 * success, 1 if a continued fraction did not settle within MAX_DEPTH or lost
 * every digit.
 *
 * H+'/H+ = p + iq is taken at L = 0, where an attractive field puts r = a in
 * no barrier: at large l inside the centrifugal barrier q / |p| ~ (F/G)^2 and
 * the fraction at l keeps correspondingly few digits. With f_0 from CF1 at 0,
 * the Wronskian q (F_0^2 + G_0^2) = 1 gives F_0, G_0; G (dominant upwards) is
 * carried to l by the l-recurrences (DLMF 33.4)
 *   u_L = (S_L u_{L-1} - u'_{L-1}) / R_L,   u'_L = R_L u_{L-1} - S_L u_L,
 *   S_L = L/rho + eta/L,  R_L = sqrt(1 + eta^2/L^2),
 * and F_l from CF1 at l and F'G - FG' = 1: F_l = 1 / (f_l G_l - G_l'). */
int ref_coulomb_open(int l, double eta_d, double rho_d, double *out)
{
    Q eta = eta_d, rho = rho_d;
    Q fl, f0;
    int sl, s0;
    if (cf1_converged(l, eta, rho, rho_d, &fl, &sl)) return 1;
    if (cf1_converged(0, eta, rho, rho_d, &f0, &s0)) return 1;
    Q p0, q0, p1, q1;
    int N = 64 + 2 * (int)fabs(eta_d), agree = 0;
    cf2_at_depth(0, eta, rho, N, &p0, &q0);
    while (agree < 2) {
        N *= 2;
        if (N > MAX_DEPTH) return 1;
        cf2_at_depth(0, eta, rho, N, &p1, &q1);
        Q scale = qabs(p1) + qabs(q1);
        agree = (qabs(p1 - p0) + qabs(q1 - q0) <= CONV * scale) ? agree + 1 : 0;
        p0 = p1;
        q0 = q1;
    }
    Q p = p1, q = q1;
    if (!(q > 0)) return 1;
    Q F0 = qsqrt(q / ((f0 - p) * (f0 - p) + q * q));
    if (s0 < 0) F0 = -F0;
    Q G = (f0 - p) * F0 / q;
    Q Gp = p * G - q * F0;
    for (int L = 1; L <= l; ++L) {
        Q S = (Q)L / rho + eta / (Q)L;
        Q R = qsqrt(1 + (eta / (Q)L) * (eta / (Q)L));
        Q Gn = (S * G - Gp) / R;
        Gp = R * G - S * Gn;
        G = Gn;
    }
    Q F = 1 / (fl * G - Gp);
    if ((F < 0) != (sl < 0)) return 1;    /* CF1's sign and the Wronskian disagree */
    Q Fp = fl * F;
    out[0] = (double)F;
    out[1] = (double)Fp;
    out[2] = (double)G;
    out[3] = (double)Gp;
    for (int j = 0; j < 4; ++j)
        if (!isfinite(out[j])) return 1;
    return 0;
}

/* ---- closed channels ------------------------------------------------ */

/* rho_0 = U(al+1,be,x)/U(al,be,x) from rho_N = 0 and
 * rho_n = -1 / ((be - 2 al - 2n - 2 - x) + (al+n+1)(al+n+2-be) rho_{n+1}). */
static Q uratio_at_depth(Q al, Q be, Q x, int N)
{
    Q r = 0;
    for (int n = N - 1; n >= 0; --n) {
        Q nn = (Q)n;
        r = -1 / ((be - 2 * al - 2 * nn - 2 - x) + (al + nn + 1) * (al + nn + 2 - be) * r);
    }
    return r;
}

/* d/dx ln W_{nu,L+1/2}(x) at one L from the U recurrence in a. */
static int whit_logderiv_at(int L, Q nu, Q x, double nu_d, Q *y)
{
    Q al = (Q)(L + 1) - nu, be = (Q)(2 * L + 2);
    /* The minimal solution only separates once n is past nu + L: start
     * there and require three successive doublings to agree. */
    int N = 64 + 2 * ((int)nu_d + L), agree = 0;
    Q r0 = uratio_at_depth(al, be, x, N), r1 = r0;
    while (agree < 2) {
        N *= 2;
        if (N > MAX_DEPTH) return 1;
        r1 = uratio_at_depth(al, be, x, N);
        agree = (qabs(r1 - r0) <= CONV * qabs(r1)) ? agree + 1 : 0;
        r0 = r1;
    }
    Q upu = -(al / x) * (1 + (be - al - 1) * r1);
    *y = -(Q)1 / 2 + (Q)(L + 1) / x + upu;
    return 0;
}

/* d/dx ln W_{nu,l+1/2}(x). Returns 0 on success.
 *
 * With r = a inside the inner centrifugal barrier (large l, small x) the
 * continued fraction at l loses up to ~45 digits, while at low l it is well
 * conditioned. So the log-derivative is taken at a starting l_s and carried
 * to l with the Coulomb ladder operator (DLMF 33.4 in r-units, scaled to x):
 *   theta_{L+1} ~ T theta_L - theta_L',  theta_{L+1}' ~ c theta_L - T theta_{L+1},
 *   T = (L+1)/x - nu/(2(L+1)),  c = -1/4 + nu^2/(4(L+1)^2),
 * i.e. y_{L+1} = c/(T - y_L) - T. The operator annihilates the decaying
 * solution when nu = L+1, so l_s is chosen with l_s + 1 >= nu + 1/2 whenever
 * nu <= l + 1/2 (no step comes within 1/2 of that case). */
int ref_whittaker_logderiv(int l, double nu_d, double x_d, double *out)
{
    Q nu = nu_d, x = x_d;
    int ls = 0;
    if (nu_d <= l + 0.5) {
        ls = (int)ceil(nu_d - 0.5);
        if (ls < 0) ls = 0;
        if (ls > l) ls = l;
    }
    Q y;
    if (whit_logderiv_at(ls, nu, x, nu_d, &y)) return 1;
    for (int L = ls; L < l; ++L) {
        Q L1 = (Q)(L + 1);
        Q T = L1 / x - nu / (2 * L1);
        Q c = -(Q)1 / 4 + nu * nu / (4 * L1 * L1);
        y = c / (T - y) - T;
    }
    *out = (double)y;
    return 0;
}

/* ---- energy-analytic regular solution (MQDT) ------------------------ */

/* out = {f(r), df/dr}. Frobenius series f = N_f sum_k c_k r^{k+l+1},
 * k(k+2l+1) c_k = -2z c_{k-1} - eps c_{k-2}, c_0 = 1,
 * N_f = (2 pi z)^{1/2} (2z)^l / (2l+1)!. Returns 0 on success. */
int ref_regular_analytic(int l, double z_d, double eps_d, double r_d, double *out)
{
    Q z = z_d, eps = eps_d, r = r_d;
    Q Nf = qsqrt(2 * Q_PI * z);
    for (int j = 0; j < l; ++j) Nf *= 2 * z;
    for (int j = 2; j <= 2 * l + 1; ++j) Nf /= (Q)j;
    Q cm2 = 0, cm1 = 1;               /* c_{k-2}, c_{k-1} */
    Q rp = 1;                         /* r^k */
    Q rl = 1;
    for (int j = 0; j < l; ++j) rl *= r; /* r^l */
    Q sum = r * rl, dsum = (Q)(l + 1) * rl;
    Q maxterm = qabs(sum);
    int quiet = 0;
    for (int k = 1; k < 100000; ++k) {
        Q ck = (-2 * z * cm1 - eps * cm2) / ((Q)k * (Q)(k + 2 * l + 1));
        rp *= r;
        Q t = ck * rp * r * rl;
        Q dt = ck * (Q)(k + l + 1) * rp * rl;
        sum += t;
        dsum += dt;
        if (qabs(t) > maxterm) maxterm = qabs(t);
        if (qabs(t) <= (Q)1e-36 * maxterm && qabs(dt) * r <= (Q)1e-36 * maxterm * (Q)(k + l + 1))
            ++quiet;
        else
            quiet = 0;
        if (quiet >= 3 && k > 8) {
            out[0] = (double)(Nf * sum);
            out[1] = (double)(Nf * dsum);
            return 0;
        }
        cm2 = cm1;
        cm1 = ck;
    }
    return 1;
}

/* ---- batched entry points (one call per array, to keep ctypes cheap) ---- */

int ref_coulomb_open_batch(int n, const int *l, const double *eta, const double *rho,
                           double *out, int *status)
{
    int bad = 0;
    for (int i = 0; i < n; ++i) {
        status[i] = ref_coulomb_open(l[i], eta[i], rho[i], out + 4 * i);
        bad += status[i] != 0;
    }
    return bad;
}

int ref_whittaker_logderiv_batch(int n, const int *l, const double *nu, const double *x,
                                 double *out, int *status)
{
    int bad = 0;
    for (int i = 0; i < n; ++i) {
        status[i] = ref_whittaker_logderiv(l[i], nu[i], x[i], out + i);
        bad += status[i] != 0;
    }
    return bad;
}

int ref_regular_analytic_batch(int n, const int *l, const double *z, const double *eps,
                               const double *r, double *out, int *status)
{
    int bad = 0;
    for (int i = 0; i < n; ++i) {
        status[i] = ref_regular_analytic(l[i], z[i], eps[i], r[i], out + 2 * i);
        bad += status[i] != 0;
    }
    return bad;
}
