// Step (b): asymptotic channel functions at r = a, one thread per (energy, channel).
//
// The outer-region equation (Section "Overview", Eq. radial, U = 0, Rydberg units)
//   u'' + (eps + 2z/r - l(l+1)/r^2) u = 0,   eps = E - e_i,
// is the Coulomb wave equation in rho = k r, eta = -z/k for an open channel
// (eps = k^2 > 0) and Whittaker's equation in x = 2 kappa r, nu = z/kappa for a
// closed channel (eps = -kappa^2 < 0).
//
// Open channel (Steed's method, FP64):
//   1. CF1 for f_l = F_l'/F_l at the channel's own l by modified Lentz. The
//      Lentz ratios D_n = B_{n-1}/B_n are ratios of a solution of the l-recurrence
//      that vanishes at l; for large n it is a positive multiple of F_l G_{l+n},
//      and G > 0 deep in the barrier, so prod sign(D_n) = sign(F_l).
//   2. F is carried down to l = 0 by the l-recurrences (stable: F is minimal
//      upwards), giving F_0'/F_0 up to one common scale.
//   3. CF2 for H+'/H+ = p + iq at l = 0, where r = a is never inside a barrier
//      for an attractive potential. Forward Lentz only finds the depth n at
//      which the fraction settles; the value is then taken bottom-up from
//      depth 2n + 20, which avoids the rounding that forward Lentz accumulates
//      on the slowly converging fractions near threshold (|eta| >> 1, rho << 1)
//      (double precision loses ~1e-10 there otherwise).
//   4. The Wronskian q (F^2 + G^2) = 1 fixes |F_0|; G_0 = (F_0' - p F_0)/q.
//   5. G is carried up to l by the l-recurrences (stable: G is dominant upwards).
//   Energy normalisation: s = F/sqrt(k), s' = sqrt(k) F', c = G/sqrt(k), c' = sqrt(k) G'.
//
// Closed channel: the log-derivative L = theta'/theta of the decaying solution
// theta ~ W_{nu,l+1/2}(2 kappa r) from CF2 continued to imaginary k
// (k = i kappa, eta = i nu, rho = i kappa a), which is real:
//   L = -kappa + (nu + Phi)/a,  Phi = a_1/(b_1 - a_2/(b_2 - ...)),
//   a_n = (L0 + n - nu)(n - 1 - L0 - nu),  b_n = 2(kappa a - nu + n),
// evaluated at a low l = L0 and carried to l with the Coulomb ladder operator
//   y_{L+1} = c/(T - y_L) - T,  T = (L+1)/a - z/(L+1),  c = eps + z^2/(L+1)^2.
// The fraction at the channel's own l loses up to ~13 digits (more near
// threshold) when r = a lies inside the inner centrifugal barrier; the ladder
// is stable upwards there. L0 = 0 unless nu <= l + 1/2, where the operator
// would pass near its null case nu = L+1; then L0 = ceil(nu - 1/2).
// Output pair (theta, theta') scaled to theta^2 + (a theta')^2 = 1.
//
// MQDT (Section "namelist stgf MQDT variables"): a closed channel with
// nu >= max(l + nu_margin, fnumin), |sin pi nu| >= 1e-3 and kappa a <=
// kappa_a_max is eliminated by quantum-defect theory (more deeply closed
// channels make f and g differ by exp(2 kappa a) at r = a, and the
// elimination would lose that factor in precision). It needs the energy-analytic regular solution
// f -> (2 pi z)^{1/2} (2z)^l r^{l+1}/(2l+1)! (r -> 0), from its Frobenius
// series in double-double (the series cancels by up to ~1e10 at r = a), and g
// defined by theta ~ f cos(pi nu) - g sin(pi nu) with f'g - fg' = 1:
//   theta-hat(a) = sin(pi nu) / (f L - f'),  theta-hat'(a) = L theta-hat(a),
//   g = (f cos(pi nu) - theta-hat) / sin(pi nu),  g' likewise.
//
// Channel tables (built once per partial wave from the same continued
// fractions, when the context asks for them; see thr_nodes_kernel,
// open_table_kernel, closed_table_kernel): at fixed r = a the pair
// f = s / sqrt(A), g~ = c sqrt(A), A = prod_{p=1..l} (1 + p^2 eps / z^2), is
// analytic in eps across the threshold (on the closed side f is the
// energy-analytic regular solution and g~ the g above at half-integer nu,
// theta ~ A f cos(pi nu) - g~ sin(pi nu)). Near a threshold the pair is
// interpolated from 16 nodes straddling it; open pairs beyond come from
// Chebyshev expansions in k, closed pairs deep enough (kappa a >= 6) from
// expansions of the direction of (theta, a theta') in nu. Each table is
// checked against direct values at build time, and pairs a table does not
// cover keep the continued fractions.
#include <math.h>

#include <cmath>

#include "dd.cuh"
#include "rcp.cuh"
#include "rm_internal.cuh"

namespace rmgb {
namespace {

constexpr int CF_MAXIT = 1 << 20;
constexpr double TINY = 1e-300;
constexpr double CF_TOL = 4e-16;
// A CF2 that settles within this many forward steps is taken from its
// forward Lentz value (few roundings, and a fast-converging fraction leaves
// no significant tail); slower ones are re-evaluated backwards from depth
// 2n + 20.
#ifndef RM_CF2_FAST_DEPTH
#define RM_CF2_FAST_DEPTH 32
#endif
constexpr int CF2_FAST_DEPTH = RM_CF2_FAST_DEPTH;

struct Cf1 {
    double f;
    int sgn;
    int ok;
    int iters;
};

// The continued fractions are evaluated through their numerators and
// denominators (Wallis recurrences), A_n = b_n A_{n-1} + a_n A_{n-2} and the
// same for B, forwards for the convergents A_n / B_n, or backwards,
// (p, q) <- (a_m q, p + b_m q) from (0, 1) at depth N, for the tail value
// p / q. Each step is then one or two dependent FMAs instead of a reciprocal
// chain, which matters because the deep fractions near thresholds are serial
// chains of hundreds to thousands of steps. Every 8 steps the quantities are
// rescaled by a power of two (exact; the ratios are unchanged) and the
// forward convergence test is applied.
constexpr int CF_CHECK = 8;

// 2^k with k chosen so that s * 2^k lies in [1, 2) (s > 0 finite; clamped
// to the normal range).
__device__ __forceinline__ double pow2_rescale(double s)
{
    const int ex = (int)((__double_as_longlong(s) >> 52) & 0x7ff);
    int se = 2046 - ex;
    se = se < 1 ? 1 : (se > 2046 ? 2046 : se);
    return __longlong_as_double((long long)se << 52);
}

// f_l = S_{l+1} + K(a_n / b_n), a_n = -(1 + eta^2/(l+n)^2), b_n = S_{l+n} + S_{l+n+1},
// S_L = L/rho + eta/L. sign(F_l) = sign(B_n): the ratios B_{n-1}/B_n are
// ratios of a solution of the l-recurrence that vanishes at l; for large n it
// is a positive multiple of F_l G_{l+n}, and G > 0 deep in the barrier.
__device__ Cf1 cf1_lentz(int l, double eta, double rho)
{
    const double irho = 1.0 / rho;
    const double L1 = l + 1.0;
    double er = eta / L1;            // eta / (l + n), carried to the next iteration
    double S = L1 * irho + er;
    double A2 = 1.0, B2 = 0.0;       // A_{n-2}, B_{n-2}
    double A1 = S, B1 = 1.0;         // A_{n-1}, B_{n-1}
    for (int n = 1; n < CF_MAXIT; ++n) {
        const double Ln1 = l + n + 1.0;
        const double er1 = eta * rcp_nr(Ln1);
        const double Snext = Ln1 * irho + er1;
        const double an = -fma(er, er, 1.0);
        const double bn = S + Snext;
        const double A = fma(bn, A1, an * A2);
        const double B = fma(bn, B1, an * B2);
        A2 = A1;
        B2 = B1;
        A1 = A;
        B1 = B;
        S = Snext;
        er = er1;
        if (n % CF_CHECK == 0) {
            const double sc = pow2_rescale(fmax(fmax(fabs(A1), fabs(B1)), fmax(fabs(A2), fabs(B2))));
            A1 *= sc;
            B1 *= sc;
            A2 *= sc;
            B2 *= sc;
            const double f = A1 / B1, fp = A2 / B2;
            if (fabs(f - fp) < CF_TOL * fabs(fp)) return {f, B1 < 0.0 ? -1 : 1, 1, n};
        }
    }
    return {0.0, 1, 0, CF_MAXIT};
}

// p + iq = H+'/H+ at l = 0: i(1 - eta/rho) + (i/rho) K,  K = K(a_m / b_m),
// a_m = (m + i eta)(m - 1 + i eta), b_m = 2(rho - eta) + 2 i m.
// The forward convergents of the tail K' = b_1 + K_{m>=2}(a_m / b_m) give
// K = a_1 / K' when they settle within CF2_FAST_DEPTH steps; otherwise the
// depth n reached sets a backward evaluation of K from depth 2n + 20.
__device__ int cf2_open_l0(double eta, double rho, double *p, double *q, int *depth)
{
    const double br = 2.0 * (rho - eta);
    double A2r = 1.0, A2i = 0.0, B2r = 0.0, B2i = 0.0;
    double A1r = br, A1i = 2.0, B1r = 1.0, B1i = 0.0;
    double fr = br, fi = 2.0;
    int n = 2;
    bool conv = false;
    for (; n < CF_MAXIT; ++n) {
        const double m = n;
        const double ar = m * (m - 1.0) - eta * eta;
        const double ai = eta * (2.0 * m - 1.0);
        const double bi = 2.0 * m;
        const double tAr = fma(ar, A2r, -ai * A2i), tAi = fma(ar, A2i, ai * A2r);
        const double tBr = fma(ar, B2r, -ai * B2i), tBi = fma(ar, B2i, ai * B2r);
        const double Ar = fma(br, A1r, fma(-bi, A1i, tAr));
        const double Ai = fma(br, A1i, fma(bi, A1r, tAi));
        const double Br = fma(br, B1r, fma(-bi, B1i, tBr));
        const double Bi = fma(br, B1i, fma(bi, B1r, tBi));
        A2r = A1r; A2i = A1i; B2r = B1r; B2i = B1i;
        A1r = Ar; A1i = Ai; B1r = Br; B1i = Bi;
        if (n % CF_CHECK == 0) {
            const double mx = fmax(fmax(fmax(fabs(A1r), fabs(A1i)), fmax(fabs(B1r), fabs(B1i))),
                                   fmax(fmax(fabs(A2r), fabs(A2i)), fmax(fabs(B2r), fabs(B2i))));
            const double sc = pow2_rescale(mx);
            A1r *= sc; A1i *= sc; B1r *= sc; B1i *= sc;
            A2r *= sc; A2i *= sc; B2r *= sc; B2i *= sc;
            const double d1 = 1.0 / (B1r * B1r + B1i * B1i), d2 = 1.0 / (B2r * B2r + B2i * B2i);
            fr = (A1r * B1r + A1i * B1i) * d1;
            fi = (A1i * B1r - A1r * B1i) * d1;
            const double gr = (A2r * B2r + A2i * B2i) * d2;
            const double gi = (A2i * B2r - A2r * B2i) * d2;
            if (fabs(fr - gr) + fabs(fi - gi) < CF_TOL * (fabs(gr) + fabs(gi))) {
                conv = true;
                break;
            }
        }
    }
    *depth = n;
    if (!conv) return 0;
    if (n <= CF2_FAST_DEPTH) {
        // K = a_1 / K',  a_1 = -eta^2 + i eta
        const double ar = -eta * eta, ai = eta;
        const double dm = 1.0 / (fr * fr + fi * fi);
        *p = -((ai * fr - ar * fi) * dm) / rho;
        *q = (1.0 - eta / rho) + ((ar * fr + ai * fi) * dm) / rho;
        return 1;
    }
    const int N = 2 * n + 20;
    double pr = 0.0, pi = 0.0, qr = 1.0, qi = 0.0;
    for (int m_ = N; m_ >= 1; --m_) {
        const double m = m_;
        const double ar = m * (m - 1.0) - eta * eta;
        const double ai = eta * (2.0 * m - 1.0);
        const double bi = 2.0 * m;
        // (p, q) <- (a_m q, p + b_m q)
        const double npr = fma(ar, qr, -ai * qi), npi = fma(ar, qi, ai * qr);
        const double nqr = fma(br, qr, fma(-bi, qi, pr));
        const double nqi = fma(br, qi, fma(bi, qr, pi));
        pr = npr; pi = npi; qr = nqr; qi = nqi;
        if (m_ % CF_CHECK == 0) {
            const double sc = pow2_rescale(fmax(fmax(fabs(pr), fabs(pi)), fmax(fabs(qr), fabs(qi))));
            pr *= sc; pi *= sc; qr *= sc; qi *= sc;
        }
    }
    const double dm = 1.0 / (qr * qr + qi * qi);
    const double vr = (pr * qr + pi * qi) * dm, vi = (pi * qr - pr * qi) * dm;
    *p = -vi / rho;
    *q = (1.0 - eta / rho) + vr / rho;
    return 1;
}

// Closed-channel log-derivative (r-units) at l = L0 from CF2 at imaginary k.
// The forward convergents of the tail K' = b_1 - a_2/(b_2 - a_3/(...)) give
// Phi = a_1 / K' when they settle within CF2_FAST_DEPTH steps; otherwise the
// depth n reached sets a backward evaluation from depth 2n + 20.
__device__ int cf2_closed(int L0, double nu, double kap, double a, double *y, int *depth)
{
    const double base = kap * a - nu;
    auto an = [&](int m) { return (L0 + m - nu) * (m - 1.0 - L0 - nu); };
    double A2 = 1.0, B2 = 0.0, A1 = 2.0 * (base + 1.0), B1 = 1.0;
    double f = A1;
    int n = 2;
    bool conv = false;
    for (; n < CF_MAXIT; ++n) {
        const double num = -an(n);
        const double den = 2.0 * (base + n);
        const double A = fma(den, A1, num * A2);
        const double B = fma(den, B1, num * B2);
        A2 = A1;
        B2 = B1;
        A1 = A;
        B1 = B;
        if (n % CF_CHECK == 0) {
            const double sc = pow2_rescale(fmax(fmax(fabs(A1), fabs(B1)), fmax(fabs(A2), fabs(B2))));
            A1 *= sc;
            B1 *= sc;
            A2 *= sc;
            B2 *= sc;
            f = A1 / B1;
            const double fp = A2 / B2;
            if (fabs(f - fp) < CF_TOL * fabs(fp)) {
                conv = true;
                break;
            }
        }
    }
    *depth = n;
    if (!conv) return 0;
    if (n <= CF2_FAST_DEPTH) {
        *y = -kap + (nu + an(1) / f) / a;
        return 1;
    }
    const int N = 2 * n + 20;
    double pp = 0.0, qq = 1.0;
    for (int m = N; m >= 2; --m) {
        // (p, q) <- (num_m q, p + den_m q)
        const double np_ = -an(m) * qq;
        qq = fma(2.0 * (base + m), qq, pp);
        pp = np_;
        if (m % CF_CHECK == 0) {
            const double sc = pow2_rescale(fmax(fabs(pp), fabs(qq)));
            pp *= sc;
            qq *= sc;
        }
    }
    const double phi = an(1) / (2.0 * (base + 1.0) + pp / qq);
    *y = -kap + (nu + phi) / a;
    return 1;
}

// Thread (i, e) with the energy index fastest: a warp covers 32 consecutive
// energies of one channel (same l and threshold, nearby eta and rho), so its
// lanes take the same branch and similar continued-fraction depths.
// Energy-analytic regular solution f(r), f'(r) (see above). Terms
// t_k = c_k r^k with k(k+2l+1) c_k = -2z c_{k-1} - eps c_{k-2}, c_0 = 1.
__device__ int regular_analytic(int l, double z, double eps, double r, double *f, double *fp)
{
    const dd zr = two_prod(-2.0 * z, r);                 // -2 z r
    const dd er2 = dd_mul_d(two_prod(-eps, r), r);       // -eps r^2
    dd tm2 = dd_make(0.0), tm1 = dd_make(1.0);
    dd S = dd_make(1.0), Sp = dd_make((double)(l + 1));
    double tmax = 1.0;
    int quiet = 0;
    for (int k = 1; k < 100000; ++k) {
        dd t = dd_add(dd_mul(zr, tm1), dd_mul(er2, tm2));
        t = dd_div_d(t, (double)k * (double)(k + 2 * l + 1));
        S = dd_add(S, t);
        Sp = dd_add(Sp, dd_mul_d(t, (double)(k + l + 1)));
        const double at = fabs(t.hi);
        tmax = fmax(tmax, at);
        if (at <= 1e-33 * tmax) {
            if (++quiet >= 3 && k > 8) {
                double Nf = sqrt(2.0 * M_PI * z);
                for (int j = 0; j < l; ++j) Nf *= 2.0 * z;
                for (int j = 2; j <= 2 * l + 1; ++j) Nf /= (double)j;
                double rl = 1.0;
                for (int j = 0; j < l; ++j) rl *= r;
                *f = Nf * rl * r * dd_to_d(S);
                *fp = Nf * rl * dd_to_d(Sp);
                return 1;
            }
        } else {
            quiet = 0;
        }
        tm2 = tm1;
        tm1 = t;
    }
    return 0;
}

// STATS: instead of the channel data, record per (energy, channel) the
// iteration counts of the continued fractions: {kind, CF1 iterations, CF2
// forward iterations (the backward pass then takes 2n + 20 steps), l - L0
// ladder steps for a closed channel or l for an open one}.
#ifndef RM_CHANFN_BS
#define RM_CHANFN_BS 128
#endif
#ifndef RM_CHANFN_MINB
#define RM_CHANFN_MINB 1
#endif
constexpr int CHANFN_BS = RM_CHANFN_BS;   // threads per block of the channel kernel
constexpr int CH_THR_INTERP = 3;          // work-record kind of an interpolated pair
constexpr int CH_OPEN_TABLE = 4;          // work-record kind of an open pair from its table
constexpr int CH_CLOSED_TABLE = 5;        // work-record kind of a closed pair from its table
constexpr double CHANFN_DEEP_EPS = 2.5e-5;   // |eps| / max(z^2, 1) below this: a deep pair
constexpr int CHANFN_DEEP_CAP = 1 << 14;     // capacity of the deep-pair list

// Pairs (energy, channel) this close to their threshold have the deepest
// continued fractions (depth ~ z / (|eps| a) steps: thousands to millions,
// each a serial chain of dependent FP64 operations). Where the channel's
// near-threshold table covers them they cost an interpolation; the others
// (no tables: z = 0, an FP64 context, or a table that failed its check) are
// listed, their energies marked, and a separate kernel (on a second stream)
// evaluates them while the main stream forms R and solves every unmarked
// energy; the marked energies are solved after it.
__device__ __forceinline__ bool chanfn_deep(const PwDev &pw, int i, double eps, double eps_thr)
{
    if (!(fabs(eps) < CHANFN_DEEP_EPS * fmax(pw.z * pw.z, 1.0)) || fabs(eps) < eps_thr) return false;
    return !(pw.thr && fabs(eps) < pw.thr[i].zone);   // covered by the channel's table
}

__global__ void chanfn_deep_mark_kernel(PwDev pw, const double *__restrict__ E, int nE, double eps_thr,
                                        int *__restrict__ count, int *__restrict__ list,
                                        int *__restrict__ defer)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nE * pw.n) return;
    const int i = (int)(idx / nE);
    const int e = (int)(idx - (long long)i * nE);
    if (chanfn_deep(pw, i, E[e] - pw.e_thr[i], eps_thr)) {
        const int k = atomicAdd(count, 1);
        if (k < CHANFN_DEEP_CAP) list[k] = (int)idx;
        defer[e] = 1;
    }
}

// Open channel at eps > 0 (Steed's method, steps 1-5 above): energy-
// normalised s, s', c, c' at r = a. Returns 0 if a fraction did not converge;
// it1 / d2: CF1 iterations and CF2 forward depth.
__device__ __forceinline__ int open_channel(int l, double eps, double z, double a, double *s, double *sp,
                                            double *c, double *cp, int *it1, int *d2)
{
    const double k = sqrt(eps);
    const double eta = -z / k;
    const double rho = k * a;
    Cf1 c1 = cf1_lentz(l, eta, rho);
    double p, q;
    *d2 = 0;
    const int ok2 = cf2_open_l0(eta, rho, &p, &q, d2);
    *it1 = c1.iters;
    if (!c1.ok || !ok2) return 0;
    // F_l, F_l' up to a common scale, carried down to l = 0
    const double Fl = (double)c1.sgn, Fpl = c1.f * Fl;
    double F = Fl, Fp = Fpl;
    for (int L = l; L >= 1; --L) {
        const double SL = L / rho + eta / L;
        const double RL = sqrt(1.0 + (eta / L) * (eta / L));
        const double Fm = (SL * F + Fp) / RL;
        Fp = SL * Fm - RL * F;
        F = Fm;
    }
    const double f0 = Fp / F;
    double F0 = sqrt(q / ((f0 - p) * (f0 - p) + q * q));
    if (F < 0.0) F0 = -F0;
    const double scale = F0 / F;
    double G = scale * (Fp - p * F) / q;
    double Gp = p * G - q * F0;
    for (int L = 0; L < l; ++L) {
        const double L1 = L + 1.0;
        const double S1 = L1 / rho + eta / L1;
        const double R1 = sqrt(1.0 + (eta / L1) * (eta / L1));
        const double Gn = (S1 * G - Gp) / R1;
        Gp = R1 * G - S1 * Gn;
        G = Gn;
    }
    const double sk = sqrt(k);
    *s = scale * Fl / sk;
    *sp = scale * Fpl * sk;
    *c = G / sk;
    *cp = Gp * sk;
    return 1;
}

// Closed channel at eps < 0: log-derivative y = theta'/theta of the decaying
// solution at r = a (CF2 at l = L0, then the ladder to l). Returns 0 if the
// fraction did not converge; d2: its forward depth, *L0o: L0.
__device__ __forceinline__ int closed_channel(int l, double eps, double z, double a, double *y, int *d2,
                                              int *L0o)
{
    const double kap = sqrt(-eps);
    const double nu = z / kap;
    int L0 = 0;
    if (nu <= l + 0.5) {
        L0 = (int)ceil(nu - 0.5);
        L0 = L0 < 0 ? 0 : (L0 > l ? l : L0);
    }
    *L0o = L0;
    *d2 = 0;
    double yy;
    if (!cf2_closed(L0, nu, kap, a, &yy, d2)) return 0;
    for (int L = L0; L < l; ++L) {
        const double L1 = L + 1.0;
        const double T = L1 / a - z / L1;
        const double c = eps + (z / L1) * (z / L1);
        yy = c / (T - yy) - T;
    }
    *y = yy;
    return 1;
}

// A(eps, l) = prod_{p=1..l} (1 + p^2 eps / z^2).
__device__ __forceinline__ double a_factor(int l, double eps, double z)
{
    const double u = eps / (z * z);
    double A = 1.0;
    for (int p = 1; p <= l; ++p) A = fma(A * (double)(p * p), u, A);
    return A;
}

// Barycentric interpolation of the table's four quantities at eps.
__device__ __forceinline__ void thr_interp(const ThrNodes &T, double eps, double v[4])
{
    double num0 = 0.0, num1 = 0.0, num2 = 0.0, num3 = 0.0, den = 0.0;
#pragma unroll 4
    for (int j = 0; j < THR_NODES; ++j) {
        const double d = eps - T.x[j];
        if (d == 0.0) {
            for (int q = 0; q < 4; ++q) v[q] = T.y[q][j];
            return;
        }
        const double t = T.w[j] * rcp_nr(d);
        den += t;
        num0 = fma(t, T.y[0][j], num0);
        num1 = fma(t, T.y[1][j], num1);
        num2 = fma(t, T.y[2][j], num2);
        num3 = fma(t, T.y[3][j], num3);
    }
    const double id = 1.0 / den;
    v[0] = num0 * id;
    v[1] = num1 * id;
    v[2] = num2 * id;
    v[3] = num3 * id;
}

// Node spacing of a channel's near-threshold table: small against the
// energy scale on which the channel functions at r = a change (~ sqrt(z) /
// a^1.5) and against the distance z^2 / (l + 1)^2 to the nearest
// singularity of g~ (at nu = l); the table covers |eps| < THR_ZONE h. A
// table is used only if leave-one-out interpolation of its four innermost
// nodes agrees with their values to THR_LOO_TOL (relative to each
// quantity's largest node value). The open-side table of the channel starts
// where that zone ends, at k0 = sqrt(THR_ZONE h).
constexpr double THR_C1 = 0.0164, THR_C2 = 0.05, THR_ZONE = 4.0, THR_LOO_TOL = 1e-9;
__device__ __forceinline__ double thr_spacing(int l, double z, double a)
{
    return fmin(THR_C1 * sqrt(z) / (a * sqrt(a)), THR_C2 * z * z / ((l + 1.0) * (l + 1.0)));
}

// The four open-side quantities of channel i at k from its table (segment
// q, local coordinate u in [-1, 1]), by Clenshaw's recurrence.
__device__ __forceinline__ void otab_eval(const PwDev &pw, int i, int q, double u, double v[4])
{
    const double *c = pw.otab + ((size_t)i * pw.otab_nseg + q) * 4 * OTAB_M;
    double b1[4] = {0.0, 0.0, 0.0, 0.0}, b2[4] = {0.0, 0.0, 0.0, 0.0};
    const double u2 = 2.0 * u;
#pragma unroll 1
    for (int m = OTAB_M - 1; m >= 1; --m) {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const double b0 = fma(u2, b1[f], c[f * OTAB_M + m] - b2[f]);
            b2[f] = b1[f];
            b1[f] = b0;
        }
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) v[f] = fma(u, b1[f], c[f * OTAB_M] - b2[f]);
}

// The closed-side direction (theta, a theta') of channel i at nu from its
// table (segment q, local coordinate u), by Clenshaw's recurrence.
__device__ __forceinline__ void ctab_eval(const PwDev &pw, int i, int q, int sub, double u, double v[2])
{
    const double *c = pw.ctab + (((size_t)i * pw.ctab_nseg + q) * CTAB_SUB + sub) * 2 * OTAB_M;
    double b1[2] = {0.0, 0.0}, b2[2] = {0.0, 0.0};
    const double u2 = 2.0 * u;
#pragma unroll 1
    for (int m = OTAB_M - 1; m >= 1; --m) {
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const double b0 = fma(u2, b1[f], c[f * OTAB_M + m] - b2[f]);
            b2[f] = b1[f];
            b1[f] = b0;
        }
    }
#pragma unroll
    for (int f = 0; f < 2; ++f) v[f] = fma(u, b1[f], c[f * OTAB_M] - b2[f]);
}

// Channel data of pair idx = i nE + e.
template <bool MQDT, bool STATS>
__device__ void chanfn_pair(const PwDev &pw, const double *__restrict__ E, int nE, const Opts &o,
                            ChanFn *__restrict__ out, int *__restrict__ status, int4 *__restrict__ work,
                            long long idx)
{
    const int n = pw.n;
    const int i = (int)(idx / nE);
    const int e = (int)(idx - (long long)i * nE);
    const double eps = E[e] - pw.e_thr[i];
    const int l = pw.l[i];
    const double a = pw.a, z = pw.z;
    ChanFn r = {0.0, 0.0, 0.0, 0.0, 0.0, CH_CLOSED, 0};
    int bad = RM_OK;
    // k - k0 on the channel's open-side table (-1: no table)
    const double kr = (eps > 0.0 && pw.otab && !pw.otab_bad[i]) ? sqrt(eps) - sqrt(THR_ZONE * thr_spacing(l, z, a))
                                                                 : -1.0;
    // cell of the channel's closed-side table (-1: none, or a cell without
    // coefficients); closed channels of the quantum-defect set take f and g
    int cq = -1;
    if (eps < 0.0 && pw.ctab && -eps >= THR_ZONE * thr_spacing(l, z, a) &&
        !(MQDT && z / sqrt(-eps) >= fmax(l + o.nu_margin, o.fnumin) && sqrt(-eps) * a <= o.kappa_a_max)) {
        const double nr = z / sqrt(-eps) - pw.ctab_nu_lo;
        if (nr >= 0.0 && nr < pw.ctab_nseg * pw.ctab_dnu) {
            const int q = min((int)floor(nr / pw.ctab_dnu), pw.ctab_nseg - 1);
            if (pw.ctab_nsub[(size_t)i * pw.ctab_nseg + q] > 0) cq = q;
        }
    }
    if (fabs(eps) < o.eps_thr) {
        bad = RM_ETHRESHOLD;
    } else if (pw.thr && fabs(eps) < pw.thr[i].zone) {
        // near the threshold: from the channel's interpolation table
        if (STATS) work[(size_t)e * n + i] = make_int4(CH_THR_INTERP, 0, 0, l);
        double v[4];
        thr_interp(pw.thr[i], eps, v);
        const double A = a_factor(l, eps, z);
        if (eps > 0.0) {
            const double sA = sqrt(A), isA = 1.0 / sA;
            r.s = v[0] * sA;
            r.sp = v[1] * sA;
            r.gh = v[2] * isA;
            r.ghp = v[3] * isA;
            r.kind = CH_OPEN;
        } else {
            const double kap = sqrt(-eps);
            const double nu = z / kap;
            double sb, cb;
            sincospi(nu, &sb, &cb);
            if (MQDT && nu >= fmax(l + o.nu_margin, o.fnumin) && kap * a <= o.kappa_a_max && fabs(sb) >= 1e-3) {
                // g = g~ + (1 - A) f cot(pi nu), from theta ~ f cos(pi nu) - g sin(pi nu)
                const double ct = (1.0 - A) * cb / sb;
                r.s = v[0];
                r.sp = v[1];
                r.gh = fma(ct, v[0], v[2]);
                r.ghp = fma(ct, v[1], v[3]);
                r.tanb = sb / cb;
                r.kind = CH_MQDT;
            } else {
                const double th = fma(A * v[0], cb, -v[2] * sb);
                const double thp = fma(A * v[1], cb, -v[3] * sb);
                const double nrm = 1.0 / sqrt(fma(th, th, (a * thp) * (a * thp)));
                r.gh = fabs(th) * nrm;
                r.ghp = (th < 0.0 ? -thp : thp) * nrm;
            }
        }
    } else if (kr >= 0.0 && kr < pw.otab_nseg * pw.otab_dk) {
        // open, from the channel's table (k >= k0: nearer ones are in the
        // near-threshold zone, handled above, or the table there was refused)
        if (STATS) work[(size_t)e * n + i] = make_int4(CH_OPEN_TABLE, 0, 0, l);
        const int q = max(0, min((int)floor(kr / pw.otab_dk), pw.otab_nseg - 1));
        const double u = fma(2.0 / pw.otab_dk, kr - q * pw.otab_dk, -1.0);
        double v[4];
        otab_eval(pw, i, q, u, v);
        const double sA = sqrt(a_factor(l, eps, z)), isA = 1.0 / sA;
        r.s = v[0] * sA;
        r.sp = v[1] * sA;
        r.gh = v[2] * isA;
        r.ghp = v[3] * isA;
        r.kind = CH_OPEN;
    } else if (eps > 0.0) {
        int it1 = 0, d2 = 0;
        const int ok = open_channel(l, eps, z, a, &r.s, &r.sp, &r.gh, &r.ghp, &it1, &d2);
        if (STATS) work[(size_t)e * n + i] = make_int4(CH_OPEN, it1, d2, l);
        if (!ok) bad = RM_ECF_NOCONV;
        else r.kind = CH_OPEN;
    } else if (cq >= 0) {
        // closed (decaying condition), from the channel's table
        if (STATS) work[(size_t)e * n + i] = make_int4(CH_CLOSED_TABLE, 0, 0, l);
        const double nr = z / sqrt(-eps) - pw.ctab_nu_lo;
        const int q = cq;
        const int ns = pw.ctab_nsub[(size_t)i * pw.ctab_nseg + q];
        const double w = pw.ctab_dnu / ns;
        const double fr = nr - q * pw.ctab_dnu;
        const int sub = min((int)floor(fr / w), ns - 1);
        const double u = fma(2.0 / w, fr - sub * w, -1.0);
        double v[2];
        ctab_eval(pw, i, q, sub, u, v);
        // theta > 0, theta^2 + (a theta')^2 = 1
        const double nrm = 1.0 / sqrt(fma(v[0], v[0], v[1] * v[1]));
        r.gh = fabs(v[0]) * nrm;
        r.ghp = (v[0] < 0.0 ? -v[1] : v[1]) * nrm / a;
    } else {
        double y;
        int d2 = 0, L0 = 0;
        const int okc = closed_channel(l, eps, z, a, &y, &d2, &L0);
        if (STATS) work[(size_t)e * n + i] = make_int4(CH_CLOSED, 0, d2, l - L0);
        if (!okc) {
            bad = RM_ECF_NOCONV;
        } else {
            const double nrm = 1.0 / sqrt(1.0 + (a * y) * (a * y));
            r.gh = nrm;
            r.ghp = y * nrm;
            const double kap = sqrt(-eps);
            const double nu = z / kap;
            if (MQDT && nu >= fmax(l + o.nu_margin, o.fnumin) && kap * a <= o.kappa_a_max) {
                double sb, cb;
                sincospi(nu, &sb, &cb);
                if (fabs(sb) >= 1e-3) {
                    double f, fp;
                    if (!regular_analytic(l, z, eps, a, &f, &fp)) {
                        bad = RM_ECF_NOCONV;
                    } else {
                        const double th = sb / (f * y - fp), thp = y * th;
                        r.gh = (f * cb - th) / sb;
                        r.ghp = (fp * cb - thp) / sb;
                        r.s = f;
                        r.sp = fp;
                        r.tanb = sb / cb;
                        r.kind = CH_MQDT;
                    }
                }
            }
        }
    }
    if (STATS) {
        if (fabs(eps) < o.eps_thr) work[(size_t)e * n + i] = make_int4(-1, 0, 0, 0);
        return;
    }
    out[(size_t)e * n + i] = r;
    if (bad != RM_OK) atomicCAS(status + e, RM_OK, bad);
}

// One block of 32 threads per channel: threads 0-7 the closed-side nodes
// (half-integer nu, descending, so x ascends), 8-15 the open side
// (eps = h, 2h, ... 8h); thread 0 then forms the weights and checks them.
__global__ void __launch_bounds__(32) thr_nodes_kernel(PwDev pw, ThrNodes *__restrict__ tab)
{
    constexpr int M = THR_NODES / 2;
    __shared__ double xs[THR_NODES], ys[4][THR_NODES];
    __shared__ int okn[THR_NODES];
    const int i = blockIdx.x, t = threadIdx.x;
    const int l = pw.l[i];
    const double z = pw.z, a = pw.a;
    const double h = thr_spacing(l, z, a);
    if (t < THR_NODES) {
        double x, v[4] = {0.0, 0.0, 0.0, 0.0};
        int ok = 0;
        if (t >= M) {
            x = h * (t - M + 1);
            int it1, d2;
            ok = open_channel(l, x, z, a, &v[0], &v[1], &v[2], &v[3], &it1, &d2);
            const double sA = sqrt(a_factor(l, x, z));
            v[0] /= sA;
            v[1] /= sA;
            v[2] *= sA;
            v[3] *= sA;
        } else {
            // node j = M - t: the half-integer nu nearest below z / sqrt(j h),
            // at least 1 below the previous node's
            const int j = M - t;
            double nu = 0.0;
            for (int q = 1; q <= j; ++q) {
                const double c = floor(z / sqrt(h * q)) + 0.5;
                nu = (q == 1) ? c : fmin(nu - 1.0, c);
            }
            x = -(z / nu) * (z / nu);
            double y, f, fp;
            int d2, L0;
            ok = nu > 0.0 && closed_channel(l, x, z, a, &y, &d2, &L0) && regular_analytic(l, z, x, a, &f, &fp);
            if (ok) {
                // at half-integer nu, theta ~ g~ and f'g~ - f g~' = 1
                v[2] = -1.0 / (f * y - fp);
                v[3] = y * v[2];
                v[0] = f;
                v[1] = fp;
            }
        }
        for (int q = 0; q < 4; ++q) ok = ok && isfinite(v[q]);
        xs[t] = x;
        for (int q = 0; q < 4; ++q) ys[q][t] = v[q];
        okn[t] = ok;
    }
    __syncthreads();
    if (t != 0) return;
    ThrNodes &T = tab[i];
    bool valid = z > 0.0 && h > 0.0;
    for (int j = 0; j < THR_NODES; ++j) valid = valid && okn[j];
    for (int j = 0; j < THR_NODES; ++j) {
        double p = 1.0;
        for (int k = 0; k < THR_NODES; ++k)
            if (k != j) p *= xs[j] - xs[k];
        T.x[j] = xs[j];
        T.w[j] = 1.0 / p;
        for (int q = 0; q < 4; ++q) T.y[q][j] = ys[q][j];
    }
    if (valid) {
        for (int q = 0; q < 4 && valid; ++q) {
            double mx = 0.0;
            for (int j = 0; j < THR_NODES; ++j) mx = fmax(mx, fabs(ys[q][j]));
            for (int k = M - 2; k <= M + 1; ++k) {
                double num = 0.0, den = 0.0;
                for (int j = 0; j < THR_NODES; ++j) {
                    if (j == k) continue;
                    const double tw = T.w[j] * (xs[j] - xs[k]) / (xs[k] - xs[j]);
                    num += tw * ys[q][j];
                    den += tw;
                }
                if (!(fabs(num / den - ys[q][k]) <= THR_LOO_TOL * mx)) valid = false;
            }
        }
    }
    T.h = h;
    T.zone = valid ? THR_ZONE * h : 0.0;
}

// With deep_count != nullptr, the listed deep pairs are skipped (when the
// list did not overflow): chanfn_deep_kernel takes them.
template <bool MQDT, bool STATS>
__global__ void __launch_bounds__(CHANFN_BS, RM_CHANFN_MINB)
    chanfn_kernel(PwDev pw, const double *__restrict__ E, int nE, Opts o, ChanFn *__restrict__ out,
                  int *__restrict__ status, int4 *__restrict__ work, const int *__restrict__ deep_count)
{
    const int n = pw.n;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nE * n) return;
    if (deep_count && *deep_count <= CHANFN_DEEP_CAP) {
        const int i0 = (int)(idx / nE);
        const int e0 = (int)(idx - (long long)i0 * nE);
        if (chanfn_deep(pw, i0, E[e0] - pw.e_thr[i0], o.eps_thr)) return;
    }
    chanfn_pair<MQDT, STATS>(pw, E, nE, o, out, status, work, idx);
}

// One thread per listed deep pair.
template <bool MQDT>
__global__ void __launch_bounds__(64)
    chanfn_deep_kernel(PwDev pw, const double *__restrict__ E, int nE, Opts o, ChanFn *__restrict__ out,
                       int *__restrict__ status, const int *__restrict__ deep_count,
                       const int *__restrict__ list)
{
    const int cnt = *deep_count;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (cnt > CHANFN_DEEP_CAP || k >= cnt) return;
    chanfn_pair<MQDT, false>(pw, E, nE, o, out, status, nullptr, list[k]);
}

__global__ void nearpole_kernel(PwDev pw, const double *__restrict__ E, int nE,
                                int *__restrict__ status)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nE) return;
    const double x = E[e];
    const double tol = 1e-12 * fmax(1.0, fabs(x));
    int lo = 0, hi = pw.N;  // first index with Ek >= x
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (pw.Ek[mid] < x) lo = mid + 1; else hi = mid;
    }
    bool near = (lo < pw.N && fabs(pw.Ek[lo] - x) < tol) ||
                (lo > 0 && fabs(pw.Ek[lo - 1] - x) < tol);
    if (near) atomicCAS(status + e, RM_OK, RM_ENEAR_POLE);
}

__global__ void export_kernel(PwDev pw, const double *__restrict__ E, int nE,
                              const ChanFn *__restrict__ cf, double *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nE * pw.n) return;
    const ChanFn c = cf[i];
    const bool open = E[i / pw.n] - pw.e_thr[i % pw.n] > 0.0;
    out[4 * i + 0] = open ? c.s : c.gh;
    out[4 * i + 1] = open ? c.sp : c.ghp;
    out[4 * i + 2] = open ? c.gh : 0.0;
    out[4 * i + 3] = open ? c.ghp : 0.0;
}

// Segment q of channel i's open-side table: the four quantities at the
// OTAB_M Chebyshev points x_j = cos(pi (j + 1/2) / M) of k in [q dk, (q + 1)
// dk) (continued fractions), their Chebyshev coefficients
// c_m = (2/M) sum_j y_j cos(pi m (j + 1/2) / M) (c_0 halved), and a check of
// the expansion against direct values at x = -0.5 and 0.5 (relative to the
// segment's largest node value); a failure marks the channel bad.
constexpr double OTAB_CHECK_TOL = 1e-12;
__global__ void __launch_bounds__(64) open_table_kernel(PwDev pw, double *__restrict__ coef, int *__restrict__ bad)
{
    constexpr int M = OTAB_M;
    __shared__ double ys[4][M + 2];
    __shared__ double cs[4][M];
    __shared__ int okn[M + 2];
    const int q = blockIdx.x, i = blockIdx.y, t = threadIdx.x;
    const int l = pw.l[i];
    const double z = pw.z, a = pw.a, dk = pw.otab_dk;
    if (t < M + 2) {
        const double x = t < M ? cospi((t + 0.5) / M) : (t == M ? -0.5 : 0.5);
        const double k = sqrt(THR_ZONE * thr_spacing(l, z, a)) + dk * (q + 0.5 * (x + 1.0));
        const double eps = k * k;
        double v[4];
        int it1, d2;
        int ok = open_channel(l, eps, z, a, &v[0], &v[1], &v[2], &v[3], &it1, &d2);
        const double sA = sqrt(a_factor(l, eps, z));
        v[0] /= sA;
        v[1] /= sA;
        v[2] *= sA;
        v[3] *= sA;
        for (int f = 0; f < 4; ++f) {
            ok = ok && isfinite(v[f]);
            ys[f][t] = v[f];
        }
        okn[t] = ok;
    }
    __syncthreads();
    if (t < 4 * M) {
        const int f = t / M, m = t - (t / M) * M;
        double c = 0.0;
        for (int j = 0; j < M; ++j) c = fma(ys[f][j], cospi(m * (j + 0.5) / M), c);
        c *= 2.0 / M;
        if (m == 0) c *= 0.5;
        cs[f][m] = c;
        coef[((size_t)i * pw.otab_nseg + q) * 4 * M + f * M + m] = c;
    }
    __syncthreads();
    if (t < 8) {
        const int f = t & 3, h = t >> 2;
        const double x = h ? 0.5 : -0.5;
        double b1 = 0.0, b2 = 0.0;
        for (int m = M - 1; m >= 1; --m) {
            const double b0 = fma(2.0 * x, b1, cs[f][m] - b2);
            b2 = b1;
            b1 = b0;
        }
        const double val = fma(x, b1, cs[f][0] - b2);
        double mx = 0.0;
        bool ok = okn[M + h];
        for (int j = 0; j < M; ++j) {
            mx = fmax(mx, fabs(ys[f][j]));
            ok = ok && okn[j];
        }
        if (!ok || !(fabs(val - ys[f][M + h]) <= OTAB_CHECK_TOL * mx)) bad[i] = 1;
    }
}

// Cell q of channel i's closed-side table: the direction (1, a L) of
// (theta, a theta') at the OTAB_M Chebyshev points in nu of each of ns equal
// sub-segments, made continuous along each (each node's sign chosen to agree
// with its neighbour's), Chebyshev coefficients, and a check of the
// expansion's direction against direct values at x = -0.6, 0.1 and 0.7 of
// every sub-segment (sine of the angle between them within
// CTAB_CHECK_TOL). ns = 1, 2, 4, 8, 16 in turn; the first that passes is
// kept, and a cell that fails at 16 gets nsub = 0: its pairs keep the
// continued fractions. The direction turns by about pi per unit nu, but
// where r = a lies in the classically allowed region of the decaying
// solution (kappa a of a few) it does so through narrow peaks of its rate
// that no modest expansion holds; deeper, it is smooth. So the table stops
// at kappa a = CTAB_KA_MIN (or the near-threshold zone, if nearer); cells
// beyond are not computed (nsub = 0).
constexpr double CTAB_CHECK_TOL = 5e-13;
__global__ void __launch_bounds__(128) closed_table_kernel(PwDev pw, double *__restrict__ coef,
                                                            unsigned char *__restrict__ nsub)
{
    constexpr int M = OTAB_M, P = M + 3;
    __shared__ double ys[CTAB_SUB][2][P];
    __shared__ double cs[CTAB_SUB][2][M];
    __shared__ int okn[CTAB_SUB][P];
    __shared__ int pass;
    const int q = blockIdx.x, i = blockIdx.y, t = threadIdx.x;
    const int l = pw.l[i];
    const double z = pw.z, a = pw.a;
    const double nu0 = pw.ctab_nu_lo + q * pw.ctab_dnu;
    const double nu_hi = fmin(z / sqrt(THR_ZONE * thr_spacing(l, z, a)), z * a / CTAB_KA_MIN);
    double *cq = coef + ((size_t)i * pw.ctab_nseg + q) * CTAB_SUB * 2 * M;
    unsigned char *nq = nsub + (size_t)i * pw.ctab_nseg + q;
    if (nu0 >= nu_hi) {
        if (t == 0) *nq = 0;
        return;
    }
    for (int ns = 1; ns <= CTAB_SUB; ns *= 2) {
        const double w = pw.ctab_dnu / ns;
        for (int k = t; k < ns * P; k += blockDim.x) {
            const int sb = k / P, j = k - (k / P) * P;
            const double x = j < M ? cospi((j + 0.5) / M) : (j == M ? -0.6 : (j == M + 1 ? 0.1 : 0.7));
            const double nu = nu0 + w * (sb + 0.5 * (x + 1.0));
            const double kap = z / nu;
            double y = 0.0;
            int d2, L0;
            const int ok = closed_channel(l, -kap * kap, z, a, &y, &d2, &L0);
            const double nrm = 1.0 / sqrt(1.0 + (a * y) * (a * y));
            ys[sb][0][j] = nrm;
            ys[sb][1][j] = a * y * nrm;
            okn[sb][j] = ok && isfinite(y);
        }
        if (t == 0) pass = 1;
        __syncthreads();
        if (t < ns) {
            for (int j = 1; j < M; ++j) {   // nodes in order of x: continuous signs
                const double dot = ys[t][0][j] * ys[t][0][j - 1] + ys[t][1][j] * ys[t][1][j - 1];
                if (dot < 0.0) {
                    ys[t][0][j] = -ys[t][0][j];
                    ys[t][1][j] = -ys[t][1][j];
                }
            }
        }
        __syncthreads();
        for (int k = t; k < ns * 2 * M; k += blockDim.x) {
            const int sb = k / (2 * M), r = k - (k / (2 * M)) * 2 * M, f = r / M, m = r - (r / M) * M;
            double c = 0.0;
            for (int j = 0; j < M; ++j) c = fma(ys[sb][f][j], cospi(m * (j + 0.5) / M), c);
            c *= 2.0 / M;
            if (m == 0) c *= 0.5;
            cs[sb][f][m] = c;
        }
        __syncthreads();
        for (int k = t; k < ns * 3; k += blockDim.x) {
            const int sb = k / 3, h = k - (k / 3) * 3;
            const double x = h == 0 ? -0.6 : (h == 1 ? 0.1 : 0.7);
            double v[2];
            for (int f = 0; f < 2; ++f) {
                double b1 = 0.0, b2 = 0.0;
                for (int m = M - 1; m >= 1; --m) {
                    const double b0 = fma(2.0 * x, b1, cs[sb][f][m] - b2);
                    b2 = b1;
                    b1 = b0;
                }
                v[f] = fma(x, b1, cs[sb][f][0] - b2);
            }
            bool ok = okn[sb][M + h];
            for (int j = 0; j < M; ++j) ok = ok && okn[sb][j];
            const double nv = sqrt(v[0] * v[0] + v[1] * v[1]);
            const double sn = fabs(v[0] * ys[sb][1][M + h] - v[1] * ys[sb][0][M + h]) / nv;
            if (!ok || !(sn <= CTAB_CHECK_TOL)) pass = 0;
        }
        __syncthreads();
        if (pass) {
            for (int k = t; k < ns * 2 * M; k += blockDim.x) {
                const int sb = k / (2 * M), r = k - (k / (2 * M)) * 2 * M;
                cq[sb * 2 * M + r] = cs[sb][r / M][r - (r / M) * M];
            }
            if (t == 0) *nq = (unsigned char)ns;
            return;
        }
        __syncthreads();
    }
    if (t == 0) *nq = 0;
}

}  // namespace

double closed_table_nu_hi(double z, double a, int l_max)
{
    double nu = 0.0;
    for (int l = 0; l <= l_max; ++l) {
        const double h = std::fmin(THR_C1 * std::sqrt(z) / (a * std::sqrt(a)), THR_C2 * z * z / ((l + 1.0) * (l + 1.0)));
        nu = std::fmax(nu, z / std::sqrt(THR_ZONE * h));
    }
    return std::fmin(nu, z * a / CTAB_KA_MIN);
}

cudaError_t launch_closed_table(const PwDev &pw, double *coef, unsigned char *nsub, cudaStream_t s)
{
    if (pw.n == 0 || pw.ctab_nseg == 0) return cudaSuccess;
    PwDev d = pw;
    d.thr = nullptr;
    d.otab = nullptr;
    d.otab_bad = nullptr;
    d.ctab = nullptr;
    d.ctab_nsub = nullptr;
    closed_table_kernel<<<dim3(pw.ctab_nseg, pw.n), 128, 0, s>>>(d, coef, nsub);
    return cudaGetLastError();
}

cudaError_t launch_chanfn(const PwDev &pw, const double *E, int nE, const Opts &o, int mqdt,
                          ChanFn *cf, int *status, const int *deep_ws, cudaStream_t s)
{
    const long long total = (long long)nE * pw.n;
    if (total == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((total + CHANFN_BS - 1) / CHANFN_BS);
    if (mqdt)
        chanfn_kernel<true, false><<<grid, CHANFN_BS, 0, s>>>(pw, E, nE, o, cf, status, nullptr, deep_ws);
    else
        chanfn_kernel<false, false><<<grid, CHANFN_BS, 0, s>>>(pw, E, nE, o, cf, status, nullptr, deep_ws);
    return cudaGetLastError();
}

size_t chanfn_deep_ws_bytes(int nE) { return (size_t)(1 + CHANFN_DEEP_CAP + nE) * sizeof(int); }

cudaError_t launch_chanfn_deep_mark(const PwDev &pw, const double *E, int nE, const Opts &o, int *deep_ws,
                                    cudaStream_t s)
{
    const long long total = (long long)nE * pw.n;
    cudaError_t e = cudaMemsetAsync(deep_ws, 0, chanfn_deep_ws_bytes(nE), s);
    if (e != cudaSuccess || total == 0) return e;
    chanfn_deep_mark_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
        pw, E, nE, o.eps_thr, deep_ws, deep_ws + 1, deep_ws + 1 + CHANFN_DEEP_CAP);
    return cudaGetLastError();
}

cudaError_t launch_chanfn_deep(const PwDev &pw, const double *E, int nE, const Opts &o, int mqdt, ChanFn *cf,
                               int *status, const int *deep_ws, cudaStream_t s)
{
    if ((long long)nE * pw.n == 0) return cudaSuccess;
    const unsigned grid = (CHANFN_DEEP_CAP + 63) / 64;
    if (mqdt)
        chanfn_deep_kernel<true><<<grid, 64, 0, s>>>(pw, E, nE, o, cf, status, deep_ws, deep_ws + 1);
    else
        chanfn_deep_kernel<false><<<grid, 64, 0, s>>>(pw, E, nE, o, cf, status, deep_ws, deep_ws + 1);
    return cudaGetLastError();
}

int chanfn_deep_cap() { return CHANFN_DEEP_CAP; }

double chanfn_deep_eps(double z) { return CHANFN_DEEP_EPS * fmax(z * z, 1.0); }

cudaError_t launch_open_table(const PwDev &pw, double *coef, int *bad, cudaStream_t s)
{
    if (pw.n == 0 || pw.otab_nseg == 0) return cudaSuccess;
    cudaError_t err = cudaMemsetAsync(bad, 0, sizeof(int) * (size_t)pw.n, s);
    if (err != cudaSuccess) return err;
    PwDev d = pw;
    d.thr = nullptr;
    d.otab = nullptr;
    d.otab_bad = nullptr;
    open_table_kernel<<<dim3(pw.otab_nseg, pw.n), 64, 0, s>>>(d, coef, bad);
    return cudaGetLastError();
}

cudaError_t launch_thr_nodes(const PwDev &pw, ThrNodes *tab, cudaStream_t s)
{
    if (pw.n == 0) return cudaSuccess;
    PwDev d = pw;
    d.thr = nullptr;
    thr_nodes_kernel<<<pw.n, 32, 0, s>>>(d, tab);
    return cudaGetLastError();
}

cudaError_t launch_chanfn_work(const PwDev &pw, const double *E, int nE, const Opts &o, int4 *work,
                               cudaStream_t s)
{
    const long long total = (long long)nE * pw.n;
    if (total == 0) return cudaSuccess;
    chanfn_kernel<false, true><<<(unsigned)((total + CHANFN_BS - 1) / CHANFN_BS), CHANFN_BS, 0, s>>>(
        pw, E, nE, o, nullptr, nullptr, work, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_nearpole(const PwDev &pw, const double *E, int nE, int *status, cudaStream_t s)
{
    if (nE == 0) return cudaSuccess;
    nearpole_kernel<<<(nE + 255) / 256, 256, 0, s>>>(pw, E, nE, status);
    return cudaGetLastError();
}

cudaError_t launch_chanfn_export(const PwDev &pw, const double *E, int nE, const ChanFn *cf,
                                 double *out, cudaStream_t s)
{
    const int count = nE * pw.n;
    if (count == 0) return cudaSuccess;
    export_kernel<<<(count + 255) / 256, 256, 0, s>>>(pw, E, nE, cf, out);
    return cudaGetLastError();
}

}  // namespace rmgb
