// Outer-region propagation with the long-range multipole potential
// (Section "Overview", Eq. radial with U != 0; namelist variables ipert and
// mzpts): the coupled radial functions are carried by Numerov's method from
// the inner-region boundary r0 = a to the asymptotic radius r1 and matched
// there.
//
// In Rydberg units
//   u_i'' = sum_j W_ij(r) u_j,  W(r) = diag(l_i(l_i+1)/r^2 - 2z/r - eps_i) + U(r),
//   U(r) = sum_{lambda=1..lambda_max} A^lambda / r^(lambda+1)  (A^lambda symmetric).
// The R-matrix at a fixes the solution matrix Psi by Psi(a) = R(a),
// a Psi'(a) - b Psi(a) = 1, and R(r1) = Psi(r1) [r1 Psi'(r1) - b Psi(r1)]^{-1}
// (symmetric; it replaces R(a) in the matching, done at r1).
//
// Numerov on the grid r_k = a + k h, h = (r1 - a) / N, with T_k = (h^2/12) W(r_k)
// and t_k = T_k Psi_k:
//   Psi_{k+1} - 2 Psi_k + Psi_{k-1} = t_{k+1} + 10 t_k + t_{k-1},
// carried in summed form (D_k = Psi_k - Psi_{k-1}, which keeps the rounding
// of the second difference from accumulating):
//   F = Psi_k + D_k + 10 t_k + t_{k-1},   t_{k+1} = T_{k+1} (1 - T_{k+1})^{-1} F,
//   D_{k+1} = D_k + t_{k+1} + 10 t_k + t_{k-1},   Psi_{k+1} = Psi_k + D_{k+1},
// with T (1 - T)^{-1} F = T F + T^2 F + O(T^3 F): the truncation is O(h^6)
// per step, the order of Numerov's own local error. Psi_1 comes from four
// classical Runge-Kutta steps of h/4; Psi'(r1) from the O(h^4) central formula
//   Psi'_N = (Psi_{N+1} - Psi_{N-1}) / (2h) - (t_{N+1} - t_{N-1}) / h
// (one step past r1). The state (Psi, D, t_k, t_{k-1}) is linear in the basis
// of solutions, and R does not depend on that basis, so every 1/kappa_max of
// radius the state is right-multiplied by G^{-1}, G = r D/h - b Psi (about
// r Psi' - b Psi): closed channels growing as exp(kappa r) never swamp the
// other columns. One CTA of NT threads per energy, FP64; a step costs two
// products T X (2 n^3 FMA) and one build of W: the kernel runs on the FP64
// pipe.
#include <math.h>

#include "dense_smem.cuh"
#include "rm_internal.cuh"

namespace rmgb {
namespace {

// One energy per CTA of NTP threads, n <= NMAX: a thread owns the elements
// q = tid + c NTP, c < QN = NMAX^2 / NTP, of every n x n matrix (NTP = 256,
// QN = 4 up to 32 channels; NTP = 512, QN = 8 up to 64 channels).
// QN is the share of the several-energies kernel below (256 threads).
constexpr int PROP_QN = 4;
constexpr int PROP_START_SUB = 4;   // Runge-Kutta steps of h/4 to Psi_1

// scale W(r) at the owned elements into Wd: sum_lambda A^lambda
// r^-(lambda+1) plus the diagonal l(l+1)/r^2 - 2z/r - eps.
template <int NTP, int QN>
__device__ __forceinline__ void build_w(double *Wd, const double *As, const double *eps_s, const double *lt_s,
                                        int n, int lmax, double z, double r, double scale, int tid)
{
    const int n2 = n * n;
    const double ir = 1.0 / r;
#pragma unroll
    for (int c = 0; c < QN; ++c) {
        const int q = tid + c * NTP;
        if (q < n2) {
            const int i = q / n, j = q - (q / n) * n;
            double u = 0.0, rp = ir * ir;
            for (int lam = 0; lam < lmax; ++lam) {
                u = fma(As[lam * n2 + q], rp, u);
                rp *= ir;
            }
            if (i == j) u += lt_s[i] * ir * ir - 2.0 * z * ir - eps_s[i];
            Wd[q] = scale * u;
        }
    }
}

// (X S) at the owned elements, the QN dot products interleaved.
template <int NTP, int QN>
__device__ __forceinline__ void mat_times(double (&kq)[QN], const double *X, const double *S, int n, int tid)
{
    const int n2 = n * n;
    int wi[QN], sj[QN];
#pragma unroll
    for (int c = 0; c < QN; ++c) {
        const int q = min(tid + c * NTP, n2 - 1);
        wi[c] = (q / n) * n;
        sj[c] = q - wi[c];
        kq[c] = 0.0;
    }
#pragma unroll 2
    for (int k = 0; k < n; ++k) {
#pragma unroll
        for (int c = 0; c < QN; ++c) kq[c] = fma(X[wi[c] + k], S[k * n + sj[c]], kq[c]);
    }
}

// nsub classical Runge-Kutta steps of hh from r_start on (psi, dps) in
// registers. Scratch S0, S1 (stage inputs of Psi), W0, W1 (W at the step's
// start and middle); on return S0 holds Psi. Starts and ends with a barrier.
template <int NTP, int QN>
__device__ void rk4_steps(double (&psi)[QN], double (&dps)[QN], double *S0, double *S1, double *W0,
                          double *W1, const double *As, const double *eps_s, const double *lt_s, int n, int lmax,
                          double z, double r_start, double hh, int nsub, int tid)
{
    const int n2 = n * n;
    const double h2 = 0.5 * hh, h3 = hh / 3.0, h6 = hh / 6.0;
    double yp[QN], yq[QN], tq[QN], kq[QN];
    __syncthreads();
#pragma unroll
    for (int c = 0; c < QN; ++c)
        if (tid + c * NTP < n2) S0[tid + c * NTP] = psi[c];
    build_w<NTP, QN>(W0, As, eps_s, lt_s, n, lmax, z, r_start, 1.0, tid);
    __syncthreads();
    for (int s = 0; s < nsub; ++s) {
        const double r0 = r_start + s * hh;
        mat_times<NTP, QN>(kq, W0, S0, n, tid);                  // stage 1
#pragma unroll
        for (int c = 0; c < QN; ++c) {
            const int q = tid + c * NTP;
            yp[c] = fma(h6, dps[c], psi[c]);
            yq[c] = fma(h6, kq[c], dps[c]);
            tq[c] = fma(h2, kq[c], dps[c]);
            if (q < n2) S1[q] = fma(h2, dps[c], psi[c]);
        }
        build_w<NTP, QN>(W1, As, eps_s, lt_s, n, lmax, z, r0 + h2, 1.0, tid);
        __syncthreads();
        mat_times<NTP, QN>(kq, W1, S1, n, tid);                  // stage 2
#pragma unroll
        for (int c = 0; c < QN; ++c) {
            const int q = tid + c * NTP;
            const double kp = tq[c];
            yp[c] = fma(h3, kp, yp[c]);
            yq[c] = fma(h3, kq[c], yq[c]);
            tq[c] = fma(h2, kq[c], dps[c]);
            if (q < n2) S0[q] = fma(h2, kp, psi[c]);
        }
        __syncthreads();
        mat_times<NTP, QN>(kq, W1, S0, n, tid);                  // stage 3
#pragma unroll
        for (int c = 0; c < QN; ++c) {
            const int q = tid + c * NTP;
            const double kp = tq[c];
            yp[c] = fma(h3, kp, yp[c]);
            yq[c] = fma(h3, kq[c], yq[c]);
            tq[c] = fma(hh, kq[c], dps[c]);
            if (q < n2) S1[q] = fma(hh, kp, psi[c]);
        }
        build_w<NTP, QN>(W0, As, eps_s, lt_s, n, lmax, z, r0 + hh, 1.0, tid);
        __syncthreads();
        mat_times<NTP, QN>(kq, W0, S1, n, tid);                  // stage 4
#pragma unroll
        for (int c = 0; c < QN; ++c) {
            const int q = tid + c * NTP;
            psi[c] = fma(h6, tq[c], yp[c]);
            dps[c] = fma(h6, kq[c], yq[c]);
            if (q < n2) S0[q] = psi[c];
        }
        __syncthreads();
    }
}

// Writes [ G^T | 1 ] (n x 2n, row stride 2n + 1) over M from G at the owned
// elements and leaves G^{-T} in its right half (M[j ld + n + k] =
// (G^{-1})_kj). The caller has passed a barrier since M was last read.
// False if G is singular.
template <int NTP, int QN>
__device__ bool invert_owned(const double (&g)[QN], double *M, int n, ElimShared *esh, int tid)
{
    const int n2 = n * n, ld = 2 * n + 1;
    for (int q = tid; q < n * ld; q += NTP) M[q] = 0.0;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < QN; ++c) {
        const int q = tid + c * NTP;
        if (q < n2) {
            const int i = q / n, j = q - (q / n) * n;
            M[j * ld + i] = g[c];
            if (i == j) M[j * ld + n + i] = 1.0;
        }
    }
    if (tid == 0) esh->bad = 0;
    __syncthreads();
    block_eliminate<double, NTP>(M, ld, n, 2 * n, esh);
    if (esh->bad) return false;
    block_backsub<double, NTP>(M, ld, n, n, n, 0);
    return true;
}

// x <- x G^{-1} at the owned elements, with G^{-T} in M (as invert_owned
// leaves it) and SX (n^2 doubles, disjoint from M) as staging.
template <int NTP, int QN>
__device__ void times_ginv(double (&x)[QN], const double *M, double *SX, int n, int tid)
{
    const int n2 = n * n, ld = 2 * n + 1;
#pragma unroll
    for (int c = 0; c < QN; ++c)
        if (tid + c * NTP < n2) SX[tid + c * NTP] = x[c];
    __syncthreads();
#pragma unroll
    for (int c = 0; c < QN; ++c) {
        const int q = min(tid + c * NTP, n2 - 1);
        const int i = q / n, j = q - (q / n) * n;
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc = fma(SX[i * n + k], M[j * ld + n + k], acc);
        x[c] = acc;
    }
    __syncthreads();
}

template <int NTP, int QN, int NMAX>
__global__ void __launch_bounds__(NTP, NTP == 256 ? 2 : 1) propagate_kernel(PwDev pw, const double *__restrict__ E,
                                                          const double *__restrict__ A, int lmax, double r1,
                                                          int steps, double *__restrict__ Rp,
                                                          int *__restrict__ status)
{
    extern __shared__ double sm[];
    __shared__ double eps_s[NMAX], lt_s[NMAX];
    __shared__ ElimShared esh;
    const int e = blockIdx.x, tid = threadIdx.x;
    const int n = pw.n, n2 = n * n;
    if (status[e] != RM_OK) return;
    // SF (F), SG (T F), TA / TB (T_{k+1}, alternating by step), then A; the
    // restarts use the first 4 n^2 doubles as scratch
    double *SF = sm, *SG = sm + n2, *TA = sm + 2 * n2, *TB = sm + 3 * n2, *As = sm + 4 * n2;
    const double a = pw.a, b = pw.b, z = pw.z, x = E[e];
    double *Re = Rp + (size_t)e * tri_ld(n);
    for (int q = tid; q < lmax * n2; q += NTP) As[q] = A[q];
    for (int i = tid; i < n; i += NTP) {
        eps_s[i] = x - pw.e_thr[i];
        lt_s[i] = (double)pw.l[i] * (pw.l[i] + 1);
    }
    const double h = (r1 - a) / steps, t12 = h * h / 12.0;
    double psi[QN], dl[QN], tp[QN], tpp[QN], kq[QN];
#pragma unroll
    for (int c = 0; c < QN; ++c) {
        const int q = tid + c * NTP;
        psi[c] = dl[c] = 0.0;
        if (q < n2) {
            const int i = q / n, j = q - (q / n) * n;
            psi[c] = Re[i <= j ? tri_idx(i, j, n) : tri_idx(j, i, n)];
            dl[c] = ((i == j ? 1.0 : 0.0) + b * psi[c]) / a;    // Psi'(a) for the starter
            SF[q] = psi[c];
        }
    }
    __syncthreads();
    // t_0 = T_0 Psi_0
    build_w<NTP, QN>(TA, As, eps_s, lt_s, n, lmax, z, a, t12, tid);
    __syncthreads();
    mat_times<NTP, QN>(tpp, TA, SF, n, tid);
    // Psi_1 (dl: Psi'(a) in, then D_1 = Psi_1 - Psi_0), t_1 = T_1 Psi_1
    {
        double p0[QN];
#pragma unroll
        for (int c = 0; c < QN; ++c) p0[c] = psi[c];
        rk4_steps<NTP, QN>(psi, dl, SF, SG, TA, TB, As, eps_s, lt_s, n, lmax, z, a, h / PROP_START_SUB, PROP_START_SUB,
                  tid);
#pragma unroll
        for (int c = 0; c < QN; ++c) dl[c] = psi[c] - p0[c];
    }
    build_w<NTP, QN>(TA, As, eps_s, lt_s, n, lmax, z, a + h, t12, tid);
    __syncthreads();
    mat_times<NTP, QN>(tp, TA, SF, n, tid);
    // restart every `sector` steps, a sector being 1 / kappa_max long,
    // kappa_max^2 = max_i (l_i(l_i+1)/a^2 - eps_i)
    int sector = steps;
    {
        double k2 = 0.0;
        for (int i = 0; i < n; ++i) k2 = fmax(k2, lt_s[i] / (a * a) - eps_s[i]);
        const double m = k2 > 0.0 ? 1.0 / (sqrt(k2) * h) : (double)steps;
        sector = m >= (double)steps ? steps : max(1, (int)m);
    }
    __syncthreads();
    for (int k = 1; k <= steps; ++k) {
        double *Tk = (k & 1) ? TB : TA;
        // F and T_{k+1}
#pragma unroll
        for (int c = 0; c < QN; ++c) {
            const int q = tid + c * NTP;
            if (q < n2) SF[q] = psi[c] + dl[c] + fma(10.0, tp[c], tpp[c]);
        }
        build_w<NTP, QN>(Tk, As, eps_s, lt_s, n, lmax, z, a + (k + 1) * h, t12, tid);
        __syncthreads();
        // T F
        mat_times<NTP, QN>(kq, Tk, SF, n, tid);
#pragma unroll
        for (int c = 0; c < QN; ++c)
            if (tid + c * NTP < n2) SG[tid + c * NTP] = kq[c];
        __syncthreads();
        // t_{k+1} = T F + T (T F); D, Psi; shift t
        double g2[QN];
        mat_times<NTP, QN>(g2, Tk, SG, n, tid);
        const bool last = k == steps;
#pragma unroll
        for (int c = 0; c < QN; ++c) {
            const double tn = kq[c] + g2[c];
            const double d = dl[c] + tn + fma(10.0, tp[c], tpp[c]);
            if (!last) {
                dl[c] = d;
                psi[c] += d;
                tpp[c] = tp[c];
                tp[c] = tn;
            } else {
                // Psi_N = psi (before the step) and Psi'_N from Psi_{N+1} =
                // psi + d, Psi_{N-1} = psi - dl, t_{N+1} = tn, t_{N-1} = tpp
                dl[c] = (d + dl[c]) / (2.0 * h) - (tn - tpp[c]) / h;
            }
        }
        if (k % sector == 0 && k + 1 < steps) {
            // right-multiply the state by G^{-1}, G = r D / h - b Psi
            const double r = a + (k + 1) * h;
            double g[QN];
#pragma unroll
            for (int c = 0; c < QN; ++c) g[c] = fma(r / h, dl[c], -b * psi[c]);
            __syncthreads();
            if (!invert_owned<NTP, QN>(g, sm, n, &esh, tid)) {
                if (tid == 0) atomicCAS(status + e, RM_OK, RM_ESINGULAR);
                return;
            }
            double *SX = sm + 3 * n2;
            times_ginv<NTP, QN>(psi, sm, SX, n, tid);
            times_ginv<NTP, QN>(dl, sm, SX, n, tid);
            times_ginv<NTP, QN>(tp, sm, SX, n, tid);
            times_ginv<NTP, QN>(tpp, sm, SX, n, tid);
        }
    }
    // R(r1) = Psi_N (r1 Psi'_N - b Psi_N)^{-1}, written symmetrised
    double g[QN];
#pragma unroll
    for (int c = 0; c < QN; ++c) g[c] = fma(r1, dl[c], -b * psi[c]);
    __syncthreads();
    if (!invert_owned<NTP, QN>(g, sm, n, &esh, tid)) {
        if (tid == 0) atomicCAS(status + e, RM_OK, RM_ESINGULAR);
        return;
    }
    double *SX = sm + 3 * n2;
    times_ginv<NTP, QN>(psi, sm, SX, n, tid);
#pragma unroll
    for (int c = 0; c < QN; ++c)
        if (tid + c * NTP < n2) SX[tid + c * NTP] = psi[c];
    __syncthreads();
    for (int q = tid; q < tri_count(n); q += NTP) {
        int i, j;
        tri_pair(q, n, i, j);
        Re[tri_idx(i, j, n)] = 0.5 * (SX[i * n + j] + SX[j * n + i]);
    }
}

// ---- several energies per CTA (n <= PROP_SMALL_MAXN) ----
// G = prop_groups(n) energies share a CTA: element qt = tid + c NT of the
// CTA's G n^2 belongs to energy group g = qt / n^2 (matrices stored group
// after group), so the products, the builds of T and the Numerov updates are
// the kernel above with group offsets, and the renormalisations and the
// final solve eliminate each group's [G^T | 1] in one warp (rows on lanes),
// the warps taking the groups in turn. Every group runs the same steps;
// groups past nE or with a failed status compute on a clamped copy and write
// nothing.
constexpr int PROP_SMALL_MAXN = 16;
constexpr int PROP_MAX_GROUPS = 64;

__host__ __device__ inline int prop_groups(int n)
{
    const int g = (NT * PROP_QN) / (n * n);
    return g < 1 ? 1 : (g > PROP_MAX_GROUPS ? PROP_MAX_GROUPS : g);
}

__device__ __forceinline__ void build_w_g(double *Wd, const double *As, const double *eps_s, const double *lt_s,
                                          int n, int GT, int lmax, double z, double r, double scale, int tid)
{
    const int n2 = n * n;
    const double ir = 1.0 / r;
#pragma unroll
    for (int c = 0; c < PROP_QN; ++c) {
        const int qt = tid + c * NT;
        if (qt < GT) {
            const int g = qt / n2, ql = qt - g * n2;
            const int i = ql / n, j = ql - (ql / n) * n;
            double u = 0.0, rp = ir * ir;
            for (int lam = 0; lam < lmax; ++lam) {
                u = fma(As[lam * n2 + ql], rp, u);
                rp *= ir;
            }
            if (i == j) u += lt_s[i] * ir * ir - 2.0 * z * ir - eps_s[g * n + i];
            Wd[qt] = scale * u;
        }
    }
}

__device__ __forceinline__ void mat_times_g(double (&kq)[PROP_QN], const double *X, const double *S, int n, int GT,
                                            int tid)
{
    const int n2 = n * n;
    int wi[PROP_QN], sj[PROP_QN];
#pragma unroll
    for (int c = 0; c < PROP_QN; ++c) {
        const int qt = min(tid + c * NT, GT - 1);
        const int g = qt / n2, ql = qt - g * n2;
        const int i = ql / n;
        wi[c] = g * n2 + i * n;
        sj[c] = g * n2 + (ql - i * n);
        kq[c] = 0.0;
    }
    for (int k = 0; k < n; ++k) {
#pragma unroll
        for (int c = 0; c < PROP_QN; ++c) kq[c] = fma(X[wi[c] + k], S[sj[c] + k * n], kq[c]);
    }
}

// rk4_steps with group offsets (see there).
__device__ void rk4_steps_g(double (&psi)[PROP_QN], double (&dps)[PROP_QN], double *S0, double *S1, double *W0,
                            double *W1, const double *As, const double *eps_s, const double *lt_s, int n, int GT,
                            int lmax, double z, double r_start, double hh, int nsub, int tid)
{
    const double h2 = 0.5 * hh, h3 = hh / 3.0, h6 = hh / 6.0;
    double yp[PROP_QN], yq[PROP_QN], tq[PROP_QN], kq[PROP_QN];
    __syncthreads();
#pragma unroll
    for (int c = 0; c < PROP_QN; ++c)
        if (tid + c * NT < GT) S0[tid + c * NT] = psi[c];
    build_w_g(W0, As, eps_s, lt_s, n, GT, lmax, z, r_start, 1.0, tid);
    __syncthreads();
    for (int s = 0; s < nsub; ++s) {
        const double r0 = r_start + s * hh;
        mat_times_g(kq, W0, S0, n, GT, tid);
#pragma unroll
        for (int c = 0; c < PROP_QN; ++c) {
            const int q = tid + c * NT;
            yp[c] = fma(h6, dps[c], psi[c]);
            yq[c] = fma(h6, kq[c], dps[c]);
            tq[c] = fma(h2, kq[c], dps[c]);
            if (q < GT) S1[q] = fma(h2, dps[c], psi[c]);
        }
        build_w_g(W1, As, eps_s, lt_s, n, GT, lmax, z, r0 + h2, 1.0, tid);
        __syncthreads();
        mat_times_g(kq, W1, S1, n, GT, tid);
#pragma unroll
        for (int c = 0; c < PROP_QN; ++c) {
            const int q = tid + c * NT;
            const double kp = tq[c];
            yp[c] = fma(h3, kp, yp[c]);
            yq[c] = fma(h3, kq[c], yq[c]);
            tq[c] = fma(h2, kq[c], dps[c]);
            if (q < GT) S0[q] = fma(h2, kp, psi[c]);
        }
        __syncthreads();
        mat_times_g(kq, W1, S0, n, GT, tid);
#pragma unroll
        for (int c = 0; c < PROP_QN; ++c) {
            const int q = tid + c * NT;
            const double kp = tq[c];
            yp[c] = fma(h3, kp, yp[c]);
            yq[c] = fma(h3, kq[c], yq[c]);
            tq[c] = fma(hh, kq[c], dps[c]);
            if (q < GT) S1[q] = fma(hh, kp, psi[c]);
        }
        build_w_g(W0, As, eps_s, lt_s, n, GT, lmax, z, r0 + hh, 1.0, tid);
        __syncthreads();
        mat_times_g(kq, W0, S1, n, GT, tid);
#pragma unroll
        for (int c = 0; c < PROP_QN; ++c) {
            const int q = tid + c * NT;
            psi[c] = fma(h6, tq[c], yp[c]);
            dps[c] = fma(h6, kq[c], yq[c]);
            if (q < GT) S0[q] = psi[c];
        }
        __syncthreads();
    }
}

// Gauss-Jordan with partial pivoting of the n x 2n matrix M (row stride
// 2n + 1, n <= 32) by one warp, row r on lane r: [G^T | 1] -> [1 | G^{-T}].
// Warp-uniform result: false on a zero or non-finite pivot.
__device__ bool warp_gauss_jordan(double *M, int n, int lane)
{
    const unsigned full = 0xffffffffu;
    const int ld = 2 * n + 1, w = 2 * n;
    for (int c = 0; c < n; ++c) {
        double v = (lane >= c && lane < n) ? fabs(M[lane * ld + c]) : -1.0;
        int idx = lane;
        for (int off = 16; off > 0; off >>= 1) {
            const double ov = __shfl_down_sync(full, v, off);
            const int oi = __shfl_down_sync(full, idx, off);
            if (ov > v || (ov == v && oi < idx)) {
                v = ov;
                idx = oi;
            }
        }
        v = __shfl_sync(full, v, 0);
        const int p = __shfl_sync(full, idx, 0);
        if (!(v > 0.0) || !isfinite(v)) return false;
        if (p != c) {
            for (int col = lane; col < w; col += 32) {
                const double t = M[c * ld + col];
                M[c * ld + col] = M[p * ld + col];
                M[p * ld + col] = t;
            }
        }
        __syncwarp();
        const double inv = 1.0 / M[c * ld + c];
        __syncwarp();
        for (int col = lane; col < w; col += 32) M[c * ld + col] *= inv;
        __syncwarp();
        if (lane < n && lane != c) {
            const double f = M[lane * ld + c];
            for (int col = c; col < w; ++col) M[lane * ld + col] = fma(-f, M[c * ld + col], M[lane * ld + col]);
        }
        __syncwarp();
    }
    return true;
}

// Per group: M_g (at sm + g n (2n + 1)) <- [G_g^T | 1] from gv at the owned
// elements, then [1 | G_g^{-T}]; a group whose G is singular is marked in
// gbad. Starts after the caller's barrier; ends with a barrier.
__device__ void invert_groups(const double (&gv)[PROP_QN], double *sm, int n, int G, int *gbad, int tid)
{
    const int n2 = n * n, ld = 2 * n + 1, GT = G * n2;
    for (int q = tid; q < G * n * ld; q += NT) sm[q] = 0.0;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < PROP_QN; ++c) {
        const int qt = tid + c * NT;
        if (qt < GT) {
            const int g = qt / n2, ql = qt - g * n2;
            const int i = ql / n, j = ql - (ql / n) * n;
            double *M = sm + g * n * ld;
            M[j * ld + i] = gv[c];
            if (i == j) M[j * ld + n + i] = 1.0;
        }
    }
    __syncthreads();
    const int lane = tid & 31;
    for (int g = tid >> 5; g < G; g += NT / 32)
        if (!warp_gauss_jordan(sm + g * n * ld, n, lane) && lane == 0) gbad[g] = 1;
    __syncthreads();
}

// x <- x G_g^{-1} at the owned elements (G_g^{-T} in M_g as invert_groups
// leaves it), staged through SX (G n^2 doubles past the M_g).
__device__ void times_ginv_g(double (&x)[PROP_QN], const double *sm, double *SX, int n, int GT, int tid)
{
    const int n2 = n * n, ld = 2 * n + 1;
#pragma unroll
    for (int c = 0; c < PROP_QN; ++c)
        if (tid + c * NT < GT) SX[tid + c * NT] = x[c];
    __syncthreads();
#pragma unroll
    for (int c = 0; c < PROP_QN; ++c) {
        const int qt = min(tid + c * NT, GT - 1);
        const int g = qt / n2, ql = qt - g * n2;
        const int i = ql / n, j = ql - (ql / n) * n;
        const double *M = sm + g * n * ld;
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc = fma(SX[g * n2 + i * n + k], M[j * ld + n + k], acc);
        x[c] = acc;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(NT, 2) propagate_small_kernel(PwDev pw, const double *__restrict__ E, int nE,
                                                                const double *__restrict__ A, int lmax, double r1,
                                                                int steps, double *__restrict__ Rp,
                                                                int *__restrict__ status)
{
    extern __shared__ double sm[];
    __shared__ double eps_s[PROP_MAX_GROUPS * 4], lt_s[PROP_SMALL_MAXN];
    __shared__ int gvalid[PROP_MAX_GROUPS], gbad[PROP_MAX_GROUPS];
    const int tid = threadIdx.x;
    const int n = pw.n, n2 = n * n, G = prop_groups(n), GT = G * n2;
    const int e0 = blockIdx.x * G;
    double *SF = sm, *SG = sm + GT, *TA = sm + 2 * GT, *TB = sm + 3 * GT, *As = sm + 4 * GT;
    const double a = pw.a, b = pw.b, z = pw.z;
    for (int q = tid; q < lmax * n2; q += NT) As[q] = A[q];
    for (int q = tid; q < G * n; q += NT) {
        const int g = q / n, i = q - g * n;
        eps_s[q] = E[min(e0 + g, nE - 1)] - pw.e_thr[i];
    }
    for (int i = tid; i < n; i += NT) lt_s[i] = (double)pw.l[i] * (pw.l[i] + 1);
    for (int g = tid; g < G; g += NT) {
        gvalid[g] = e0 + g < nE && status[e0 + g] == RM_OK;
        gbad[g] = 0;
    }
    const double h = (r1 - a) / steps, t12 = h * h / 12.0;
    double psi[PROP_QN], dl[PROP_QN], tp[PROP_QN], tpp[PROP_QN], kq[PROP_QN];
#pragma unroll
    for (int c = 0; c < PROP_QN; ++c) {
        const int qt = tid + c * NT;
        psi[c] = dl[c] = 0.0;
        if (qt < GT) {
            const int g = qt / n2, ql = qt - g * n2;
            const int i = ql / n, j = ql - (ql / n) * n;
            const double *Re = Rp + (size_t)min(e0 + g, nE - 1) * tri_ld(n);
            psi[c] = Re[i <= j ? tri_idx(i, j, n) : tri_idx(j, i, n)];
            dl[c] = ((i == j ? 1.0 : 0.0) + b * psi[c]) / a;
            SF[qt] = psi[c];
        }
    }
    __syncthreads();
    build_w_g(TA, As, eps_s, lt_s, n, GT, lmax, z, a, t12, tid);
    __syncthreads();
    mat_times_g(tpp, TA, SF, n, GT, tid);
    {
        double p0[PROP_QN];
#pragma unroll
        for (int c = 0; c < PROP_QN; ++c) p0[c] = psi[c];
        rk4_steps_g(psi, dl, SF, SG, TA, TB, As, eps_s, lt_s, n, GT, lmax, z, a, h / PROP_START_SUB,
                    PROP_START_SUB, tid);
#pragma unroll
        for (int c = 0; c < PROP_QN; ++c) dl[c] = psi[c] - p0[c];
    }
    build_w_g(TA, As, eps_s, lt_s, n, GT, lmax, z, a + h, t12, tid);
    __syncthreads();
    mat_times_g(tp, TA, SF, n, GT, tid);
    int sector = steps;
    {
        double k2 = 0.0;
        for (int q = 0; q < G * n; ++q) k2 = fmax(k2, lt_s[q % n] / (a * a) - eps_s[q]);
        const double m = k2 > 0.0 ? 1.0 / (sqrt(k2) * h) : (double)steps;
        sector = m >= (double)steps ? steps : max(1, (int)m);
    }
    __syncthreads();
    double *SX = sm + 3 * GT;
    for (int k = 1; k <= steps; ++k) {
        double *Tk = (k & 1) ? TB : TA;
#pragma unroll
        for (int c = 0; c < PROP_QN; ++c) {
            const int q = tid + c * NT;
            if (q < GT) SF[q] = psi[c] + dl[c] + fma(10.0, tp[c], tpp[c]);
        }
        build_w_g(Tk, As, eps_s, lt_s, n, GT, lmax, z, a + (k + 1) * h, t12, tid);
        __syncthreads();
        mat_times_g(kq, Tk, SF, n, GT, tid);
#pragma unroll
        for (int c = 0; c < PROP_QN; ++c)
            if (tid + c * NT < GT) SG[tid + c * NT] = kq[c];
        __syncthreads();
        double g2[PROP_QN];
        mat_times_g(g2, Tk, SG, n, GT, tid);
        const bool last = k == steps;
#pragma unroll
        for (int c = 0; c < PROP_QN; ++c) {
            const double tn = kq[c] + g2[c];
            const double d = dl[c] + tn + fma(10.0, tp[c], tpp[c]);
            if (!last) {
                dl[c] = d;
                psi[c] += d;
                tpp[c] = tp[c];
                tp[c] = tn;
            } else {
                dl[c] = (d + dl[c]) / (2.0 * h) - (tn - tpp[c]) / h;
            }
        }
        if (k % sector == 0 && k + 1 < steps) {
            const double r = a + (k + 1) * h;
            double gv[PROP_QN];
#pragma unroll
            for (int c = 0; c < PROP_QN; ++c) gv[c] = fma(r / h, dl[c], -b * psi[c]);
            __syncthreads();
            invert_groups(gv, sm, n, G, gbad, tid);
            times_ginv_g(psi, sm, SX, n, GT, tid);
            times_ginv_g(dl, sm, SX, n, GT, tid);
            times_ginv_g(tp, sm, SX, n, GT, tid);
            times_ginv_g(tpp, sm, SX, n, GT, tid);
        }
    }
    double gv[PROP_QN];
#pragma unroll
    for (int c = 0; c < PROP_QN; ++c) gv[c] = fma(r1, dl[c], -b * psi[c]);
    __syncthreads();
    invert_groups(gv, sm, n, G, gbad, tid);
    times_ginv_g(psi, sm, SX, n, GT, tid);
#pragma unroll
    for (int c = 0; c < PROP_QN; ++c)
        if (tid + c * NT < GT) SX[tid + c * NT] = psi[c];
    __syncthreads();
    const int tc = tri_count(n);
    for (int q = tid; q < G * tc; q += NT) {
        const int g = q / tc;
        if (!gvalid[g] || gbad[g]) continue;
        int i, j;
        tri_pair(q - g * tc, n, i, j);
        double *Re = Rp + (size_t)(e0 + g) * tri_ld(n);
        Re[tri_idx(i, j, n)] = 0.5 * (SX[g * n2 + i * n + j] + SX[g * n2 + j * n + i]);
    }
    for (int g = tid; g < G; g += NT)
        if (gvalid[g] && gbad[g]) atomicCAS(status + e0 + g, RM_OK, RM_ESINGULAR);
}

}  // namespace

bool propagate_fits(int n, int lmax)
{
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        optin = 227 * 1024;
    }
    return propagate_smem(n, lmax) <= (size_t)optin;
}

size_t propagate_smem(int n, int lmax)
{
    const int gt = n <= PROP_SMALL_MAXN ? prop_groups(n) * n * n : n * n;
    return ((size_t)4 * gt + (size_t)lmax * n * n) * sizeof(double);
}

cudaError_t launch_propagate(const PwDev &pw, const double *E, int nE, const double *A, int lmax, double r1,
                             int steps, double *Rp, int *status, cudaStream_t s)
{
    if (pw.n > PROP_MAXN || lmax < 0 || lmax > PROP_MAX_LAMBDA || steps < 2 || !propagate_fits(pw.n, lmax))
        return cudaErrorInvalidValue;
    if (nE == 0) return cudaSuccess;
    const size_t smem = propagate_smem(pw.n, lmax);
    if (pw.n <= PROP_SMALL_MAXN) {
        cudaError_t err =
            cudaFuncSetAttribute(propagate_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        const int G = prop_groups(pw.n);
        propagate_small_kernel<<<(nE + G - 1) / G, NT, smem, s>>>(pw, E, nE, A, lmax, r1, steps, Rp, status);
        return cudaGetLastError();
    }
    if (pw.n <= 32) {
        cudaError_t err =
            cudaFuncSetAttribute(propagate_kernel<256, 4, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        propagate_kernel<256, 4, 32><<<nE, 256, smem, s>>>(pw, E, A, lmax, r1, steps, Rp, status);
        return cudaGetLastError();
    }
    cudaError_t err =
        cudaFuncSetAttribute(propagate_kernel<512, 8, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    propagate_kernel<512, 8, 64><<<nE, 512, smem, s>>>(pw, E, A, lmax, r1, steps, Rp, status);
    return cudaGetLastError();
}

}  // namespace rmgb
