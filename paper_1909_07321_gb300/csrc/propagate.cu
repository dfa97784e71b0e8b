// Outer-region propagation with the long-range multipole potential
// (Section "Overview", Eq. radial with U != 0; namelist variable ipert): the
// coupled radial functions are carried from the inner-region boundary r0 = a
// to the asymptotic radius r1 and matched there.
//
// In Rydberg units
//   u_i'' = sum_j W_ij(r) u_j,  W(r) = diag(l_i(l_i+1)/r^2 - 2z/r - eps_i) + U(r),
//   U(r) = sum_{lambda=1..lambda_max} A^lambda / r^(lambda+1)  (A^lambda symmetric).
// The R-matrix at a fixes the solution matrix Psi by Psi(a) = R(a),
// a Psi'(a) - b Psi(a) = 1; Psi and Psi' are integrated to r1 by the
// classical fourth-order Runge-Kutta method with a fixed number of steps,
// and R(r1) = Psi(r1) [r1 Psi'(r1) - b Psi(r1)]^{-1} (symmetric; it replaces
// R(a) in the matching, done at r1). One CTA of NT threads per energy, all
// matrices in shared memory, FP64.
#include <math.h>

#include "dense_smem.cuh"
#include "rm_internal.cuh"

namespace rmgb {
namespace {

// Shared memory: Psi, Psi', their RK4 accumulators, the stage inputs, W Psi
// and W (8 n^2 doubles), then the coefficients A (lambda_max n^2).
__global__ void __launch_bounds__(NT) propagate_kernel(PwDev pw, const double *__restrict__ E,
                                                      const double *__restrict__ A, int lmax, double r1,
                                                      int steps, double *__restrict__ Rp, int *__restrict__ status)
{
    extern __shared__ double sm[];
    __shared__ double eps_s[PROP_MAXN], lt_s[PROP_MAXN];
    __shared__ ElimShared esh;
    const int e = blockIdx.x, tid = threadIdx.x;
    const int n = pw.n, n2 = n * n;
    if (status[e] != RM_OK) return;
    double *Psi = sm, *P = sm + n2, *Yp = sm + 2 * n2, *Yq = sm + 3 * n2;
    double *Tp = sm + 4 * n2, *Tq = sm + 5 * n2, *Kq = sm + 6 * n2, *Wm = sm + 7 * n2;
    double *As = sm + 8 * n2;
    const double a = pw.a, b = pw.b, z = pw.z, x = E[e];
    double *Re = Rp + (size_t)e * tri_ld(n);
    for (int q = tid; q < lmax * n2; q += NT) As[q] = A[q];
    for (int i = tid; i < n; i += NT) {
        eps_s[i] = x - pw.e_thr[i];
        lt_s[i] = (double)pw.l[i] * (pw.l[i] + 1);
    }
    for (int q = tid; q < n2; q += NT) {
        const int i = q / n, j = q - (q / n) * n;
        const double r = Re[i <= j ? tri_idx(i, j, n) : tri_idx(j, i, n)];
        Psi[q] = r;
        P[q] = ((i == j ? 1.0 : 0.0) + b * r) / a;
    }
    __syncthreads();
    const double h = (r1 - a) / steps;
    // RK4: stage inputs (Tp, Tq), slopes (Tq, W Tp); weights and offsets
    const double cw[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    const double dn[4] = {0.5, 0.5, 1.0, 0.0};
    const double off[4] = {0.0, 0.5, 0.5, 1.0};
    for (int s = 0; s < steps; ++s) {
        const double r0 = a + s * h;
#pragma unroll
        for (int st = 0; st < 4; ++st) {
            const double r = r0 + off[st] * h;
            const double *ip = st == 0 ? Psi : Tp;   // stage input
            const double *iq = st == 0 ? P : Tq;
            // W(r)
            const double ir = 1.0 / r;
            for (int q = tid; q < n2; q += NT) {
                const int i = q / n, j = q - (q / n) * n;
                double u = 0.0, rp = ir * ir;
                for (int lam = 0; lam < lmax; ++lam) {
                    u = fma(As[lam * n2 + q], rp, u);
                    rp *= ir;
                }
                if (i == j) u += lt_s[i] * ir * ir - 2.0 * z * ir - eps_s[i];
                Wm[q] = u;
            }
            __syncthreads();
            // W Tp
            for (int q = tid; q < n2; q += NT) {
                const int i = q / n, j = q - (q / n) * n;
                double acc = 0.0;
                for (int k = 0; k < n; ++k) acc = fma(Wm[i * n + k], ip[k * n + j], acc);
                Kq[q] = acc;
            }
            __syncthreads();
            // accumulate and form the next stage's input
            const double wh = cw[st] * h, dh = dn[st] * h;
            for (int q = tid; q < n2; q += NT) {
                const double kp = iq[q], kq = Kq[q];
                Yp[q] = (st == 0 ? Psi[q] : Yp[q]) + wh * kp;
                Yq[q] = (st == 0 ? P[q] : Yq[q]) + wh * kq;
                if (st < 3) {
                    Tp[q] = Psi[q] + dh * kp;
                    Tq[q] = P[q] + dh * kq;
                }
            }
            __syncthreads();
        }
        double *t0 = Psi, *t1 = P;
        Psi = Yp;
        P = Yq;
        Yp = t0;
        Yq = t1;
    }
    // R(r1)^T = (r1 Psi' - b Psi)^{-T} Psi^T: eliminate [ (r1 Psi' - b Psi)^T | Psi^T ]
    // (n x 2n, over Tp..Kq, which hold 3 n^2 doubles)
    double *M = Tp;
    const int ld = 2 * n + 1;
    for (int q = tid; q < n2; q += NT) {
        const int i = q / n, j = q - (q / n) * n;
        M[j * ld + i] = r1 * P[q] - b * Psi[q];
        M[j * ld + n + i] = Psi[q];
    }
    if (tid == 0) esh.bad = 0;
    __syncthreads();
    block_eliminate<double>(M, ld, n, 2 * n, &esh);
    if (esh.bad) {
        if (tid == 0) atomicCAS(status + e, RM_OK, RM_ESINGULAR);
        return;
    }
    block_backsub<double>(M, ld, n, n, n, 0);
    for (int q = tid; q < tri_count(n); q += NT) {
        int i, j;
        tri_pair(q, n, i, j);
        Re[tri_idx(i, j, n)] = 0.5 * (M[i * ld + n + j] + M[j * ld + n + i]);
    }
}

}  // namespace

size_t propagate_smem(int n, int lmax) { return (size_t)(8 + lmax) * n * n * sizeof(double); }

cudaError_t launch_propagate(const PwDev &pw, const double *E, int nE, const double *A, int lmax, double r1,
                             int steps, double *Rp, int *status, cudaStream_t s)
{
    if (pw.n > PROP_MAXN || lmax < 0 || lmax > PROP_MAX_LAMBDA || steps < 1) return cudaErrorInvalidValue;
    if (nE == 0) return cudaSuccess;
    const size_t smem = propagate_smem(pw.n, lmax);
    cudaError_t err = cudaFuncSetAttribute(propagate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    propagate_kernel<<<nE, NT, smem, s>>>(pw, E, A, lmax, r1, steps, Rp, status);
    return cudaGetLastError();
}

}  // namespace rmgb
