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
// R(a) in the matching, done at r1). The integration restarts from R(r) at
// sector boundaries 1 / kappa_max apart (R does not depend on the basis of
// solutions carried), so that closed channels growing as exp(kappa r) do not
// swamp the other columns. One CTA of NT threads per energy, FP64.
// A step costs four products W Psi (4 n^3 FMA) and two builds of W: the
// kernel runs on the FP64 pipe.
#include <math.h>

#include "dense_smem.cuh"
#include "rm_internal.cuh"

namespace rmgb {
namespace {

// Elements of an n x n matrix one thread owns (q = tid + c NT, c < PROP_QN).
constexpr int PROP_QN = (PROP_MAXN * PROP_MAXN + NT - 1) / NT;

// W(r) at the owned elements into Wd: sum_lambda A^lambda r^-(lambda+1) plus
// the diagonal l(l+1)/r^2 - 2z/r - eps.
__device__ __forceinline__ void build_w(double *Wd, const double *As, const double *eps_s, const double *lt_s,
                                        int n, int lmax, double z, double r, int tid)
{
    const int n2 = n * n;
    const double ir = 1.0 / r;
#pragma unroll
    for (int c = 0; c < PROP_QN; ++c) {
        const int q = tid + c * NT;
        if (q < n2) {
            const int i = q / n, j = q - (q / n) * n;
            double u = 0.0, rp = ir * ir;
            for (int lam = 0; lam < lmax; ++lam) {
                u = fma(As[lam * n2 + q], rp, u);
                rp *= ir;
            }
            if (i == j) u += lt_s[i] * ir * ir - 2.0 * z * ir - eps_s[i];
            Wd[q] = u;
        }
    }
}

// (W S) at the owned elements, the PROP_QN dot products interleaved.
__device__ __forceinline__ void w_times(double (&kq)[PROP_QN], const double *Wd, const double *S, int n, int tid)
{
    const int n2 = n * n;
    int wi[PROP_QN], sj[PROP_QN];
#pragma unroll
    for (int c = 0; c < PROP_QN; ++c) {
        const int q = min(tid + c * NT, n2 - 1);
        wi[c] = (q / n) * n;
        sj[c] = q - wi[c];
        kq[c] = 0.0;
    }
#pragma unroll 2
    for (int k = 0; k < n; ++k) {
#pragma unroll
        for (int c = 0; c < PROP_QN; ++c) kq[c] = fma(Wd[wi[c] + k], S[k * n + sj[c]], kq[c]);
    }
}

// Psi <- Psi G^{-1}, Psi' <- Psi' G^{-1} with G = r Psi' - b Psi at the
// owned elements (then Psi = R(r) and r Psi' - b Psi = 1), by eliminating
// [ G^T | Psi^T ] over M (n x 2n, row stride 2n + 1; the caller's 3 n^2
// doubles of scratch). The new Psi also goes to S. False if G is singular.
__device__ bool restart_from_r(double (&psi)[PROP_QN], double (&dps)[PROP_QN], double *S, double *M, int n,
                               double b, double r, ElimShared *esh, int tid)
{
    const int n2 = n * n, ld = 2 * n + 1;
#pragma unroll
    for (int c = 0; c < PROP_QN; ++c) {
        const int q = tid + c * NT;
        if (q < n2) {
            const int i = q / n, j = q - (q / n) * n;
            M[j * ld + i] = r * dps[c] - b * psi[c];
            M[j * ld + n + i] = psi[c];
        }
    }
    if (tid == 0) esh->bad = 0;
    __syncthreads();
    block_eliminate<double>(M, ld, n, 2 * n, esh);
    if (esh->bad) return false;
    block_backsub<double>(M, ld, n, n, n, 0);
#pragma unroll
    for (int c = 0; c < PROP_QN; ++c) {
        const int q = tid + c * NT;
        if (q < n2) {
            const int i = q / n, j = q - (q / n) * n;
            psi[c] = M[j * ld + n + i];
            dps[c] = ((i == j ? 1.0 : 0.0) + b * psi[c]) / r;
            S[q] = psi[c];
        }
    }
    __syncthreads();
    return true;
}

// One CTA per energy. The solution Psi and its derivative at the owned
// elements stay in registers with the RK4 accumulators; shared memory holds
// what the products W S read across threads: the stage input of Psi (two
// buffers, alternating by stage) and W (two buffers: at r0 and r0 + h/2;
// W(r0 + h) is built over the first once stage 1 is done with it), then the
// coefficients A. One barrier per stage.
__global__ void __launch_bounds__(NT, 2) propagate_kernel(PwDev pw, const double *__restrict__ E,
                                                          const double *__restrict__ A, int lmax, double r1,
                                                          int steps, double *__restrict__ Rp,
                                                          int *__restrict__ status)
{
    extern __shared__ double sm[];
    __shared__ double eps_s[PROP_MAXN], lt_s[PROP_MAXN];
    __shared__ ElimShared esh;
    const int e = blockIdx.x, tid = threadIdx.x;
    const int n = pw.n, n2 = n * n;
    if (status[e] != RM_OK) return;
    double *S0 = sm, *S1 = sm + n2, *W0 = sm + 2 * n2, *W1 = sm + 3 * n2, *As = sm + 4 * n2;
    const double a = pw.a, b = pw.b, z = pw.z, x = E[e];
    double *Re = Rp + (size_t)e * tri_ld(n);
    for (int q = tid; q < lmax * n2; q += NT) As[q] = A[q];
    for (int i = tid; i < n; i += NT) {
        eps_s[i] = x - pw.e_thr[i];
        lt_s[i] = (double)pw.l[i] * (pw.l[i] + 1);
    }
    double psi[PROP_QN], dps[PROP_QN], yp[PROP_QN], yq[PROP_QN], tq[PROP_QN], kq[PROP_QN];
#pragma unroll
    for (int c = 0; c < PROP_QN; ++c) {
        const int q = tid + c * NT;
        psi[c] = dps[c] = yp[c] = yq[c] = tq[c] = 0.0;
        if (q < n2) {
            const int i = q / n, j = q - (q / n) * n;
            psi[c] = Re[i <= j ? tri_idx(i, j, n) : tri_idx(j, i, n)];
            dps[c] = ((i == j ? 1.0 : 0.0) + b * psi[c]) / a;
            S0[q] = psi[c];
        }
    }
    __syncthreads();
    build_w(W0, As, eps_s, lt_s, n, lmax, z, a, tid);
    const double h = (r1 - a) / steps, h2 = 0.5 * h, h3 = h / 3.0, h6 = h / 6.0;
    // restart from R every `sector` steps, a sector being 1 / kappa_max long,
    // kappa_max^2 = max_i (l_i(l_i+1)/a^2 - eps_i)
    int sector = steps;
    {
        double k2 = 0.0;
        for (int i = 0; i < n; ++i) k2 = fmax(k2, lt_s[i] / (a * a) - eps_s[i]);
        const double m = k2 > 0.0 ? 1.0 / (sqrt(k2) * h) : (double)steps;
        sector = m >= (double)steps ? steps : max(1, (int)m);
    }
    __syncthreads();
    for (int s = 0; s < steps; ++s) {
        const double r0 = a + s * h;
        // stage 1 at r0: input Psi (S0), W0; writes the stage-2 input to S1
        w_times(kq, W0, S0, n, tid);
#pragma unroll
        for (int c = 0; c < PROP_QN; ++c) {
            const int q = tid + c * NT;
            yp[c] = fma(h6, dps[c], psi[c]);
            yq[c] = fma(h6, kq[c], dps[c]);
            tq[c] = fma(h2, kq[c], dps[c]);
            if (q < n2) S1[q] = fma(h2, dps[c], psi[c]);
        }
        build_w(W1, As, eps_s, lt_s, n, lmax, z, r0 + h2, tid);
        __syncthreads();
        // stage 2 at r0 + h/2: input S1, W1; writes the stage-3 input to S0
        w_times(kq, W1, S1, n, tid);
#pragma unroll
        for (int c = 0; c < PROP_QN; ++c) {
            const int q = tid + c * NT;
            const double kp = tq[c];
            yp[c] = fma(h3, kp, yp[c]);
            yq[c] = fma(h3, kq[c], yq[c]);
            tq[c] = fma(h2, kq[c], dps[c]);
            if (q < n2) S0[q] = fma(h2, kp, psi[c]);
        }
        __syncthreads();
        // stage 3 at r0 + h/2: input S0, W1; writes the stage-4 input to S1
        // and W(r0 + h) over W0
        w_times(kq, W1, S0, n, tid);
#pragma unroll
        for (int c = 0; c < PROP_QN; ++c) {
            const int q = tid + c * NT;
            const double kp = tq[c];
            yp[c] = fma(h3, kp, yp[c]);
            yq[c] = fma(h3, kq[c], yq[c]);
            tq[c] = fma(h, kq[c], dps[c]);
            if (q < n2) S1[q] = fma(h, kp, psi[c]);
        }
        build_w(W0, As, eps_s, lt_s, n, lmax, z, r0 + h, tid);
        __syncthreads();
        // stage 4 at r0 + h: input S1, W0; the new Psi goes to S0
        w_times(kq, W0, S1, n, tid);
#pragma unroll
        for (int c = 0; c < PROP_QN; ++c) {
            const int q = tid + c * NT;
            psi[c] = fma(h6, tq[c], yp[c]);
            dps[c] = fma(h6, kq[c], yq[c]);
            if (q < n2) S0[q] = psi[c];
        }
        __syncthreads();
        if ((s + 1) % sector == 0 && s + 1 < steps) {
            // R(r) = Psi (r Psi' - b Psi)^{-1} does not depend on the basis
            // of solutions Psi holds: continue from Psi = R(r),
            // r Psi' - b Psi = 1, so that growing closed channels never
            // swamp the other columns
            const double r = a + (s + 1) * h;
            if (!restart_from_r(psi, dps, S0, S1, n, b, r, &esh, tid)) {
                if (tid == 0) atomicCAS(status + e, RM_OK, RM_ESINGULAR);
                return;
            }
            build_w(W0, As, eps_s, lt_s, n, lmax, z, r, tid);
            __syncthreads();
        }
    }
    // R(r1) = Psi (r1 Psi' - b Psi)^{-1}, written symmetrised
    if (!restart_from_r(psi, dps, S0, S1, n, b, r1, &esh, tid)) {
        if (tid == 0) atomicCAS(status + e, RM_OK, RM_ESINGULAR);
        return;
    }
    for (int q = tid; q < tri_count(n); q += NT) {
        int i, j;
        tri_pair(q, n, i, j);
        Re[tri_idx(i, j, n)] = 0.5 * (S0[i * n + j] + S0[j * n + i]);
    }
}

}  // namespace

size_t propagate_smem(int n, int lmax) { return (size_t)(4 + lmax) * n * n * sizeof(double); }

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
