// Steps (c) and (d) for n <= SOLVE_SMALL_MAXN channels: one CTA per energy,
// everything in shared memory, FP64.
//
// (c) Matching (Section "Overview", Eq. match). Channels split into the set P
// whose amplitudes are unknowns of K (open channels, plus in MQDT mode the
// closed channels eliminated by quantum-defect theory) and the remaining
// closed channels, which keep their decaying boundary condition. With
// psi_ij = S_i delta_ij + Ghat_i X_ij (S, Ghat = s, c open; f, g MQDT; theta
// decaying, no S), psi(a) = R (a psi'(a) - b psi(a)) gives
//   [diag(Ghat) - R diag(a Ghat' - b Ghat)] X = -[diag(S) - R diag(a S' - b S)] P.
// Unknowns are ordered decaying-closed first, so after Gaussian elimination
// with partial pivoting of [A | B] the P unknowns are the trailing rows of
// the triangular system: back-substitution runs over those rows only, giving
// K_u = X[P rows] (the physical K in direct mode).
// MQDT (Section "namelist stgf MQDT variables", iqdt): with o = open and
// c = eliminated channels of P,
//   K = K_oo - K_oc (K_cc + diag(tan pi nu))^{-1} K_co.
//
// (d) T = 2iK(1 - iK)^{-1} (Section "Glossary of terms") in real form. K is
// symmetric, so with M = 1 + K^2 (SPD), X = M^{-1} K and Y = M^{-1} K^2 =
// 1 - M^{-1}:
//   T = -2Y + 2iX,  |T_ab|^2 = 4 (X_ab^2 + Y_ab^2).
// M^{-1} by the symmetric sweep operator; X from one product (upper
// triangle: X is symmetric). Then for target levels I <= J, one thread owns
// Omega_IJ(E) and adds g sum_{a in I, b in J} |T_ab|^2 in a fixed order, so
// the accumulation is deterministic (no atomics).
// The FP32 variant of the mixed-precision path is solve_f32.cu.
#include <math.h>

#include "dense_smem.cuh"
#include "rm_internal.cuh"

namespace rmgb {
namespace {

__global__ void __launch_bounds__(NT) solve_small_kernel(
    PwDev pw, const double *__restrict__ E, const ChanFn *__restrict__ cfa,
    const double *__restrict__ Ra, int *__restrict__ status, double *__restrict__ K_out,
    int *__restrict__ n_open_out, double *__restrict__ omega, int n_tri, int mqdt_layout,
    const int *__restrict__ deep_ws, int deep_cap, int pass, double *__restrict__ ku_out,
    int *__restrict__ ku_np)
{
    // Energies holding a deep (near-threshold) channel pair are solved in
    // pass 1, after their channel data is complete; the others in pass 0.
    if (deep_ws) {
        const bool deferred = deep_ws[0] <= deep_cap && deep_ws[1 + deep_cap + blockIdx.x] != 0;
        if (pass == 0 ? deferred : !deferred) return;
    }
    extern __shared__ double sm[];
    __shared__ int col_chan[SOLVE_SMALL_MAXN];   // unknown column -> channel
    __shared__ int open_pos[SOLVE_SMALL_MAXN];   // channel -> open position (-1 otherwise)
    __shared__ int qpos[SOLVE_SMALL_MAXN];       // MQDT channel k -> its position in P
    __shared__ int opos[SOLVE_SMALL_MAXN];       // open channel k -> its position in P
    __shared__ double vcol[SOLVE_SMALL_MAXN];
    __shared__ int s_no, s_np, s_nq;
    __shared__ ElimShared esh;

    const int e = blockIdx.x;
    const int n = pw.n;
    const int tid = threadIdx.x;
    const double x = E[e];
    const ChanFn *cf = cfa + (size_t)e * n;
    const double *Rp = Ra + (size_t)e * tri_ld(n);   // packed upper triangle
    const bool ok_status = status[e] == RM_OK;

    if (tid == 0) {
        int no = 0;
        for (int i = 0; i < n; ++i) no += (x - pw.e_thr[i] > 0.0);
        if (n_open_out) n_open_out[e] = no;
        s_no = no;
        esh.bad = 0;
        if (ok_status) {
            int np = 0;
            for (int i = 0; i < n; ++i) np += (cf[i].kind != CH_CLOSED);
            const int ncl = n - np;
            int pc = 0, pp = 0, po = 0, pq = 0;
            for (int i = 0; i < n; ++i) {
                const int k = cf[i].kind;
                if (k == CH_CLOSED) {
                    col_chan[pc++] = i;
                    open_pos[i] = -1;
                } else {
                    col_chan[ncl + pp] = i;
                    if (k == CH_OPEN) {
                        open_pos[i] = po;
                        opos[po++] = pp;
                    } else {
                        open_pos[i] = -1;
                        qpos[pq++] = pp;
                    }
                    ++pp;
                }
            }
            s_np = np;
            s_nq = pq;
        }
    }
    __syncthreads();
    const int no = s_no;
    if (!ok_status || no == 0) return;
    const int np = s_np, nq = s_nq, ncl = n - np;

    const int w = n + np;        // augmented width
    const int ld = w + 1;        // padded row stride
    using Real = double;
    Real *M = sm;
    const double a = pw.a, b = pw.b;

    // ---- assemble [A | B] -------------------------------------------------
    for (int q = tid; q < n * w; q += NT) {
        const int r = q / w, c = q - (q / w) * w;
        double v;
        if (c < n) {
            const int j = col_chan[c];
            const ChanFn cj = cf[j];
            v = -Rp[r <= j ? tri_idx(r, j, n) : tri_idx(j, r, n)] * (a * cj.ghp - b * cj.gh);
            if (r == j) v += cj.gh;
        } else {
            const int o = col_chan[ncl + (c - n)];
            const ChanFn co = cf[o];
            v = Rp[r <= o ? tri_idx(r, o, n) : tri_idx(o, r, n)] * (a * co.sp - b * co.s);
            if (r == o) v -= co.s;
        }
        M[r * ld + c] = (Real)v;
    }
    __syncthreads();

    block_eliminate<Real>(M, ld, n, w, &esh);
    if (esh.bad) {
        if (tid == 0) status[e] = RM_ESINGULAR;
        return;
    }
    block_backsub<Real>(M, ld, n, n, np, ncl);   // K_u = rows ncl.. of the RHS columns
    if (ku_out) {
        // K_u itself (P channels in channel order), for interpolation between energies
        for (int q = tid; q < np * np; q += NT) {
            const int p = q / np, r = q - (q / np) * np;
            ku_out[(size_t)e * n * n + (size_t)p * n + r] = (double)M[(ncl + p) * ld + n + r];
        }
        if (tid == 0) ku_np[e] = np;
        return;
    }

    const int lk = no + 1;
    double *Kp;   // K (no x no, symmetrised), row stride kld
    double *Mi;   // M = 1 + K^2, then M^{-1} (no x no), row stride mld
    int kld, mld;
    if (nq == 0) {
        double *Md = reinterpret_cast<double *>(sm);
        // Direct mode (or no eliminated channel at this energy): K = K_u sits
        // in rows ncl.. / columns n.. of the augmented matrix; it is
        // symmetrised in place, and M takes columns 0.. of the same rows (the
        // eliminated part is no longer read). Only the augmented matrix is
        // needed in shared memory.
        Kp = Md + ncl * ld + n;
        kld = ld;
        Mi = Md + ncl * ld;
        mld = ld;
        const int nsym0 = no * (no + 1) / 2;
        for (int q = tid; q < nsym0; q += NT) {
            int p, r;
            tri_pair(q, no, p, r);
            const double kpr = Kp[p * kld + r], krp = Kp[r * kld + p];
            if (K_out) {
                K_out[(size_t)e * n * n + (size_t)p * n + r] = kpr;
                K_out[(size_t)e * n * n + (size_t)r * n + p] = krp;
            }
            const double v = 0.5 * (kpr + krp);
            Kp[p * kld + r] = v;
            Kp[r * kld + p] = v;
        }
        __syncthreads();
    } else {
        if (!mqdt_layout) {   // direct-mode launch: never produced by the channel kernel
            if (tid == 0) status[e] = RM_ESINGULAR;
            return;
        }
        // Shared layout: [region A: n(2n+2) doubles][region B: n(n+1) doubles].
        double *Ks = sm + (size_t)n * (2 * n + 2);   // region B
        const Real *Mq = M;
        // ---- MQDT elimination of the nq channels --------------------------
        const int lu = np + 1;
        double *Ku = Ks;           // K_u (np x np) in region B
        for (int q = tid; q < np * np; q += NT) {
            const int p = q / np, r = q - (q / np) * np;
            Ku[p * lu + r] = (double)Mq[(ncl + p) * ld + n + r];
        }
        for (int i = tid; i < nq; i += NT) vcol[i] = cf[col_chan[ncl + qpos[i]]].tanb;
        __syncthreads();
        if (!mqdt_eliminate(Ku, lu, no, nq, qpos, opos, vcol, sm, Ks,
                            K_out ? K_out + (size_t)e * n * n : nullptr, n, &esh)) {
            if (tid == 0) status[e] = RM_ESINGULAR;
            return;
        }
        Kp = Ks;
        kld = lk;
        Mi = sm;
        mld = lk;
    }
    if (!omega) return;

    if (!t_omega(pw, x, Kp, kld, Mi, mld, no, open_pos, vcol, omega + (size_t)e * n_tri, &esh)) {
        if (tid == 0) status[e] = RM_ESINGULAR;
        return;
    }
}

}  // namespace

int solve_small_max_n() { return SOLVE_SMALL_MAXN; }

// Direct mode needs only the augmented matrix n x (2n + 1); MQDT mode also
// holds K_u and the elimination system.
size_t solve_small_smem(int n, int mqdt, int f32)
{
    if (f32) return (size_t)n * n * sizeof(float);
    if (!mqdt) return (size_t)n * (2 * n + 1) * sizeof(double);
    const size_t aug = (size_t)n * (2 * n + 2);
    const size_t ks = (size_t)n * (n + 1);
    return (aug + ks) * sizeof(double);
}

cudaError_t launch_solve_small(const PwDev &pw, const double *E, int nE, const ChanFn *cf,
                               const double *R, int *status, double *K_out, int *n_open_out,
                               double *omega, int n_tri, int mqdt, int f32, const int *deep_ws, int pass,
                               cudaStream_t s, double *ku_out, int *ku_np)
{
    if (pw.n > SOLVE_SMALL_MAXN || (f32 && mqdt) || (f32 && ku_out)) return cudaErrorInvalidValue;
    if (nE == 0) return cudaSuccess;
    if (f32) return launch_solve_f32(pw, E, nE, cf, R, status, K_out, n_open_out, omega, n_tri, deep_ws, pass, s);
    const size_t smem = solve_small_smem(pw.n, mqdt, 0);
    const int cap = chanfn_deep_cap();
    cudaError_t err =
        cudaFuncSetAttribute(solve_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    solve_small_kernel<<<nE, NT, smem, s>>>(pw, E, cf, R, status, K_out, n_open_out, omega, n_tri, mqdt ? 1 : 0,
                                            deep_ws, cap, pass, ku_out, ku_np);
    return cudaGetLastError();
}

}  // namespace rmgb
