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
#include <math.h>

#include <type_traits>

#include "rm_internal.cuh"

namespace rmgb {
namespace {

constexpr int SOLVE_SMALL_MAXN = 96;
constexpr int NT = 256;

struct ElimShared {
    int piv;
    int bad;
    double pivinv;
};

// In-place Gaussian elimination with partial pivoting of the first `rows`
// columns of the rows x w matrix M (row stride ld), whole block, in the
// element type T (double, or float for the FP32 matching). Sets sh->bad on a
// zero or non-finite pivot.
template <typename T>
__device__ void block_eliminate(T *M, int ld, int rows, int w, ElimShared *sh)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int c = 0; c < rows; ++c) {
        if (warp == 0) {
            T best = -1;
            int bi = c;
            for (int r = c + lane; r < rows; r += 32) {
                const T v = fabs(M[r * ld + c]);
                if (v > best) { best = v; bi = r; }
            }
            for (int off = 16; off > 0; off >>= 1) {
                const T ob = __shfl_down_sync(0xffffffffu, best, off);
                const int oi = __shfl_down_sync(0xffffffffu, bi, off);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (lane == 0) {
                sh->piv = bi;
                const double pv = (double)M[bi * ld + c];
                if (!(best > 0) || !isfinite(pv)) sh->bad = 1;
                sh->pivinv = 1.0 / pv;
            }
        }
        __syncthreads();
        const int p = sh->piv;
        if (p != c) {
            for (int q = c + tid; q < w; q += NT) {
                const T t = M[c * ld + q];
                M[c * ld + q] = M[p * ld + q];
                M[p * ld + q] = t;
            }
            __syncthreads();
        }
        // trailing update; G threads share a row and form its multiplier once
        // (the multipliers are not stored: every right-hand side is in the
        // augmented matrix), so there is no separate scaling pass or barrier
        constexpr int G = 4;
        const T pinv = (T)sh->pivinv;
        const int nr = rows - c - 1;
        const T *prow = M + c * ld;
        for (int q = tid; q < nr * G; q += NT) {
            const int r = c + 1 + q / G, j = q - (q / G) * G;
            T *row = M + r * ld;
            const T f = row[c] * pinv;
            for (int cc = c + 1 + j; cc < w; cc += G) row[cc] = fma(-f, prow[cc], row[cc]);
        }
        __syncthreads();
    }
}

// Back-substitution of the upper-triangular rows x rows system in M for the
// n_rhs right-hand sides in columns rhs0.., over rows t = rows-1 .. row_lo,
// in place; one thread per right-hand side.
template <typename T>
__device__ void block_backsub(T *M, int ld, int rows, int rhs0, int n_rhs, int row_lo)
{
    for (int qq = threadIdx.x; qq < n_rhs; qq += NT) {
        const int cq = rhs0 + qq;
        for (int t = rows - 1; t >= row_lo; --t) {
            T s = M[t * ld + cq];
            for (int u = t + 1; u < rows; ++u) s = fma(-M[t * ld + u], M[u * ld + cq], s);
            M[t * ld + cq] = s / M[t * ld + t];
        }
    }
    __syncthreads();
}

// In-place inverse of the symmetric positive definite m x m matrix A (row
// stride ld) by the sweep operator: Gauss-Jordan elimination without
// pivoting (which SPD matrices do not need), keeping the symmetry, so only
// the upper triangle is read and updated (m^3 flops instead of 2 m^3). Step
// k, with d = a_kk and v_i = a_ik / d: a_ij -= v_i v_j d (i, j != k),
// a_ik = v_i, a_kk = -1/d; after all m steps the upper triangle holds
// -A^{-1}, which is then negated and mirrored into the full matrix.
// v is shared scratch of m doubles. Sets sh->bad if a pivot is not positive.
__device__ void spd_sweep_inverse(double *A, int ld, int m, double *v, ElimShared *sh)
{
    const int tid = threadIdx.x;
    constexpr int G = 8;                        // threads per pair of rows
    const int ngroups = (m + 1) / 2;            // rows g and m-1-g share a group
    for (int k = 0; k < m; ++k) {
        const double d = A[k * ld + k];
        if (!(d > 0.0) || !isfinite(d)) {       // the same value in every thread
            if (tid == 0) sh->bad = 1;
            return;
        }
        const double dinv = 1.0 / d;
        for (int i = tid; i < m; i += NT)
            v[i] = (i == k) ? 0.0 : ((i < k) ? A[i * ld + k] : A[k * ld + i]) * dinv;
        __syncthreads();
        for (int q = tid; q < ngroups * G; q += NT) {
            const int g = q / G, t = q - (q / G) * G;
            for (int h = 0; h < 2; ++h) {
                const int i = h ? m - 1 - g : g;
                if (h && i == g) break;
                double *row = A + i * ld;
                const double vi = v[i];
                for (int j = i + t; j < m; j += G) {
                    if (i == k) row[j] = (j == k) ? -dinv : v[j];
                    else if (j == k) row[j] = vi;
                    else row[j] = fma(-vi * d, v[j], row[j]);
                }
            }
        }
        __syncthreads();
    }
    // A^{-1} = -(upper triangle), mirrored
    for (int q = tid; q < m * m; q += NT) {
        const int i = q / m, j = q - (q / m) * m;
        if (i > j) A[i * ld + j] = -A[j * ld + i];
    }
    __syncthreads();
    for (int q = tid; q < m * m; q += NT) {
        const int i = q / m, j = q - (q / m) * m;
        if (i <= j) A[i * ld + j] = -A[i * ld + j];
    }
    __syncthreads();
}

// Row-wise upper-triangle index q -> (p, r), p <= r < m.
__device__ __forceinline__ void tri_pair(int q, int m, int &p, int &r)
{
    const float t = (float)(2 * m + 1);
    int pp = (int)((t - sqrtf(fmaxf(t * t - 8.0f * (float)q, 0.0f))) * 0.5f);
    if (pp < 0) pp = 0;
    while (pp > 0 && pp * m - (pp * (pp - 1)) / 2 > q) --pp;
    while ((pp + 1) * m - ((pp + 1) * pp) / 2 <= q) ++pp;
    p = pp;
    r = pp + (q - (pp * m - (pp * (pp - 1)) / 2));
}

// Shared-memory bytes of region A in the FP32-matching layout: the float
// augmented matrix n x (2n + 1), later M^{-1} (at most n x (n + 1) doubles).
__host__ __device__ inline size_t f32_region_a(int n)
{
    const size_t aug = (size_t)n * (2 * n + 1) * sizeof(float);
    const size_t mi = (size_t)n * (n + 1) * sizeof(double);
    return ((aug > mi ? aug : mi) + 15) & ~(size_t)15;
}

// F32: the matching system is eliminated in FP32 (direct mode only; the T
// step and Omega stay FP64).
template <bool F32>
__global__ void __launch_bounds__(NT) solve_small_kernel(
    PwDev pw, const double *__restrict__ E, const ChanFn *__restrict__ cfa,
    const double *__restrict__ Ra, int *__restrict__ status, double *__restrict__ K_out,
    int *__restrict__ n_open_out, double *__restrict__ omega, int n_tri, int mqdt_layout,
    const int *__restrict__ deep_ws, int deep_cap, int pass)
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
    __shared__ int piv[SOLVE_SMALL_MAXN];
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
    using Real = typename std::conditional<F32, float, double>::type;
    Real *M = reinterpret_cast<Real *>(sm);
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

    const int lk = no + 1;
    double *Kp;   // K (no x no, symmetrised), row stride kld
    double *Mi;   // M = 1 + K^2, then M^{-1} (no x no), row stride mld
    int kld, mld;
    if (F32) {
        if (nq > 0) {   // FP32 matching is launched for direct mode only
            if (tid == 0) status[e] = RM_ESINGULAR;
            return;
        }
        // K (FP64) into region B, then M^{-1} over the float matrix in region A
        Kp = reinterpret_cast<double *>(reinterpret_cast<char *>(sm) + f32_region_a(n));
        kld = lk;
        const int nsym0 = no * (no + 1) / 2;
        for (int q = tid; q < nsym0; q += NT) {
            int p, r;
            tri_pair(q, no, p, r);
            const double kpr = (double)M[(ncl + p) * ld + n + r];
            const double krp = (double)M[(ncl + r) * ld + n + p];
            if (K_out) {
                K_out[(size_t)e * n * n + (size_t)p * n + r] = kpr;
                K_out[(size_t)e * n * n + (size_t)r * n + p] = krp;
            }
            const double v = 0.5 * (kpr + krp);
            Kp[p * kld + r] = v;
            Kp[r * kld + p] = v;
        }
        __syncthreads();
        Mi = sm;
        mld = lk;
    } else if (nq == 0) {
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
        __syncthreads();
        // [K_cc + diag(tan pi nu) | K_co] in region A
        const int w2 = nq + no, ld2 = w2 + 1;
        double *C = sm;
        for (int q = tid; q < nq * w2; q += NT) {
            const int i = q / w2, j = q - (q / w2) * w2;
            double v;
            if (j < nq) {
                v = Ku[qpos[i] * lu + qpos[j]];
                if (i == j) v += cf[col_chan[ncl + qpos[i]]].tanb;
            } else {
                v = Ku[qpos[i] * lu + opos[j - nq]];
            }
            C[i * ld2 + j] = v;
        }
        __syncthreads();
        block_eliminate<double>(C, ld2, nq, w2, &esh);
        if (esh.bad) {
            if (tid == 0) status[e] = RM_ESINGULAR;
            return;
        }
        block_backsub<double>(C, ld2, nq, nq, no, 0);   // Y = (K_cc + tan)^{-1} K_co
        // K = K_oo - K_oc Y, after [C | Y] in region A
        double *Kd = sm + (size_t)nq * ld2;
        for (int q = tid; q < no * no; q += NT) {
            const int s2 = q / no, t = q - (q / no) * no;
            double v = Ku[opos[s2] * lu + opos[t]];
            for (int i = 0; i < nq; ++i) v = fma(-Ku[opos[s2] * lu + qpos[i]], C[i * ld2 + nq + t], v);
            Kd[s2 * lk + t] = v;
        }
        __syncthreads();
        for (int q = tid; q < no * no; q += NT) {
            const int p = q / no, r = q - (q / no) * no;
            const double kpr = Kd[p * lk + r];
            Ks[p * lk + r] = 0.5 * (kpr + Kd[r * lk + p]);   // overwrites K_u, no longer read
            if (K_out) K_out[(size_t)e * n * n + (size_t)p * n + r] = kpr;
        }
        __syncthreads();
        Kp = Ks;
        kld = lk;
        Mi = sm;
        mld = lk;
    }
    if (!omega) return;

    // ---- M = 1 + K^2 (upper triangle, mirrored), inverted in place ----------
    const int nsym = no * (no + 1) / 2;
    for (int q = tid; q < nsym; q += NT) {
        int p, r;
        tri_pair(q, no, p, r);
        double s = (p == r) ? 1.0 : 0.0;
        for (int u = 0; u < no; ++u) s = fma(Kp[p * kld + u], Kp[u * kld + r], s);
        Mi[p * mld + r] = s;
        Mi[r * mld + p] = s;
    }
    __syncthreads();
    spd_sweep_inverse(Mi, mld, no, vcol, &esh);
    if (esh.bad) {
        if (tid == 0) status[e] = RM_ESINGULAR;
        return;
    }

    // ---- Omega_IJ += g sum_{a in I, b in J} |T_ab|^2 -------------------------
    // |T_ab|^2 = 4 (X_ab^2 + Y_ab^2), X = K M^{-1}, Y = 1 - M^{-1}, each pair
    // formed where it is summed (taken with a <= b: both are symmetric).
    const int nl = pw.n_levels;
    const int npair = nl * (nl + 1) / 2;
    double *om = omega + (size_t)e * n_tri;
    const double g = pw.g;
    for (int q = tid; q < npair; q += NT) {
        int I, J;
        tri_pair(q, nl, I, J);
        if (!(x - pw.lev_thr[I] > 0.0) || !(x - pw.lev_thr[J] > 0.0)) continue;
        double s = 0.0;
        for (int ia = pw.lev_start[I]; ia < pw.lev_start[I + 1]; ++ia) {
            const int pa0 = open_pos[pw.lev_chan[ia]];
            for (int ib = pw.lev_start[J]; ib < pw.lev_start[J + 1]; ++ib) {
                const int pb0 = open_pos[pw.lev_chan[ib]];
                const int pa = min(pa0, pb0), pb = max(pa0, pb0);
                double xv = 0.0;
                for (int u = 0; u < no; ++u) xv = fma(Kp[pa * kld + u], Mi[u * mld + pb], xv);
                const double yv =
                    ((pa == pb) ? 1.0 : 0.0) - 0.5 * (Mi[pa * mld + pb] + Mi[pb * mld + pa]);
                s += 4.0 * (xv * xv + yv * yv);
            }
        }
        om[q] += g * s;
    }
}

}  // namespace

int solve_small_max_n() { return SOLVE_SMALL_MAXN; }

// Direct mode needs only the augmented matrix n x (2n + 1); MQDT mode also
// holds K_u and the elimination system; FP32 matching keeps the float matrix
// (then M^{-1}) beside K.
size_t solve_small_smem(int n, int mqdt, int f32)
{
    if (f32) return f32_region_a(n) + (size_t)n * (n + 1) * sizeof(double);
    if (!mqdt) return (size_t)n * (2 * n + 1) * sizeof(double);
    const size_t aug = (size_t)n * (2 * n + 2);
    const size_t ks = (size_t)n * (n + 1);
    return (aug + ks) * sizeof(double);
}

cudaError_t launch_solve_small(const PwDev &pw, const double *E, int nE, const ChanFn *cf,
                               const double *R, int *status, double *K_out, int *n_open_out,
                               double *omega, int n_tri, int mqdt, int f32, const int *deep_ws, int pass,
                               cudaStream_t s)
{
    if (pw.n > SOLVE_SMALL_MAXN || (f32 && mqdt)) return cudaErrorInvalidValue;
    if (nE == 0) return cudaSuccess;
    const size_t smem = solve_small_smem(pw.n, mqdt, f32);
    const int cap = chanfn_deep_cap();
    cudaError_t err;
    if (f32) {
        err = cudaFuncSetAttribute(solve_small_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem);
        if (err != cudaSuccess) return err;
        solve_small_kernel<true><<<nE, NT, smem, s>>>(pw, E, cf, R, status, K_out, n_open_out, omega,
                                                      n_tri, 0, deep_ws, cap, pass);
    } else {
        err = cudaFuncSetAttribute(solve_small_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem);
        if (err != cudaSuccess) return err;
        solve_small_kernel<false><<<nE, NT, smem, s>>>(pw, E, cf, R, status, K_out, n_open_out, omega,
                                                       n_tri, mqdt ? 1 : 0, deep_ws, cap, pass);
    }
    return cudaGetLastError();
}

}  // namespace rmgb
