// Dense linear algebra on one matrix per CTA in shared memory (256 threads;
// the elimination and back-substitution take the block size as NTH),
// shared by the per-energy solvers: Gaussian elimination with partial
// pivoting and back-substitution (FP64 or FP32), the symmetric sweep
// inverse, the MQDT closed-channel elimination and the T-matrix / collision
// strength step. Every routine is called by the whole block and ends with a
// barrier.
#pragma once

#include "rcp.cuh"

#include <math.h>

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
template <typename T, int NTH = NT>
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
            for (int q = c + tid; q < w; q += NTH) {
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
        for (int q = tid; q < nr * G; q += NTH) {
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
template <typename T, int NTH = NT>
__device__ void block_backsub(T *M, int ld, int rows, int rhs0, int n_rhs, int row_lo)
{
    for (int qq = threadIdx.x; qq < n_rhs; qq += NTH) {
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

// Complex FP32 reciprocal 1/d = conj(d) / |d|^2 and product. d is first
// scaled by a power of two (exact) so that its larger component lies in
// [1, 2) and |d|^2 can neither overflow nor underflow; the scale is applied
// again to the result. A zero, infinite or NaN d gives a non-finite result.
__device__ __forceinline__ float2 crcp_f(float2 d)
{
    const float m = fmaxf(fabsf(d.x), fabsf(d.y));
    const int ex = min((__float_as_int(m) >> 23) & 0xff, 253);   // biased exponent of m
    const float sc = __int_as_float((254 - ex) << 23);            // 2^(127 - ex)
    const float xr = d.x * sc, xi = d.y * sc;
    const float t = rcp_nr_f(fmaf(xr, xr, xi * xi)) * sc;   // |d'|^2 in [1, 8)
    return make_float2(xr * t, -xi * t);
}

__device__ __forceinline__ float2 cmul_f(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
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

// MQDT elimination (Section "namelist stgf MQDT variables"):
//   K = K_oo - K_oc (K_cc + diag(tq))^{-1} K_co
// from K_u (np x np, row stride lu) with the eliminated channels at P
// positions qpos[0..nq) and the open ones at opos[0..no); tq[i] is the
// diagonal term of eliminated channel i (tan pi nu). scratch holds
// nq (nq + no + 1) + no (no + 1) doubles. K is written symmetrised to Ks
// (row stride no + 1; Ks may be K_u's storage, which is not read after the
// product is formed) and, unsymmetrised, to K_row (row stride ldo) when not
// null. Returns false (sh->bad set) if K_cc + diag(tq) is singular.
__device__ bool mqdt_eliminate(const double *Ku, int lu, int no, int nq, const int *qpos, const int *opos,
                               const double *tq, double *scratch, double *Ks, double *K_row, int ldo,
                               ElimShared *sh)
{
    const int tid = threadIdx.x;
    const int w2 = nq + no, ld2 = w2 + 1, lk = no + 1;
    double *C = scratch;
    for (int q = tid; q < nq * w2; q += NT) {
        const int i = q / w2, j = q - (q / w2) * w2;
        double v;
        if (j < nq) {
            v = Ku[qpos[i] * lu + qpos[j]];
            if (i == j) v += tq[i];
        } else {
            v = Ku[qpos[i] * lu + opos[j - nq]];
        }
        C[i * ld2 + j] = v;
    }
    __syncthreads();
    block_eliminate<double>(C, ld2, nq, w2, sh);
    if (sh->bad) return false;
    block_backsub<double>(C, ld2, nq, nq, no, 0);   // Y = (K_cc + tq)^{-1} K_co
    double *Kd = scratch + (size_t)nq * ld2;
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
        Ks[p * lk + r] = 0.5 * (kpr + Kd[r * lk + p]);
        if (K_row) K_row[(size_t)p * ldo + r] = kpr;
    }
    __syncthreads();
    return true;
}

// Step (d) for one energy (Section "Glossary of terms"): T = 2iK(1 - iK)^{-1}
// in real form. K is symmetric, so with M = 1 + K^2 (SPD), X = M^{-1} K and
// Y = M^{-1} K^2 = 1 - M^{-1}: |T_ab|^2 = 4 (X_ab^2 + Y_ab^2). M^{-1} by the
// symmetric sweep; X formed pair by pair inside the collision-strength sum:
// for target levels I <= J open at energy x, one thread owns Omega_IJ and
// adds g sum_{a in I, b in J} |T_ab|^2 in a fixed order (deterministic).
// Kp: K (no x no, row stride kld); Mi: no x no scratch (row stride mld);
// open_pos maps a channel to its open position. Returns false (sh->bad set)
// if M is not positive definite to working precision.
__device__ bool t_omega(const PwDev &pw, double x, const double *Kp, int kld, double *Mi, int mld, int no,
                        const int *open_pos, double *vcol, double *om, ElimShared *sh)
{
    const int tid = threadIdx.x;
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
    spd_sweep_inverse(Mi, mld, no, vcol, sh);
    if (sh->bad) return false;
    const int nl = pw.n_levels;
    const int npair = nl * (nl + 1) / 2;
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
    return true;
}

}  // namespace
}  // namespace rmgb
