// Steps (c) and (d) for any channel count, working matrices in global memory
// (used above the shared-memory solver's limit). Same mathematics as
// solve_small.cu (Section "Overview", Eq. match; Section "namelist stgf MQDT
// variables"; Section "Glossary of terms"), organised as a chain of batched
// kernels over a block of energies:
//
//   classify      per energy: open set, P set (open + MQDT-eliminated),
//                 unknown ordering (decaying-closed first)
//   assemble      [A | B] (n x (n + n_p)) from packed R and channel data
//   lu            CTA per energy: blocked right-looking Gaussian elimination
//                 with partial pivoting (panel width 32, full-row swaps),
//                 then blocked back-substitution of the trailing rows only
//   extract       K_u = X[P rows]; direct mode: K = K_u
//   mqdt          [K_cc + diag(tan pi nu) | K_co] -> lu -> K = K_oo - K_oc Y
//   T             [1 + K^2 | K] -> lu -> X, Y = K X, |T|^2 = 4 (X^2 + Y^2)
//   omega         thread per (energy, level pair I <= J), fixed summation order
//
// FP64 by default. With the FP32 matching option (rm_opts.solve_precision =
// RM_FP32) the matching system is assembled and solved in FP32 and the T step
// inverts 1 - iK in FP32 complex arithmetic (dense_global_f32.cuh: one CTA per
// energy, blocked LU with partial pivoting; blocked sweep of the complex
// symmetric 1 - iK), while the MQDT elimination, K and Omega stay FP64:
//
//   order         the energies by decreasing n_p: the LU's and the sweep's
//                 CTAs take them in that order (longest first)
//   assemble_f32  [A | 0 | B] in FP32 (right-hand sides from a 4-aligned column)
//   lu32          X = A^{-1} B for the P rows
//   extract_f32   K_u (FP64) = X[P rows]; direct mode: K = K_u
//   mqdt          as above (FP64)
//   zbuild        Z = 1 - iK (FP32 complex)
//   zsweep        Z -> -(1 - iK)^{-1};  T = 2 (1 - iK)^{-1} - 2
//   t2z           |T_ab|^2 = 4 |Z_ab + delta_ab|^2 (symmetrised, FP64)
//
// Per-energy sizes differ (n_o, n_p vary with E); every kernel reads them from
// the per-energy descriptors and idles outside them.
#include <math.h>

#include <algorithm>

#include "dense_global_f32.cuh"
#include "rm_internal.cuh"

namespace rmgb {
namespace {

constexpr int NTH = 256;
constexpr int PNB = 32;     // LU panel width
constexpr int GT = 64;      // GEMM / update tile
constexpr int GK = 16;      // GEMM k-chunk

// Per-energy layout of the workspace (doubles): [aug: n(2n+1)][ku: n^2][ks: n^2],
// each slot rounded to 256 bytes (the FP32 kernels read it by float4)
__host__ __device__ inline size_t slot_doubles(int n)
{
    return ((size_t)n * (2 * n + 1) + 2 * (size_t)n * n + 31) & ~(size_t)31;
}

struct EnergyDims {
    int no, np, nq, ncl;   // np < 0: energy skipped (failed status or no open channel)
};

// ---- classify -----------------------------------------------------------

__global__ void classify_kernel(PwDev pw, const double *__restrict__ E, int nE,
                                const ChanFn *__restrict__ cfa, const int *__restrict__ status,
                                EnergyDims *dims, int *col_chan, int *open_pos, int *qpos,
                                int *opos, int *n_open_out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nE) return;
    const int n = pw.n;
    const double x = E[e];
    int no = 0;
    for (int i = 0; i < n; ++i) no += (x - pw.e_thr[i] > 0.0);
    if (n_open_out) n_open_out[e] = no;
    EnergyDims d = {no, -1, 0, 0};
    if (status[e] == RM_OK && no > 0) {
        const ChanFn *cf = cfa + (size_t)e * n;
        int np = 0;
        for (int i = 0; i < n; ++i) np += (cf[i].kind != CH_CLOSED);
        const int ncl = n - np;
        int pc = 0, pp = 0, po = 0, pq = 0;
        int *cc = col_chan + (size_t)e * n, *op = open_pos + (size_t)e * n;
        int *qp = qpos + (size_t)e * n, *oq = opos + (size_t)e * n;
        for (int i = 0; i < n; ++i) {
            const int k = cf[i].kind;
            if (k == CH_CLOSED) {
                cc[pc++] = i;
                op[i] = -1;
            } else {
                cc[ncl + pp] = i;
                if (k == CH_OPEN) {
                    op[i] = po;
                    oq[po++] = pp;
                } else {
                    op[i] = -1;
                    qp[pq++] = pp;
                }
                ++pp;
            }
        }
        d.np = np;
        d.nq = pq;
        d.ncl = ncl;
    }
    dims[e] = d;
}

// ---- CTA order of the per-energy FP32 kernels ------------------------------

// order[0 .. nE) = the energies by decreasing n_p (the matching system's
// right-hand sides; the LU's cost grows with n_p, the T step's with n_o^3 and
// n_o <= n_p), skipped energies last: the longest CTAs start first, so the
// short ones fill the SMs at the end of the launch (longest-processing-time
// order). One CTA; a counting sort over the n + 2 keys in shared memory
// (dynamic, (n + 2) ints). The order among equal keys is arbitrary: every CTA
// computes its own energy, so the results do not depend on it.
__global__ void order_kernel(int n, int nE, const EnergyDims *__restrict__ dims, int *order)
{
    extern __shared__ int hist[];
    const int nb = n + 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto bin = [&](int e) {
        const int np = dims[e].np;
        return np < 0 ? n + 1 : n - min(np, n);
    };
    for (int b = tid; b < nb; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    for (int e = tid; e < nE; e += blockDim.x) atomicAdd(&hist[bin(e)], 1);
    __syncthreads();
    if (warp == 0) {   // exclusive prefix sum, 32 bins at a time
        int run = 0;
        for (int base = 0; base < nb; base += 32) {
            const int b = base + lane;
            const int v = b < nb ? hist[b] : 0;
            int incl = v;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += t;
            }
            if (b < nb) hist[b] = run + incl - v;
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    __syncthreads();
    for (int e = tid; e < nE; e += blockDim.x) order[atomicAdd(&hist[bin(e)], 1)] = e;
}

// ---- assemble [A | B] -----------------------------------------------------

__global__ void assemble_kernel(PwDev pw, int nE, const ChanFn *__restrict__ cfa,
                                const double *__restrict__ Ra, const EnergyDims *__restrict__ dims,
                                const int *__restrict__ col_chan, double *ws)
{
    const int e = blockIdx.y;
    const EnergyDims d = dims[e];
    if (d.np < 0) return;
    const int n = pw.n, w = n + d.np, ld = w + 1;
    double *M = ws + (size_t)e * slot_doubles(n);
    const ChanFn *cf = cfa + (size_t)e * n;
    const double *Rp = Ra + (size_t)e * tri_ld(n);
    const int *cc = col_chan + (size_t)e * n;
    const double a = pw.a, b = pw.b;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < (long long)n * w;
         q += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(q / w), c = (int)(q - (q / w) * w);
        double v;
        if (c < n) {
            const int j = cc[c];
            const ChanFn cj = cf[j];
            v = -Rp[r <= j ? tri_idx(r, j, n) : tri_idx(j, r, n)] * (a * cj.ghp - b * cj.gh);
            if (r == j) v += cj.gh;
        } else {
            const int o = cc[d.ncl + (c - n)];
            const ChanFn co = cf[o];
            v = Rp[r <= o ? tri_idx(r, o, n) : tri_idx(o, r, n)] * (a * co.sp - b * co.s);
            if (r == o) v -= co.s;
        }
        M[(size_t)r * ld + c] = v;
    }
}

// ---- blocked LU with partial pivoting, then back-substitution --------------

struct LuJob {
    double *M;     // rows x w, row stride ld
    int ld, rows, w, row_lo;   // rows <= 0: skip; back-substitute rows [row_lo, rows)
};

__device__ double block_max_abs_row(const double *M, int ld, int c, int r0, int rows, int *arg,
                                    double *red_v, int *red_i)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double best = -1.0;
    int bi = r0;
    for (int r = r0 + tid; r < rows; r += NTH) {
        const double v = fabs(M[(size_t)r * ld + c]);
        if (v > best || (v == best && r < bi)) { best = v; bi = r; }
    }
    for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) {
        red_v[warp] = best;
        red_i[warp] = bi;
    }
    __syncthreads();
    if (tid == 0) {
        for (int k = 1; k < NTH / 32; ++k)
            if (red_v[k] > red_v[0] || (red_v[k] == red_v[0] && red_i[k] < red_i[0])) {
                red_v[0] = red_v[k];
                red_i[0] = red_i[k];
            }
    }
    __syncthreads();
    *arg = red_i[0];
    const double v = red_v[0];
    __syncthreads();
    return v;
}

// C[r0.., c0..] -= L[r0.., k0..k0+kb) * U[k0..k0+kb), c0..], tiles of 64 x 64
// staged in shared memory (each thread 4 x 4 outputs).
__device__ void block_rank_update(double *M, int ld, int r0, int r1, int c0, int c1, int k0, int kb,
                                  double (*Ls)[GT + 1], double (*Us)[GT + 1])
{
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int tr = r0; tr < r1; tr += GT) {
        for (int tc = c0; tc < c1; tc += GT) {
            __syncthreads();
            for (int q = tid; q < GT * PNB; q += NTH) {
                const int rr = q / PNB, kk = q - (q / PNB) * PNB;
                const int gr = tr + rr;
                Ls[kk][rr] = (gr < r1 && kk < kb) ? M[(size_t)gr * ld + k0 + kk] : 0.0;
                const int kr = q / GT, cc = q - (q / GT) * GT;
                const int gc = tc + cc;
                Us[kr][cc] = (kr < kb && gc < c1) ? M[(size_t)(k0 + kr) * ld + gc] : 0.0;
            }
            __syncthreads();
            double acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
            for (int kk = 0; kk < kb; ++kk) {
                double av[4], bv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) av[i] = Ls[kk][ty * 4 + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) bv[j] = Us[kk][tx * 4 + j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int gr = tr + ty * 4 + i;
                if (gr >= r1) continue;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int gc = tc + tx * 4 + j;
                    if (gc < c1) M[(size_t)gr * ld + gc] -= acc[i][j];
                }
            }
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(NTH) lu_kernel(const LuJob *__restrict__ jobs, int *status)
{
    __shared__ double Ls[PNB][GT + 1];
    __shared__ double Us[PNB][GT + 1];
    __shared__ double red_v[NTH / 32];
    __shared__ int red_i[NTH / 32];
    __shared__ int s_bad;
    const LuJob job = jobs[blockIdx.x];
    if (job.rows <= 0) return;
    double *M = job.M;
    const int ld = job.ld, n = job.rows, w = job.w;
    const int tid = threadIdx.x;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int k0 = 0; k0 < n; k0 += PNB) {
        const int kb = min(PNB, n - k0);
        // panel: columns k0 .. k0+kb-1, unblocked, full-row swaps
        for (int c = k0; c < k0 + kb; ++c) {
            int piv;
            const double best = block_max_abs_row(M, ld, c, c, n, &piv, red_v, red_i);
            const double pv = M[(size_t)piv * ld + c];
            if (!(best > 0.0) || !isfinite(pv)) {
                if (tid == 0) s_bad = 1;
                break;
            }
            if (piv != c) {
                for (int q = tid; q < w; q += NTH) {
                    const double t = M[(size_t)c * ld + q];
                    M[(size_t)c * ld + q] = M[(size_t)piv * ld + q];
                    M[(size_t)piv * ld + q] = t;
                }
                __syncthreads();
            }
            const double pinv = 1.0 / pv;
            for (int r = c + 1 + tid; r < n; r += NTH) M[(size_t)r * ld + c] *= pinv;
            __syncthreads();
            // rank-1 update of the rest of the panel
            const int nc = k0 + kb - c - 1, nr = n - c - 1;
            for (int q = tid; q < nr * nc; q += NTH) {
                const int r = c + 1 + q / nc, cc = c + 1 + (q - (q / nc) * nc);
                M[(size_t)r * ld + cc] = fma(-M[(size_t)r * ld + c], M[(size_t)c * ld + cc],
                                             M[(size_t)r * ld + cc]);
            }
            __syncthreads();
        }
        __syncthreads();
        if (s_bad) break;
        // U12 = L11^{-1} A12 (unit lower triangular), columns k0+kb .. w-1
        for (int cc = k0 + kb + tid; cc < w; cc += NTH) {
            for (int i = 1; i < kb; ++i) {
                double s = M[(size_t)(k0 + i) * ld + cc];
                for (int j = 0; j < i; ++j)
                    s = fma(-M[(size_t)(k0 + i) * ld + k0 + j], M[(size_t)(k0 + j) * ld + cc], s);
                M[(size_t)(k0 + i) * ld + cc] = s;
            }
        }
        __syncthreads();
        // trailing update A22 -= L21 U12
        if (k0 + kb < n) block_rank_update(M, ld, k0 + kb, n, k0 + kb, w, k0, kb, Ls, Us);
    }
    if (s_bad) {
        if (tid == 0) atomicCAS(status + blockIdx.x, RM_OK, RM_ESINGULAR);
        return;
    }
    // blocked back-substitution of rows [row_lo, n) for RHS columns [n, w)
    const int lo = job.row_lo;
    int t1 = n;
    while (t1 > lo) {
        const int t0 = max(lo, t1 - PNB);
        // solve the diagonal block rows t0..t1-1 (one thread per RHS column)
        for (int cq = n + tid; cq < w; cq += NTH) {
            for (int t = t1 - 1; t >= t0; --t) {
                double s = M[(size_t)t * ld + cq];
                for (int u = t + 1; u < t1; ++u) s = fma(-M[(size_t)t * ld + u], M[(size_t)u * ld + cq], s);
                M[(size_t)t * ld + cq] = s / M[(size_t)t * ld + t];
            }
        }
        __syncthreads();
        // rows lo..t0-1 -= U[lo..t0, t0..t1) X[t0..t1, :]
        if (t0 > lo) block_rank_update(M, ld, lo, t0, n, w, t0, t1 - t0, Ls, Us);
        t1 = t0;
    }
}

// ---- batched GEMM: C = alpha A B + beta C (+ I) ---------------------------

struct GemmJob {
    const double *A;
    const double *B;
    double *C;
    int lda, ldb, ldc, m, n, k;
    double alpha, beta;
    int add_identity;
};

__global__ void __launch_bounds__(NTH) gemm_kernel(const GemmJob *__restrict__ jobs)
{
    const GemmJob j = jobs[blockIdx.z];
    if (j.m <= 0 || j.n <= 0) return;
    const int r0 = blockIdx.y * GT, c0 = blockIdx.x * GT;
    if (r0 >= j.m || c0 >= j.n) return;
    __shared__ double As[GK][GT + 1];
    __shared__ double Bs[GK][GT + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int k0 = 0; k0 < j.k; k0 += GK) {
        for (int q = tid; q < GT * GK; q += NTH) {
            const int rr = q / GK, kk = q - (q / GK) * GK;
            const int gr = r0 + rr, gk = k0 + kk;
            As[kk][rr] = (gr < j.m && gk < j.k) ? j.A[(size_t)gr * j.lda + gk] : 0.0;
            const int kr = q / GT, cc = q - (q / GT) * GT;
            const int gk2 = k0 + kr, gc = c0 + cc;
            Bs[kr][cc] = (gk2 < j.k && gc < j.n) ? j.B[(size_t)gk2 * j.ldb + gc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int gr = r0 + ty * 4 + a;
        if (gr >= j.m) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int gc = c0 + tx * 4 + b;
            if (gc >= j.n) continue;
            double v = j.alpha * acc[a][b];
            if (j.beta != 0.0) v += j.beta * j.C[(size_t)gr * j.ldc + gc];
            if (j.add_identity && gr == gc) v += 1.0;
            j.C[(size_t)gr * j.ldc + gc] = v;
        }
    }
}

// ---- per-energy job set-up and elementwise steps ----------------------------

// pointers of one energy's slot
struct Slot {
    double *aug, *ku, *ks;
};
__device__ __forceinline__ Slot slot_of(double *ws, int n, int e)
{
    double *base = ws + (size_t)e * slot_doubles(n);
    return {base, base + (size_t)n * (2 * n + 1), base + (size_t)n * (2 * n + 1) + (size_t)n * n};
}

// An energy whose elimination turned out singular takes no further part.
__global__ void prune_kernel(int nE, const int *status, EnergyDims *dims)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nE && status[e] != RM_OK) dims[e].np = -1;
}

__global__ void jobs_match_kernel(int n, int nE, const EnergyDims *dims, double *ws, LuJob *lu)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nE) return;
    const EnergyDims d = dims[e];
    LuJob j = {nullptr, 0, 0, 0, 0};
    if (d.np >= 0) {
        const Slot s = slot_of(ws, n, e);
        j = {s.aug, n + d.np + 1, n, n + d.np, d.ncl};
    }
    lu[e] = j;
}

// K_u -> ku (np x np, ld np); if no channel is MQDT-eliminated, K = K_u -> ks
// (symmetrised, ld no) and K_out.
__global__ void extract_kernel(int n, int nE, const EnergyDims *dims, double *ws, double *K_out)
{
    const int e = blockIdx.y;
    const EnergyDims d = dims[e];
    if (d.np < 0) return;
    const Slot s = slot_of(ws, n, e);
    const int ld = n + d.np + 1;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < d.np * d.np; q += gridDim.x * blockDim.x) {
        const int p = q / d.np, r = q - (q / d.np) * d.np;
        const double v = s.aug[(size_t)(d.ncl + p) * ld + n + r];
        s.ku[(size_t)p * d.np + r] = v;
        if (d.nq == 0) {
            s.ks[(size_t)p * d.no + r] = 0.5 * (v + s.aug[(size_t)(d.ncl + r) * ld + n + p]);
            if (K_out) K_out[(size_t)e * n * n + (size_t)p * n + r] = v;
        }
    }
}

// MQDT: [K_cc + diag(tan pi nu) | K_co] into aug (nq x (nq + no), ld nq+no+1),
// K_oo into ks, K_oc into the aug area after it.
__global__ void mqdt_build_kernel(int n, int nE, const EnergyDims *dims, const ChanFn *cfa,
                                  const int *col_chan, const int *qpos, const int *opos, double *ws,
                                  LuJob *lu, GemmJob *gj)
{
    const int e = blockIdx.y;
    const EnergyDims d = dims[e];
    const bool act = d.np >= 0 && d.nq > 0;
    const Slot s = slot_of(ws, n, e);
    const int w2 = d.nq + d.no, ld2 = w2 + 1;
    double *koc = s.aug + (size_t)d.nq * ld2;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        LuJob j = {nullptr, 0, 0, 0, 0};
        GemmJob g = {nullptr, nullptr, nullptr, 0, 0, 0, 0, 0, 0, 0.0, 0.0, 0};
        if (act) {
            j = {s.aug, ld2, d.nq, w2, 0};
            // ks = K_oo - K_oc Y,  Y in aug columns nq.. (ld ld2)
            g = {koc, s.aug + d.nq, s.ks, d.nq, ld2, d.no, d.no, d.no, d.nq, -1.0, 1.0, 0};
        }
        lu[e] = j;
        gj[e] = g;
    }
    if (!act) return;
    const int *qp = qpos + (size_t)e * n, *op = opos + (size_t)e * n, *cc = col_chan + (size_t)e * n;
    const ChanFn *cf = cfa + (size_t)e * n;
    const int np = d.np;
    const int total = d.nq * w2 + d.no * d.no + d.no * d.nq;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        if (q < d.nq * w2) {
            const int i = q / w2, jj = q - (q / w2) * w2;
            double v;
            if (jj < d.nq) {
                v = s.ku[(size_t)qp[i] * np + qp[jj]];
                if (i == jj) v += cf[cc[d.ncl + qp[i]]].tanb;
            } else {
                v = s.ku[(size_t)qp[i] * np + op[jj - d.nq]];
            }
            s.aug[(size_t)i * ld2 + jj] = v;
        } else if (q < d.nq * w2 + d.no * d.no) {
            const int t = q - d.nq * w2;
            const int a = t / d.no, b = t - (t / d.no) * d.no;
            s.ks[(size_t)a * d.no + b] = s.ku[(size_t)op[a] * np + op[b]];
        } else {
            const int t = q - d.nq * w2 - d.no * d.no;
            const int a = t / d.nq, b = t - (t / d.nq) * d.nq;
            koc[(size_t)a * d.nq + b] = s.ku[(size_t)op[a] * np + qp[b]];
        }
    }
}

// After the MQDT GEMM: K (ks, unsymmetrised) -> K_out, then symmetrise in place
// via the ku area.
__global__ void mqdt_finish_kernel(int n, int nE, const EnergyDims *dims, double *ws, double *K_out)
{
    const int e = blockIdx.y;
    const EnergyDims d = dims[e];
    if (d.np < 0 || d.nq == 0) return;
    const Slot s = slot_of(ws, n, e);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < d.no * d.no; q += gridDim.x * blockDim.x) {
        const int p = q / d.no, r = q - (q / d.no) * d.no;
        const double v = s.ks[(size_t)p * d.no + r];
        if (K_out) K_out[(size_t)e * n * n + (size_t)p * n + r] = v;
        s.ku[(size_t)p * d.no + r] = 0.5 * (v + s.ks[(size_t)r * d.no + p]);
    }
}

__global__ void mqdt_copyback_kernel(int n, int nE, const EnergyDims *dims, double *ws)
{
    const int e = blockIdx.y;
    const EnergyDims d = dims[e];
    if (d.np < 0 || d.nq == 0) return;
    const Slot s = slot_of(ws, n, e);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < d.no * d.no; q += gridDim.x * blockDim.x)
        s.ks[q] = s.ku[q];
}

// T step set-up: aug = [ (1 + K^2) | K ] (no x 2 no, ld 2no+1); the K^2 GEMM
// writes the left half, this kernel the right half and the jobs.
__global__ void t_build_kernel(int n, int nE, const EnergyDims *dims, double *ws, LuJob *lu,
                               GemmJob *gj)
{
    const int e = blockIdx.y;
    const EnergyDims d = dims[e];
    const bool act = d.np >= 0;
    const Slot s = slot_of(ws, n, e);
    const int ld = 2 * d.no + 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        LuJob j = {nullptr, 0, 0, 0, 0};
        GemmJob g = {nullptr, nullptr, nullptr, 0, 0, 0, 0, 0, 0, 0.0, 0.0, 0};
        if (act) {
            j = {s.aug, ld, d.no, 2 * d.no, 0};
            g = {s.ks, s.ks, s.aug, d.no, d.no, ld, d.no, d.no, d.no, 1.0, 0.0, 1};
        }
        lu[e] = j;
        gj[e] = g;
    }
    if (!act) return;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < d.no * d.no; q += gridDim.x * blockDim.x) {
        const int p = q / d.no, r = q - (q / d.no) * d.no;
        s.aug[(size_t)p * ld + d.no + r] = s.ks[q];
    }
}

// Y = K X into ku (ld no), X in aug columns no.. (ld 2no+1)
__global__ void y_jobs_kernel(int n, int nE, const EnergyDims *dims, double *ws, GemmJob *gj)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nE) return;
    const EnergyDims d = dims[e];
    GemmJob g = {nullptr, nullptr, nullptr, 0, 0, 0, 0, 0, 0, 0.0, 0.0, 0};
    if (d.np >= 0) {
        const Slot s = slot_of(ws, n, e);
        g = {s.ks, s.aug + d.no, s.ku, d.no, 2 * d.no + 1, d.no, d.no, d.no, d.no, 1.0, 0.0, 0};
    }
    gj[e] = g;
}

// |T|^2 = 4 (X^2 + Y^2) with X, Y symmetrised; written over ks (ld no).
__global__ void t2_kernel(int n, int nE, const EnergyDims *dims, double *ws)
{
    const int e = blockIdx.y;
    const EnergyDims d = dims[e];
    if (d.np < 0) return;
    const Slot s = slot_of(ws, n, e);
    const int ld = 2 * d.no + 1;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < d.no * d.no; q += gridDim.x * blockDim.x) {
        const int p = q / d.no, r = q - (q / d.no) * d.no;
        const double x = 0.5 * (s.aug[(size_t)p * ld + d.no + r] + s.aug[(size_t)r * ld + d.no + p]);
        const double y = 0.5 * (s.ku[(size_t)p * d.no + r] + s.ku[(size_t)r * d.no + p]);
        s.ks[q] = 4.0 * (x * x + y * y);
    }
}

__global__ void omega_kernel(PwDev pw, const double *__restrict__ E, int nE,
                             const EnergyDims *__restrict__ dims, const int *__restrict__ open_pos,
                             double *ws, double *omega, int n_tri)
{
    const int e = blockIdx.y;
    const EnergyDims d = dims[e];
    if (d.np < 0) return;
    const int n = pw.n, nl = pw.n_levels;
    const Slot s = slot_of(ws, n, e);
    const double x = E[e];
    const int *op = open_pos + (size_t)e * n;
    double *om = omega + (size_t)e * n_tri;
    const int npair = nl * (nl + 1) / 2;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < npair; q += gridDim.x * blockDim.x) {
        int I = 0, rem = q;
        while (rem >= nl - I) { rem -= nl - I; ++I; }
        const int J = I + rem;
        if (!(x - pw.lev_thr[I] > 0.0) || !(x - pw.lev_thr[J] > 0.0)) continue;
        double sum = 0.0;
        for (int ia = pw.lev_start[I]; ia < pw.lev_start[I + 1]; ++ia) {
            const int pa = op[pw.lev_chan[ia]];
            for (int ib = pw.lev_start[J]; ib < pw.lev_start[J + 1]; ++ib) {
                const int pb = op[pw.lev_chan[ib]];
                sum += s.ks[(size_t)pa * d.no + pb];
            }
        }
        om[q] += pw.g * sum;
    }
}

// ---- FP32 path ---------------------------------------------------------------

// [A | 0 | B] in FP32: A = diag(Ghat) - R diag(a Ghat' - b Ghat), B as in
// assemble_kernel, right-hand sides from column rhs0(n), zero padding.
__global__ void assemble_f32_kernel(PwDev pw, int nE, const ChanFn *__restrict__ cfa,
                                    const double *__restrict__ Ra, const EnergyDims *__restrict__ dims,
                                    const int *__restrict__ col_chan, double *ws)
{
    const int e = blockIdx.y;
    const EnergyDims d = dims[e];
    if (d.np < 0) return;
    const int n = pw.n, rhs = f32d::rhs0(n), ld = f32d::aug_ld(n, d.np);
    float *M = reinterpret_cast<float *>(slot_of(ws, n, e).aug);
    const ChanFn *cf = cfa + (size_t)e * n;
    const double *Rp = Ra + (size_t)e * tri_ld(n);
    const int *cc = col_chan + (size_t)e * n;
    const double a = pw.a, b = pw.b;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < (long long)n * ld;
         q += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(q / ld), c = (int)(q - (q / ld) * ld);
        double v = 0.0;
        if (c < n) {
            const int j = cc[c];
            const ChanFn cj = cf[j];
            v = -Rp[r <= j ? tri_idx(r, j, n) : tri_idx(j, r, n)] * (a * cj.ghp - b * cj.gh);
            if (r == j) v += cj.gh;
        } else if (c >= rhs && c < rhs + d.np) {
            const int o = cc[d.ncl + (c - rhs)];
            const ChanFn co = cf[o];
            v = Rp[r <= o ? tri_idx(r, o, n) : tri_idx(o, r, n)] * (a * co.sp - b * co.s);
            if (r == o) v -= co.s;
        }
        M[(size_t)r * ld + c] = (float)v;
    }
}

template <int PB>
__global__ void __launch_bounds__(f32d::NTH, 1) lu32_kernel(int n, const EnergyDims *__restrict__ dims, double *ws,
                                                            int *status, const int *__restrict__ order)
{
    extern __shared__ float4 fsm4[];
    const int e = order[blockIdx.x];
    const EnergyDims d = dims[e];
    if (d.np < 0) return;
    float *M = reinterpret_cast<float *>(slot_of(ws, n, e).aug);
    const int rhs = f32d::rhs0(n);
    if (!f32d::lu32_factor_solve<PB>(M, f32d::aug_ld(n, d.np), n, rhs + d.np, rhs, d.ncl,
                                     reinterpret_cast<float *>(fsm4)))
        if (threadIdx.x == 0) atomicCAS(status + e, RM_OK, RM_ESINGULAR);
}

// K_u (FP64, np x np) = X[P rows]; without MQDT-eliminated channels also K
// (symmetrised into ks, as written into K_out).
__global__ void extract_f32_kernel(int n, int nE, const EnergyDims *dims, double *ws, double *K_out)
{
    const int e = blockIdx.y;
    const EnergyDims d = dims[e];
    if (d.np < 0) return;
    const Slot s = slot_of(ws, n, e);
    const float *M = reinterpret_cast<const float *>(s.aug);
    const int ld = f32d::aug_ld(n, d.np), rhs = f32d::rhs0(n);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < d.np * d.np; q += gridDim.x * blockDim.x) {
        const int p = q / d.np, r = q - (q / d.np) * d.np;
        const double v = (double)M[(size_t)(d.ncl + p) * ld + rhs + r];
        s.ku[(size_t)p * d.np + r] = v;
        if (d.nq == 0) {
            s.ks[(size_t)p * d.no + r] = 0.5 * (v + (double)M[(size_t)(d.ncl + r) * ld + rhs + p]);
            if (K_out) K_out[(size_t)e * n * n + (size_t)p * n + r] = v;
        }
    }
}

// Z = 1 - iK (FP32 complex, row stride z_ld(no), zero padding) from K in ks.
__global__ void zbuild_kernel(int n, int nE, const EnergyDims *dims, double *ws)
{
    const int e = blockIdx.y;
    const EnergyDims d = dims[e];
    if (d.np < 0) return;
    const Slot s = slot_of(ws, n, e);
    float2 *Z = reinterpret_cast<float2 *>(s.aug);
    const int ldz = f32d::z_ld(d.no);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < d.no * ldz; q += gridDim.x * blockDim.x) {
        const int p = q / ldz, r = q - (q / ldz) * ldz;
        float2 v = make_float2(0.f, 0.f);
        if (r < d.no) v = make_float2(p == r ? 1.f : 0.f, (float)(-s.ks[(size_t)p * d.no + r]));
        Z[q] = v;
    }
}

template <int PB>
__global__ void __launch_bounds__(f32d::NTH, 1) zsweep_kernel(int n, const EnergyDims *__restrict__ dims, double *ws,
                                                              int *status, const int *__restrict__ order)
{
    extern __shared__ float4 fsm4[];
    const int e = order[blockIdx.x];
    const EnergyDims d = dims[e];
    if (d.np < 0) return;
    float2 *Z = reinterpret_cast<float2 *>(slot_of(ws, n, e).aug);
    if (!f32d::zsweep_invert<PB>(Z, f32d::z_ld(d.no), d.no, reinterpret_cast<float2 *>(fsm4)))
        if (threadIdx.x == 0) atomicCAS(status + e, RM_OK, RM_ESINGULAR);
}

// |T_ab|^2 = 4 |W_ab - delta_ab|^2 with W = (1 - iK)^{-1} = -Z (upper triangle
// of Z, so |T|^2 is symmetric), into ks.
__global__ void t2z_kernel(int n, int nE, const EnergyDims *dims, double *ws)
{
    const int e = blockIdx.y;
    const EnergyDims d = dims[e];
    if (d.np < 0) return;
    const Slot s = slot_of(ws, n, e);
    const float2 *Z = reinterpret_cast<const float2 *>(s.aug);
    const int ldz = f32d::z_ld(d.no);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < d.no * d.no; q += gridDim.x * blockDim.x) {
        const int p = q / d.no, r = q - (q / d.no) * d.no;
        const float2 u = Z[(size_t)min(p, r) * ldz + max(p, r)];   // upper triangle
        const double ur = (double)u.x + (p == r ? 1.0 : 0.0), ui = u.y;
        s.ks[q] = 4.0 * (ur * ur + ui * ui);
    }
}

int max_dyn_smem()
{
    static int v = -1;
    if (v < 0) {
        int dev = 0, x = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&x, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
            cudaGetLastError();
            x = 48 * 1024;
        }
        v = x;
    }
    return v;
}

// Panel widths that fit shared memory for n channels (0: none fits).
int lu_pb(int n)
{
    if (f32d::lu_smem<32>(n) <= (size_t)max_dyn_smem()) return 32;
    if (f32d::lu_smem<16>(n) <= (size_t)max_dyn_smem()) return 16;
    return 0;
}
int z_pb(int m)
{
    if (f32d::z_smem<16>(m) <= (size_t)max_dyn_smem()) return 16;
    if (f32d::z_smem<8>(m) <= (size_t)max_dyn_smem()) return 8;
    return 0;
}

template <class K> cudaError_t set_smem(K kern, size_t bytes)
{
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

bool solve_large_f32_supported(int n) { return lu_pb(n) > 0 && z_pb(n) > 0; }

size_t solve_large_bytes_per_energy(int n)
{
    return slot_doubles(n) * sizeof(double) + sizeof(EnergyDims) + 4 * (size_t)n * sizeof(int) +
           sizeof(LuJob) + sizeof(GemmJob) + sizeof(int) + 64;
}

// Runs steps (c) and (d) for a block of nE energies. ws must hold
// solve_large_bytes_per_energy(n) * nE bytes. Returns the first CUDA error.
cudaError_t launch_solve_large(const PwDev &pw, const double *E, int nE, const ChanFn *cf,
                               const double *R, int *status, double *K_out, int *n_open_out,
                               double *omega, int n_tri, void *ws_raw, int *launches,
                               cudaStream_t st, int f32)
{
    if (f32 && !solve_large_f32_supported(pw.n)) return cudaErrorInvalidValue;
    if (nE == 0) return cudaSuccess;
    const int n = pw.n;
    char *p = static_cast<char *>(ws_raw);
    double *ws = reinterpret_cast<double *>(p);
    p += slot_doubles(n) * sizeof(double) * nE;
    EnergyDims *dims = reinterpret_cast<EnergyDims *>(p);
    p += sizeof(EnergyDims) * nE;
    int *col_chan = reinterpret_cast<int *>(p);
    int *open_pos = col_chan + (size_t)n * nE;
    int *qpos = open_pos + (size_t)n * nE;
    int *opos = qpos + (size_t)n * nE;
    p += 4 * (size_t)n * nE * sizeof(int);
    p = reinterpret_cast<char *>(((uintptr_t)p + 15) & ~(uintptr_t)15);
    LuJob *lu = reinterpret_cast<LuJob *>(p);
    p += sizeof(LuJob) * nE;
    p = reinterpret_cast<char *>(((uintptr_t)p + 15) & ~(uintptr_t)15);
    GemmJob *gj = reinterpret_cast<GemmJob *>(p);
    p += sizeof(GemmJob) * nE;
    p = reinterpret_cast<char *>(((uintptr_t)p + 15) & ~(uintptr_t)15);
    int *order = reinterpret_cast<int *>(p);

    const int eg = (nE + 127) / 128;
    int L = 0;
    cudaError_t err;
#define LAUNCH_OK()                                   \
    do {                                              \
        ++L;                                          \
        if ((err = cudaGetLastError()) != cudaSuccess) \
            return err;                               \
    } while (0)
    classify_kernel<<<eg, 128, 0, st>>>(pw, E, nE, cf, status, dims, col_chan, open_pos, qpos, opos,
                                        n_open_out);
    LAUNCH_OK();
    const int xb = (int)std::min<long long>(64, ((long long)n * 2 * n + NTH - 1) / NTH);
    const int xb2 = (int)std::min<long long>(64, ((long long)n * n + NTH - 1) / NTH);
    if (f32) {
        order_kernel<<<1, 1024, (size_t)(n + 2) * sizeof(int), st>>>(n, nE, dims, order);
        LAUNCH_OK();
        assemble_f32_kernel<<<dim3(xb, nE), NTH, 0, st>>>(pw, nE, cf, R, dims, col_chan, ws);
        LAUNCH_OK();
        const int pb = lu_pb(n);
        if (pb == 32) {
            const size_t sm = f32d::lu_smem<32>(n);
            if ((err = set_smem(lu32_kernel<32>, sm)) != cudaSuccess) return err;
            lu32_kernel<32><<<nE, f32d::NTH, sm, st>>>(n, dims, ws, status, order);
        } else {
            const size_t sm = f32d::lu_smem<16>(n);
            if ((err = set_smem(lu32_kernel<16>, sm)) != cudaSuccess) return err;
            lu32_kernel<16><<<nE, f32d::NTH, sm, st>>>(n, dims, ws, status, order);
        }
        LAUNCH_OK();
        prune_kernel<<<eg, 128, 0, st>>>(nE, status, dims);
        LAUNCH_OK();
        extract_f32_kernel<<<dim3(xb2, nE), NTH, 0, st>>>(n, nE, dims, ws, K_out);
        LAUNCH_OK();
    } else {
        assemble_kernel<<<dim3(xb, nE), NTH, 0, st>>>(pw, nE, cf, R, dims, col_chan, ws);
        LAUNCH_OK();
        jobs_match_kernel<<<eg, 128, 0, st>>>(n, nE, dims, ws, lu);
        LAUNCH_OK();
        lu_kernel<<<nE, NTH, 0, st>>>(lu, status);
        LAUNCH_OK();
        prune_kernel<<<eg, 128, 0, st>>>(nE, status, dims);
        LAUNCH_OK();
        extract_kernel<<<dim3(xb2, nE), NTH, 0, st>>>(n, nE, dims, ws, K_out);
        LAUNCH_OK();
    }
    const int tiles = (n + GT - 1) / GT;
    // MQDT elimination (no-op for energies without eliminated channels)
    mqdt_build_kernel<<<dim3(xb2, nE), NTH, 0, st>>>(n, nE, dims, cf, col_chan, qpos, opos, ws, lu, gj);
    LAUNCH_OK();
    lu_kernel<<<nE, NTH, 0, st>>>(lu, status);
    LAUNCH_OK();
    prune_kernel<<<eg, 128, 0, st>>>(nE, status, dims);
    LAUNCH_OK();
    gemm_kernel<<<dim3(tiles, tiles, nE), NTH, 0, st>>>(gj);
    LAUNCH_OK();
    mqdt_finish_kernel<<<dim3(xb2, nE), NTH, 0, st>>>(n, nE, dims, ws, K_out);
    LAUNCH_OK();
    mqdt_copyback_kernel<<<dim3(xb2, nE), NTH, 0, st>>>(n, nE, dims, ws);
    LAUNCH_OK();
    if (omega && f32) {
        zbuild_kernel<<<dim3(xb2, nE), NTH, 0, st>>>(n, nE, dims, ws);
        LAUNCH_OK();
        const int pb = z_pb(n);
        if (pb == 16) {
            const size_t sm = f32d::z_smem<16>(n);
            if ((err = set_smem(zsweep_kernel<16>, sm)) != cudaSuccess) return err;
            zsweep_kernel<16><<<nE, f32d::NTH, sm, st>>>(n, dims, ws, status, order);
        } else {
            const size_t sm = f32d::z_smem<8>(n);
            if ((err = set_smem(zsweep_kernel<8>, sm)) != cudaSuccess) return err;
            zsweep_kernel<8><<<nE, f32d::NTH, sm, st>>>(n, dims, ws, status, order);
        }
        LAUNCH_OK();
        prune_kernel<<<eg, 128, 0, st>>>(nE, status, dims);
        LAUNCH_OK();
        t2z_kernel<<<dim3(xb2, nE), NTH, 0, st>>>(n, nE, dims, ws);
        LAUNCH_OK();
        const int nl = pw.n_levels;
        const int xb3 = (int)std::min<long long>(64, ((long long)nl * (nl + 1) / 2 + NTH - 1) / NTH);
        omega_kernel<<<dim3(xb3, nE), NTH, 0, st>>>(pw, E, nE, dims, open_pos, ws, omega, n_tri);
        LAUNCH_OK();
    } else if (omega) {
        t_build_kernel<<<dim3(xb2, nE), NTH, 0, st>>>(n, nE, dims, ws, lu, gj);
        LAUNCH_OK();
        gemm_kernel<<<dim3(tiles, tiles, nE), NTH, 0, st>>>(gj);   // 1 + K^2
        LAUNCH_OK();
        lu_kernel<<<nE, NTH, 0, st>>>(lu, status);                // X = (1 + K^2)^{-1} K
        LAUNCH_OK();
        prune_kernel<<<eg, 128, 0, st>>>(nE, status, dims);
        LAUNCH_OK();
        y_jobs_kernel<<<eg, 128, 0, st>>>(n, nE, dims, ws, gj);
        LAUNCH_OK();
        gemm_kernel<<<dim3(tiles, tiles, nE), NTH, 0, st>>>(gj);   // Y = K X
        LAUNCH_OK();
        t2_kernel<<<dim3(xb2, nE), NTH, 0, st>>>(n, nE, dims, ws);
        LAUNCH_OK();
        const int nl = pw.n_levels;
        const int xb3 = (int)std::min<long long>(64, ((long long)nl * (nl + 1) / 2 + NTH - 1) / NTH);
        omega_kernel<<<dim3(xb3, nE), NTH, 0, st>>>(pw, E, nE, dims, open_pos, ws, omega, n_tri);
        LAUNCH_OK();
    }
#undef LAUNCH_OK
    if (launches) *launches += L;
    return cudaSuccess;
}

}  // namespace rmgb
