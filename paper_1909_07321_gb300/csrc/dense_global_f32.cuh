// FP32 dense kernels of the global-memory solver's mixed-precision path
// (rm_opts.solve_precision = RM_FP32, channel counts above the shared-memory
// solver's limit). One CTA of 512 threads works on one energy's matrices in
// global memory:
//
//   lu32_factor_solve   [A | B] -> solves A X = B for the trailing rows of X
//                       (the matching system, Section "Overview", Eq. match):
//                       blocked right-looking LU with partial pivoting. The
//                       current panel of PB columns (all rows below its
//                       diagonal) is held in shared memory, column-major, and
//                       factored there (two barriers per column: the row
//                       update of one column carries the pivot search of the
//                       next); its row interchanges are applied to the
//                       columns to its right as one permutation per panel;
//                       U12 = L11^{-1} A12 is solved one column per thread;
//                       the trailing matrix takes the rank-PB update
//                       A22 -= L21 U12 in tiles of 128 x 128 with 4 x 8
//                       register tiles per thread (the U12 strips staged in
//                       two shared buffers in turn). Back-substitution of the
//                       requested rows runs in the same blocked form, upwards.
//   zsweep_invert       Z <- -Z^{-1} for a complex symmetric Z whose
//                       Hermitian part is positive definite (Z = 1 - iK, the
//                       T step of Section "Glossary of terms"): the sweep
//                       operator applied PB pivots at a time, no pivoting
//                       (every leading block of such a Z is nonsingular).
//                       Per block of pivots K: the PB x PB block is swept in
//                       shared memory (B -> -B^{-1}), the panel
//                       P = Z[:, K] B^{-1} is formed in shared memory, every
//                       other entry takes Z_ij -= P_i Z_Kj (rank-PB complex
//                       update in tiles of 128 x 64, 4 x 4 per thread), and
//                       Z[:, K], Z[K, :] become P and P^T. Z stays symmetric,
//                       so only the upper triangle is kept current: tiles
//                       wholly below the diagonal are skipped and every read
//                       takes the entry (min(i, j), max(i, j)).
//
// Both kernels read and write their matrix through global memory (L2), with
// no waits other than __syncthreads. A zero or non-finite pivot marks the
// energy RM_ESINGULAR and the CTA returns.
#pragma once

#include <math.h>

#include "rm_internal.cuh"

namespace rmgb {
namespace f32d {

constexpr int NTH = 512;
constexpr int NWARP = NTH / 32;
constexpr int UW = 128;    // real strip width (columns)
constexpr int UWC = 64;    // complex strip width (columns)

// Layout of the real augmented matrix of n unknowns and np right-hand sides:
// columns [0, n) A, [n, rhs0(n)) zero, [rhs0(n), rhs0(n) + np) B, zero up to ld.
__host__ __device__ inline int rhs0(int n) { return (n + 3) & ~3; }
__host__ __device__ inline int aug_ld(int n, int np) { return (rhs0(n) + np + 3) & ~3; }
// Column stride of the shared-memory panel (4 mod 32 floats: the row-wise
// panel load hits 4-way bank conflicts at most, float4 reads stay aligned).
__host__ __device__ inline int lu_npad(int n) { return ((rhs0(n) + 31) & ~31) + 4; }
// Complex matrix of order m: row stride, and the panel's column stride.
__host__ __device__ inline int z_ld(int m) { return (m + 3) & ~3; }
__host__ __device__ inline int z_npad(int m) { return ((m + 7) & ~7) + 8; }

template <int PB> __host__ __device__ inline size_t lu_smem(int n)
{
    const size_t f = (size_t)PB * lu_npad(n) + 2 * (size_t)PB * (UW + 4);
    // perm [npad], move lists [2 PB], counters [8], reduction keys
    // [NWARP x 64 bit], reduction values [NWARP], and slack
    const size_t i = (size_t)lu_npad(n) + 2 * PB + 8 + 3 * NWARP + 16;
    return f * sizeof(float) + i * sizeof(int);
}

template <int PB> __host__ __device__ inline size_t z_smem(int m)
{
    return ((size_t)PB * z_npad(m) + (size_t)PB * (UWC + 2) + (size_t)PB * (PB + 1)) * sizeof(float2);
}

// Packed key of a pivot candidate: larger magnitude first, then lower row.
// Magnitudes are non-negative floats, whose bit patterns order as integers;
// a NaN counts as +infinity (it is then caught as a non-finite pivot).
__device__ __forceinline__ unsigned long long piv_key(float v, int r)
{
    float m = fabsf(v);
    if (m != m) m = __int_as_float(0x7f800000);
    return ((unsigned long long)__float_as_uint(m) << 32) | (unsigned)(0x7fffffff - r);
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long k)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, k, off);
        k = o > k ? o : k;
    }
    return k;
}

// ---- real blocked LU ---------------------------------------------------------

// C[rows, cols c0..c0+128) -= Lp[0..PB)[rows] * Us[0..PB)[cols] for rows
// [rlo, rhi), stored only where row in [rstore, rhi) and col < ld. Lp is the
// column-major panel (stride npad), Us the staged strip (stride UW + 4).
// Thread (ty, tx) = (tid / 16, tid % 16) takes rows 4 ty .. 4 ty + 3 of each
// 128-row tile and columns 4 tx .. 4 tx + 3 and 64 + 4 tx .. 64 + 4 tx + 3
// (a quarter-warp's float4 reads of Us hit distinct banks).
template <int PB>
__device__ __forceinline__ void lu_update_strip(float *M, int ld, int rlo, int rhi, int rstore, int c0,
                                                const float *Lp, int npad, const float *Us)
{
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int cb[2] = {c0 + 4 * tx, c0 + 64 + 4 * tx};
    // C tile of rows rb .. rb + 3 into v (zero outside [rstore, rhi) or past ld)
    auto load = [&](int rb, float (&v)[4][8]) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = rb + i;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                if (r < rhi && r >= rstore && cb[h] < ld)
                    q = *reinterpret_cast<const float4 *>(M + (size_t)r * ld + cb[h]);
                v[i][4 * h + 0] = q.x;
                v[i][4 * h + 1] = q.y;
                v[i][4 * h + 2] = q.z;
                v[i][4 * h + 3] = q.w;
            }
        }
    };
    // the next row tile's C is loaded while this one is updated
    float acc[4][8], nxt[4][8];
    int rb = rlo + ty * 4;
    if (rb < rhi) load(rb, acc);
    for (int r0 = rlo; r0 < rhi; r0 += 128, rb += 128) {
        if (rb >= rhi) break;
        if (rb + 128 < rhi) load(rb + 128, nxt);
        const bool full = rb + 3 < rhi;
#pragma unroll 4
        for (int k = 0; k < PB; ++k) {
            float a[4], b[8];
            if (full) {
                const float4 a0 = *reinterpret_cast<const float4 *>(Lp + k * npad + rb);
                a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = (rb + i < rhi) ? Lp[k * npad + rb + i] : 0.f;
            }
            const float4 b0 = *reinterpret_cast<const float4 *>(Us + k * (UW + 4) + 4 * tx);
            const float4 b1 = *reinterpret_cast<const float4 *>(Us + k * (UW + 4) + 64 + 4 * tx);
            b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
            b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(-a[i], b[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = rb + i;
            if (r >= rhi || r < rstore) continue;
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (cb[h] < ld)
                    *reinterpret_cast<float4 *>(M + (size_t)r * ld + cb[h]) =
                        make_float4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2], acc[i][4 * h + 3]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = nxt[i][j];
    }
}

// Rows [rlo, rhi) (stored from rstore), columns [c_lo, w): C -= Lp[0..PB) x
// U, where U = rows [u0, u0 + PB) of M (final). Strips of 128 columns, their
// U staged in two shared buffers in turn (one barrier per strip).
template <int PB>
__device__ void lu_update_rows(float *M, int ld, int u0, int kb, int rlo, int rhi, int rstore, int c_lo, int w,
                               const float *Lp, int npad, float *Us)
{
    const int tid = threadIdx.x;
    const int nstrip = (w - c_lo + UW - 1) / UW;
    auto stage = [&](int s, float *buf) {
        const int c0 = c_lo + s * UW;
        for (int q = tid; q < PB * UW; q += NTH) {
            const int k = q / UW, jj = q - (q / UW) * UW;
            const int c = c0 + jj;
            buf[k * (UW + 4) + jj] = (k < kb && c < w) ? M[(size_t)(u0 + k) * ld + c] : 0.f;
        }
    };
    stage(0, Us);
    __syncthreads();
    for (int s = 0; s < nstrip; ++s) {
        float *cur = Us + (s & 1) * PB * (UW + 4);
        if (s + 1 < nstrip) stage(s + 1, Us + ((s + 1) & 1) * PB * (UW + 4));
        lu_update_strip<PB>(M, ld, rlo, rhi, rstore, c_lo + s * UW, Lp, npad, cur);
        __syncthreads();
    }
}

// Solves A X = B in place for the n x w augmented matrix M (row stride ld,
// A in columns [0, n), right-hand sides in [rhs, w), zero padding between and
// after), leaving X in rows [row_lo, n) of the right-hand-side columns.
// Returns false if a pivot is zero or not finite.
template <int PB>
__device__ bool lu32_factor_solve(float *M, int ld, int n, int w, int rhs, int row_lo, float *smem)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int npad = lu_npad(n);
    float *Lp = smem;
    float *Us = Lp + (size_t)PB * npad;
    int *perm = reinterpret_cast<int *>(Us + 2 * PB * (UW + 4));
    int *mv_dst = perm + npad;
    int *mv_src = mv_dst + PB;
    int *sh_int = mv_src + PB;                 // [0]: move count, [1]: bad
    unsigned long long *red = reinterpret_cast<unsigned long long *>(sh_int + 8);   // [NWARP]
    float *red_val = reinterpret_cast<float *>(red + NWARP);                        // [NWARP]

    for (int k0 = 0; k0 < n; k0 += PB) {
        const int kb = min(PB, n - k0);
        // panel rows [k0, n), columns [k0, k0 + kb) -> Lp[j][r]
        for (int q = tid; q < (n - k0) * kb; q += NTH) {
            const int r = k0 + q / kb, j = q - (q / kb) * kb;
            Lp[j * npad + r] = M[(size_t)r * ld + k0 + j];
        }
        for (int r = k0 + tid; r < n; r += NTH) perm[r] = r;
        if (tid == 0) sh_int[0] = 0;
        __syncthreads();
        // pivot candidates of the panel's first column
        {
            unsigned long long key = 0ull;
            float kv = 0.f;
            for (int r = k0 + tid; r < n; r += NTH) {
                const float v = Lp[r];
                const unsigned long long kk = piv_key(v, r);
                if (kk > key) {
                    key = kk;
                    kv = v;
                }
            }
            const unsigned long long wk = warp_max_u64(key);
            const unsigned ball = __ballot_sync(0xffffffffu, key == wk && wk != 0ull);
            if (lane == 0) red[warp] = wk;
            if (ball && lane == __ffs(ball) - 1) red_val[warp] = kv;
        }
        __syncthreads();
        for (int j = 0; j < kb; ++j) {
            const int c = k0 + j;
            unsigned long long best = red[0];
            float pv = red_val[0];
#pragma unroll
            for (int q = 1; q < NWARP; ++q)
                if (red[q] > best) {
                    best = red[q];
                    pv = red_val[q];
                }
            const int p = 0x7fffffff - (int)(unsigned)(best & 0xffffffffu);
            const bool bad = best == 0ull || !(fabsf(pv) > 0.f) || !isfinite(pv);
            if (!bad && p != c) {
                if (tid < kb) {
                    const float t = Lp[tid * npad + c];
                    Lp[tid * npad + c] = Lp[tid * npad + p];
                    Lp[tid * npad + p] = t;
                }
                if (tid == PB) {
                    const int t = perm[c];
                    perm[c] = perm[p];
                    perm[p] = t;
                }
            }
            __syncthreads();
            if (bad) return false;
            // multipliers and the rank-1 update of the panel's remaining
            // columns; each thread's rows of column j + 1 are final here, so
            // their pivot candidates are taken on the way
            const float ipv = 1.0f / pv;
            unsigned long long key = 0ull;
            float kv = 0.f;
            for (int r = c + 1 + tid; r < n; r += NTH) {
                const float l = Lp[j * npad + r] * ipv;
                Lp[j * npad + r] = l;
                for (int jj = j + 1; jj < kb; ++jj)
                    Lp[jj * npad + r] = fmaf(-l, Lp[jj * npad + c], Lp[jj * npad + r]);
                if (j + 1 < kb) {
                    const float v = Lp[(j + 1) * npad + r];
                    const unsigned long long kk = piv_key(v, r);
                    if (kk > key) {
                        key = kk;
                        kv = v;
                    }
                }
            }
            if (j + 1 < kb) {
                const unsigned long long wk = warp_max_u64(key);
                const unsigned ball = __ballot_sync(0xffffffffu, key == wk && wk != 0ull);
                if (lane == 0) red[warp] = wk;
                if (ball && lane == __ffs(ball) - 1) red_val[warp] = kv;
            }
            __syncthreads();
        }
        // rows [k0, k0 + kb) of the panel (U11 and the unit-lower L11) to
        // global memory; rows moved below the panel by its interchanges
        for (int q = tid; q < kb * kb; q += NTH) {
            const int i = q / kb, j = q - (q / kb) * kb;
            M[(size_t)(k0 + i) * ld + k0 + j] = Lp[j * npad + k0 + i];
        }
        for (int r = k0 + kb + tid; r < n; r += NTH)
            if (perm[r] != r) {
                const int s = atomicAdd(&sh_int[0], 1);
                mv_dst[s] = r;
                mv_src[s] = perm[r];
            }
        __syncthreads();
        const int nmv = sh_int[0];
        if (k0 + kb >= w) continue;
        // trailing columns: interchanges and U12 = L11^{-1} A12, one thread per
        // column; U12 goes to rows [k0, k0 + kb) of global memory
        for (int c = k0 + kb + tid; c < w; c += NTH) {
            float x[PB];
            // The new rows k0 .. k0 + kb come from perm[], which may name rows
            // below the panel; those rows are then move destinations, so they
            // are read first. A row below the panel only ever receives a row
            // of [k0, k0 + kb) (a position of the panel is never swapped
            // again once its pivot is chosen), and those rows are written
            // last, so the moves need no further ordering.
#pragma unroll
            for (int j = 0; j < PB; ++j) x[j] = j < kb ? M[(size_t)perm[k0 + j] * ld + c] : 0.f;
            for (int i0 = 0; i0 < nmv; i0 += 8) {
                float y[8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (i0 + i < nmv) y[i] = M[(size_t)mv_src[i0 + i] * ld + c];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (i0 + i < nmv) M[(size_t)mv_dst[i0 + i] * ld + c] = y[i];
            }
#pragma unroll
            for (int j = 1; j < PB; ++j) {
                if (j < kb) {
                    float sum = x[j];
#pragma unroll
                    for (int i = 0; i < PB; ++i)
                        if (i < j) sum = fmaf(-Lp[i * npad + k0 + j], x[i], sum);
                    x[j] = sum;
                }
            }
#pragma unroll
            for (int j = 0; j < PB; ++j)
                if (j < kb) M[(size_t)(k0 + j) * ld + c] = x[j];
        }
        __syncthreads();
        if (k0 + kb < n) lu_update_rows<PB>(M, ld, k0, kb, k0 + kb, n, k0 + kb, k0 + kb, w, Lp, npad, Us);
    }
    // back-substitution of rows [row_lo, n) for the right-hand sides
    const int rs = row_lo & ~3;
    int t1 = n;
    while (t1 > row_lo) {
        const int t0 = max(row_lo, t1 - PB);
        const int tb = t1 - t0;
        for (int q = tid; q < (t1 - rs) * tb; q += NTH) {
            const int r = rs + q / tb, j = q - (q / tb) * tb;
            Lp[j * npad + r] = r >= row_lo ? M[(size_t)r * ld + t0 + j] : 0.f;
        }
        __syncthreads();
        for (int c = rhs + tid; c < w; c += NTH) {
            float x[PB];
#pragma unroll
            for (int j = 0; j < PB; ++j) x[j] = j < tb ? M[(size_t)(t0 + j) * ld + c] : 0.f;
#pragma unroll
            for (int i = PB - 1; i >= 0; --i) {
                if (i < tb) {
                    float sum = x[i];
#pragma unroll
                    for (int j = 0; j < PB; ++j)
                        if (j > i && j < tb) sum = fmaf(-Lp[j * npad + t0 + i], x[j], sum);
                    x[i] = sum / Lp[i * npad + t0 + i];
                }
            }
#pragma unroll
            for (int j = 0; j < PB; ++j)
                if (j < tb) M[(size_t)(t0 + j) * ld + c] = x[j];
        }
        __syncthreads();
        if (t0 > row_lo) lu_update_rows<PB>(M, ld, t0, PB, rs, t0, row_lo, rhs, w, Lp, npad, Us);
        t1 = t0;
    }
    return true;
}

// ---- complex symmetric sweep -------------------------------------------------

__device__ __forceinline__ float2 cfma_neg(float2 a, float2 b, float2 c)
{
    // c - a b
    c.x = fmaf(-a.x, b.x, fmaf(a.y, b.y, c.x));
    c.y = fmaf(-a.x, b.y, fmaf(-a.y, b.x, c.y));
    return c;
}

__device__ __forceinline__ float2 crcp_safe(float2 d)
{
    const float s = fmaxf(fabsf(d.x), fabsf(d.y));
    const float xr = d.x / s, xi = d.y / s;
    const float t = 1.0f / (s * fmaf(xr, xr, xi * xi));
    return make_float2(xr * t, -xi * t);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Entry (i, j) of a symmetric Z of which only the upper triangle is current.
__device__ __forceinline__ float2 zu(const float2 *Z, int ldz, int i, int j)
{
    return i <= j ? Z[(size_t)i * ldz + j] : Z[(size_t)j * ldz + i];
}

// Z (m x m complex symmetric, row stride ldz, zero padding to ldz) <- -Z^{-1}
// in its upper triangle (the lower triangle is left stale).
template <int PB>
__device__ bool zsweep_invert(float2 *Z, int ldz, int m, float2 *smem)
{
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int npz = z_npad(m);
    float2 *Lp = smem;
    float2 *Us = Lp + (size_t)PB * npz;
    float2 *Bs = Us + PB * (UWC + 2);
    for (int k0 = 0; k0 < m; k0 += PB) {
        const int kb = min(PB, m - k0);
        if (tid < PB * PB) {
            const int i = tid / PB, j = tid - (tid / PB) * PB;
            Bs[i * (PB + 1) + j] = (i < kb && j < kb) ? zu(Z, ldz, k0 + i, k0 + j) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        // sweep of the diagonal block: B -> -B^{-1}
        for (int p = 0; p < kb; ++p) {
            const float2 d = Bs[p * (PB + 1) + p];
            const bool bad = !(fabsf(d.x) + fabsf(d.y) > 0.f) || !isfinite(d.x) || !isfinite(d.y);
            if (bad) return false;   // the same decision in every thread
            const float2 dinv = crcp_safe(d);
            float2 v = make_float2(0.f, 0.f);
            const int i = tid / PB, j = tid - (tid / PB) * PB;
            const bool own = tid < PB * PB && i < kb && j < kb;
            if (own) {
                if (i == p && j == p) {
                    v = make_float2(-dinv.x, -dinv.y);
                } else if (i == p) {
                    v = cmul(Bs[p * (PB + 1) + j], dinv);
                } else if (j == p) {
                    v = cmul(Bs[i * (PB + 1) + p], dinv);
                } else {
                    v = cfma_neg(cmul(Bs[i * (PB + 1) + p], dinv), Bs[p * (PB + 1) + j], Bs[i * (PB + 1) + j]);
                }
            }
            __syncthreads();
            if (own) Bs[i * (PB + 1) + j] = v;
            __syncthreads();
        }
        // panel P_i = Z[i, K] B^{-1} = -Z[i, K] Bs for rows i outside K
        for (int i = tid; i < m; i += NTH) {
            float2 P[PB];
#pragma unroll
            for (int k = 0; k < PB; ++k) P[k] = make_float2(0.f, 0.f);
            if (i < k0 || i >= k0 + kb) {
#pragma unroll
                for (int q = 0; q < PB; ++q) {
                    if (q < kb) {
                        const float2 zq = zu(Z, ldz, i, k0 + q);
#pragma unroll
                        for (int k = 0; k < PB; ++k) P[k] = cfma_neg(zq, Bs[q * (PB + 1) + k], P[k]);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < PB; ++k) Lp[k * npz + i] = (k < kb) ? P[k] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        // Z_ij -= P_i Z_Kj for i, j outside K, i <= j (tiles of 128 x 64
        // wholly below the diagonal are skipped), 64 columns at a time
        for (int c0 = 0; c0 < m; c0 += UWC) {
            for (int q = tid; q < PB * UWC; q += NTH) {
                const int k = q / UWC, jj = q - (q / UWC) * UWC;
                const int c = c0 + jj;
                const bool in = k < kb && c < m && (c < k0 || c >= k0 + kb);
                Us[k * (UWC + 2) + jj] = in ? zu(Z, ldz, k0 + k, c) : make_float2(0.f, 0.f);
            }
            __syncthreads();
            const int cb[2] = {c0 + 2 * tx, c0 + 32 + 2 * tx};
            const int r_end = min(m, c0 + UWC);   // row tiles starting past this are below the diagonal
            auto zload = [&](int rb, float2 (&v)[4][4]) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int r = rb + i;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (r < m && cb[h] < ldz) q = *reinterpret_cast<const float4 *>(Z + (size_t)r * ldz + cb[h]);
                        v[i][2 * h] = make_float2(q.x, q.y);
                        v[i][2 * h + 1] = make_float2(q.z, q.w);
                    }
                }
            };
            float2 acc[4][4], nxt[4][4];
            int rb = ty * 4;
            if (rb < m) zload(rb, acc);
            for (int r0 = 0; r0 < r_end; r0 += 128, rb += 128) {
                if (rb >= m) break;
                if (r0 + 128 < r_end && rb + 128 < m) zload(rb + 128, nxt);
#pragma unroll 4
                for (int k = 0; k < PB; ++k) {
                    float2 a[4], b[4];
                    const float4 a0 = *reinterpret_cast<const float4 *>(Lp + k * npz + rb);
                    const float4 a1 = *reinterpret_cast<const float4 *>(Lp + k * npz + rb + 2);
                    a[0] = make_float2(a0.x, a0.y);
                    a[1] = make_float2(a0.z, a0.w);
                    a[2] = make_float2(a1.x, a1.y);
                    a[3] = make_float2(a1.z, a1.w);
                    const float4 b0 = *reinterpret_cast<const float4 *>(Us + k * (UWC + 2) + 2 * tx);
                    const float4 b1 = *reinterpret_cast<const float4 *>(Us + k * (UWC + 2) + 32 + 2 * tx);
                    b[0] = make_float2(b0.x, b0.y);
                    b[1] = make_float2(b0.z, b0.w);
                    b[2] = make_float2(b1.x, b1.y);
                    b[3] = make_float2(b1.z, b1.w);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = cfma_neg(a[i], b[j], acc[i][j]);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int r = rb + i;
                    if (r >= m) continue;
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        if (cb[h] < ldz)
                            *reinterpret_cast<float4 *>(Z + (size_t)r * ldz + cb[h]) =
                                make_float4(acc[i][2 * h].x, acc[i][2 * h].y, acc[i][2 * h + 1].x,
                                            acc[i][2 * h + 1].y);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = nxt[i][j];
            }
            __syncthreads();
        }
        // upper-triangle positions of Z[i, K] = P_i and Z[K, i] = P_i^T, and
        // Z[K, K] = -B^{-1}
        for (int i = tid; i < k0; i += NTH) {
#pragma unroll
            for (int k = 0; k < PB; ++k)
                if (k < kb) Z[(size_t)i * ldz + k0 + k] = Lp[k * npz + i];
        }
        for (int q = tid; q < kb * (m - k0 - kb); q += NTH) {
            const int k = q / (m - k0 - kb), i = k0 + kb + (q - (q / (m - k0 - kb)) * (m - k0 - kb));
            Z[(size_t)(k0 + k) * ldz + i] = Lp[k * npz + i];
        }
        if (tid < PB * PB) {
            const int i = tid / PB, j = tid - (tid / PB) * PB;
            if (i < kb && j < kb) Z[(size_t)(k0 + i) * ldz + k0 + j] = Bs[i * (PB + 1) + j];
        }
        __syncthreads();
    }
    return true;
}

}  // namespace f32d
}  // namespace rmgb
