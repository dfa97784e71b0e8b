// Steps (c) and (d) in FP32 for the mixed-precision path (direct mode,
// n <= SOLVE_SMALL_MAXN): one CTA of 16 x 16 threads per energy, with both
// matrices held in registers.
//
// (c) Matching (Section "Overview", Eq. match), as in solve_small.cu: with
// the channels ordered closed first, then open (the set P),
//   [diag(Ghat) - R diag(a Ghat' - b Ghat)] X = -[diag(S) - R diag(a S' - b S)] P,
// K = X[P rows]. Thread (tx, ty) = (tid / 16, tid % 16) holds rows ty + 16 i
// and columns tx + 16 j of the n x (n + n_o) augmented matrix, so the 16
// owners of a column form one half-warp. Gauss-Jordan elimination with
// partial pivoting, the pivot rows left in place (implicit pivoting): for
// column c its half-warp finds the pivot row p among the rows not yet used
// (largest magnitude to 2^-17, lowest index among those) by one max-reduction
// and publishes the multipliers and p; after one barrier every thread takes the pivot row's values
// for its columns by a shuffle from the lane of its own half-warp that holds
// row p, and every other row r (used or not) takes a_rj -= (a_rc / a_pc) a_pj
// for j > c. After n columns the unknowns are x_c = a_{p(c), rhs} / a_{p(c), c},
// with no back-substitution.
//
// (d) T = 2iK(1 - iK)^{-1} = 2(1 - iK)^{-1} - 2 (Section "Glossary of
// terms"): 1 - iK (complex, K symmetrised) in registers in the same 16 x 16
// layout, inverted in place by the sweep operator (Gauss-Jordan without
// pivoting: its Hermitian part is the identity, so every pivot has a
// positive real part); the matrix is symmetric, so each step publishes one
// column and needs one barrier. The sweep leaves W = -(1 - iK)^{-1}, and
// |T_ab|^2 = 4 |W_ab + delta_ab|^2. For target levels I <= J one thread owns
// Omega_IJ(E) and adds g sum_{a in I, b in J} |T_ab|^2 in FP64, in a fixed
// order (deterministic, no atomics).
#include <math.h>

#include "dense_smem.cuh"
#include "rm_internal.cuh"

namespace rmgb {
namespace {

constexpr int G16 = 16;                          // thread grid 16 x 16
constexpr int MAXN = SOLVE_SMALL_MAXN;

// Element k of a register array for an index k that is the same in every
// thread of the warp: a uniform branch per case keeps the array in
// registers (a runtime subscript would move it to local memory).
template <int N, typename T>
__device__ __forceinline__ T pick(const T (&v)[N], int k)
{
    T r = v[0];
#pragma unroll
    for (int q = 1; q < N; ++q)
        if (k == q) r = v[q];
    return r;
}

// One step of the sweep on pivot k, after the pivot column has been
// published: z_ij -= v_i u_j, then column k <- v, row k <- v^T and the pivot
// <- -1/d (v = u / d, u = column k before the step; uniform tile indices).
template <int TR>
__device__ __forceinline__ void sweep_apply(float2 (&z)[TR][TR], int k, int tx, int ty, const float2 *vc,
                                            const float2 *uc, float2 dinv)
{
    const int kk = k >> 4;
    float2 vi[TR], uj[TR];
#pragma unroll
    for (int i = 0; i < TR; ++i) {
        vi[i] = vc[ty + G16 * i];
        uj[i] = uc[tx + G16 * i];
    }
#pragma unroll
    for (int i = 0; i < TR; ++i) {
#pragma unroll
        for (int j = 0; j < TR; ++j) {
            float2 zz = z[i][j];
            zz.x = fmaf(-vi[i].x, uj[j].x, fmaf(vi[i].y, uj[j].y, zz.x));
            zz.y = fmaf(-vi[i].x, uj[j].y, fmaf(-vi[i].y, uj[j].x, zz.y));
            z[i][j] = zz;
        }
    }
    if (tx == (k & 15)) {
#pragma unroll
        for (int j = 0; j < TR; ++j)
            if (kk == j) {
#pragma unroll
                for (int i = 0; i < TR; ++i) z[i][j] = vi[i];
            }
    }
    if (ty == (k & 15)) {
#pragma unroll
        for (int i = 0; i < TR; ++i)
            if (kk == i) {
#pragma unroll
                for (int j = 0; j < TR; ++j) {
                    const int c = tx + G16 * j;
                    z[i][j] = (c == k) ? make_float2(-dinv.x, -dinv.y) : vc[c];
                }
            }
    }
}

// Shared buffers of the T step's sweep (two per buffer: published pivot
// columns alternate between steps), row stride `stride`.
struct SweepShared {
    float2 *ucol, *vcol, *ucol2, *vcol2;
    float2 *dbuf, *dinvbuf, *dbuf2, *dinvbuf2;
    int stride;
};

// T step for n_o <= 16 TS open channels (TS tiles per side in registers,
// no padding tiles beyond them): W = -(1 - iK)^{-1} by the complex sweep, and
// |T_ab|^2 = 4 |W_ab + delta_ab|^2 written over K in Pm. Returns false (in
// every thread) if a pivot is zero or not finite.
template <int TS>
__device__ __forceinline__ bool t_sweep(float *Pm, int no, int tid, int lane, int tx, int ty, unsigned hmask,
                                        const SweepShared &sh)
{
    const unsigned full = 0xffffffffu;
    float2 z[TS][TS];
#pragma unroll
    for (int i = 0; i < TS; ++i) {
        const int r = ty + G16 * i;
#pragma unroll
        for (int j = 0; j < TS; ++j) {
            const int c = tx + G16 * j;
            float2 v = make_float2(0.0f, 0.0f);
            if (r < no && c < no) v = make_float2(r == c ? 1.0f : 0.0f, -0.5f * (Pm[r * no + c] + Pm[c * no + r]));
            z[i][j] = v;
        }
    }
    // Pivots in pairs (k even, k + 1) as in the elimination: the owner warp
    // finds d1 = z_kk and v1 = column k / d1 (lanes 0-15), brings column k + 1
    // through the step on k (lanes 16-31: w_i = z_i,k+1 - v1_i z_k+1,k, and
    // w_k = z_k+1,k / d1), takes d2 = w_k+1, and publishes both; every thread
    // then applies both steps after one barrier.
    int k_first_single = 0;
    for (int k = 0; k + 1 < no; k += 2) {
        const int buf = (k >> 1) & 1;
        const int kk = k >> 4;
        if ((tx >> 1) == ((k & 15) >> 1)) {
            float2 u[TS];
#pragma unroll
            for (int i = 0; i < TS; ++i) u[i] = pick<TS>(z[i], kk);
            const float2 ukk = pick<TS>(u, kk);
            float2 d1, uk1;
            d1.x = __shfl_sync(full, ukk.x, k & 15);
            d1.y = __shfl_sync(full, ukk.y, k & 15);
            uk1.x = __shfl_sync(full, ukk.x, (k + 1) & 15);   // z_{k+1,k}
            uk1.y = __shfl_sync(full, ukk.y, (k + 1) & 15);
            const float2 dinv1 = crcp_f(d1);
            float2 w[TS];
#pragma unroll
            for (int i = 0; i < TS; ++i) {
                const float2 v1 = cmul_f(u[i], dinv1);
                float2 vA;
                vA.x = __shfl_xor_sync(full, v1.x, 16);
                vA.y = __shfl_xor_sync(full, v1.y, 16);
                const int r = ty + G16 * i;
                const float2 uv = cmul_f(vA, uk1);
                w[i] = (r == k) ? cmul_f(uk1, dinv1) : make_float2(u[i].x - uv.x, u[i].y - uv.y);
                if ((tx & 1) == 0 && r < no) {
                    sh.ucol[buf * sh.stride + r] = u[i];
                    sh.vcol[buf * sh.stride + r] = v1;
                }
            }
            const float2 wk1 = pick<TS>(w, kk);
            float2 d2;
            d2.x = __shfl_sync(full, wk1.x, 16 + ((k + 1) & 15));
            d2.y = __shfl_sync(full, wk1.y, 16 + ((k + 1) & 15));
            const float2 dinv2 = crcp_f(d2);
            if (tx & 1) {
#pragma unroll
                for (int i = 0; i < TS; ++i) {
                    const int r = ty + G16 * i;
                    if (r < no) {
                        sh.ucol2[buf * sh.stride + r] = w[i];
                        sh.vcol2[buf * sh.stride + r] = cmul_f(w[i], dinv2);
                    }
                }
            }
            if (lane == 0) {
                sh.dbuf[buf] = d1;
                sh.dinvbuf[buf] = dinv1;
                sh.dbuf2[buf] = d2;
                sh.dinvbuf2[buf] = dinv2;
            }
        }
        __syncthreads();
        const float2 d1 = sh.dbuf[buf], d2 = sh.dbuf2[buf];
        if (!(fabsf(d1.x) + fabsf(d1.y) > 0.0f) || !isfinite(d1.x) || !isfinite(d1.y) ||
            !(fabsf(d2.x) + fabsf(d2.y) > 0.0f) || !isfinite(d2.x) || !isfinite(d2.y)) {
            return false;
        }
        sweep_apply<TS>(z, k, tx, ty, sh.vcol + buf * sh.stride, sh.ucol + buf * sh.stride, sh.dinvbuf[buf]);
        sweep_apply<TS>(z, k + 1, tx, ty, sh.vcol2 + buf * sh.stride, sh.ucol2 + buf * sh.stride, sh.dinvbuf2[buf]);
        k_first_single = k + 2;
    }
    for (int k = k_first_single; k < no; ++k) {
        const int buf = (k >> 1) & 1;
        const int kk = k >> 4;
        if (tx == (k & 15)) {
            // column k's half-warp: u, the pivot d = u_k, and v = u / d
            float2 u[TS];
#pragma unroll
            for (int i = 0; i < TS; ++i) u[i] = pick<TS>(z[i], kk);
            const float2 uk = pick<TS>(u, kk);
            float2 d;
            d.x = __shfl_sync(hmask, uk.x, k & 15, 16);
            d.y = __shfl_sync(hmask, uk.y, k & 15, 16);
            const float2 dinv = crcp_f(d);
#pragma unroll
            for (int i = 0; i < TS; ++i) {
                const int r = ty + G16 * i;
                if (r < no) {
                    sh.ucol[buf * sh.stride + r] = u[i];
                    sh.vcol[buf * sh.stride + r] = cmul_f(u[i], dinv);
                }
            }
            if (ty == 0) {
                sh.dbuf[buf] = d;
                sh.dinvbuf[buf] = dinv;
            }
        }
        __syncthreads();
        const float2 d = sh.dbuf[buf];
        if (!(fabsf(d.x) + fabsf(d.y) > 0.0f) || !isfinite(d.x) || !isfinite(d.y)) {
            return false;
        }
        sweep_apply<TS>(z, k, tx, ty, sh.vcol + buf * sh.stride, sh.ucol + buf * sh.stride, sh.dinvbuf[buf]);
    }
    __syncthreads();   // every read of K in Pm is done
#pragma unroll
    for (int i = 0; i < TS; ++i) {
        const int r = ty + G16 * i;
#pragma unroll
        for (int j = 0; j < TS; ++j) {
            const int c = tx + G16 * j;
            if (r < no && c < no) {
                const float re = z[i][j].x + (r == c ? 1.0f : 0.0f), im = z[i][j].y;
                Pm[r * no + c] = 4.0f * fmaf(re, re, im * im);
            }
        }
    }
    __syncthreads();

    return true;
}

// The T step with the smallest tile count that holds n_o (ts = ceil(n_o / 16),
// the same in every thread).
template <int TS, int TMAX>
__device__ __forceinline__ bool t_sweep_dispatch(int ts, float *Pm, int no, int tid, int lane, int tx, int ty,
                                                 unsigned hmask, const SweepShared &sh)
{
    if constexpr (TS < TMAX) {
        if (ts <= TS) return t_sweep<TS>(Pm, no, tid, lane, tx, ty, hmask, sh);
        return t_sweep_dispatch<TS + 1, TMAX>(ts, Pm, no, tid, lane, tx, ty, hmask, sh);
    } else {
        return t_sweep<TMAX>(Pm, no, tid, lane, tx, ty, hmask, sh);
    }
}

template <int TR, int TC>
__global__ void __launch_bounds__(NT, TR >= 6 ? 2 : 4) solve_f32_kernel(
    PwDev pw, const double *__restrict__ E, const ChanFn *__restrict__ cfa, const double *__restrict__ Ra,
    int *__restrict__ status, double *__restrict__ K_out, int *__restrict__ n_open_out,
    double *__restrict__ omega, int n_tri, const int *__restrict__ deep_ws, int deep_cap, int pass)
{
    static_assert(TC == 2 * TR && G16 * TR <= MAXN, "tile shape");
    if (deep_ws) {
        const bool deferred = deep_ws[0] <= deep_cap && deep_ws[1 + deep_cap + blockIdx.x] != 0;
        if (pass == 0 ? deferred : !deferred) return;
    }
    extern __shared__ float fsm[];                // [packed R of this energy][K, later |T|^2 (n_o x n_o)]
    float *Rs = fsm;
    float *Pm = fsm + tri_ld(pw.n);
    __shared__ int col_chan[MAXN];                // unknown column -> channel
    __shared__ int open_pos[MAXN];                // channel -> position in P (-1: closed)
    __shared__ float colv[MAXN], dgv[MAXN];       // unknown column: a Ghat' - b Ghat, Ghat
    __shared__ float rsv[MAXN], rss[MAXN];        // right-hand side k: a S' - b S, S
    __shared__ int kind_s[MAXN];
    __shared__ float colbuf[2][G16 * TR];         // multipliers a_rc / a_pc (0 for the pivot row)
    __shared__ float colbuf2[2][G16 * TR];        // second column of a pair
    __shared__ int pbuf[2], pbuf2[2];
    __shared__ float pvbuf[2], pvbuf2[2];
    __shared__ unsigned used_s[(G16 * TR + 31) / 32];
    __shared__ float2 vcol[2][G16 * TR];
    __shared__ float2 dbuf[2], dinvbuf[2], dbuf2[2], dinvbuf2[2];
    __shared__ float2 vcol2[2][G16 * TR], ucol2[2][G16 * TR];
    __shared__ int rowpos[G16 * TR];
    __shared__ float pivval[MAXN];
    __shared__ float2 ucol[2][G16 * TR];
    __shared__ double lev_thr_s[MAXN];
    __shared__ int lev_start_s[MAXN + 1], lev_chan_s[MAXN];
    __shared__ int s_no, s_np;

    const int e = blockIdx.x;
    const int n = pw.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = tid >> 4, ty = tid & 15;
    const double x = E[e];
    const ChanFn *cf = cfa + (size_t)e * n;
    const double *Rp = Ra + (size_t)e * tri_ld(n);
    if (status[e] != RM_OK) {
        if (tid == 0 && n_open_out) {
            int no = 0;
            for (int i = 0; i < n; ++i) no += (x - pw.e_thr[i] > 0.0);
            n_open_out[e] = no;
        }
        return;
    }

    // ---- channel order: closed first, then P (open), by warp prefix counts
    for (int i = tid; i < n; i += NT) kind_s[i] = cf[i].kind;
    for (int r = tid; r < G16 * TR; r += NT) {
        for (int q = 0; q < 2; ++q) {
            ucol[q][r] = make_float2(0.0f, 0.0f);
            vcol[q][r] = make_float2(0.0f, 0.0f);
            ucol2[q][r] = make_float2(0.0f, 0.0f);
            vcol2[q][r] = make_float2(0.0f, 0.0f);
        }
    }
    if (tid < (G16 * TR + 31) / 32) used_s[tid] = 0u;
    // R of this energy and the level tables, by coalesced loads
    for (int q = tid; q < tri_ld(n); q += NT) Rs[q] = (float)Rp[q];
    const int nl = pw.n_levels;
    const bool lev_sm = nl <= MAXN;    // more levels than that (some without channels): read them in place
    if (lev_sm) {
        for (int q = tid; q < nl; q += NT) lev_thr_s[q] = pw.lev_thr[q];
        for (int q = tid; q <= nl; q += NT) lev_start_s[q] = pw.lev_start[q];
    }
    for (int q = tid; q < n; q += NT) lev_chan_s[q] = pw.lev_chan[q];
    __syncthreads();
    const double *lthr = lev_sm ? lev_thr_s : pw.lev_thr;
    const int *lstart = lev_sm ? lev_start_s : pw.lev_start;
    if (warp == 0) {
        int ncl_run = 0, np_run = 0, no_run = 0;
        for (int base = 0; base < n; base += 32) {
            const int i = base + lane;
            const bool in = i < n;
            const bool closed = in && kind_s[i] == CH_CLOSED;
            const bool pch = in && !closed;
            const unsigned bc = __ballot_sync(0xffffffffu, closed);
            const unsigned bp = __ballot_sync(0xffffffffu, pch);
            const unsigned bo = __ballot_sync(0xffffffffu, in && x - pw.e_thr[i] > 0.0);
            const unsigned lt = (1u << lane) - 1u;
            if (closed) {
                col_chan[ncl_run + __popc(bc & lt)] = i;
                open_pos[i] = -1;
            }
            if (pch) open_pos[i] = np_run + __popc(bp & lt);
            ncl_run += __popc(bc);
            np_run += __popc(bp);
            no_run += __popc(bo);
        }
        if (lane == 0) {
            s_np = np_run;
            s_no = no_run;
            if (n_open_out) n_open_out[e] = no_run;
        }
    }
    __syncthreads();
    const int np = s_np, no = s_no, ncl = n - np;
    if (no == 0) return;
    if (np != no) {   // direct mode: P is the open set
        if (tid == 0) status[e] = RM_ESINGULAR;
        return;
    }
    for (int i = tid; i < n; i += NT)
        if (open_pos[i] >= 0) col_chan[ncl + open_pos[i]] = i;
    __syncthreads();
    const double a = pw.a, b = pw.b;
    for (int c = tid; c < n; c += NT) {
        const ChanFn cj = cf[col_chan[c]];
        colv[c] = (float)(a * cj.ghp - b * cj.gh);
        dgv[c] = (float)cj.gh;
        if (c >= ncl) {
            rsv[c - ncl] = (float)(a * cj.sp - b * cj.s);
            rss[c - ncl] = (float)cj.s;
        }
    }
    __syncthreads();

    // ---- assemble the tile of [A | B] (FP32, as it is eliminated) -----------
    const int w = n + np;
    float t[TR][TC];
#pragma unroll
    for (int i = 0; i < TR; ++i) {
        const int r = ty + G16 * i;
#pragma unroll
        for (int j = 0; j < TC; ++j) {
            const int c = tx + G16 * j;
            float v = 0.0f;
            if (r < n && c < w) {
                if (c < n) {
                    const int ch = col_chan[c];
                    v = -Rs[r <= ch ? tri_idx(r, ch, n) : tri_idx(ch, r, n)] * colv[c];
                    if (r == ch) v += dgv[c];
                } else {
                    const int k = c - n;
                    const int ch = col_chan[ncl + k];
                    v = Rs[r <= ch ? tri_idx(r, ch, n) : tri_idx(ch, r, n)] * rsv[k];
                    if (r == ch) v -= rss[k];
                }
            }
            t[i][j] = v;
        }
    }

    // ---- Gauss-Jordan elimination, implicit partial pivoting -----------------
    // Columns are taken in pairs (c even, c + 1): their owner half-warps form
    // one warp (lanes 0-15 column c, 16-31 column c + 1), which finds pivot
    // p1 of column c, brings column c + 1 up to date with it by shuffles,
    // finds its pivot p2, and publishes both multiplier columns; after one
    // barrier every thread applies both eliminations in turn (the first
    // leaves row p2 as a_p2j - m1_p2 a_p1j, the pivot row of the second).
    const unsigned hmask = (lane & 16) ? 0xffff0000u : 0x0000ffffu;
    const unsigned full = 0xffffffffu;
    int c_first_single = 0;
    for (int c = 0; c + 1 < n; c += 2) {
        const int buf = (c >> 1) & 1;
        const int jc = c >> 4;
        if ((tx >> 1) == ((c & 15) >> 1)) {
            float v[TR];
            unsigned key = 0u;
#pragma unroll
            for (int i = 0; i < TR; ++i) {
                v[i] = pick<TC>(t[i], jc);
                const int r = ty + G16 * i;
                const bool used = (used_s[r >> 5] >> (r & 31)) & 1u;
                const unsigned kv = (__float_as_uint(fabsf(v[i])) & ~0x7fu) | (unsigned)(127 - r);
                if (r < n && !used && kv > key) key = kv;
            }
            key = __reduce_max_sync(hmask, key);
            const unsigned keyA = __shfl_sync(full, key, 0);
            const int p1 = keyA ? 127 - (int)(keyA & 0x7fu) : 0;
            const float at_p1 = pick<TR>(v, p1 >> 4);
            const float pv1 = __shfl_sync(full, at_p1, p1 & 15);
            const float u1 = __shfl_sync(full, at_p1, 16 + (p1 & 15));   // a_{p1, c+1}
            const float ipv1 = __frcp_rn(pv1);
            float m1[TR], v2[TR];
            unsigned key2 = 0u;
#pragma unroll
            for (int i = 0; i < TR; ++i) {
                const int r = ty + G16 * i;
                m1[i] = (r == p1) ? 0.0f : v[i] * ipv1;
                const float mA = __shfl_xor_sync(full, m1[i], 16);
                v2[i] = fmaf(-mA, u1, v[i]);
                const bool used = ((used_s[r >> 5] >> (r & 31)) & 1u) || r == p1;
                const unsigned kv = (__float_as_uint(fabsf(v2[i])) & ~0x7fu) | (unsigned)(127 - r);
                if (r < n && !used && kv > key2) key2 = kv;
            }
            key2 = __reduce_max_sync(hmask, key2);
            const unsigned keyB = __shfl_sync(full, key2, 16);
            const int p2 = keyB ? 127 - (int)(keyB & 0x7fu) : 0;
            const float pv2 = __shfl_sync(full, pick<TR>(v2, p2 >> 4), 16 + (p2 & 15));
            const float ipv2 = __frcp_rn(pv2);
            if ((tx & 1) == 0) {
#pragma unroll
                for (int i = 0; i < TR; ++i) colbuf[buf][ty + G16 * i] = m1[i];
            } else {
#pragma unroll
                for (int i = 0; i < TR; ++i) {
                    const int r = ty + G16 * i;
                    colbuf2[buf][r] = (r == p2) ? 0.0f : v2[i] * ipv2;
                }
            }
            if (lane == 0) {
                pbuf[buf] = p1;
                pvbuf[buf] = pv1;
                pbuf2[buf] = p2;
                pvbuf2[buf] = pv2;
                used_s[p1 >> 5] |= 1u << (p1 & 31);
                used_s[p2 >> 5] |= 1u << (p2 & 31);
                rowpos[p1] = c;
                rowpos[p2] = c + 1;
                pivval[c] = pv1;
                pivval[c + 1] = pv2;
            }
        }
        __syncthreads();
        const int p1 = pbuf[buf], p2 = pbuf2[buf];
        const float pv1 = pvbuf[buf], pv2 = pvbuf2[buf];
        if (!(fabsf(pv1) > 0.0f) || !isfinite(pv1) || !(fabsf(pv2) > 0.0f) || !isfinite(pv2)) {
            if (tid == 0) status[e] = RM_ESINGULAR;
            return;
        }
        // first elimination (row p1); it turns row p2 into its reduced form
        // a_p2j - m1_p2 a_p1j, which the second elimination then uses
        const int ip1 = p1 >> 4, src1 = (lane & 16) | (p1 & 15);
        const int ip2 = p2 >> 4, src2 = (lane & 16) | (p2 & 15);
        float rb[TC];
#pragma unroll
        for (int i = 0; i < TR; ++i) {
            if (ip1 == i) {
#pragma unroll
                for (int j = 0; j < TC; ++j) rb[j] = __shfl_sync(full, t[i][j], src1);
            }
        }
#pragma unroll
        for (int i = 0; i < TR; ++i) {
            const float f1 = colbuf[buf][ty + G16 * i];
#pragma unroll
            for (int j = 0; j < TC; ++j) t[i][j] = fmaf(-f1, rb[j], t[i][j]);
        }
#pragma unroll
        for (int i = 0; i < TR; ++i) {
            if (ip2 == i) {
#pragma unroll
                for (int j = 0; j < TC; ++j) rb[j] = __shfl_sync(full, t[i][j], src2);
            }
        }
#pragma unroll
        for (int i = 0; i < TR; ++i) {
            const float f2 = colbuf2[buf][ty + G16 * i];
#pragma unroll
            for (int j = 0; j < TC; ++j) t[i][j] = fmaf(-f2, rb[j], t[i][j]);
        }
        c_first_single = c + 2;
    }
    for (int c = c_first_single; c < n; ++c) {
        const int buf = (c >> 1) & 1;
        if (tx == (c & 15)) {
            // the column's half-warp: pivot row by shuffles, then the multipliers
            const int jc = c >> 4;
            float v[TR];
            // pivot: one max-reduction over keys |v| (low 7 mantissa bits
            // replaced by 127 - r, so rows within 2^-17 of the largest
            // magnitude tie and the lowest one wins); unused rows only
            unsigned key = 0u;
#pragma unroll
            for (int i = 0; i < TR; ++i) {
                v[i] = pick<TC>(t[i], jc);
                const int r = ty + G16 * i;
                const bool used = (used_s[r >> 5] >> (r & 31)) & 1u;
                const unsigned kv = (__float_as_uint(fabsf(v[i])) & ~0x7fu) | (unsigned)(127 - r);
                if (r < n && !used && kv > key) key = kv;
            }
            key = __reduce_max_sync(hmask, key);
            const int p = key ? 127 - (int)(key & 0x7fu) : 0;
            const float pv = __shfl_sync(hmask, pick<TR>(v, p >> 4), p & 15, 16);
            const float ipv = __frcp_rn(pv);
#pragma unroll
            for (int i = 0; i < TR; ++i) {
                const int r = ty + G16 * i;
                colbuf[buf][r] = (r == p) ? 0.0f : v[i] * ipv;
            }
            if (ty == 0) {
                pbuf[buf] = p;
                pvbuf[buf] = pv;
                used_s[p >> 5] |= 1u << (p & 31);
                rowpos[p] = c;
                pivval[c] = pv;
            }
        }
        __syncthreads();
        const int p = pbuf[buf];
        const float pv = pvbuf[buf];
        if (!(fabsf(pv) > 0.0f) || !isfinite(pv)) {   // the same in every thread
            if (tid == 0) status[e] = RM_ESINGULAR;
            return;
        }
        // row p's values for this thread's columns, from the lane of this
        // half-warp that holds row p. Columns <= c and the padding take the
        // update too: they are never read again (padding stays zero, as row
        // p's padding is zero); the pivot row's multiplier is zero.
        const int ip = p >> 4, src = (lane & 16) | (p & 15);
        float rb[TC];
#pragma unroll
        for (int i = 0; i < TR; ++i) {
            if (ip == i) {
#pragma unroll
                for (int j = 0; j < TC; ++j) rb[j] = __shfl_sync(0xffffffffu, t[i][j], src);
            }
        }
#pragma unroll
        for (int i = 0; i < TR; ++i) {
            const float f = colbuf[buf][ty + G16 * i];
#pragma unroll
            for (int j = 0; j < TC; ++j) t[i][j] = fmaf(-f, rb[j], t[i][j]);
        }
    }
    __syncthreads();

    // ---- K_u = x of the P unknowns, into Pm (n_o x n_o, row = unknown) -------
#pragma unroll
    for (int i = 0; i < TR; ++i) {
        const int r = ty + G16 * i;
        const int u = r < n ? rowpos[r] : -1;
        if (u >= ncl) {
            const float dinv = 1.0f / pivval[u];
#pragma unroll
            for (int j = 0; j < TC; ++j) {
                const int col = tx + G16 * j;
                if (col >= n && col < w) Pm[(u - ncl) * no + (col - n)] = t[i][j] * dinv;
            }
        }
    }
    __syncthreads();
    if (K_out) {
        for (int q = tid; q < no * no; q += NT) {
            const int p = q / no, r = q - (q / no) * no;
            K_out[(size_t)e * n * n + (size_t)p * n + r] = (double)Pm[q];
        }
    }
    if (!omega) return;

    // ---- T step: W = -(1 - iK)^{-1} by the complex sweep in registers --------
    {
        const SweepShared sh = {&ucol[0][0], &vcol[0][0], &ucol2[0][0], &vcol2[0][0],
                                dbuf, dinvbuf, dbuf2, dinvbuf2, G16 * TR};
        if (!t_sweep_dispatch<1, TR>((no + 15) >> 4, Pm, no, tid, lane, tx, ty, hmask, sh)) {
            if (tid == 0) status[e] = RM_ESINGULAR;
            return;
        }
    }

    // ---- Omega ----------------------------------------------------------------
    const int npair = nl * (nl + 1) / 2;
    const double g = pw.g;
    double *om = omega + (size_t)e * n_tri;
    for (int q = tid; q < npair; q += NT) {
        int I, J;
        tri_pair(q, nl, I, J);
        if (!(x - lthr[I] > 0.0) || !(x - lthr[J] > 0.0)) continue;
        double s = 0.0;
        for (int ia = lstart[I]; ia < lstart[I + 1]; ++ia) {
            const int pa = open_pos[lev_chan_s[ia]];
            for (int ib = lstart[J]; ib < lstart[J + 1]; ++ib)
                s += (double)Pm[pa * no + open_pos[lev_chan_s[ib]]];
        }
        om[q] += g * s;
    }
}

template <int TR, int TC>
cudaError_t launch_tile(const PwDev &pw, const double *E, int nE, const ChanFn *cf, const double *R, int *status,
                        double *K_out, int *n_open_out, double *omega, int n_tri, const int *deep_ws, int pass,
                        cudaStream_t s)
{
    const size_t smem = ((size_t)tri_ld(pw.n) + (size_t)pw.n * pw.n) * sizeof(float);
    cudaError_t err =
        cudaFuncSetAttribute(solve_f32_kernel<TR, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    solve_f32_kernel<TR, TC><<<nE, NT, smem, s>>>(pw, E, cf, R, status, K_out, n_open_out, omega, n_tri, deep_ws,
                                                  chanfn_deep_cap(), pass);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_solve_f32(const PwDev &pw, const double *E, int nE, const ChanFn *cf, const double *R,
                             int *status, double *K_out, int *n_open_out, double *omega, int n_tri,
                             const int *deep_ws, int pass, cudaStream_t s)
{
    if (pw.n > MAXN) return cudaErrorInvalidValue;
    if (nE == 0) return cudaSuccess;
    if (pw.n <= 32) return launch_tile<2, 4>(pw, E, nE, cf, R, status, K_out, n_open_out, omega, n_tri, deep_ws, pass, s);
    if (pw.n <= 64) return launch_tile<4, 8>(pw, E, nE, cf, R, status, K_out, n_open_out, omega, n_tri, deep_ws, pass, s);
    return launch_tile<6, 12>(pw, E, nE, cf, R, status, K_out, n_open_out, omega, n_tri, deep_ws, pass, s);
}

}  // namespace rmgb
