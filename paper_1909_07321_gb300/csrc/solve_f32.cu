// Steps (c) and (d) in FP32 for the mixed-precision path (direct mode,
// n <= SOLVE_SMALL_MAXN): one CTA of 16 x 16 threads per energy, with both
// matrices held in registers.
//
// (c) Matching (Section "Overview", Eq. match), as in solve_small.cu: with
// the channels ordered closed first, then open (the set P),
//   [diag(Ghat) - R diag(a Ghat' - b Ghat)] X = -[diag(S) - R diag(a S' - b S)] P,
// K = X[P rows]. Thread (ty, tx) holds rows ty + 16 i and columns tx + 16 j
// of the n x (n + n_o) augmented matrix. Gauss-Jordan elimination with
// partial pivoting, the pivot rows left in place (implicit pivoting): for
// column c the owners publish the column, every warp finds the same pivot
// row p among the rows not yet used (largest magnitude, lowest index on
// ties), the owners of row p publish it, and every other row r (used or not)
// takes a_rj -= (a_rc / a_pc) a_pj for j > c. After n columns the unknowns
// are x_c = a_{p(c), rhs} / a_{p(c), c}, with no back-substitution; only the
// pivot column and row pass through shared memory.
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

template <int TR, int TC>
__global__ void __launch_bounds__(NT) solve_f32_kernel(
    PwDev pw, const double *__restrict__ E, const ChanFn *__restrict__ cfa, const double *__restrict__ Ra,
    int *__restrict__ status, double *__restrict__ K_out, int *__restrict__ n_open_out,
    double *__restrict__ omega, int n_tri, const int *__restrict__ deep_ws, int deep_cap, int pass)
{
    static_assert(TC == 2 * TR && G16 * TR <= MAXN, "tile shape");
    if (deep_ws) {
        const bool deferred = deep_ws[0] <= deep_cap && deep_ws[1 + deep_cap + blockIdx.x] != 0;
        if (pass == 0 ? deferred : !deferred) return;
    }
    extern __shared__ float Pm[];                 // K, later |T|^2 (n_o x n_o)
    __shared__ int col_chan[MAXN];                // unknown column -> channel
    __shared__ int open_pos[MAXN];                // channel -> position in P (-1: closed)
    __shared__ double colv[MAXN], dgv[MAXN];      // unknown column: a Ghat' - b Ghat, Ghat
    __shared__ double rsv[MAXN], rss[MAXN];       // right-hand side k: a S' - b S, S
    __shared__ int kind_s[MAXN];
    __shared__ float colbuf[2][G16 * TR];
    __shared__ float rowbuf[2][G16 * TC];
    __shared__ int done_s[G16 * TR];
    __shared__ int rowpos[G16 * TR];
    __shared__ float pivval[MAXN];
    __shared__ float2 ucol[2][G16 * TR];
    __shared__ int s_no, s_np;

    const int e = blockIdx.x;
    const int n = pw.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ty = tid >> 4, tx = tid & 15;
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
        done_s[r] = 0;
        ucol[0][r] = make_float2(0.0f, 0.0f);
        ucol[1][r] = make_float2(0.0f, 0.0f);
    }
    __syncthreads();
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
        colv[c] = a * cj.ghp - b * cj.gh;
        dgv[c] = cj.gh;
        if (c >= ncl) {
            rsv[c - ncl] = a * cj.sp - b * cj.s;
            rss[c - ncl] = cj.s;
        }
    }
    __syncthreads();

    // ---- assemble the tile of [A | B] ----------------------------------------
    const int w = n + np;
    float t[TR][TC];
#pragma unroll
    for (int i = 0; i < TR; ++i) {
        const int r = ty + G16 * i;
#pragma unroll
        for (int j = 0; j < TC; ++j) {
            const int c = tx + G16 * j;
            double v = 0.0;
            if (r < n && c < w) {
                if (c < n) {
                    const int ch = col_chan[c];
                    const double Rv = Rp[r <= ch ? tri_idx(r, ch, n) : tri_idx(ch, r, n)];
                    v = -Rv * colv[c];
                    if (r == ch) v += dgv[c];
                } else {
                    const int k = c - n;
                    const int ch = col_chan[ncl + k];
                    const double Rv = Rp[r <= ch ? tri_idx(r, ch, n) : tri_idx(ch, r, n)];
                    v = Rv * rsv[k];
                    if (r == ch) v -= rss[k];
                }
            }
            t[i][j] = (float)v;
        }
    }

    // ---- Gauss-Jordan elimination, implicit partial pivoting -----------------
    for (int c = 0; c < n; ++c) {
        const int buf = c & 1;
        if (tx == (c & 15)) {
            const int jc = c >> 4;
#pragma unroll
            for (int i = 0; i < TR; ++i) {
                // select chains, not t[i][jc]: a runtime index would move the tile to local memory
                float v = t[i][0];
#pragma unroll
                for (int j = 1; j < TC; ++j) v = (j == jc) ? t[i][j] : v;
                colbuf[buf][ty + G16 * i] = v;
            }
        }
        __syncthreads();
        // pivot: largest |a_rc| among unused rows, lowest row on ties (every warp alike)
        float best = -1.0f;
        int bi = 0x7fffffff;
        for (int r = lane; r < n; r += 32) {
            const float v = done_s[r] ? -1.0f : fabsf(colbuf[buf][r]);
            if (v > best || (v == best && r < bi)) {
                best = v;
                bi = r;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, off);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        const int p = bi;
        const float pv = colbuf[buf][p];
        if (!(fabsf(pv) > 0.0f) || !isfinite(pv)) {   // the same in every thread
            if (tid == 0) status[e] = RM_ESINGULAR;
            return;
        }
        if (ty == (p & 15)) {
            const int ip = p >> 4;
#pragma unroll
            for (int j = 0; j < TC; ++j) {
                float v = t[0][j];
#pragma unroll
                for (int i = 1; i < TR; ++i) v = (i == ip) ? t[i][j] : v;
                const int col = tx + G16 * j;
                if (col > c && col < w) rowbuf[buf][col] = v;
            }
        }
        __syncthreads();
        if (tid == 0) {
            done_s[p] = 1;
            rowpos[p] = c;
            pivval[c] = pv;
        }
        const float ipv = 1.0f / pv;
        float rb[TC];
#pragma unroll
        for (int j = 0; j < TC; ++j) {
            const int col = tx + G16 * j;
            rb[j] = (col > c && col < w) ? rowbuf[buf][col] : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < TR; ++i) {
            const int r = ty + G16 * i;
            if (r < n && r != p) {
                const float f = colbuf[buf][r] * ipv;
#pragma unroll
                for (int j = 0; j < TC; ++j) t[i][j] = fmaf(-f, rb[j], t[i][j]);
            }
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
    float2 z[TR][TR];
#pragma unroll
    for (int i = 0; i < TR; ++i) {
        const int r = ty + G16 * i;
#pragma unroll
        for (int j = 0; j < TR; ++j) {
            const int c = tx + G16 * j;
            float2 v = make_float2(0.0f, 0.0f);
            if (r < no && c < no) v = make_float2(r == c ? 1.0f : 0.0f, -0.5f * (Pm[r * no + c] + Pm[c * no + r]));
            z[i][j] = v;
        }
    }
    for (int k = 0; k < no; ++k) {
        const int buf = k & 1;
        if (tx == (k & 15)) {
            const int jk = k >> 4;
#pragma unroll
            for (int i = 0; i < TR; ++i) {
                const int r = ty + G16 * i;
                float2 v = z[i][0];
#pragma unroll
                for (int j = 1; j < TR; ++j) v = (j == jk) ? z[i][j] : v;
                if (r < no) ucol[buf][r] = v;
            }
        }
        __syncthreads();
        const float2 d = ucol[buf][k];
        if (!(fabsf(d.x) + fabsf(d.y) > 0.0f) || !isfinite(d.x) || !isfinite(d.y)) {
            if (tid == 0) status[e] = RM_ESINGULAR;
            return;
        }
        const float2 dinv = crcp_f(d);
        float2 ui[TR], uj[TR];
#pragma unroll
        for (int i = 0; i < TR; ++i) {
            ui[i] = cmul_f(ucol[buf][ty + G16 * i], dinv);     // v_i = u_i / d
            uj[i] = ucol[buf][tx + G16 * i];
        }
#pragma unroll
        for (int i = 0; i < TR; ++i) {
            const int r = ty + G16 * i;
#pragma unroll
            for (int j = 0; j < TR; ++j) {
                const int c = tx + G16 * j;
                float2 zz = z[i][j];
                zz.x = fmaf(-ui[i].x, uj[j].x, fmaf(ui[i].y, uj[j].y, zz.x));
                zz.y = fmaf(-ui[i].x, uj[j].y, fmaf(-ui[i].y, uj[j].x, zz.y));
                if (c == k) zz = ui[i];
                if (r == k) zz = (c == k) ? make_float2(-dinv.x, -dinv.y) : cmul_f(uj[j], dinv);
                z[i][j] = zz;
            }
        }
    }
    __syncthreads();   // every read of K in Pm is done
#pragma unroll
    for (int i = 0; i < TR; ++i) {
        const int r = ty + G16 * i;
#pragma unroll
        for (int j = 0; j < TR; ++j) {
            const int c = tx + G16 * j;
            if (r < no && c < no) {
                const float re = z[i][j].x + (r == c ? 1.0f : 0.0f), im = z[i][j].y;
                Pm[r * no + c] = 4.0f * fmaf(re, re, im * im);
            }
        }
    }
    __syncthreads();

    // ---- Omega ----------------------------------------------------------------
    const int nl = pw.n_levels;
    const int npair = nl * (nl + 1) / 2;
    const double g = pw.g;
    double *om = omega + (size_t)e * n_tri;
    for (int q = tid; q < npair; q += NT) {
        int I, J;
        tri_pair(q, nl, I, J);
        if (!(x - pw.lev_thr[I] > 0.0) || !(x - pw.lev_thr[J] > 0.0)) continue;
        double s = 0.0;
        for (int ia = pw.lev_start[I]; ia < pw.lev_start[I + 1]; ++ia) {
            const int pa = open_pos[pw.lev_chan[ia]];
            for (int ib = pw.lev_start[J]; ib < pw.lev_start[J + 1]; ++ib)
                s += (double)Pm[pa * no + open_pos[pw.lev_chan[ib]]];
        }
        om[q] += g * s;
    }
}

template <int TR, int TC>
cudaError_t launch_tile(const PwDev &pw, const double *E, int nE, const ChanFn *cf, const double *R, int *status,
                        double *K_out, int *n_open_out, double *omega, int n_tri, const int *deep_ws, int pass,
                        cudaStream_t s)
{
    const size_t smem = (size_t)pw.n * pw.n * sizeof(float);
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
