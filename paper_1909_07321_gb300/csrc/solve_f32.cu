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
// column c the pivot row p is the largest magnitude among the rows not yet
// used (to 2^-17, lowest index among those), every other row r (used or not)
// takes a_rj -= m_r a_pj, m_r = a_rc (1 / a_pc), for j > c (the reciprocal
// by rcp.approx and one Newton-Raphson step, within one ulp; a pivot below
// the smallest normal number counts as zero). After n columns the unknowns
// are x_c = a_{p(c), rhs} / a_{p(c), c}, with no back-substitution.
//
// The columns are eliminated in blocks of KBG. The block's columns are
// copied to shared memory and one warp (lane l holds rows l + 32 s) runs the
// KBG steps on them alone: pivot by one warp max-reduction, multipliers, and
// the step's update of the block's later columns. It publishes the KBG pivot
// rows and multiplier columns; after one barrier every thread applies the
// KBG steps to its columns past the block in the same order (the pivot row's
// values for a thread's columns come from the thread of its half-warp that
// holds that row, through shared memory). Every element therefore takes the
// same operations, in the same order, as in the column-by-column
// elimination, with two barriers per KBG columns instead of one per column;
// columns left of the block and the padding beyond n + n_o are not touched.
// The serial part of every block is one warp's, so the throughput comes from
// the energies resident on an SM: block sizes and tiles are chosen to keep a
// thread within 64 registers, four CTAs per SM, up to 64 channels.
//
// (d) T = 2iK(1 - iK)^{-1} = 2(1 - iK)^{-1} - 2 (Section "Glossary of
// terms"): 1 - iK (complex, K symmetrised) in registers in the same 16 x 16
// layout, inverted in place by the sweep operator (Gauss-Jordan without
// pivoting: its Hermitian part is the identity, so every pivot has a
// positive real part). One sweep step on pivot k with u = column k and
// d = u_k, v = u / d: z_ij -= v_i u_j, then column k <- v, row k <- v^T and
// z_kk <- -1/d. The pivots are taken in blocks the same way: one warp sweeps
// the block's columns through its KB steps and publishes each step's u and v;
// every thread then applies z_ij -= v_i u_j for the KB steps and takes the
// block's rows and columns from the swept block (the matrix is symmetric).
// The sweep leaves W = -(1 - iK)^{-1}, and |T_ab|^2 = 4 |W_ab + delta_ab|^2.
// For target levels I <= J one thread owns Omega_IJ(E) and adds
// g sum_{a in I, b in J} |T_ab|^2, the level pair's sum in FP32 (as the
// values; relative error <= |I||J| 2^-24) and the addition to Omega in FP64
// by one atomic add, the only addition to that entry in the launch: launches
// on a stream are ordered, so the sum over partial waves is deterministic,
// and the add needs no read of Omega by the kernel.
#include <math.h>

#include "dense_smem.cuh"
#include "rm_internal.cuh"

namespace rmgb {
namespace {

constexpr int G16 = 16;                          // thread grid 16 x 16
constexpr int MAXN = SOLVE_SMALL_MAXN;
constexpr int KBG = 4;                           // columns per elimination block
constexpr float kMinNormal = 1.17549435e-38f;    // smallest normal FP32 number: smaller pivots count as zero

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

// Element [s][q] of a 2-D register array, s uniform, q a compile-time index.
template <int S, int Q, typename T>
__device__ __forceinline__ T pick_s(const T (&v)[S][Q], int s, int q)
{
    T r = v[0][q];
#pragma unroll
    for (int k = 1; k < S; ++k)
        if (s == k) r = v[k][q];
    return r;
}

__device__ __forceinline__ float2 shfl2(float2 v, int src)
{
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// Loads TR consecutive floats (f, 16-byte aligned) by vector loads.
template <int TR>
__device__ __forceinline__ void load_row(float (&f)[TR], const float *src)
{
#pragma unroll
    for (int i = 0; i < TR; i += 4) {
        if (i + 4 <= TR) {
            const float4 v = *reinterpret_cast<const float4 *>(src + i);
            f[i] = v.x, f[i + 1] = v.y, f[i + 2] = v.z, f[i + 3] = v.w;
        } else {
            const float2 v = *reinterpret_cast<const float2 *>(src + i);
            f[i] = v.x, f[i + 1] = v.y;
        }
    }
}

// Whether the elimination steps skip the tiles left of the block and the
// padding tiles (uniform branches) or update every tile.
constexpr bool kSkipTiles = true;

// One elimination step on this thread's tiles: the thread of the half-warp
// that holds pivot row p writes its values for the half-warp's columns to rb,
// then t_ij -= f_i rb_j (f: the step's multipliers for this thread's rows).
template <int TR, int TC, int TRP>
__device__ __forceinline__ void gj_step(float (&t)[TR][TC], int p, const float *fq, float *rb, int ty, int jlo,
                                        int jhi)
{
    if (ty == (p & 15)) {
        const int ip = p >> 4;
#pragma unroll
        for (int i = 0; i < TR; ++i)
            if (ip == i) {
#pragma unroll
                for (int j = 0; j < TC; j += 4)
                    *reinterpret_cast<float4 *>(rb + j) = make_float4(t[i][j], t[i][j + 1], t[i][j + 2], t[i][j + 3]);
            }
    }
    __syncwarp();
    float f[TR], u[TC];
    load_row<TR>(f, fq);
    load_row<TC>(u, rb);
#pragma unroll
    for (int j = 0; j < TC; ++j) {
        if (!kSkipTiles || (j >= jlo && j < jhi)) {
#pragma unroll
            for (int i = 0; i < TR; ++i) t[i][j] = fmaf(-f[i], u[j], t[i][j]);
        }
    }
}

// The same step on tiles J0..TC-1 (J0 fixed at compile time: no per-tile
// conditions; padding tiles past n + n_o hold zeros in every row, the pivot
// row's too, and stay zero). Only the quads of rb from J0's on are written.
template <int TR, int TC, int TRP, int J0>
__device__ __forceinline__ void gj_step_from(float (&t)[TR][TC], int p, const float *fq, float *rb, int ty)
{
    constexpr int JQ = J0 & ~3;
    if (ty == (p & 15)) {
        const int ip = p >> 4;
#pragma unroll
        for (int i = 0; i < TR; ++i)
            if (ip == i) {
#pragma unroll
                for (int j = JQ; j < TC; j += 4)
                    *reinterpret_cast<float4 *>(rb + j) = make_float4(t[i][j], t[i][j + 1], t[i][j + 2], t[i][j + 3]);
            }
    }
    __syncwarp();
    float f[TR], u[TC];
    load_row<TR>(f, fq);
#pragma unroll
    for (int j = JQ; j < TC; j += 4) {
        const float4 v = *reinterpret_cast<const float4 *>(rb + j);
        u[j] = v.x, u[j + 1] = v.y, u[j + 2] = v.z, u[j + 3] = v.w;
    }
#pragma unroll
    for (int j = J0; j < TC; ++j) {
#pragma unroll
        for (int i = 0; i < TR; ++i) t[i][j] = fmaf(-f[i], u[j], t[i][j]);
    }
}

// A full block's KBG steps on tiles j0..TC-1, the first live tile dispatched
// to a compile-time J0 (one branch per block instead of one per tile and step).
template <int TR, int TC, int TRP, int KB, int J0 = 0>
__device__ __forceinline__ void gj_block_from(int j0, float (&t)[TR][TC], const int (&pk)[KB], const float *mbt,
                                              float *rbt, int ty)
{
    if constexpr (J0 + 1 < TC) {
        if (j0 > J0) return gj_block_from<TR, TC, TRP, KB, J0 + 1>(j0, t, pk, mbt, rbt, ty);
    }
#pragma unroll
    for (int q = 0; q < KB; ++q)
        gj_step_from<TR, TC, TRP, J0>(t, pk[q], mbt + q * G16 * TRP, rbt + (q & 1) * G16 * TC, ty);
}

// Shared-memory layout of the blocked elimination and sweep for TR row tiles
// (sizes in floats; both phases use the same buffer one after the other).
template <int TR, int TC>
struct BlkLayout {
    static constexpr int ROWS = G16 * TR;
    static constexpr int TRP = (TR + 3) & ~3;     // per-thread row values, padded for vector loads
    // elimination: block columns [KBG][ROWS], multipliers [KBG][16][TRP],
    // pivot-row values [2][16][TC]
    static constexpr int GJ = KBG * ROWS + KBG * G16 * TRP + 2 * G16 * TC;
    // sweep (float2): block columns and swept block [KBT][ROWS] each, u and v
    // [KBT][16][VST] each (VST = TRP + 2: rows of consecutive ty start in
    // different banks), KBT <= 8
    static constexpr int VST = TRP + 2;
    static constexpr int SW = 2 * (2 * 8 * ROWS + 2 * 8 * G16 * VST);
    static constexpr int FLOATS = GJ > SW ? GJ : SW;
};

// Loads TS consecutive complex values (16-byte aligned) by vector loads.
template <int TS>
__device__ __forceinline__ void load_cvec(float2 (&v)[TS], const float2 *src)
{
#pragma unroll
    for (int i = 0; i < TS; i += 2) {
        if (i + 2 <= TS) {
            const float4 w = *reinterpret_cast<const float4 *>(src + i);
            v[i] = make_float2(w.x, w.y), v[i + 1] = make_float2(w.z, w.w);
        } else {
            v[i] = src[i];
        }
    }
}

// One sweep step on this thread's tiles: z_ij -= v_i u_j (v for its rows,
// u for its columns).
template <int TS>
__device__ __forceinline__ void sweep_step(float2 (&z)[TS][TS], const float2 *vq, const float2 *uq)
{
    float2 vi[TS], uj[TS];
    load_cvec<TS>(vi, vq);
    load_cvec<TS>(uj, uq);
#pragma unroll
    for (int i = 0; i < TS; ++i) {
#pragma unroll
        for (int j = 0; j < TS; ++j) {
            float2 zz = z[i][j];
            zz.x = fmaf(-vi[i].x, uj[j].x, fmaf(vi[i].y, uj[j].y, zz.x));
            zz.y = fmaf(-vi[i].x, uj[j].y, fmaf(-vi[i].y, uj[j].x, zz.y));
            z[i][j] = zz;
        }
    }
}

// T step for n_o <= 16 TS open channels (TS tiles per side in registers),
// pivots in blocks of KBT: W = -(1 - iK)^{-1} by the complex sweep, and
// |T_ab|^2 = 4 |W_ab + delta_ab|^2 written over K in Pm. Returns false (in
// every thread) if a pivot is zero or not finite.
template <int TS, int TR, int TC, int KBT>
__device__ __forceinline__ bool t_sweep(float *Pm, int no, int lane, int warp, int tx, int ty, float *xs,
                                        int *s_bad)
{
    using L = BlkLayout<TR, TC>;
    constexpr int ROWS = L::ROWS, VST = L::VST;
    constexpr int RWT = (G16 * TS + 31) / 32;     // rows per lane of the sweeping warp
    float2 *zp = reinterpret_cast<float2 *>(xs);  // [KBT][ROWS] the block's columns
    float2 *zf = zp + 8 * ROWS;                   // [KBT][ROWS] the swept block
    float2 *Vb = zf + 8 * ROWS;                   // [KBT][16][VST] v by (ty, i)
    float2 *Ub = Vb + 8 * G16 * VST;              // [KBT][16][VST] u by (tx, j)
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
    for (int k0 = 0; k0 < no; k0 += KBT) {
        const int kb = min(KBT, no - k0);
        const int jb = k0 >> 4, tx0 = k0 & 15;
        if (tx >= tx0 && tx < tx0 + kb) {
            float2 *col = zp + (tx - tx0) * ROWS;
#pragma unroll
            for (int i = 0; i < TS; ++i) col[ty + G16 * i] = pick<TS>(z[i], jb);
        }
        __syncthreads();
        if (warp == 0) {
            float2 a[RWT][KBT];
            bool bad = false;   // a zero or non-finite pivot in this block (the same in every lane)
#pragma unroll
            for (int s = 0; s < RWT; ++s) {
                const int r = lane + 32 * s;
#pragma unroll
                for (int q = 0; q < KBT; ++q)
                    a[s][q] = (q < kb && r < G16 * TS) ? zp[q * ROWS + r] : make_float2(0.0f, 0.0f);
            }
#pragma unroll
            for (int q = 0; q < KBT; ++q) {
                if (q < kb) {
                    const int kq = k0 + q;
                    const float2 d = shfl2(pick_s(a, kq >> 5, q), kq & 31);
                    bad |= !(fabsf(d.x) + fabsf(d.y) > 0.0f) || !isfinite(d.x) || !isfinite(d.y);
                    const float2 dinv = crcp_f(d);
                    float2 v[RWT];
#pragma unroll
                    for (int s = 0; s < RWT; ++s) {
                        const int r = lane + 32 * s;
                        v[s] = cmul_f(a[s][q], dinv);
                        if (r < G16 * TS) {
                            const int idx = (q * G16 + (r & 15)) * VST + (r >> 4);
                            Ub[idx] = a[s][q];
                            Vb[idx] = v[s];
                        }
                    }
#pragma unroll
                    for (int q2 = 0; q2 < KBT; ++q2) {
                        if (q2 != q && q2 < kb) {
                            const int k2 = k0 + q2;
                            const float2 u2 = shfl2(pick_s(a, k2 >> 5, q), k2 & 31);   // z_{k2, kq}
                            const float2 vk2 = cmul_f(u2, dinv);
#pragma unroll
                            for (int s = 0; s < RWT; ++s) {
                                const int r = lane + 32 * s;
                                float2 zz = a[s][q2];
                                zz.x = fmaf(-v[s].x, u2.x, fmaf(v[s].y, u2.y, zz.x));
                                zz.y = fmaf(-v[s].x, u2.y, fmaf(-v[s].y, u2.x, zz.y));
                                a[s][q2] = (r == kq) ? vk2 : zz;
                            }
                        }
                    }
#pragma unroll
                    for (int s = 0; s < RWT; ++s) {
                        const int r = lane + 32 * s;
                        a[s][q] = (r == kq) ? make_float2(-dinv.x, -dinv.y) : v[s];
                    }
                }
            }
#pragma unroll
            for (int s = 0; s < RWT; ++s) {
                const int r = lane + 32 * s;
#pragma unroll
                for (int q = 0; q < KBT; ++q)
                    if (q < kb && r < G16 * TS) zf[q * ROWS + r] = a[s][q];
            }
            if (lane == 0) *s_bad = bad;
        }
        __syncthreads();
        if (*s_bad) return false;   // the same in every thread
        if (kb == KBT) {
#pragma unroll
            for (int q = 0; q < KBT; ++q) sweep_step<TS>(z, Vb + (q * G16 + ty) * VST, Ub + (q * G16 + tx) * VST);
        } else {
            for (int q = 0; q < kb; ++q) sweep_step<TS>(z, Vb + (q * G16 + ty) * VST, Ub + (q * G16 + tx) * VST);
        }
        // the block's rows, then its columns, from the swept block (so that an
        // entry in both keeps the swept column's value)
        if (ty >= tx0 && ty < tx0 + kb) {
            const float2 *col = zf + (ty - tx0) * ROWS;
#pragma unroll
            for (int i = 0; i < TS; ++i)
                if (i == jb) {
#pragma unroll
                    for (int j = 0; j < TS; ++j) z[i][j] = col[tx + G16 * j];
                }
        }
        if (tx >= tx0 && tx < tx0 + kb) {
            const float2 *col = zf + (tx - tx0) * ROWS;
#pragma unroll
            for (int j = 0; j < TS; ++j)
                if (j == jb) {
#pragma unroll
                    for (int i = 0; i < TS; ++i) z[i][j] = col[ty + G16 * i];
                }
        }
    }
    __syncthreads();   // every read of K in Pm and of the buffers is done
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

// Pivots per sweep block for TS tiles (the sweeping warp holds TS x TS
// complex tile values and its block of columns at the same time, within the
// 64 registers a thread has at four CTAs per SM).
template <int TS>
struct SweepBlock {
    static constexpr int value = TS <= 2 ? 4 : 2;
};

// The T step with the smallest tile count that holds n_o (ts = ceil(n_o / 16),
// the same in every thread).
template <int TS, int TR, int TC>
__device__ __forceinline__ bool t_sweep_dispatch(int ts, float *Pm, int no, int lane, int warp, int tx, int ty,
                                                 float *xs, int *s_bad)
{
    if constexpr (TS < TR) {
        if (ts <= TS) return t_sweep<TS, TR, TC, SweepBlock<TS>::value>(Pm, no, lane, warp, tx, ty, xs, s_bad);
        return t_sweep_dispatch<TS + 1, TR, TC>(ts, Pm, no, lane, warp, tx, ty, xs, s_bad);
    } else {
        return t_sweep<TR, TR, TC, SweepBlock<TR>::value>(Pm, no, lane, warp, tx, ty, xs, s_bad);
    }
}

template <int TR, int TC>
__global__ void __launch_bounds__(NT, TR >= 6 ? 2 : 4) solve_f32_kernel(
    PwDev pw, const double *__restrict__ E, const ChanFn *__restrict__ cfa, const double *__restrict__ Ra,
    int *__restrict__ status, double *__restrict__ K_out, int *__restrict__ n_open_out,
    double *__restrict__ omega, int n_tri, const int *__restrict__ deep_ws, int deep_cap, int pass)
{
    static_assert(TC == 2 * TR && G16 * TR <= MAXN, "tile shape");
    using L = BlkLayout<TR, TC>;
    constexpr int ROWS = L::ROWS, TRP = L::TRP;
    constexpr int RWG = (ROWS + 31) / 32;         // rows per lane of the factoring warp
    if (deep_ws) {
        const bool deferred = deep_ws[0] <= deep_cap && deep_ws[1 + deep_cap + blockIdx.x] != 0;
        if (pass == 0 ? deferred : !deferred) return;
    }
    extern __shared__ float fsm[];                // [packed R of this energy][K, later |T|^2 (n_o x n_o)]
    float *Rs = fsm;
    float *Pm = fsm + tri_ld(pw.n);
    __shared__ __align__(16) float xs[L::FLOATS]; // the elimination's, then the sweep's block buffers
    __shared__ int col_chan[MAXN];                // unknown column -> channel
    __shared__ int open_pos[MAXN];                // channel -> position in P (-1: closed)
    __shared__ float cv_s[MAXN], dg_s[MAXN];      // channel: a Ghat' - b Ghat, Ghat (its unknown's column)
    __shared__ float sv_s[MAXN], ss_s[MAXN];      // channel: a S' - b S, S (its right-hand side)
    __shared__ int kind_s[MAXN];
    __shared__ bool open_s[MAXN];                 // channel open at this energy
    __shared__ __align__(16) int pbk[KBG];        // the block's pivot rows
    __shared__ int s_bad;                         // the block has a zero or non-finite pivot
    __shared__ int rowpos[ROWS];
    __shared__ float pivval[MAXN];
    __shared__ bool lev_open_s[MAXN];             // level open at this energy
    __shared__ int lev_start_s[MAXN + 1], lev_chan_s[MAXN];
    __shared__ int olev[MAXN];                    // the levels open at this energy, ascending
    __shared__ int s_no, s_np, s_nlo;

    const int e = blockIdx.x;
    const int n = pw.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = tid >> 4, ty = tid & 15;
    const double x = E[e];
    const ChanFn *cf = cfa + (size_t)e * n;
    const double *Rp = Ra + (size_t)e * tri_ld(n);
    const int st_e = status[e];
    const double a = pw.a, b = pw.b;
    const int nl = pw.n_levels;
    const int npair = nl * (nl + 1) / 2;
    double *om = omega ? omega + (size_t)e * n_tri : nullptr;
    // this energy's channel data (as the matrix entries need them), R and the
    // level tables into shared memory, every load issued before the first barrier
    for (int i = tid; i < n; i += NT) {
        const ChanFn c = cf[i];
        kind_s[i] = c.kind;
        cv_s[i] = (float)(a * c.ghp - b * c.gh);
        dg_s[i] = (float)c.gh;
        sv_s[i] = (float)(a * c.sp - b * c.s);
        ss_s[i] = (float)c.s;
        open_s[i] = x - pw.e_thr[i] > 0.0;
    }
    if (st_e != RM_OK) {
        if (tid == 0 && n_open_out) {
            int no = 0;
            for (int i = 0; i < n; ++i) no += (x - pw.e_thr[i] > 0.0);
            n_open_out[e] = no;
        }
        return;
    }
    {
        // R in batches of RB loads in flight per thread (each conversion waits
        // for its load)
        constexpr int RB = 8;
        const int m = tri_ld(n);
        for (int q0 = tid; q0 < m; q0 += RB * NT) {
            double v[RB];
#pragma unroll
            for (int k = 0; k < RB; ++k) {
                const int q = q0 + k * NT;
                v[k] = q < m ? Rp[q] : 0.0;
            }
#pragma unroll
            for (int k = 0; k < RB; ++k) {
                const int q = q0 + k * NT;
                if (q < m) Rs[q] = (float)v[k];
            }
        }
    }
    const bool lev_sm = nl <= MAXN;    // more levels than that (some without channels): read them in place
    if (lev_sm) {
        for (int q = tid; q < nl; q += NT) lev_open_s[q] = x - pw.lev_thr[q] > 0.0;
        for (int q = tid; q <= nl; q += NT) lev_start_s[q] = pw.lev_start[q];
    }
    for (int q = tid; q < n; q += NT) lev_chan_s[q] = pw.lev_chan[q];
    __syncthreads();
    const int *lstart = lev_sm ? lev_start_s : pw.lev_start;

    // ---- channel order: closed first, then P (open), by warp prefix counts
    if (warp == 0) {
        int ncl_run = 0, np_run = 0, no_run = 0;
        for (int base = 0; base < n; base += 32) {
            const int i = base + lane;
            const bool in = i < n;
            const bool closed = in && kind_s[i] == CH_CLOSED;
            const bool pch = in && !closed;
            const unsigned bc = __ballot_sync(0xffffffffu, closed);
            const unsigned bp = __ballot_sync(0xffffffffu, pch);
            const unsigned bo = __ballot_sync(0xffffffffu, in && open_s[i]);
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
        if (lev_sm) {
            int nlo_run = 0;
            for (int base = 0; base < nl; base += 32) {
                const int q = base + lane;
                const bool op = q < nl && lev_open_s[q];
                const unsigned bo = __ballot_sync(0xffffffffu, op);
                if (op) olev[nlo_run + __popc(bo & ((1u << lane) - 1u))] = q;
                nlo_run += __popc(bo);
            }
            if (lane == 0) s_nlo = nlo_run;
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
                    v = -Rs[r <= ch ? tri_idx(r, ch, n) : tri_idx(ch, r, n)] * cv_s[ch];
                    if (r == ch) v += dg_s[ch];
                } else {
                    const int ch = col_chan[ncl + c - n];
                    v = Rs[r <= ch ? tri_idx(r, ch, n) : tri_idx(ch, r, n)] * sv_s[ch];
                    if (r == ch) v -= ss_s[ch];
                }
            }
            t[i][j] = v;
        }
    }

    // ---- Gauss-Jordan elimination in blocks of KBG columns --------------------
    float *pan = xs;                              // [KBG][ROWS] the block's columns
    float *mb = xs + KBG * ROWS;                  // [KBG][16][TRP] multipliers, by (ty, i)
    float *rowb = mb + KBG * G16 * TRP;           // [2][16][TC] pivot-row values, by column class
    const unsigned full = 0xffffffffu;
    const int jhi = (w + G16 - 1) >> 4;           // tiles holding a column < n + n_o
    // factoring warp: row lane + 32 s takes part in the pivot search while
    // umask[s] is all ones (rows < n not yet used); rtag[s] = 127 - row
    unsigned umask[RWG], rtag[RWG];
#pragma unroll
    for (int s = 0; s < RWG; ++s) {
        umask[s] = lane + 32 * s < n ? ~0u : 0u;
        rtag[s] = (unsigned)(127 - (lane + 32 * s));
    }
    for (int c0 = 0; c0 < n; c0 += KBG) {
        const int kb = min(KBG, n - c0);
        const int jb = c0 >> 4, tx0 = c0 & 15;
        if (tx >= tx0 && tx < tx0 + kb) {
            float *col = pan + (tx - tx0) * ROWS;
#pragma unroll
            for (int i = 0; i < TR; ++i) col[ty + G16 * i] = pick<TC>(t[i], jb);
        }
        __syncthreads();
        if (warp == 0) {
            float a[RWG][KBG];
            int myp = 0;
            float mypv = 0.0f;
#pragma unroll
            for (int s = 0; s < RWG; ++s) {
                const int r = lane + 32 * s;
#pragma unroll
                for (int q = 0; q < KBG; ++q) a[s][q] = (q < kb && r < ROWS) ? pan[q * ROWS + r] : 0.0f;
            }
#pragma unroll
            for (int q = 0; q < KBG; ++q) {
                if (q < kb) {
                    // pivot: one max-reduction over keys |v| (low 7 mantissa bits
                    // replaced by 127 - r, so rows within 2^-17 of the largest
                    // magnitude tie and the lowest one wins); unused rows only
                    unsigned key = 0u;
#pragma unroll
                    for (int s = 0; s < RWG; ++s)
                        key = max(key, ((__float_as_uint(a[s][q]) & 0x7fffff80u) | rtag[s]) & umask[s]);
                    key = __reduce_max_sync(full, key);
                    const int p = key ? 127 - (int)(key & 0x7fu) : 0;
                    const int ps = p >> 5, pl = p & 31;
                    const float pv = __shfl_sync(full, pick_s(a, ps, q), pl);
                    const float ipv = rcp_nr_f(pv);
                    float m[RWG];
#pragma unroll
                    for (int s = 0; s < RWG; ++s) {
                        const int r = lane + 32 * s;
                        m[s] = (r == p) ? 0.0f : a[s][q] * ipv;
                        if (r < ROWS) mb[(q * G16 + (r & 15)) * TRP + (r >> 4)] = m[s];
                    }
#pragma unroll
                    for (int q2 = q + 1; q2 < KBG; ++q2) {
                        if (q2 < kb) {
                            const float u = __shfl_sync(full, pick_s(a, ps, q2), pl);
#pragma unroll
                            for (int s = 0; s < RWG; ++s) a[s][q2] = fmaf(-m[s], u, a[s][q2]);
                        }
                    }
                    if (lane == pl) {
#pragma unroll
                        for (int s = 0; s < RWG; ++s)
                            if (ps == s) umask[s] = 0u;
                    }
                    if (lane == q) {
                        myp = p;
                        mypv = pv;
                    }
                }
            }
            if (lane < kb) {   // lane q records step q
                pbk[lane] = myp;
                rowpos[myp] = c0 + lane;
                pivval[c0 + lane] = mypv;
            }
            const unsigned badq =
                __ballot_sync(full, lane < kb && (!(fabsf(mypv) >= kMinNormal) || !isfinite(mypv)));
            if (lane == 0) s_bad = badq != 0u;
        }
        __syncthreads();
        if (s_bad) {   // the same in every thread
            if (tid == 0) status[e] = RM_ESINGULAR;
            return;
        }
        // the block's steps on this thread's columns past the block (tiles
        // jlo..jhi-1; columns of tile jlo left of the block's end take the
        // update too, and are never read again)
        const int jlo = (c0 + kb) >> 4;
        if (kb == KBG) {
            int pk[KBG];
#pragma unroll
            for (int q = 0; q < KBG; q += 4) {
                const int4 v4 = *reinterpret_cast<const int4 *>(pbk + q);
                pk[q] = v4.x, pk[q + 1] = v4.y, pk[q + 2] = v4.z, pk[q + 3] = v4.w;
            }
            gj_block_from<TR, TC, TRP, KBG>(jlo, t, pk, mb + ty * TRP, rowb + tx * TC, ty);
        } else {
            for (int q = 0; q < kb; ++q)
                gj_step<TR, TC, TRP>(t, pbk[q], mb + (q * G16 + ty) * TRP, rowb + ((q & 1) * G16 + tx) * TC, ty,
                                     jlo, jhi);
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
    if (!t_sweep_dispatch<1, TR, TC>((no + 15) >> 4, Pm, no, lane, warp, tx, ty, xs, &s_bad)) {
        if (tid == 0) status[e] = RM_ESINGULAR;
        return;
    }

    // ---- Omega ----------------------------------------------------------------
    const double g = pw.g;
    // the level pair's |I||J| values of |T|^2, summed in FP32 like them
    auto pair_sum = [&](int I, int J) {
        float s = 0.0f;
        for (int ia = lstart[I]; ia < lstart[I + 1]; ++ia) {
            const int pa = open_pos[lev_chan_s[ia]];
            for (int ib = lstart[J]; ib < lstart[J + 1]; ++ib) s += Pm[pa * no + open_pos[lev_chan_s[ib]]];
        }
        return s;
    };
    if (lev_sm) {
        // open level pairs I <= J only: warp w takes the rows of the open-level
        // triangle w, w + 8, ..., its lanes the row's pairs
        const int nlo = s_nlo;
        for (int ip = warp; ip < nlo; ip += NT / 32) {
            const int I = olev[ip];
            for (int jp = ip + lane; jp < nlo; jp += 32) {
                const int J = olev[jp];
                atomicAdd(om + tri_idx(I, J, nl), g * (double)pair_sum(I, J));   // the only addition in this launch
            }
        }
    } else {
        for (int q = tid; q < npair; q += NT) {
            int I, J;
            tri_pair(q, nl, I, J);
            if (!(x - pw.lev_thr[I] > 0.0 && x - pw.lev_thr[J] > 0.0)) continue;
            atomicAdd(om + q, g * (double)pair_sum(I, J));   // the only addition to om[q] in this launch
        }
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
