// Step (a), FP64: R_ij(E) = (1/2a) sum_k w_ik w_jk / (E_k - E)  (Section "Overview",
// Eq. rmatrix), the upper triangle of each energy's R in the packed layout
// (tri_idx, stride tri_ld(n)).
//
// This is the plain-FP64 baseline the mixed-precision path is measured
// against. Only the upper triangle is computed (tiles with tile_j >= tile_i)
// and stored, so every R is exactly symmetric. d_k = 1/(E_k - E) is formed
// once per (tile, k) in shared memory and folded into the j-operand.
#include "rm_internal.cuh"

namespace rmgb {
namespace {

// n < 32: one thread per (energy, i <= j), plain loop over poles.
__global__ void form_r_naive(PwDev pw, const double *__restrict__ E, int nE,
                             double *__restrict__ R)
{
    const int n = pw.n;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nE * n * n) return;
    const int e = (int)(idx / ((long long)n * n));
    const int ij = (int)(idx - (long long)e * n * n);
    const int i = ij / n, j = ij - (ij / n) * n;
    if (i > j) return;
    const double x = E[e];
    const double *wi = pw.W + (size_t)i * pw.N;
    const double *wj = pw.W + (size_t)j * pw.N;
    double acc = 0.0;
    for (int k = 0; k < pw.N; ++k) acc = fma(wi[k], wj[k] / (pw.Ek[k] - x), acc);
    acc *= 0.5 / pw.a;
    R[(size_t)e * tri_ld(n) + tri_idx(i, j, n)] = acc;
}

constexpr int TB = 64;   // output tile
constexpr int TK = 16;   // pole chunk
constexpr int TT = 4;    // outputs per thread per dimension

// n >= 32: CTA per (energy, 64x64 upper tile); 256 threads x 4x4 outputs.
// Off-diagonal tiles: thread (ty, tx) = (tid/16, tid%16) owns rows 4ty.., cols
// 4tx... Diagonal tiles: the 32x32 quadrant below the diagonal is not needed,
// so whole warps are assigned to the three upper quadrants (2 warps each) and
// warps 6-7 sit out; the FP64 pipe is not spent on discarded outputs.
__global__ void __launch_bounds__(256) form_r_tiled(PwDev pw, const double *__restrict__ E,
                                                    double *__restrict__ R)
{
    const int ti = blockIdx.y, tj = blockIdx.x;
    if (tj < ti) return;
    const int e = blockIdx.z;
    const int n = pw.n, N = pw.N;
    const int i0 = ti * TB, j0 = tj * TB;
    __shared__ double Wi[TK][TB + 1];
    __shared__ double Wj[TK][TB + 1];
    __shared__ double dk[TK];
    const int tid = threadIdx.x;
    int tx = tid & 15, ty = tid >> 4;
    bool active = true;
    if (ti == tj) {
        const int w = tid >> 5, l = tid & 31;
        const int quad = w >> 1;             // 0: (0,0), 1: (0,1), 2: (1,1), 3: idle
        const int sub = (w & 1) * 32 + l;    // 64 threads per 32x32 quadrant
        const int qy = (quad == 2) ? 1 : 0, qx = (quad == 0) ? 0 : 1;
        ty = qy * 8 + (sub >> 3);
        tx = qx * 8 + (sub & 7);
        active = quad < 3;
    }
    const double x = E[e];
    double acc[TT][TT];
#pragma unroll
    for (int a = 0; a < TT; ++a)
#pragma unroll
        for (int b = 0; b < TT; ++b) acc[a][b] = 0.0;

    for (int k0 = 0; k0 < N; k0 += TK) {
        if (tid < TK) {
            const int k = k0 + tid;
            dk[tid] = (k < N) ? 1.0 / (pw.Ek[k] - x) : 0.0;
        }
        __syncthreads();
        // 64 rows x 16 poles per operand: 4 elements per thread, k fastest
#pragma unroll
        for (int t = 0; t < (TB * TK) / 256; ++t) {
            const int q = tid + t * 256;
            const int r = q / TK, c = q - (q / TK) * TK;
            const int k = k0 + c;
            const int gi = i0 + r, gj = j0 + r;
            Wi[c][r] = (gi < n && k < N) ? pw.W[(size_t)gi * N + k] : 0.0;
            Wj[c][r] = (gj < n && k < N) ? pw.W[(size_t)gj * N + k] * dk[c] : 0.0;
        }
        __syncthreads();
        if (active) {
#pragma unroll
        for (int c = 0; c < TK; ++c) {
            double av[TT], bv[TT];
#pragma unroll
            for (int a = 0; a < TT; ++a) av[a] = Wi[c][ty * TT + a];
#pragma unroll
            for (int b = 0; b < TT; ++b) bv[b] = Wj[c][tx * TT + b];
#pragma unroll
            for (int a = 0; a < TT; ++a)
#pragma unroll
                for (int b = 0; b < TT; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        }
        __syncthreads();
    }
    if (!active) return;
    const double h = 0.5 / pw.a;
    double *Re = R + (size_t)e * tri_ld(n);
#pragma unroll
    for (int a = 0; a < TT; ++a) {
        const int i = i0 + ty * TT + a;
#pragma unroll
        for (int b = 0; b < TT; ++b) {
            const int j = j0 + tx * TT + b;
            if (i < n && j < n && i <= j) Re[tri_idx(i, j, n)] = acc[a][b] * h;
        }
    }
}

}  // namespace

cudaError_t launch_form_r_fp64(const PwDev &pw, const double *E, int nE, double *R,
                               cudaStream_t s)
{
    if (nE == 0) return cudaSuccess;
    if (pw.n < 32) {
        const long long total = (long long)nE * pw.n * pw.n;
        form_r_naive<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(pw, E, nE, R);
    } else {
        const int t = (pw.n + TB - 1) / TB;
        dim3 grid(t, t, nE);
        form_r_tiled<<<grid, 256, 0, s>>>(pw, E, R);
    }
    return cudaGetLastError();
}

}  // namespace rmgb
