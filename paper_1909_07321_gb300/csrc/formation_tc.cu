// Step (a) in mixed precision on tcgen05 tensor cores (Section "Overview",
// Eq. rmatrix, split as the spec precision plan asks: bulk products in
// low precision with FP32 accumulation, near-pole terms in FP64).
//
// For every energy e of a block and every channel pair p = (i <= j):
//   R_packed[e][p] = sum_k D[e][k] P[p][k],   D[e][k] = 1/(E_k - E_e),
//                                             P[p][k] = w_ik w_jk / (2a),
// one GEMM over all energies of the block (M = energies, N = pairs,
// K = poles). Both operands are split x = hi + lo with hi, lo in the MMA
// input type (bf16, or tf32 carried in fp32), and the product is taken as
// hi*hi + hi*lo + lo*hi with FP32 accumulation in tensor memory; lo*lo is
// dropped. Terms with |E_k - E_e| < delta are zeroed in D and added later in
// FP64 by the near-pole fix-up kernel.
//
// Kernel layout (one persistent CTA per SM, 192 threads):
//   warp 0, one lane : TMA producer (D tile 128 x BK, P tile BN x BK, hi and
//                      lo, 128-byte swizzle) into a ring of STAGES stages,
//   warp 1           : allocates 2 BN TMEM columns; one lane issues
//                      tcgen05.mma (M = 128, N = BN) into one of two
//                      accumulators,
//   warps 2..5       : epilogue; each reads its 32-lane quadrant of the
//                      accumulator with tcgen05.ld, converts to FP64 and
//                      stores R_packed rows.
// Every mbarrier wait is bounded (about 2 s by %globaltimer); a wait that
// gives up sets *err_flag, and every role then drains and exits, so the host
// sees an error instead of a hung GPU.
#include <cuda_bf16.h>
#include <stdint.h>

#include "tc_sm103.cuh"

namespace rmgb {
namespace {

constexpr int BM = 128;            // energies per tile (TMEM lanes)
constexpr int NTHREADS = 192;
constexpr int ROW_BYTES = TC_ROW_BYTES;
constexpr int A_TILE = BM * ROW_BYTES;   // 16 KB

// Tile variants (pairs per tile BN, ring depth STAGES): 256 x 2 stages (96
// KB per stage), 128 x 3 and 128 x 2 (64 KB per stage); chosen per partial
// wave by the context's autotuner, 256 x 2 otherwise.
template <int BN> struct PairTile {
    static constexpr int B_TILE = BN * ROW_BYTES;
    static constexpr int STAGE_BYTES = 2 * (A_TILE + B_TILE);   // hi + lo of both operands
    static constexpr int TMEM_COLS = 2 * BN;                    // two accumulators
};

template <int KIND, int BN, int STAGES>
__global__ void __launch_bounds__(NTHREADS, 1)
    form_r_tc_kernel(const __grid_constant__ CUtensorMap tmDh, const __grid_constant__ CUtensorMap tmDl,
                     const __grid_constant__ CUtensorMap tmPh, const __grid_constant__ CUtensorMap tmPl,
                     double *__restrict__ Rp, int ldR, int nE, int n_pairs, int n_kb, int n_ntiles,
                     int n_tiles, int *err_flag, unsigned long long probe_ns)
{
    if (probe_ns) {
        // bounded-wait self-test: nothing allocated or in flight yet
        __shared__ uint64_t probe;
        if (threadIdx.x == 0) wait_probe(&probe, probe_ns, err_flag);
        __syncthreads();
        return;
    }
    constexpr int B_TILE = PairTile<BN>::B_TILE;
    constexpr int STAGE_BYTES = PairTile<BN>::STAGE_BYTES;
    constexpr int TMEM_COLS = PairTile<BN>::TMEM_COLS;
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte alignment for the 128-byte swizzle atoms
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *accf = empty + STAGES;
    uint64_t *acce = accf + 2;
    uint64_t *done = acce + 2;
    uint32_t *tmem_slot = (uint32_t *)(done + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 4);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, TMEM_COLS);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer ----
            int stage = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < n_tiles; t += gridDim.x) {
                const int m0 = (t / n_ntiles) * BM, n0 = (t % n_ntiles) * BN;
                for (int kb = 0; kb < n_kb; ++kb) {
                    if (!mbar_wait(&empty[stage], ph ^ 1u, err_flag)) { ok = false; break; }
                    uint8_t *st = smem + stage * STAGE_BYTES;
                    mbar_expect_tx(&full[stage], STAGE_BYTES);
                    const int kx = kb * (ROW_BYTES / (KIND == TC_BF16X3 ? 2 : 4));
                    tma_load_2d(smem_u32(st), &tmDh, &full[stage], kx, m0);
                    tma_load_2d(smem_u32(st + A_TILE), &tmDl, &full[stage], kx, m0);
                    tma_load_2d(smem_u32(st + 2 * A_TILE), &tmPh, &full[stage], kx, n0);
                    tma_load_2d(smem_u32(st + 2 * A_TILE + B_TILE), &tmPl, &full[stage], kx, n0);
                    if (++stage == STAGES) { stage = 0; ph ^= 1u; }
                }
            }
            if (!ok) {
                // let copies already in flight land before the CTA exits
                spin_ns(2000000ull);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer ----
            const uint32_t id = idesc<KIND, BM, BN>();
            int stage = 0;
            uint32_t ph = 0;
            int acc = 0;
            uint32_t aph = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < n_tiles; t += gridDim.x) {
                if (!mbar_wait(&acce[acc], aph ^ 1u, err_flag)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(acc * BN);
                for (int kb = 0; kb < n_kb; ++kb) {
                    if (!mbar_wait(&full[stage], ph, err_flag)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t st = smem_u32(smem + stage * STAGE_BYTES);
                    const uint64_t ah = sdesc_sw128(st), al = sdesc_sw128(st + A_TILE);
                    const uint64_t bh = sdesc_sw128(st + 2 * A_TILE);
                    const uint64_t bl = sdesc_sw128(st + 2 * A_TILE + B_TILE);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t o = (uint64_t)(ks * 32) >> 4;   // 32 bytes of K per MMA
                        umma<KIND>(d_tmem, ah + o, bh + o, id, (kb | ks) != 0);
                        umma<KIND>(d_tmem, ah + o, bl + o, id, 1u);
                        umma<KIND>(d_tmem, al + o, bh + o, id, 1u);
                    }
                    umma_commit(&empty[stage]);
                    if (++stage == STAGES) { stage = 0; ph ^= 1u; }
                }
                if (!ok) break;
                umma_commit(&accf[acc]);
                if (++acc == 2) { acc = 0; aph ^= 1u; }
            }
            // all MMAs issued by this thread complete before TMEM is freed
            umma_commit(done);
            mbar_wait(done, 0, nullptr);
        }
    } else {
        // ---- epilogue: warps 2..5 -> TMEM lane quadrant warp % 4 ----
        const int quad = warp & 3;
        int acc = 0;
        uint32_t aph = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
            if (!mbar_wait(&accf[acc], aph, err_flag)) break;
            tc_fence_after();
            const int m0 = (t / n_ntiles) * BM, n0 = (t % n_ntiles) * BN;
            const int e = m0 + quad * 32 + lane;
            double *row = Rp + (size_t)e * ldR;
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + (uint32_t)(acc * BN + c0) + ((uint32_t)(quad * 32) << 16), r);
                if (e < nE) {
                    const int p0 = n0 + c0;
                    if (p0 + 32 <= n_pairs) {
#pragma unroll
                        for (int j = 0; j < 32; j += 2) {
                            double2 v = make_double2((double)__uint_as_float(r[j]),
                                                     (double)__uint_as_float(r[j + 1]));
                            *reinterpret_cast<double2 *>(row + p0 + j) = v;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (p0 + j < n_pairs) row[p0 + j] = (double)__uint_as_float(r[j]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[acc]);
            if (++acc == 2) { acc = 0; aph ^= 1u; }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        tmem_dealloc(tmem, TMEM_COLS);
}

// ---- operand preparation ---------------------------------------------------

__device__ __forceinline__ void split_store(double x, int kind, void *hi, void *lo, size_t idx)
{
    const float f = (float)x;
    if (kind == TC_BF16X3) {
        const __nv_bfloat16 h = __float2bfloat16_rn(f);
        const __nv_bfloat16 l = __float2bfloat16_rn(f - __bfloat162float(h));
        static_cast<__nv_bfloat16 *>(hi)[idx] = h;
        static_cast<__nv_bfloat16 *>(lo)[idx] = l;
    } else {
        uint32_t hb;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(f));
        const float h = __uint_as_float(hb);
        static_cast<float *>(hi)[idx] = h;
        static_cast<float *>(lo)[idx] = f - h;
    }
}

__global__ void split_p_kernel(PwDev pw, int kind, int Kpad, void *Ph, void *Pl)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int np = tri_count(pw.n);
    if (idx >= (long long)np * Kpad) return;
    const int p = (int)(idx / Kpad), k = (int)(idx - (long long)p * Kpad);
    // invert the row-wise pair index
    int i = 0, rem = p;
    while (rem >= pw.n - i) { rem -= pw.n - i; ++i; }
    const int j = i + rem;
    const double v = (k < pw.N) ? pw.W[(size_t)i * pw.N + k] * pw.W[(size_t)j * pw.N + k] * (0.5 / pw.a) : 0.0;
    split_store(v, kind, Ph, Pl, (size_t)idx);
}

// A double as hi + lo floats (hi = x rounded, lo = the rest rounded).
__device__ __forceinline__ float2 split_hl(double x)
{
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

// E_k - E from hi + lo pairs in FP32: (hi - hi) rounds once relative to the
// difference and (lo - lo) restores what the rounding of E_k and E dropped,
// so the result is within ~2^-23 relative of E_k - E whenever |E_k - E| >=
// delta >> |E| 2^-48. The near/far decision |E_k - E| < delta of the split
// and of the FP64 near-pole terms is taken on this value, identically.
__device__ __forceinline__ float pole_den(float2 ek, float2 e) { return (ek.x - e.x) + (ek.y - e.y); }

__global__ void split_e_kernel(const double *__restrict__ E, int nE, float2 *__restrict__ e_hl)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nE) e_hl[e] = split_hl(E[e]);
}

// D_k(E) = 1/(E_k - E) for |E_k - E| >= delta (else 0: those terms are
// added in FP64 by near_pole_fixup_kernel), split hi + lo, entirely in FP32
// (pole_den, correctly rounded reciprocal): no FP64 pipe work, so the split
// does not compete with the channel functions running beside it. Thread:
// two consecutive poles of one energy (Kpad is even); grid: (pole pairs,
// energies).
template <int KIND>
__global__ void split_d_kernel(PwDev pw, const float2 *__restrict__ e_hl, int nE, float delta_f, int Kpad,
                               void *Dh, void *Dl)
{
    const int k = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (k >= Kpad) return;
    float2 ek[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) ek[h] = k + h < pw.N ? pw.Ek_hl[k + h] : make_float2(0.0f, 0.0f);
    for (int e = blockIdx.y; e < nE; e += gridDim.y) {
        const float2 x = e_hl[e];
        float d[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            d[h] = 0.0f;
            if (k + h < pw.N) {
                const float den = pole_den(ek[h], x);
                if (fabsf(den) >= delta_f) d[h] = __frcp_rn(den);
            }
        }
        const size_t idx = (size_t)e * Kpad + k;
        if (KIND == TC_BF16X3) {
            const __nv_bfloat162 hi = __floats2bfloat162_rn(d[0], d[1]);
            const float2 hf = __bfloat1622float2(hi);
            const __nv_bfloat162 lo = __floats2bfloat162_rn(d[0] - hf.x, d[1] - hf.y);
            *reinterpret_cast<__nv_bfloat162 *>(static_cast<__nv_bfloat16 *>(Dh) + idx) = hi;
            *reinterpret_cast<__nv_bfloat162 *>(static_cast<__nv_bfloat16 *>(Dl) + idx) = lo;
        } else {
            uint32_t h0, h1;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h0) : "f"(d[0]));
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h1) : "f"(d[1]));
            const float2 hi = make_float2(__uint_as_float(h0), __uint_as_float(h1));
            *reinterpret_cast<float2 *>(static_cast<float *>(Dh) + idx) = hi;
            *reinterpret_cast<float2 *>(static_cast<float *>(Dl) + idx) = make_float2(d[0] - hi.x, d[1] - hi.y);
        }
    }
}

// Near-pole terms in FP64. One thread per energy finds the poles within
// delta of E (sorted E_k, binary search) and, if there are any, appends the
// energy and its pole range to a list; then one warp per listed energy adds
// every pair's FP64 terms (lanes over j). Each energy is listed once, so the
// result does not depend on the list order.
__global__ void near_pole_range_kernel(PwDev pw, const double *__restrict__ E, int nE, double delta,
                                       int *__restrict__ count, int *__restrict__ list, int2 *__restrict__ range)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nE) return;
    const double x = E[e];
    int lo = 0, hi = pw.N;
    while (lo < hi) {          // first k with E_k > x - 2 delta (a margin for the FP32 test)
        const int mid = (lo + hi) >> 1;
        if (pw.Ek[mid] <= x - 2.0 * delta) lo = mid + 1; else hi = mid;
    }
    int k1 = lo;
    while (k1 < pw.N && pw.Ek[k1] < x + 2.0 * delta) ++k1;
    // same near/far test as split_d_kernel
    const float2 xh = split_hl(x);
    const float df = (float)delta;
    bool any = false;
    for (int k = lo; k < k1; ++k) any |= fabsf(pole_den(pw.Ek_hl[k], xh)) < df;
    if (!any) return;
    const int slot = atomicAdd(count, 1);
    list[slot] = e;
    range[slot] = make_int2(lo, k1);
}

__global__ void near_pole_fixup_kernel(PwDev pw, const double *__restrict__ E, double delta,
                                       const int *__restrict__ count, const int *__restrict__ list,
                                       const int2 *__restrict__ range, double *__restrict__ Rp)
{
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int cnt = *count;
    const int n = pw.n;
    const double h = 0.5 / pw.a;
    for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < cnt; s += nw) {
        const int e = list[s];
        const int2 kr = range[s];
        const double x = E[e];
        const float2 xh = split_hl(x);
        const float df = (float)delta;
        double *Re = Rp + (size_t)e * tri_ld(n);
        for (int i = 0; i < n; ++i) {
            double *row = Re + tri_idx(i, i, n);
            for (int j = i + lane; j < n; j += 32) {
                double acc = 0.0;
                for (int k = kr.x; k < kr.y; ++k) {
                    if (fabsf(pole_den(pw.Ek_hl[k], xh)) < df)
                        acc += pw.W[(size_t)i * pw.N + k] * pw.W[(size_t)j * pw.N + k] / (pw.Ek[k] - x);
                }
                row[j - i] += h * acc;
            }
        }
    }
}

__global__ void unpack_r_kernel(int n, int nE, const double *__restrict__ Rp, double *__restrict__ R)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nE * n * n) return;
    const int e = (int)(idx / ((long long)n * n));
    const int ij = (int)(idx - (long long)e * n * n);
    const int i = ij / n, j = ij - (ij / n) * n;
    const int a = i < j ? i : j, b = i < j ? j : i;
    R[idx] = Rp[(size_t)e * tri_ld(n) + tri_idx(a, b, n)];
}

}  // namespace

int tc_kpad(int N, int kind)
{
    const int bk = ROW_BYTES / ((kind == TC_BF16X3) ? 2 : 4);
    return ((N + bk - 1) / bk) * bk;
}

cudaError_t launch_split_p(const PwDev &pw, int kind, int Kpad, void *P_hi, void *P_lo, cudaStream_t s)
{
    const long long total = (long long)tri_count(pw.n) * Kpad;
    split_p_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(pw, kind, Kpad, P_hi, P_lo);
    return cudaGetLastError();
}

cudaError_t launch_split_d(const PwDev &pw, const double *E, int nE, double delta, int kind, int Kpad,
                           void *D_hi, void *D_lo, float2 *e_hl, cudaStream_t s)
{
    if ((long long)nE * Kpad == 0) return cudaSuccess;
    if (!pw.Ek_hl) return cudaErrorInvalidValue;
    split_e_kernel<<<(unsigned)((nE + 255) / 256), 256, 0, s>>>(E, nE, e_hl);
    const dim3 grid((unsigned)((Kpad / 2 + 255) / 256), (unsigned)(nE < 65535 ? nE : 65535));
    if (kind == TC_BF16X3)
        split_d_kernel<TC_BF16X3><<<grid, 256, 0, s>>>(pw, e_hl, nE, (float)delta, Kpad, D_hi, D_lo);
    else
        split_d_kernel<TC_TF32X3><<<grid, 256, 0, s>>>(pw, e_hl, nE, (float)delta, Kpad, D_hi, D_lo);
    return cudaGetLastError();
}

namespace {

template <int KIND, int BN, int STAGES>
cudaError_t launch_pair_variant(const void *D_hi, const void *D_lo, const void *P_hi, const void *P_lo, int nE,
                                int n_pairs, int Kpad, double *Rp, int ldR, int *err_flag, cudaStream_t s,
                                unsigned long long probe_ns)
{
    CUtensorMap mDh, mDl, mPh, mPl;
    if (!make_map(&mDh, D_hi, KIND, Kpad, nE, BM) || !make_map(&mDl, D_lo, KIND, Kpad, nE, BM) ||
        !make_map(&mPh, P_hi, KIND, Kpad, n_pairs, BN) || !make_map(&mPl, P_lo, KIND, Kpad, n_pairs, BN))
        return cudaErrorInvalidValue;
    const int bk = ROW_BYTES / ((KIND == TC_BF16X3) ? 2 : 4);
    const int n_kb = Kpad / bk;
    const int n_mt = (nE + BM - 1) / BM, n_nt = (n_pairs + BN - 1) / BN;
    const int n_tiles = n_mt * n_nt;
    const int grid = n_tiles < num_sms() ? n_tiles : num_sms();
    const size_t smem = (size_t)STAGES * PairTile<BN>::STAGE_BYTES + 1024 + 256;
    cudaError_t e = cudaFuncSetAttribute(form_r_tc_kernel<KIND, BN, STAGES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    form_r_tc_kernel<KIND, BN, STAGES><<<grid, NTHREADS, smem, s>>>(mDh, mDl, mPh, mPl, Rp, ldR, nE, n_pairs,
                                                                    n_kb, n_nt, n_tiles, err_flag, probe_ns);
    return cudaGetLastError();
}

template <int KIND>
cudaError_t launch_pair(int variant, const void *D_hi, const void *D_lo, const void *P_hi, const void *P_lo, int nE,
                        int n_pairs, int Kpad, double *Rp, int ldR, int *err_flag, cudaStream_t s,
                        unsigned long long probe_ns)
{
    switch (variant) {
    case 1:
        return launch_pair_variant<KIND, 128, 3>(D_hi, D_lo, P_hi, P_lo, nE, n_pairs, Kpad, Rp, ldR, err_flag, s,
                                                 probe_ns);
    case 2:
        return launch_pair_variant<KIND, 128, 2>(D_hi, D_lo, P_hi, P_lo, nE, n_pairs, Kpad, Rp, ldR, err_flag, s,
                                                 probe_ns);
    default:
        return launch_pair_variant<KIND, 256, 2>(D_hi, D_lo, P_hi, P_lo, nE, n_pairs, Kpad, Rp, ldR, err_flag, s,
                                                 probe_ns);
    }
}

}  // namespace

int tc_pair_variants() { return 3; }

void tc_pair_variant_shape(int variant, int *tile_n, int *stages)
{
    *tile_n = variant == 0 ? 256 : 128;
    *stages = variant == 1 ? 3 : 2;
}

cudaError_t launch_form_r_tc(int kind, const void *D_hi, const void *D_lo, const void *P_hi,
                             const void *P_lo, int nE, int n_pairs, int Kpad, double *Rp, int ldR,
                             int *err_flag, cudaStream_t s, int variant, unsigned long long probe_ns)
{
    if (nE == 0) return cudaSuccess;
    if (variant < 0 || variant >= tc_pair_variants()) return cudaErrorInvalidValue;
    if (kind == TC_BF16X3)
        return launch_pair<TC_BF16X3>(variant, D_hi, D_lo, P_hi, P_lo, nE, n_pairs, Kpad, Rp, ldR, err_flag, s,
                                      probe_ns);
    return launch_pair<TC_TF32X3>(variant, D_hi, D_lo, P_hi, P_lo, nE, n_pairs, Kpad, Rp, ldR, err_flag, s,
                                  probe_ns);
}

size_t near_pole_ws_bytes(int nE) { return 16 + (size_t)nE * (sizeof(int) + sizeof(int2)); }

cudaError_t launch_near_pole_fixup(const PwDev &pw, const double *E, int nE, double delta, double *Rp, void *ws,
                                   cudaStream_t s)
{
    if (nE == 0) return cudaSuccess;
    int *count = static_cast<int *>(ws);
    int2 *range = reinterpret_cast<int2 *>(static_cast<char *>(ws) + 16);
    int *list = reinterpret_cast<int *>(range + nE);
    cudaError_t err = cudaMemsetAsync(count, 0, sizeof(int), s);
    if (err != cudaSuccess) return err;
    near_pole_range_kernel<<<(unsigned)((nE + 255) / 256), 256, 0, s>>>(pw, E, nE, delta, count, list, range);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const int warps = nE < 4 * 152 * 8 ? nE : 4 * 152 * 8;
    near_pole_fixup_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(pw, E, delta, count, list, range, Rp);
    return cudaGetLastError();
}

cudaError_t launch_unpack_r(int n, int nE, const double *Rp, double *R, cudaStream_t s)
{
    const long long total = (long long)nE * n * n;
    if (total == 0) return cudaSuccess;
    unpack_r_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(n, nE, Rp, R);
    return cudaGetLastError();
}

}  // namespace rmgb
