// Step (a) in mixed precision for wide partial waves: Eq. rmatrix taken as
// one GEMM per energy,
//   R(E) = W diag(d(E)) W^T / (2a),   d_k(E) = 1/(E_k - E),
// on tcgen05 tensor cores. This is the per-energy form of the formation that
// the paper's Section "CUDA optimisations" offloads; the pair-operand form in
// formation_tc.cu is preferred while its w_i w_j operand fits in memory.
//
// Operands (K = poles, both K-major, 128-byte swizzle):
//   fixed  B[j][k] = w_jk, split hi/lo once per partial wave, loaded by TMA;
//   scaled A[i][k] = w_ik d_k(E), formed per energy on the fly by converter
//                    warps from an FP32 copy of W and d(E) in FP32, split
//                    hi/lo and written into the swizzled layout.
// Product hi*hi + hi*lo + lo*hi with FP32 accumulation in tensor memory.
// FP32 accumulation error grows with the number of accumulation steps, so K
// is cut into segments of 4096 poles; each segment's tile is written as an
// FP32 partial and a reduction kernel sums the segments in FP64 (fixed
// order, so R is deterministic), adds the near-pole terms |E_k - E| < delta
// in FP64 and scales by 1/2a.
//
// Work item = (K segment, pair of energies, tile 128 i x 256 j of the upper
// triangle). Persistent CTA per SM, 448 threads:
//   warp 0, one lane : TMA of the fixed tiles into a 2-stage ring,
//   warp 1           : allocates 512 TMEM columns (one 256-column
//                      accumulator per energy); one lane issues the MMAs,
//   warps 2..5       : epilogue, TMEM -> FP32 partial rows,
//   warps 6..13      : converters, scaled tiles into a 3-slot ring.
// Every mbarrier wait is bounded (about 2 s); a wait that gives up sets
// *err_flag and every role drains and exits.
#include <cuda_bf16.h>
#include <stdint.h>

#include "tc_sm103.cuh"

namespace rmgb {
namespace {

constexpr int PE_BM = 128;                 // rows i per tile (TMEM lanes)
constexpr int PE_BN = 256;                 // columns j per tile (TMEM columns)
constexpr int PE_G = 2;                    // energies per work item
constexpr int PE_BSTAGES = 2;
constexpr int PE_ASLOTS = 3;
constexpr int PE_A_TILE = PE_BM * TC_ROW_BYTES;   // 16 KB
constexpr int PE_A_SLOT = 2 * PE_A_TILE;          // hi + lo
constexpr int PE_B_TILE = PE_BN * TC_ROW_BYTES;   // 32 KB
constexpr int PE_B_STAGE = 2 * PE_B_TILE;         // hi + lo
constexpr int PE_SEG_K = 4096;             // poles per FP32 accumulation segment
constexpr int PE_NCONV = 256;              // converter threads
constexpr int PE_THREADS = 192 + PE_NCONV;
constexpr int PE_TMEM_COLS = PE_G * PE_BN;
constexpr int PE_SMEM = PE_BSTAGES * PE_B_STAGE + PE_ASLOTS * PE_A_SLOT + 1024 + 256;
constexpr int PE_MAX_JB = 32;              // n <= 8192

static_assert(PE_TMEM_COLS <= 512, "accumulators exceed tensor memory");
static_assert(PE_SMEM <= 232448, "shared memory over the per-CTA limit");

struct PeGeom {
    int n, Kpad, nE;
    int n_ib, n_jb, n_tiles;
    int n_chunks, seg_chunks, n_seg;
    int n_groups;
    long long n_items;
};

// Tiles of column block jb that hold some (i <= j): row blocks 0..count-1.
__host__ __device__ __forceinline__ int pe_col_tiles(int jb, int n_ib)
{
    const int c = ((jb + 1) * PE_BN - 1) / PE_BM + 1;
    return c < n_ib ? c : n_ib;
}

struct PeItem {
    int seg, e0, ng, t, ib, jb, c0, c1;
};

__device__ __forceinline__ PeItem pe_decode(const PeGeom &g, long long item)
{
    PeItem it;
    const long long per_seg = (long long)g.n_groups * g.n_tiles;
    it.seg = (int)(item / per_seg);
    const int rem = (int)(item - (long long)it.seg * per_seg);
    const int grp = rem / g.n_tiles;
    it.t = rem - grp * g.n_tiles;
    int t = it.t, jb = 0;
    for (int c = pe_col_tiles(0, g.n_ib); t >= c; c = pe_col_tiles(jb, g.n_ib)) {
        t -= c;
        ++jb;
    }
    it.ib = t;
    it.jb = jb;
    it.e0 = grp * PE_G;
    it.ng = min(PE_G, g.nE - it.e0);
    it.c0 = it.seg * g.seg_chunks;
    it.c1 = min(it.c0 + g.seg_chunks, g.n_chunks);
    return it;
}

// Lane 0 waits, the warp follows its verdict (keeps .sync.aligned
// instructions and __syncwarp convergent if a wait gives up).
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, int *err, int lane)
{
    int ok = 1;
    if (lane == 0) ok = mbar_wait(bar, parity, err) ? 1 : 0;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// x = w d split into the MMA input type, 16 bytes of hi and of lo.
template <int KIND> struct Split16;
template <> struct Split16<TC_BF16X3> {
    static constexpr int EPC = 8;   // elements per 16-byte chunk
    __device__ __forceinline__ static void run(const float *w, const float *d, uint4 &hi, uint4 &lo)
    {
        uint32_t h[4], l[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const float x0 = w[2 * m] * d[2 * m], x1 = w[2 * m + 1] * d[2 * m + 1];
            const __nv_bfloat162 hh = __floats2bfloat162_rn(x0, x1);
            const float2 hf = __bfloat1622float2(hh);
            const __nv_bfloat162 ll = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
            h[m] = *reinterpret_cast<const uint32_t *>(&hh);
            l[m] = *reinterpret_cast<const uint32_t *>(&ll);
        }
        hi = make_uint4(h[0], h[1], h[2], h[3]);
        lo = make_uint4(l[0], l[1], l[2], l[3]);
    }
};
template <> struct Split16<TC_TF32X3> {
    static constexpr int EPC = 4;
    __device__ __forceinline__ static void run(const float *w, const float *d, uint4 &hi, uint4 &lo)
    {
        uint32_t h[4], l[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const float x = w[m] * d[m];
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h[m]) : "f"(x));
            l[m] = __float_as_uint(x - __uint_as_float(h[m]));
        }
        hi = make_uint4(h[0], h[1], h[2], h[3]);
        lo = make_uint4(l[0], l[1], l[2], l[3]);
    }
};

template <int KIND>
__global__ void __launch_bounds__(PE_THREADS, 1)
    form_r_pe_kernel(const __grid_constant__ CUtensorMap tmWh, const __grid_constant__ CUtensorMap tmWl,
                     const float *__restrict__ W32, const float *__restrict__ D32,
                     float *__restrict__ part, const PeGeom g, int *err_flag, unsigned long long probe_ns)
{
    if (probe_ns) {
        // bounded-wait self-test: nothing allocated or in flight yet
        __shared__ uint64_t probe;
        if (threadIdx.x == 0) wait_probe(&probe, probe_ns, err_flag);
        __syncthreads();
        return;
    }
    constexpr int BK = TC_ROW_BYTES / (KIND == TC_BF16X3 ? 2 : 4);   // K per chunk
    constexpr int EPC = Split16<KIND>::EPC;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *bring = smem;
    uint8_t *aring = smem + PE_BSTAGES * PE_B_STAGE;
    uint64_t *bfull = (uint64_t *)(aring + PE_ASLOTS * PE_A_SLOT);
    uint64_t *bempty = bfull + PE_BSTAGES;
    uint64_t *afull = bempty + PE_BSTAGES;
    uint64_t *aempty = afull + PE_ASLOTS;
    uint64_t *accf = aempty + PE_ASLOTS;
    uint64_t *acce = accf + 1;
    uint64_t *done = acce + 1;
    uint32_t *tmem_slot = (uint32_t *)(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < PE_BSTAGES; ++s) {
            mbar_init(&bfull[s], 1);
            mbar_init(&bempty[s], 1);
        }
        for (int s = 0; s < PE_ASLOTS; ++s) {
            mbar_init(&afull[s], PE_NCONV / 32);
            mbar_init(&aempty[s], 1);
        }
        mbar_init(accf, 1);
        mbar_init(acce, 4);
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, PE_TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer: fixed tiles w_jk (hi, lo) ----
            int st = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (long long item = blockIdx.x; ok && item < g.n_items; item += gridDim.x) {
                const PeItem it = pe_decode(g, item);
                for (int c = it.c0; c < it.c1; ++c) {
                    if (!mbar_wait(&bempty[st], ph ^ 1u, err_flag)) { ok = false; break; }
                    uint8_t *b = bring + st * PE_B_STAGE;
                    mbar_expect_tx(&bfull[st], PE_B_STAGE);
                    tma_load_2d(smem_u32(b), &tmWh, &bfull[st], c * BK, it.jb * PE_BN);
                    tma_load_2d(smem_u32(b + PE_B_TILE), &tmWl, &bfull[st], c * BK, it.jb * PE_BN);
                    if (++st == PE_BSTAGES) { st = 0; ph ^= 1u; }
                }
            }
            if (!ok) spin_ns(2000000ull);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer ----
            const uint32_t id = idesc<KIND, PE_BM, PE_BN>();
            int bs = 0, as = 0;
            uint32_t bph = 0, aph = 0, eph = 0;
            bool ok = true;
            for (long long item = blockIdx.x; ok && item < g.n_items; item += gridDim.x) {
                const PeItem it = pe_decode(g, item);
                if (!mbar_wait(acce, eph ^ 1u, err_flag)) { ok = false; break; }
                tc_fence_after();
                for (int c = it.c0; ok && c < it.c1; ++c) {
                    if (!mbar_wait(&bfull[bs], bph, err_flag)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t b = smem_u32(bring + bs * PE_B_STAGE);
                    const uint64_t bh = sdesc_sw128(b), bl = sdesc_sw128(b + PE_B_TILE);
                    for (int j = 0; j < it.ng; ++j) {
                        if (!mbar_wait(&afull[as], aph, err_flag)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t a = smem_u32(aring + as * PE_A_SLOT);
                        const uint64_t ah = sdesc_sw128(a), al = sdesc_sw128(a + PE_A_TILE);
                        const uint32_t d = tmem + (uint32_t)(j * PE_BN);
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {
                            const uint64_t o = (uint64_t)(ks * 32) >> 4;   // 32 bytes of K per MMA
                            umma<KIND>(d, ah + o, bh + o, id, (c != it.c0 || ks != 0) ? 1u : 0u);
                            umma<KIND>(d, ah + o, bl + o, id, 1u);
                            umma<KIND>(d, al + o, bh + o, id, 1u);
                        }
                        umma_commit(&aempty[as]);
                        if (++as == PE_ASLOTS) { as = 0; aph ^= 1u; }
                    }
                    if (!ok) break;
                    umma_commit(&bempty[bs]);
                    if (++bs == PE_BSTAGES) { bs = 0; bph ^= 1u; }
                }
                if (!ok) break;
                umma_commit(accf);
                eph ^= 1u;
            }
            // all MMAs issued by this thread complete before TMEM is freed
            umma_commit(done);
            mbar_wait(done, 0, nullptr);
        }
    } else if (warp < 6) {
        // ---- epilogue: warps 2..5 -> TMEM lane quadrant warp % 4 ----
        const int quad = warp & 3;
        const int il = quad * 32 + lane;
        uint32_t fph = 0;
        for (long long item = blockIdx.x; item < g.n_items; item += gridDim.x) {
            const PeItem it = pe_decode(g, item);
            if (!warp_wait(accf, fph, err_flag, lane)) break;
            tc_fence_after();
            for (int j = 0; j < it.ng; ++j) {
                float *row = part + ((((size_t)it.seg * g.nE + it.e0 + j) * g.n_tiles + it.t) * PE_BM + il) *
                                        PE_BN;
                for (int c0 = 0; c0 < PE_BN; c0 += 32) {
                    uint32_t r[32];
                    tmem_ld32(tmem + (uint32_t)(j * PE_BN + c0) + ((uint32_t)(quad * 32) << 16), r);
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        *reinterpret_cast<uint4 *>(row + c0 + 4 * q) =
                            make_uint4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce);
            fph ^= 1u;
        }
    } else {
        // ---- converters: scaled tiles w_ik d_k(E) ----
        const int tid = threadIdx.x - 192;
        const int q = tid & 7, r0 = tid >> 3;   // 16-byte chunk q of rows r0 + 32 m
        int as = 0;
        uint32_t aph = 0;
        bool ok = true;
        for (long long item = blockIdx.x; ok && item < g.n_items; item += gridDim.x) {
            const PeItem it = pe_decode(g, item);
            for (int c = it.c0; ok && c < it.c1; ++c) {
                const int k0 = c * BK + q * EPC;
                float w[4][EPC];
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const int row = it.ib * PE_BM + r0 + 32 * m;
                    if (row < g.n) {
                        const float4 *src = reinterpret_cast<const float4 *>(W32 + (size_t)row * g.Kpad + k0);
#pragma unroll
                        for (int v = 0; v < EPC / 4; ++v) {
                            const float4 x = __ldg(src + v);
                            w[m][4 * v] = x.x;
                            w[m][4 * v + 1] = x.y;
                            w[m][4 * v + 2] = x.z;
                            w[m][4 * v + 3] = x.w;
                        }
                    } else {
#pragma unroll
                        for (int v = 0; v < EPC; ++v) w[m][v] = 0.f;
                    }
                }
                for (int j = 0; j < it.ng; ++j) {
                    if (!warp_wait(&aempty[as], aph ^ 1u, err_flag, lane)) { ok = false; break; }
                    float d[EPC];
                    const float4 *ds = reinterpret_cast<const float4 *>(D32 + (size_t)(it.e0 + j) * g.Kpad + k0);
#pragma unroll
                    for (int v = 0; v < EPC / 4; ++v) {
                        const float4 x = __ldg(ds + v);
                        d[4 * v] = x.x;
                        d[4 * v + 1] = x.y;
                        d[4 * v + 2] = x.z;
                        d[4 * v + 3] = x.w;
                    }
                    uint8_t *a = aring + as * PE_A_SLOT;
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        uint4 hi, lo;
                        Split16<KIND>::run(w[m], d, hi, lo);
                        const uint32_t off = sw128_offset(r0 + 32 * m, q);
                        *reinterpret_cast<uint4 *>(a + off) = hi;
                        *reinterpret_cast<uint4 *>(a + PE_A_TILE + off) = lo;
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&afull[as]);
                    if (++as == PE_ASLOTS) { as = 0; aph ^= 1u; }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, PE_TMEM_COLS);
}

// ---- operand preparation and reduction -------------------------------------

// Once per partial wave: W32 = (float)w, and w split hi/lo in the MMA type,
// all [n][Kpad] with zero padding past N.
__global__ void pe_prep_w_kernel(PwDev pw, int kind, int Kpad, float *W32, void *Wh, void *Wl)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)pw.n * Kpad) return;
    const int i = (int)(idx / Kpad), k = (int)(idx - (long long)i * Kpad);
    const float f = (k < pw.N) ? (float)pw.W[(size_t)i * pw.N + k] : 0.f;
    W32[idx] = f;
    if (kind == TC_BF16X3) {
        const __nv_bfloat16 h = __float2bfloat16_rn(f);
        static_cast<__nv_bfloat16 *>(Wh)[idx] = h;
        static_cast<__nv_bfloat16 *>(Wl)[idx] = __float2bfloat16_rn(f - __bfloat162float(h));
    } else {
        uint32_t hb;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(f));
        static_cast<float *>(Wh)[idx] = __uint_as_float(hb);
        static_cast<float *>(Wl)[idx] = f - __uint_as_float(hb);
    }
}

// Per energy block: d_k(E_e) in FP32, 0 where |E_k - E_e| < delta or k >= N;
// the thread of k = 0 also records the pole range [k0, k1) that can lie
// within delta of E_e (sorted E_k, binary search) for the reduction.
__global__ void pe_d32_kernel(PwDev pw, const double *__restrict__ E, int nE, double delta, int Kpad,
                              float *D32, int2 *np_range)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nE * Kpad) return;
    const int e = (int)(idx / Kpad), k = (int)(idx - (long long)e * Kpad);
    const double x = E[e];
    float d = 0.f;
    if (k < pw.N) {
        const double den = pw.Ek[k] - x;
        if (fabs(den) >= delta) d = (float)(1.0 / den);
    }
    D32[idx] = d;
    if (k == 0) {
        int lo = 0, hi = pw.N;
        while (lo < hi) {   // first k with E_k > x - delta
            const int mid = (lo + hi) >> 1;
            if (pw.Ek[mid] <= x - delta) lo = mid + 1; else hi = mid;
        }
        int k1 = lo;
        while (k1 < pw.N && pw.Ek[k1] < x + delta) ++k1;
        np_range[e] = make_int2(lo, k1);
    }
}

// R_ij for j >= i = (1/2a) [sum over segments of the FP32 partials (in FP64,
// segment order) + the FP64 terms of the poles within delta of E]. Block
// (energy e, band of PE_RROWS rows); threads along j, so both the partial
// rows and the packed output rows are read and written contiguously.
constexpr int PE_RROWS = 4;
__global__ void __launch_bounds__(256)
    pe_reduce_kernel(PwDev pw, const double *__restrict__ E, double delta, const int2 *__restrict__ np_range,
                     const float *__restrict__ part, const PeGeom g, double *__restrict__ Rp, int ldR)
{
    const int e = blockIdx.x;
    const int n = pw.n;
    __shared__ int s_off[PE_MAX_JB];
    if (threadIdx.x < g.n_jb) {
        int acc = 0;
        for (int jb = 0; jb < (int)threadIdx.x; ++jb) acc += pe_col_tiles(jb, g.n_ib);
        s_off[threadIdx.x] = acc;
    }
    __syncthreads();
    const double x = E[e];
    const int2 kr = np_range[e];
    const double h = 0.5 / pw.a;
    const size_t seg_stride = (size_t)g.nE * g.n_tiles * PE_BM * PE_BN;
    double *Re = Rp + (size_t)e * ldR;
    const int i0 = blockIdx.y * PE_RROWS;
    for (int i = i0; i < min(n, i0 + PE_RROWS); ++i) {
        const int ib = i / PE_BM, il = i - ib * PE_BM;
        double *out = Re + tri_idx(i, i, n);
        for (int j = i + threadIdx.x; j < n; j += blockDim.x) {
            const int jb = j / PE_BN;
            const float *p =
                part + (((size_t)e * g.n_tiles + s_off[jb] + ib) * PE_BM + il) * PE_BN + (j - jb * PE_BN);
            double s = 0.0;
            for (int sg = 0; sg < g.n_seg; ++sg) s += (double)__ldg(p + sg * seg_stride);
            for (int k = kr.x; k < kr.y; ++k) {
                const double den = pw.Ek[k] - x;   // same exclusion test as pe_d32_kernel
                if (fabs(den) < delta) s += pw.W[(size_t)i * pw.N + k] * pw.W[(size_t)j * pw.N + k] / den;
            }
            out[j - i] = h * s;
        }
    }
}

PeGeom pe_geom(int n, int Kpad, int kind, int nE)
{
    PeGeom g;
    const int bk = TC_ROW_BYTES / (kind == TC_BF16X3 ? 2 : 4);
    g.n = n;
    g.Kpad = Kpad;
    g.nE = nE;
    g.n_ib = (n + PE_BM - 1) / PE_BM;
    g.n_jb = (n + PE_BN - 1) / PE_BN;
    g.n_tiles = 0;
    for (int jb = 0; jb < g.n_jb; ++jb) g.n_tiles += pe_col_tiles(jb, g.n_ib);
    g.n_chunks = Kpad / bk;
    g.seg_chunks = PE_SEG_K / bk;
    g.n_seg = (g.n_chunks + g.seg_chunks - 1) / g.seg_chunks;
    g.n_groups = (nE + PE_G - 1) / PE_G;
    g.n_items = (long long)g.n_seg * g.n_groups * g.n_tiles;
    return g;
}

}  // namespace

int pe_max_n() { return PE_MAX_JB * PE_BN; }

size_t pe_bytes_per_energy(int n, int N, int kind)
{
    const int Kpad = tc_kpad(N, kind);
    const PeGeom g = pe_geom(n, Kpad, kind, 1);
    return (size_t)g.n_seg * g.n_tiles * PE_BM * PE_BN * sizeof(float) + (size_t)Kpad * sizeof(float) +
           sizeof(int2);
}

size_t pe_operand_bytes(int n, int N, int kind)
{
    const size_t Kpad = (size_t)tc_kpad(N, kind);
    const size_t es = (kind == TC_BF16X3) ? 2 : 4;
    return (size_t)n * Kpad * (sizeof(float) + 2 * es);
}

cudaError_t launch_pe_prep_w(const PwDev &pw, int kind, int Kpad, float *W32, void *Wh, void *Wl,
                             cudaStream_t s)
{
    const long long total = (long long)pw.n * Kpad;
    pe_prep_w_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(pw, kind, Kpad, W32, Wh, Wl);
    return cudaGetLastError();
}

cudaError_t launch_pe_d32(const PwDev &pw, const double *E, int nE, double delta, int Kpad, float *D32,
                          cudaStream_t s)
{
    const long long total = (long long)nE * Kpad;
    if (total == 0) return cudaSuccess;
    int2 *np_range = reinterpret_cast<int2 *>(D32 + (size_t)nE * Kpad);
    pe_d32_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(pw, E, nE, delta, Kpad, D32, np_range);
    return cudaGetLastError();
}

cudaError_t launch_form_r_pe(int kind, int n, int Kpad, const float *W32, const void *Wh, const void *Wl,
                             const float *D32, int nE, float *part, int *err_flag, cudaStream_t s,
                             unsigned long long probe_ns)
{
    if (nE == 0) return cudaSuccess;
    if (n > pe_max_n() || Kpad % 4 != 0) return cudaErrorInvalidValue;
    CUtensorMap mh, ml;
    if (!make_map(&mh, Wh, kind, Kpad, n, PE_BN) || !make_map(&ml, Wl, kind, Kpad, n, PE_BN))
        return cudaErrorInvalidValue;
    const PeGeom g = pe_geom(n, Kpad, kind, nE);
    const long long grid = g.n_items < num_sms() ? g.n_items : num_sms();
    cudaError_t e;
    if (kind == TC_BF16X3) {
        e = cudaFuncSetAttribute(form_r_pe_kernel<TC_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 PE_SMEM);
        if (e != cudaSuccess) return e;
        form_r_pe_kernel<TC_BF16X3><<<(unsigned)grid, PE_THREADS, PE_SMEM, s>>>(mh, ml, W32, D32, part, g,
                                                                                 err_flag, probe_ns);
    } else {
        e = cudaFuncSetAttribute(form_r_pe_kernel<TC_TF32X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 PE_SMEM);
        if (e != cudaSuccess) return e;
        form_r_pe_kernel<TC_TF32X3><<<(unsigned)grid, PE_THREADS, PE_SMEM, s>>>(mh, ml, W32, D32, part, g,
                                                                                 err_flag, probe_ns);
    }
    return cudaGetLastError();
}

cudaError_t launch_pe_reduce(const PwDev &pw, int kind, int Kpad, const double *E, int nE, double delta,
                             const float *D32, const float *part, double *Rp, int ldR, cudaStream_t s)
{
    if (nE == 0) return cudaSuccess;
    const PeGeom g = pe_geom(pw.n, Kpad, kind, nE);
    const int2 *np_range = reinterpret_cast<const int2 *>(D32 + (size_t)nE * Kpad);
    pe_reduce_kernel<<<dim3((unsigned)nE, (unsigned)((pw.n + PE_RROWS - 1) / PE_RROWS)), 256, 0, s>>>(
        pw, E, delta, np_range, part, g, Rp, ldR);
    return cudaGetLastError();
}

}  // namespace rmgb
