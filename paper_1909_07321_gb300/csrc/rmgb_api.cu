// C ABI of the R -> K -> Omega hot path (declared in include/rmgb.h).
//
// The context owns every device buffer: per partial wave the sorted poles,
// the surface amplitudes and the channel tables; per call a workspace sized
// by opts.mem_budget; and the Omega accumulator of the registered grid.
// A call to rm_solve_energies enqueues, per block of energies,
//   near-pole check -> channel functions -> R formation -> matching + T + Omega
// on the context stream, with no host synchronisation.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>
#include <utility>
#include <vector>

#include "rm_internal.cuh"

using namespace rmgb;

namespace {

constexpr int MAX_PW = 4096;
constexpr int MAX_L = 64;
constexpr int MAX_BLOCK_E = 32768;

// Bumped whenever any device buffer of the library is freed or moved: a
// captured CUDA graph (rm_solve_batch) holds raw pointers and is replayed
// only while the generation it was captured under is current.
std::atomic<unsigned long long> g_buf_gen{1};

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    void release()
    {
        if (p) {
            cudaFree(p);
            g_buf_gen.fetch_add(1);
        }
        p = nullptr;
        bytes = 0;
    }
    // grow-only; contents are not preserved
    cudaError_t reserve(size_t b)
    {
        if (b <= bytes) return cudaSuccess;
        release();
        cudaError_t e = cudaMalloc(&p, b);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        bytes = b;
        return cudaSuccess;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

struct PwHost {
    bool loaded = false, channels = false;
    int n = 0, N = 0, n_levels = 0;
    double a = 0, b = 0, z = 0, g = 0;
    DevBuf Ek, W, e_thr, l, level, lev_start, lev_chan, lev_thr;
    DevBuf Ek_hl;   // E_k as hi + lo floats
    // mixed-precision operand P = w_i w_j / 2a, split hi/lo (built on first use)
    DevBuf Ph, Pl;
    int p_kind = -1, p_kpad = 0;
    // per-energy formulation: W in FP32 and w split hi/lo (built on first use)
    DevBuf W32, Wh, Wl;
    int w_kind = -1;
    // formation chosen by the autotuner (rm_opts.autotune): formulation and
    // pair-kernel tile variant, and the measured ms per energy of every
    // candidate (-1: not applicable)
    bool tuned = false;
    int tune_form = 0, tune_var = 0;
    double tune_ms[4] = {-1.0, -1.0, -1.0, -1.0};
    std::vector<double> h_e_thr, h_Ek;   // host copies (thresholds, sorted poles)
    std::vector<int> h_l;
    // near-threshold interpolation tables (z > 0), built when the wave has
    // both its poles and its channels; use_deep: some near-threshold pairs
    // are not covered and go to the side stream
    DevBuf thr;
    bool use_deep = true;
    // open-side tables (z > 0): coefficients, failure flags, geometry
    DevBuf otab, otab_bad;
    double otab_dk = 0.0;
    int otab_nseg = 0;
    DevBuf ctab, ctab_nsub;
    double ctab_nu_lo = 0.0;
    int ctab_nseg = 0;
    // outer-region propagation (rm_set_multipoles): coefficients [lmax][n][n]
    // on the device, radius r1, Numerov steps; prop_lmax < 0: none
    DevBuf propA;
    int prop_lmax = -1, prop_steps = 0;
    double prop_r1 = 0.0;
    double a_match() const { return prop_lmax >= 0 ? prop_r1 : a; }
    size_t bytes() const
    {
        size_t b = 0;
        for (const DevBuf *d : {&Ek, &Ek_hl, &W, &e_thr, &l, &level, &lev_start, &lev_chan, &lev_thr, &Ph, &Pl,
                                &W32, &Wh, &Wl, &thr, &otab, &otab_bad, &ctab, &ctab_nsub, &propA})
            b += d->bytes;
        return b;
    }
    void release()
    {
        for (DevBuf *d : {&Ek, &Ek_hl, &W, &e_thr, &l, &level, &lev_start, &lev_chan, &lev_thr, &Ph, &Pl, &W32,
                          &Wh, &Wl, &thr, &otab, &otab_bad, &ctab, &ctab_nsub, &propA})
            d->release();
        prop_lmax = -1;
        use_deep = true;
        otab_nseg = 0;
        ctab_nseg = 0;
        loaded = channels = false;
        p_kind = -1;
        w_kind = -1;
        tuned = false;
    }
    PwDev dev() const
    {
        PwDev d;
        d.n = n;
        d.N = N;
        d.a = a;
        d.b = b;
        d.z = z;
        d.g = g;
        d.n_levels = n_levels;
        d.Ek = Ek.as<double>();
        d.W = W.as<double>();
        d.e_thr = e_thr.as<double>();
        d.l = l.as<int>();
        d.level = level.as<int>();
        d.lev_start = lev_start.as<int>();
        d.lev_chan = lev_chan.as<int>();
        d.lev_thr = lev_thr.as<double>();
        d.thr = thr.as<ThrNodes>();
        d.Ek_hl = Ek_hl.as<float2>();
        if (otab_nseg > 0) {
            d.otab = otab.as<double>();
            d.otab_bad = otab_bad.as<int>();
            d.otab_dk = otab_dk;
            d.otab_nseg = otab_nseg;
        }
        if (ctab_nseg > 0) {
            d.ctab = ctab.as<double>();
            d.ctab_nsub = ctab_nsub.as<unsigned char>();
            d.ctab_nu_lo = ctab_nu_lo;
            d.ctab_dnu = CTAB_DNU;
            d.ctab_nseg = ctab_nseg;
        }
        return d;
    }
    // As dev(), with a = the matching radius (r1 when the wave is propagated):
    // for the channel functions, their tables and the matching solve.
    PwDev dev_match() const
    {
        PwDev d = dev();
        d.a = a_match();
        return d;
    }
};

}  // namespace

namespace {

// One lane: a stream of work with its own workspace and Omega accumulator.
// The lanes of a context share its partial waves (poles, channels, tables and
// the low-precision operands), so work on several lanes overlaps on the
// device without loading a pole set twice. Lane 0 serves the calls without a
// lane argument.
struct Lane {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // grid and Omega accumulator
    int grid_nE = 0, grid_nlev = 0, grid_ntri = 0;
    std::vector<double> grid_host;
    DevBuf omega;
    // asynchronous read-out (rm_collision_strengths_async): a second
    // accumulator, a copy stream, and per physical buffer (cur: the active
    // one) the event after its last copy
    DevBuf omega_alt;
    cudaStream_t copy = nullptr;
    cudaEvent_t ev_solved = nullptr, ev_copied[2] = {nullptr, nullptr};
    bool copied[2] = {false, false};
    int omega_cur = 0;
    // workspace
    DevBuf wsE, wsCf, wsR, wsStatus, wsMq, wsDh, wsDl, wsErr, wsL, wsPart, wsDeep, wsNear, wsEhl;
    // coarse-mesh interpolation: node energies, statuses + orders, K_u, S_u, fine plan
    DevBuf wsQn, wsQst, wsQk, wsQs, wsQf, wsQc;
    // side stream for the deep channel pairs / the formation chain, with fork / join events
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_done = nullptr;   // after the lane's last enqueued work (rm_lane_query)
    size_t ws_bytes() const
    {
        size_t b = 0;
        for (const DevBuf *d : {&wsE, &wsCf, &wsR, &wsStatus, &wsMq, &wsDh, &wsDl, &wsErr, &wsL, &wsPart, &wsDeep,
                                &wsNear, &wsEhl, &wsQn, &wsQst, &wsQk, &wsQs, &wsQf, &wsQc})
            b += d->bytes;
        return b;
    }
    void release()
    {
        for (DevBuf *d : {&omega, &omega_alt, &wsE, &wsCf, &wsR, &wsStatus, &wsMq, &wsDh, &wsDl, &wsErr, &wsL,
                          &wsPart, &wsDeep, &wsNear, &wsEhl, &wsQn, &wsQst, &wsQk, &wsQs, &wsQf, &wsQc})
            d->release();
    }
};

constexpr int MAX_LANES = 64;

}  // namespace

namespace {

// One captured batch (rm_solve_batch): its arguments, the device pointers it
// was captured with, the buffer generation, the executable graph and the
// kernel launches it holds.
struct BatchGraph {
    std::vector<int> pws;
    int n_E = 0, mode = 0, lanes = 0;
    const double *E = nullptr;
    const void *omega = nullptr;
    unsigned long long gen = 0;
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;
};

}  // namespace

struct rm_ctx {
    rm_opts opts;
    std::vector<PwHost> pw;
    std::vector<Lane> lanes;
    std::vector<BatchGraph> graphs;
    DevBuf batchE;                 // host energies of rm_solve_batch, at a stable address
    cudaEvent_t ev_batch = nullptr;
    unsigned long long wait_probe_ns = 0;   // rm_set_wait_probe
    long long launches = 0;
    // per-phase event pairs (tracing)
    bool prof = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[RM_PH_COUNT];
    size_t ev_used[RM_PH_COUNT] = {};
    char err[512] = "no error";
};

namespace {

int fail(rm_ctx *c, int code, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? RM_ENOMEM : RM_ECUDA,   \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,      \
                        __LINE__);                                                      \
    } while (0)

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool finite_all(const double *x, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

int check_pw(rm_ctx *ctx, int pw, bool need_channels)
{
    if (!ctx) return RM_EINVAL;
    if (pw < 0 || pw >= MAX_PW) return fail(ctx, RM_EINVAL, "pw %d out of range [0, %d)", pw, MAX_PW);
    if ((int)ctx->pw.size() <= pw || !ctx->pw[pw].loaded)
        return fail(ctx, RM_ENOTLOADED, "partial wave %d has no poles loaded", pw);
    if (need_channels && !ctx->pw[pw].channels)
        return fail(ctx, RM_ENOTLOADED, "partial wave %d has no channels set", pw);
    return RM_SUCCESS;
}

template <class T> cudaError_t upload(DevBuf &d, const T *h, size_t count, cudaStream_t s)
{
    cudaError_t e = d.reserve(count * sizeof(T));
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(d.p, h, count * sizeof(T), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

// Records the start event of a traced launch of `phase` (no-op if tracing is off).
cudaError_t prof_begin(rm_ctx *ctx, int phase, cudaStream_t st = nullptr)
{
    if (!ctx->prof) return cudaSuccess;
    auto &v = ctx->ev[phase];
    size_t &u = ctx->ev_used[phase];
    if (u == v.size()) {
        cudaEvent_t a, b;
        cudaError_t e = cudaEventCreate(&a);
        if (e != cudaSuccess) return e;
        e = cudaEventCreate(&b);
        if (e != cudaSuccess) return e;
        v.push_back({a, b});
    }
    return cudaEventRecord(v[u].first, st ? st : ctx->lanes[0].stream);
}

cudaError_t prof_end(rm_ctx *ctx, int phase, cudaStream_t st = nullptr)
{
    if (!ctx->prof) return cudaSuccess;
    auto &v = ctx->ev[phase];
    size_t &u = ctx->ev_used[phase];
    cudaError_t e = cudaEventRecord(v[u].second, st ? st : ctx->lanes[0].stream);
    ++u;
    return e;
}

Opts make_opts(const rm_opts &o)
{
    Opts r;
    r.eps_thr = o.eps_thr;
    r.delta_pole = o.delta_pole;
    r.fnumin = o.fnumin;
    r.nu_margin = o.nu_margin;
    r.kappa_a_max = o.mqdt_kappa_a_max;
    return r;
}

}  // namespace

// ---------------------------------------------------------------------------

extern "C" void rm_default_opts(rm_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = RM_FP64;
    o->delta_pole = 1e-3;
    o->eps_thr = 1e-10;
    o->fnumin = 0.0;
    o->nu_margin = 0.1;
    o->device = 0;
    o->stream = nullptr;
    o->mem_budget = 0;
    o->mqdt_kappa_a_max = 5.0;
    o->solver = RM_SOLVER_AUTO;
    o->formulation = RM_FORM_AUTO;
    o->solve_precision = RM_FP64;
    o->channel_tables = -1;
    o->lanes = 1;
    o->autotune = 0;
}

extern "C" int rm_create(rm_ctx **out, const rm_opts *opts)
{
    if (!out) return RM_EINVAL;
    *out = nullptr;
    rm_opts o;
    if (opts) o = *opts; else rm_default_opts(&o);
    if (o.solver < RM_SOLVER_AUTO || o.solver > RM_SOLVER_LARGE) return RM_EINVAL;
    if (o.formulation < RM_FORM_AUTO || o.formulation > RM_FORM_ENERGY) return RM_EINVAL;
    if (o.solve_precision != RM_FP64 && o.solve_precision != RM_FP32) return RM_EINVAL;
    if (o.channel_tables < -1 || o.channel_tables > 1) return RM_EINVAL;
    if (o.channel_tables == -1) o.channel_tables = o.precision == RM_FP64 ? 0 : 1;
    if (!(o.eps_thr >= 0) || !(o.delta_pole >= 0) || !std::isfinite(o.fnumin) ||
        !(o.mqdt_kappa_a_max >= 0) ||
        !std::isfinite(o.nu_margin) ||
        (o.precision != RM_FP64 && o.precision != RM_FP32 && o.precision != RM_BF16X3))
        return RM_EINVAL;
    if (cudaSetDevice(o.device) != cudaSuccess) {
        cudaGetLastError();
        return RM_ECUDA;
    }
    if (o.mem_budget == 0) {
        size_t fr = 0, tot = 0;
        o.mem_budget = (size_t)32 << 30;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && fr / 2 < o.mem_budget) o.mem_budget = fr / 2;
        cudaGetLastError();
    }
    if (o.lanes == 0) o.lanes = 1;
    if (o.autotune != 0 && o.autotune != 1) return RM_EINVAL;
    if (o.pair_tile < 0 || o.pair_tile > tc_pair_variants()) return RM_EINVAL;
    if (o.lanes < 1 || o.lanes > MAX_LANES) return RM_EINVAL;
    rm_ctx *ctx = new (std::nothrow) rm_ctx();
    if (!ctx) return RM_ENOMEM;
    ctx->opts = o;
    ctx->lanes.resize(o.lanes);
    int lo_prio = 0, hi_prio = 0;
    cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    for (int i = 0; i < o.lanes; ++i) {
        Lane *ln = &ctx->lanes[i];
        bool ok = true;
        if (i == 0 && o.stream) {
            ln->stream = static_cast<cudaStream_t>(o.stream);
        } else {
            ok = cudaStreamCreateWithFlags(&ln->stream, cudaStreamNonBlocking) == cudaSuccess;
            ln->own_stream = ok;
        }
        ok = ok && cudaStreamCreateWithPriority(&ln->side, cudaStreamNonBlocking, hi_prio) == cudaSuccess &&
             cudaEventCreateWithFlags(&ln->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&ln->ev_join, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&ln->ev_done, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            rm_destroy(ctx);
            return RM_ECUDA;
        }
    }
    if (cudaEventCreateWithFlags(&ctx->ev_batch, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        rm_destroy(ctx);
        return RM_ECUDA;
    }
    *out = ctx;
    return RM_SUCCESS;
}

extern "C" void rm_destroy(rm_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->opts.device);
    for (Lane &l : ctx->lanes) {
        if (l.stream) cudaStreamSynchronize(l.stream);
        if (l.side) cudaStreamSynchronize(l.side);
        if (l.copy) cudaStreamSynchronize(l.copy);
    }
    for (auto &p : ctx->pw) p.release();
    for (BatchGraph &g : ctx->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    ctx->batchE.release();
    if (ctx->ev_batch) cudaEventDestroy(ctx->ev_batch);
    for (Lane &l : ctx->lanes) {
        Lane *ln = &l;
        if (ln->copy) cudaStreamDestroy(ln->copy);
        if (ln->ev_solved) cudaEventDestroy(ln->ev_solved);
        for (cudaEvent_t ev : ln->ev_copied)
            if (ev) cudaEventDestroy(ev);
        ln->release();
        if (ln->side) cudaStreamDestroy(ln->side);
        if (ln->ev_fork) cudaEventDestroy(ln->ev_fork);
        if (ln->ev_join) cudaEventDestroy(ln->ev_join);
        if (ln->ev_done) cudaEventDestroy(ln->ev_done);
        if (ln->own_stream) cudaStreamDestroy(ln->stream);
    }
    for (int p = 0; p < RM_PH_COUNT; ++p)
        for (auto &pr : ctx->ev[p]) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    delete ctx;
}

namespace {

// Near-threshold tables of wave P (its poles, a and channels are set): one
// launch, then the validity of every table is read back (once per wave).
int build_thr(rm_ctx *ctx, PwHost &P)
{
    Lane *ln = &ctx->lanes[0];
    P.thr.release();
    P.otab.release();
    P.otab_bad.release();
    P.otab_nseg = 0;
    P.ctab.release();
    P.ctab_nsub.release();
    P.ctab_nseg = 0;
    P.use_deep = true;
    if (!(P.z > 0.0) || P.n == 0 || !ctx->opts.channel_tables) return RM_SUCCESS;
    // open-side tables: segments of width OTAB_C / a in k up to OTAB_EPS_MAX Ry
    // (a: the matching radius)
    {
        const double dk = OTAB_C / P.a_match();
        const int nseg = (int)std::ceil(std::sqrt(OTAB_EPS_MAX) / dk);
        CK(P.otab.reserve(sizeof(double) * (size_t)P.n * nseg * 4 * OTAB_M));
        CK(P.otab_bad.reserve(sizeof(int) * (size_t)P.n));
        PwDev d = P.dev_match();
        d.otab_dk = dk;
        d.otab_nseg = nseg;
        CK(launch_open_table(d, P.otab.as<double>(), P.otab_bad.as<int>(), ln->stream));
        ++ctx->launches;
        P.otab_dk = dk;
        P.otab_nseg = nseg;
    }
    // closed-side tables: segments of width CTAB_DNU in nu from CTAB_EPS_MIN
    // Ry below threshold up to the channels' near-threshold zones
    {
        const int l_max = *std::max_element(P.h_l.begin(), P.h_l.end());
        const double nu_lo = P.z / std::sqrt(-CTAB_EPS_MIN);
        const double nu_hi = closed_table_nu_hi(P.z, P.a_match(), l_max);
        const int nseg = std::min(CTAB_MAX_SEG, (int)std::ceil((nu_hi - nu_lo) / CTAB_DNU));
        // at most 1 GiB of closed-side coefficients per wave (else the
        // continued fractions serve the closed pairs)
        const size_t bytes = sizeof(double) * (size_t)P.n * std::max(nseg, 0) * CTAB_SUB * 2 * OTAB_M;
        if (nseg > 0 && bytes <= ((size_t)1 << 30)) {
            CK(P.ctab.reserve(sizeof(double) * (size_t)P.n * nseg * CTAB_SUB * 2 * OTAB_M));
            CK(P.ctab_nsub.reserve((size_t)P.n * nseg));
            PwDev d = P.dev_match();
            d.ctab_nu_lo = nu_lo;
            d.ctab_dnu = CTAB_DNU;
            d.ctab_nseg = nseg;
            CK(launch_closed_table(d, P.ctab.as<double>(), P.ctab_nsub.as<unsigned char>(), ln->stream));
            ++ctx->launches;
            P.ctab_nu_lo = nu_lo;
            P.ctab_nseg = nseg;
        }
    }
    CK(P.thr.reserve(sizeof(ThrNodes) * (size_t)P.n));
    CK(launch_thr_nodes(P.dev_match(), P.thr.as<ThrNodes>(), ln->stream));
    ++ctx->launches;
    std::vector<ThrNodes> h(P.n);
    CK(cudaMemcpyAsync(h.data(), P.thr.p, sizeof(ThrNodes) * (size_t)P.n, cudaMemcpyDeviceToHost, ln->stream));
    CK(cudaStreamSynchronize(ln->stream));
    bool all = true;
    for (int i = 0; i < P.n; ++i) all = all && h[i].zone >= chanfn_deep_eps(P.z);
    P.use_deep = !all;
    return RM_SUCCESS;
}

}  // namespace

extern "C" int rm_load_poles(rm_ctx *ctx, int pw, int n_ch, int n_poles, const double *E_k,
                             const double *W, double a, double b)
{
    if (!ctx) return RM_EINVAL;
    if (pw < 0 || pw >= MAX_PW) return fail(ctx, RM_EINVAL, "pw %d out of range", pw);
    if (n_ch <= 0 || n_poles <= 0 || !E_k || !W)
        return fail(ctx, RM_EINVAL, "n_ch=%d n_poles=%d must be > 0 with non-NULL arrays", n_ch,
                    n_poles);
    if (!(a > 0) || !std::isfinite(a) || !std::isfinite(b))
        return fail(ctx, RM_EINVAL, "a=%g must be > 0 and b=%g finite", a, b);
    if (!finite_all(E_k, n_poles) || !finite_all(W, (size_t)n_ch * n_poles))
        return fail(ctx, RM_EINVAL, "non-finite pole energy or amplitude");
    CK(cudaSetDevice(ctx->opts.device));
    Lane *ln = &ctx->lanes[0];
    if ((int)ctx->pw.size() <= pw) ctx->pw.resize(pw + 1);
    PwHost &P = ctx->pw[pw];
    const bool same_n = P.loaded && P.n == n_ch;
    // sort poles (R does not depend on their order); permute W's columns alike
    std::vector<int> ord(n_poles);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return E_k[x] < E_k[y]; });
    std::vector<double> Es(n_poles), Ws((size_t)n_ch * n_poles);
    for (int k = 0; k < n_poles; ++k) Es[k] = E_k[ord[k]];
    for (int i = 0; i < n_ch; ++i)
        for (int k = 0; k < n_poles; ++k) Ws[(size_t)i * n_poles + k] = W[(size_t)i * n_poles + ord[k]];
    P.Ek.release();
    P.W.release();
    P.Ph.release();
    P.Pl.release();
    P.p_kind = -1;
    P.W32.release();
    P.Wh.release();
    P.Wl.release();
    P.w_kind = -1;
    CK(upload(P.Ek, Es.data(), Es.size(), ln->stream));
    {
        std::vector<float2> hl(n_poles);
        for (int k = 0; k < n_poles; ++k) {
            const float h = (float)Es[k];
            hl[k] = make_float2(h, (float)(Es[k] - (double)h));
        }
        P.Ek_hl.release();
        CK(upload(P.Ek_hl, hl.data(), hl.size(), ln->stream));
    }
    P.h_Ek = Es;
    CK(upload(P.W, Ws.data(), Ws.size(), ln->stream));
    P.n = n_ch;
    P.N = n_poles;
    P.a = a;
    P.b = b;
    P.loaded = true;
    if (!same_n) P.channels = false;
    // new poles (and a) clear any outer-region propagation
    P.propA.release();
    P.prop_lmax = -1;
    return P.channels ? build_thr(ctx, P) : RM_SUCCESS;
}

extern "C" int rm_set_channels(rm_ctx *ctx, int pw, const double *e_thr, const int *l, double z,
                               const int *level, int n_levels, double g_weight)
{
    int rc = check_pw(ctx, pw, false);
    if (rc) return rc;
    PwHost &P = ctx->pw[pw];
    const int n = P.n;
    if (!e_thr || !l || !level) return fail(ctx, RM_EINVAL, "NULL channel array");
    if (!(z >= 0) || !std::isfinite(z) || !std::isfinite(g_weight) || n_levels <= 0)
        return fail(ctx, RM_EINVAL, "z=%g must be >= 0, g finite, n_levels=%d > 0", z, n_levels);
    if (!finite_all(e_thr, n)) return fail(ctx, RM_EINVAL, "non-finite threshold");
    std::vector<double> lev_thr(n_levels, std::numeric_limits<double>::infinity());
    std::vector<int> cnt(n_levels, 0);
    for (int i = 0; i < n; ++i) {
        if (l[i] < 0 || l[i] > MAX_L) return fail(ctx, RM_EINVAL, "l[%d]=%d out of [0,%d]", i, l[i], MAX_L);
        if (level[i] < 0 || level[i] >= n_levels)
            return fail(ctx, RM_EINVAL, "level[%d]=%d out of [0,%d)", i, level[i], n_levels);
        double &t = lev_thr[level[i]];
        if (cnt[level[i]] && t != e_thr[i])
            return fail(ctx, RM_EINVAL, "channels of level %d have different thresholds", level[i]);
        t = e_thr[i];
        cnt[level[i]]++;
    }
    std::vector<int> start(n_levels + 1, 0), chan(n), fill(n_levels, 0);
    for (int I = 0; I < n_levels; ++I) start[I + 1] = start[I] + cnt[I];
    for (int i = 0; i < n; ++i) chan[start[level[i]] + fill[level[i]]++] = i;
    CK(cudaSetDevice(ctx->opts.device));
    Lane *ln = &ctx->lanes[0];
    CK(upload(P.e_thr, e_thr, n, ln->stream));
    CK(upload(P.l, l, n, ln->stream));
    CK(upload(P.level, level, n, ln->stream));
    CK(upload(P.lev_start, start.data(), start.size(), ln->stream));
    CK(upload(P.lev_chan, chan.data(), chan.size(), ln->stream));
    CK(upload(P.lev_thr, lev_thr.data(), lev_thr.size(), ln->stream));
    P.h_e_thr.assign(e_thr, e_thr + n);
    P.h_l.assign(l, l + n);
    P.z = z;
    P.g = g_weight;
    P.n_levels = n_levels;
    P.channels = true;
    return build_thr(ctx, P);
}

extern "C" int rm_set_multipoles(rm_ctx *ctx, int pw, int lambda_max, const double *A, double r1, int n_steps)
{
    int rc = check_pw(ctx, pw, false);
    if (rc) return rc;
    PwHost &P = ctx->pw[pw];
    const int n = P.n;
    if (lambda_max == 0) {
        P.prop_lmax = -1;
        P.prop_r1 = 0.0;
        P.prop_steps = 0;
        return P.channels ? build_thr(ctx, P) : RM_SUCCESS;
    }
    if (n > PROP_MAXN) return fail(ctx, RM_EUNSUPPORTED, "propagation takes at most %d channels (n_ch=%d)",
                                   PROP_MAXN, n);
    if (lambda_max < 0 || lambda_max > PROP_MAX_LAMBDA)
        return fail(ctx, RM_EINVAL, "lambda_max=%d out of [0,%d]", lambda_max, PROP_MAX_LAMBDA);
    if (!propagate_fits(n, lambda_max))
        return fail(ctx, RM_EUNSUPPORTED, "propagation of %d channels with lambda_max=%d needs more shared memory "
                    "than one CTA has", n, lambda_max);
    if (!A) return fail(ctx, RM_EINVAL, "NULL multipole coefficients");
    if (!std::isfinite(r1) || !(r1 >= P.a)) return fail(ctx, RM_EINVAL, "r1=%g must be >= a=%g", r1, P.a);
    if (n_steps < 2) return fail(ctx, RM_EINVAL, "n_steps=%d must be >= 2", n_steps);
    const size_t cnt = (size_t)lambda_max * n * n;
    if (!finite_all(A, cnt)) return fail(ctx, RM_EINVAL, "non-finite multipole coefficient");
    for (int lam = 0; lam < lambda_max; ++lam)
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < i; ++j)
                if (A[((size_t)lam * n + i) * n + j] != A[((size_t)lam * n + j) * n + i])
                    return fail(ctx, RM_EINVAL, "A[%d] not symmetric at (%d,%d)", lam + 1, i, j);
    CK(cudaSetDevice(ctx->opts.device));
    Lane *ln = &ctx->lanes[0];
    CK(upload(P.propA, A, cnt, ln->stream));
    P.prop_lmax = lambda_max;
    P.prop_r1 = r1;
    P.prop_steps = n_steps;
    return P.channels ? build_thr(ctx, P) : RM_SUCCESS;
}

namespace {

// Energies as a device pointer on the context stream (copies host input).
int device_energies(rm_ctx *ctx, Lane *ln, int n_E, const double *E, const double **dE)
{
    if (is_device_ptr(E)) {
        *dE = E;
        return RM_SUCCESS;
    }
    if (!finite_all(E, n_E)) return fail(ctx, RM_EINVAL, "non-finite energy");
    CK(ln->wsE.reserve((size_t)n_E * sizeof(double)));
    CK(cudaMemcpyAsync(ln->wsE.p, E, (size_t)n_E * sizeof(double), cudaMemcpyHostToDevice,
                       ln->stream));
    *dE = ln->wsE.as<double>();
    return RM_SUCCESS;
}

int tc_kind(int precision) { return precision == RM_BF16X3 ? TC_BF16X3 : TC_TF32X3; }
size_t tc_esize(int kind) { return kind == TC_BF16X3 ? 2 : 4; }

// Largest n_pairs x Kpad operand (hi + lo) the pair formulation keeps per
// partial wave; larger waves take the per-energy formulation.
constexpr size_t MAX_P_BYTES = (size_t)4 << 30;
// Automatic choice: the pair formulation up to this channel count (its tiles
// carry no padding in the pair dimension; the per-energy tiles of 128 x 256
// channels are mostly padding for small n).
constexpr int AUTO_PAIRS_MAX_N = 192;

size_t pair_operand_bytes(const PwHost &P, int kind)
{
    return (size_t)tri_count(P.n) * tc_kpad(P.N, kind) * tc_esize(kind) * 2;
}

// Formulation the context's precision and options give this partial wave.
int formulation(rm_ctx *ctx, const PwHost &P)
{
    if (ctx->opts.precision == RM_FP64) return 0;
    if (ctx->opts.formulation != RM_FORM_AUTO) return ctx->opts.formulation;
    if (P.tuned) return P.tune_form;
    const int kind = tc_kind(ctx->opts.precision);
    return (P.n <= AUTO_PAIRS_MAX_N && pair_operand_bytes(P, kind) <= MAX_P_BYTES) ? RM_FORM_PAIRS
                                                                                   : RM_FORM_ENERGY;
}

int check_precision(rm_ctx *ctx, const PwHost &P)
{
    const int f = formulation(ctx, P);
    if (f == 0) return RM_SUCCESS;
    const int kind = tc_kind(ctx->opts.precision);
    if (f == RM_FORM_PAIRS) {
        const size_t bytes = pair_operand_bytes(P, kind);
        if (bytes > MAX_P_BYTES)
            return fail(ctx, RM_EUNSUPPORTED,
                        "pair formulation of n_ch=%d, n_poles=%d needs %zu bytes of pair operands "
                        "(limit %zu); use RM_FORM_ENERGY",
                        P.n, P.N, bytes, MAX_P_BYTES);
    } else if (P.n > pe_max_n()) {
        return fail(ctx, RM_EUNSUPPORTED, "per-energy formulation takes at most %d channels (n_ch=%d)",
                    pe_max_n(), P.n);
    }
    return RM_SUCCESS;
}

bool use_large(rm_ctx *ctx, const PwHost &P)
{
    if (ctx->opts.solver == RM_SOLVER_LARGE) return true;
    if (ctx->opts.solver == RM_SOLVER_SMALL) return false;
    return P.n > solve_small_max_n();
}

int block_energies(rm_ctx *ctx, const PwHost &P)
{
    size_t per = (size_t)tri_ld(P.n) * sizeof(double) + (size_t)P.n * sizeof(ChanFn) + 64;
    if (use_large(ctx, P)) per += solve_large_bytes_per_energy(P.n);
    const int f = formulation(ctx, P);
    const int kind = tc_kind(ctx->opts.precision);
    if (f == RM_FORM_PAIRS) per += 2 * (size_t)tc_kpad(P.N, kind) * tc_esize(kind);
    if (f == RM_FORM_ENERGY) per += pe_bytes_per_energy(P.n, P.N, kind);
    size_t B = ctx->opts.mem_budget / per;
    if (B < 1) B = 1;
    if (B > MAX_BLOCK_E) B = MAX_BLOCK_E;
    return (int)B;
}

// Packed R of nE energies into R (stride tri_ld(n)), in the context's precision.
int form_r_block(rm_ctx *ctx, Lane *ln, PwHost &P, const double *E, int nE, double *R, cudaStream_t st = nullptr)
{
    if (!st) st = ln->stream;
    const PwDev d = P.dev();
    if (ctx->opts.precision == RM_FP64) {
        CK(prof_begin(ctx, RM_PH_FORM, st));
        CK(launch_form_r_fp64(d, E, nE, R, st));
        CK(prof_end(ctx, RM_PH_FORM, st));
        ctx->launches++;
        return RM_SUCCESS;
    }
    const int kind = tc_kind(ctx->opts.precision);
    const int Kpad = tc_kpad(P.N, kind);
    const size_t es = tc_esize(kind);
    if (!ln->wsErr.p) {
        CK(ln->wsErr.reserve(sizeof(int)));
        CK(cudaMemsetAsync(ln->wsErr.p, 0, sizeof(int), st));
    }
    if (formulation(ctx, P) == RM_FORM_ENERGY) {
        if (P.w_kind != kind) {
            const size_t nk = (size_t)P.n * Kpad;
            CK(P.W32.reserve(nk * sizeof(float)));
            CK(P.Wh.reserve(nk * es));
            CK(P.Wl.reserve(nk * es));
            CK(launch_pe_prep_w(d, kind, Kpad, P.W32.as<float>(), P.Wh.p, P.Wl.p, st));
            ctx->launches++;
            // complete before any lane uses the shared operand
            CK(cudaStreamSynchronize(st));
            P.w_kind = kind;
        }
        CK(ln->wsDh.reserve((size_t)nE * Kpad * sizeof(float) + (size_t)nE * sizeof(int2)));
        CK(ln->wsPart.reserve(pe_bytes_per_energy(P.n, P.N, kind) * (size_t)nE));
        CK(prof_begin(ctx, RM_PH_SPLIT, st));
        CK(launch_pe_d32(d, E, nE, ctx->opts.delta_pole, Kpad, ln->wsDh.as<float>(), st));
        CK(prof_end(ctx, RM_PH_SPLIT, st));
        CK(prof_begin(ctx, RM_PH_FORM, st));
        CK(launch_form_r_pe(kind, P.n, Kpad, P.W32.as<float>(), P.Wh.p, P.Wl.p, ln->wsDh.as<float>(), nE,
                            ln->wsPart.as<float>(), ln->wsErr.as<int>(), st, ctx->wait_probe_ns));
        CK(prof_end(ctx, RM_PH_FORM, st));
        CK(prof_begin(ctx, RM_PH_FIXUP, st));
        CK(launch_pe_reduce(d, kind, Kpad, E, nE, ctx->opts.delta_pole, ln->wsDh.as<float>(),
                            ln->wsPart.as<float>(), R,
                            tri_ld(P.n), st));
        CK(prof_end(ctx, RM_PH_FIXUP, st));
        ctx->launches += 3;
        return RM_SUCCESS;
    }
    if (P.p_kind != kind) {
        const size_t pb = (size_t)tri_count(P.n) * Kpad * es;
        CK(P.Ph.reserve(pb));
        CK(P.Pl.reserve(pb));
        CK(launch_split_p(d, kind, Kpad, P.Ph.p, P.Pl.p, st));
        ctx->launches++;
        // complete before any lane uses the shared operand
        CK(cudaStreamSynchronize(st));
        P.p_kind = kind;
        P.p_kpad = Kpad;
    }
    CK(ln->wsDh.reserve((size_t)nE * Kpad * es));
    CK(ln->wsDl.reserve((size_t)nE * Kpad * es));
    CK(prof_begin(ctx, RM_PH_SPLIT, st));
    CK(ln->wsEhl.reserve((size_t)nE * sizeof(float2)));
    CK(launch_split_d(d, E, nE, ctx->opts.delta_pole, kind, Kpad, ln->wsDh.p, ln->wsDl.p, ln->wsEhl.as<float2>(),
                      st));
    CK(prof_end(ctx, RM_PH_SPLIT, st));
    CK(prof_begin(ctx, RM_PH_FORM, st));
    CK(launch_form_r_tc(kind, ln->wsDh.p, ln->wsDl.p, P.Ph.p, P.Pl.p, nE, tri_count(P.n), Kpad, R,
                        tri_ld(P.n), ln->wsErr.as<int>(), st,
                        ctx->opts.pair_tile > 0 ? ctx->opts.pair_tile - 1 : (P.tuned ? P.tune_var : 0),
                        ctx->wait_probe_ns));
    CK(prof_end(ctx, RM_PH_FORM, st));
    CK(prof_begin(ctx, RM_PH_FIXUP, st));
    CK(ln->wsNear.reserve(near_pole_ws_bytes(nE)));
    CK(launch_near_pole_fixup(d, E, nE, ctx->opts.delta_pole, R, ln->wsNear.p, st));
    CK(prof_end(ctx, RM_PH_FIXUP, st));
    ctx->launches += 5;
    return RM_SUCCESS;
}

// After a synchronisation: a tensor-core kernel that gave up a bounded wait
// left its flag set.
int check_device_flag(rm_ctx *ctx, Lane *ln)
{
    if (!ln->wsErr.p) return RM_SUCCESS;
    int f = 0;
    CK(cudaMemcpy(&f, ln->wsErr.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (f) {
        CK(cudaMemset(ln->wsErr.p, 0, sizeof(int)));
        return fail(ctx, RM_ETIMEOUT, "a tensor-core formation kernel gave up a bounded wait");
    }
    return RM_SUCCESS;
}

// Everything a solve of n_E energies of P on lane ln reserves (the
// reservations of solve_on_lane, solve_blocks and form_r_block, in the same
// sizes), and the shared tensor-core operands, without launching the solve.
int reserve_solve(rm_ctx *ctx, Lane *ln, PwHost &P, int n_E)
{
    const bool large = use_large(ctx, P);
    const int ntri = P.n_levels * (P.n_levels + 1) / 2;
    const int B = std::min(n_E, block_energies(ctx, P));
    CK(ln->omega.reserve((size_t)n_E * ntri * sizeof(double)));
    CK(ln->wsE.reserve((size_t)n_E * sizeof(double)));
    CK(ln->wsStatus.reserve((size_t)n_E * sizeof(int)));
    CK(ln->wsCf.reserve((size_t)B * P.n * sizeof(ChanFn)));
    CK(ln->wsR.reserve((size_t)B * tri_ld(P.n) * sizeof(double)));
    if (large) CK(ln->wsL.reserve(solve_large_bytes_per_energy(P.n) * (size_t)B + 256));
    if (!large && P.use_deep) CK(ln->wsDeep.reserve(chanfn_deep_ws_bytes(B)));
    if (ctx->opts.precision == RM_FP64) return RM_SUCCESS;
    const int kind = tc_kind(ctx->opts.precision);
    const int Kpad = tc_kpad(P.N, kind);
    const size_t es = tc_esize(kind);
    if (!ln->wsErr.p) {
        CK(ln->wsErr.reserve(sizeof(int)));
        CK(cudaMemsetAsync(ln->wsErr.p, 0, sizeof(int), ln->stream));
    }
    const PwDev d = P.dev();
    if (formulation(ctx, P) == RM_FORM_ENERGY) {
        if (P.w_kind != kind) {
            const size_t nk = (size_t)P.n * Kpad;
            CK(P.W32.reserve(nk * sizeof(float)));
            CK(P.Wh.reserve(nk * es));
            CK(P.Wl.reserve(nk * es));
            CK(launch_pe_prep_w(d, kind, Kpad, P.W32.as<float>(), P.Wh.p, P.Wl.p, ln->stream));
            ctx->launches++;
            P.w_kind = kind;
        }
        CK(ln->wsDh.reserve((size_t)B * Kpad * sizeof(float) + (size_t)B * sizeof(int2)));
        CK(ln->wsPart.reserve(pe_bytes_per_energy(P.n, P.N, kind) * (size_t)B));
    } else {
        if (P.p_kind != kind) {
            const size_t pb = (size_t)tri_count(P.n) * Kpad * es;
            CK(P.Ph.reserve(pb));
            CK(P.Pl.reserve(pb));
            CK(launch_split_p(d, kind, Kpad, P.Ph.p, P.Pl.p, ln->stream));
            ctx->launches++;
            P.p_kind = kind;
            P.p_kpad = Kpad;
        }
        CK(ln->wsDh.reserve((size_t)B * Kpad * es));
        CK(ln->wsDl.reserve((size_t)B * Kpad * es));
        CK(ln->wsEhl.reserve((size_t)B * sizeof(float2)));
        CK(ln->wsNear.reserve(near_pole_ws_bytes(B)));
    }
    CK(cudaStreamSynchronize(ln->stream));
    return RM_SUCCESS;
}

// Process-wide autotuner choices: (operand type, channels, padded poles,
// energy-block bucket) -> (formulation, pair tile variant).
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tune;

// Candidate index of a (formulation, variant): pair variants 0..2, per-energy 3.
int tune_slot(int form, int var) { return form == RM_FORM_PAIRS ? var : 3; }

// Chooses the formation of wave P by timing every applicable candidate on the
// first min(n_E, 2048) energies dE (CUDA events on the lane's stream, one
// warm-up and two timed formations each), or takes the process-wide choice
// for its shape. Operands of the candidates not chosen are freed.
int tune_wave(rm_ctx *ctx, Lane *ln, PwHost &P, const double *dE, int n_E)
{
    const int kind = tc_kind(ctx->opts.precision);
    const int Kpad = tc_kpad(P.N, kind);
    const int nb = std::min(n_E, 2048);
    int bucket = 1;
    while (bucket < nb) bucket <<= 1;
    const auto key = std::make_tuple(kind, P.n, Kpad, bucket);
    std::vector<std::pair<int, int>> cand;
    if (pair_operand_bytes(P, kind) <= MAX_P_BYTES)
        for (int v = 0; v < tc_pair_variants(); ++v) cand.push_back({RM_FORM_PAIRS, v});
    if (P.n <= pe_max_n()) cand.push_back({RM_FORM_ENERGY, 0});
    if (cand.empty()) return RM_SUCCESS;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            P.tuned = true;
            P.tune_form = it->second.first;
            P.tune_var = it->second.second;
            return RM_SUCCESS;
        }
    }
    const bool prof = ctx->prof;
    ctx->prof = false;
    CK(ln->wsR.reserve((size_t)nb * tri_ld(P.n) * sizeof(double)));
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    int best = -1;
    double best_ms = 0.0;
    int rc = RM_SUCCESS;
    for (int c = 0; c < (int)cand.size() && rc == RM_SUCCESS; ++c) {
        P.tuned = true;
        P.tune_form = cand[c].first;
        P.tune_var = cand[c].second;
        rc = form_r_block(ctx, ln, P, dE, nb, ln->wsR.as<double>());
        if (rc) break;
        cudaEventRecord(a, ln->stream);
        for (int r = 0; r < 2 && rc == RM_SUCCESS; ++r) rc = form_r_block(ctx, ln, P, dE, nb, ln->wsR.as<double>());
        cudaEventRecord(b, ln->stream);
        if (cudaEventSynchronize(b) != cudaSuccess) rc = fail(ctx, RM_ECUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        const double per = ms / (2.0 * nb);
        P.tune_ms[tune_slot(cand[c].first, cand[c].second)] = per;
        if (best < 0 || per < best_ms) {
            best = c;
            best_ms = per;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->prof = prof;
    if (rc) return rc;
    P.tune_form = cand[best].first;
    P.tune_var = cand[best].second;
    if (P.tune_form != RM_FORM_PAIRS) {
        P.Ph.release();
        P.Pl.release();
        P.p_kind = -1;
    } else {
        P.W32.release();
        P.Wh.release();
        P.Wl.release();
        P.w_kind = -1;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = {P.tune_form, P.tune_var};
    return RM_SUCCESS;
}

}  // namespace

namespace {

// Registers the energy grid of the Omega accumulator (first call) or checks
// that this call uses the registered one.
int register_grid(rm_ctx *ctx, Lane *ln, const PwHost &P, int n_E, const double *E, bool dev_in)
{
    const int ntri = P.n_levels * (P.n_levels + 1) / 2;
    if (ln->grid_nE == 0) {
        CK(ln->omega.reserve((size_t)n_E * ntri * sizeof(double)));
        CK(cudaMemsetAsync(ln->omega.p, 0, (size_t)n_E * ntri * sizeof(double), ln->stream));
        ln->grid_nE = n_E;
        ln->grid_nlev = P.n_levels;
        ln->grid_ntri = ntri;
        ln->grid_host.clear();
        if (!dev_in) ln->grid_host.assign(E, E + n_E);
    } else {
        if (n_E != ln->grid_nE || P.n_levels != ln->grid_nlev)
            return fail(ctx, RM_EGRID, "grid (%d energies, %d levels) differs from registered (%d, %d)",
                        n_E, P.n_levels, ln->grid_nE, ln->grid_nlev);
        if (!dev_in && !ln->grid_host.empty() &&
            memcmp(E, ln->grid_host.data(), (size_t)n_E * sizeof(double)) != 0)
            return fail(ctx, RM_EGRID, "energies differ from the registered grid");
    }
    return RM_SUCCESS;
}

// Steps (b)-(d) for n_E device energies dE, block by block; dstatus must be
// zeroed. omega: Omega rows of these energies (nullptr: no accumulation).
// ku_out / ku_np (shared-memory solver, MQDT mode): K_u instead of K, T, Omega.
int solve_blocks(rm_ctx *ctx, Lane *ln, PwHost &P, const double *dE, int n_E, int mode, double *K_out, int *n_open_out,
                 int *dstatus, double *omega, double *ku_out = nullptr, int *ku_np = nullptr)
{
    const bool large = use_large(ctx, P);
    const int ntri = P.n_levels * (P.n_levels + 1) / 2;
    const int B = std::min(n_E, block_energies(ctx, P));
    CK(ln->wsCf.reserve((size_t)B * P.n * sizeof(ChanFn)));
    CK(ln->wsR.reserve((size_t)B * tri_ld(P.n) * sizeof(double)));
    if (large) CK(ln->wsL.reserve(solve_large_bytes_per_energy(P.n) * (size_t)B + 256));
    const PwDev d = P.dev_match();
    const Opts o = make_opts(ctx->opts);
    for (int e0 = 0; e0 < n_E; e0 += B) {
        const int nb = std::min(B, n_E - e0);
        const double *Eb = dE + e0;
        int *sb = dstatus + e0;
        CK(prof_begin(ctx, RM_PH_NEARPOLE, ln->stream));
        CK(launch_nearpole(d, Eb, nb, sb, ln->stream));
        CK(prof_end(ctx, RM_PH_NEARPOLE, ln->stream));
        // Deep (near-threshold) channel pairs go to the side stream, and the
        // energies holding them are solved after it joins (shared-memory
        // solver only).
        const bool split = !large && P.use_deep;
        int *deep = nullptr;
        if (split) {
            CK(ln->wsDeep.reserve(chanfn_deep_ws_bytes(B)));
            deep = ln->wsDeep.as<int>();
            CK(launch_chanfn_deep_mark(d, Eb, nb, o, deep, ln->stream));
            CK(cudaEventRecord(ln->ev_fork, ln->stream));
            CK(cudaStreamWaitEvent(ln->side, ln->ev_fork, 0));
            CK(launch_chanfn_deep(d, Eb, nb, o, mode == RM_MQDT, ln->wsCf.as<ChanFn>(), sb, deep, ln->side));
            CK(cudaEventRecord(ln->ev_join, ln->side));
            ctx->launches += 2;
        }
        // With no deep pairs to wait for, the formation of R (tensor pipe,
        // the longer chain: split, GEMM, near-pole terms) runs on the
        // high-priority second stream and step (b) (FP64 pipe) beside it on
        // the context's stream, filling what the formation leaves of the
        // SMs; the solve joins both.
        const bool beside = !P.use_deep;
        if (beside) {
            CK(cudaEventRecord(ln->ev_fork, ln->stream));
            CK(cudaStreamWaitEvent(ln->side, ln->ev_fork, 0));
            int rc = form_r_block(ctx, ln, P, Eb, nb, ln->wsR.as<double>(), ln->side);
            if (rc) return rc;
            CK(cudaEventRecord(ln->ev_join, ln->side));
        }
        CK(prof_begin(ctx, RM_PH_CHANFN, ln->stream));
        CK(launch_chanfn(d, Eb, nb, o, mode == RM_MQDT, ln->wsCf.as<ChanFn>(), sb, deep, ln->stream));
        CK(prof_end(ctx, RM_PH_CHANFN, ln->stream));
        ctx->launches += 2;
        if (beside) {
            CK(cudaStreamWaitEvent(ln->stream, ln->ev_join, 0));
        } else {
            int rc = form_r_block(ctx, ln, P, Eb, nb, ln->wsR.as<double>());
            if (rc) return rc;
        }
        if (P.prop_lmax >= 0) {
            // R(a) -> R(r1) once every status of the block is final (the
            // deep pairs' too), so a singular propagation never masks an
            // earlier error
            if (split) CK(cudaStreamWaitEvent(ln->stream, ln->ev_join, 0));
            CK(prof_begin(ctx, RM_PH_PROPAGATE, ln->stream));
            CK(launch_propagate(P.dev(), Eb, nb, P.propA.as<double>(), P.prop_lmax, P.prop_r1, P.prop_steps,
                                ln->wsR.as<double>(), sb, ln->stream));
            CK(prof_end(ctx, RM_PH_PROPAGATE, ln->stream));
            ++ctx->launches;
        }
        CK(prof_begin(ctx, RM_PH_SOLVE, ln->stream));
        double *Kb = K_out ? K_out + (size_t)e0 * P.n * P.n : nullptr;
        int *nob = n_open_out ? n_open_out + e0 : nullptr;
        double *omb = omega ? omega + (size_t)e0 * ntri : nullptr;
        if (large) {
            int L = 0;
            const int f32 = ctx->opts.solve_precision == RM_FP32 && !ku_out && solve_large_f32_supported(P.n);
            CK(launch_solve_large(d, Eb, nb, ln->wsCf.as<ChanFn>(), ln->wsR.as<double>(), sb, Kb, nob,
                                  omb, ntri, ln->wsL.p, &L, ln->stream, f32));
            ctx->launches += L;
        } else {
            const int f32 = mode == RM_DIRECT && ctx->opts.solve_precision == RM_FP32 && !ku_out;
            double *kub = ku_out ? ku_out + (size_t)e0 * P.n * P.n : nullptr;
            int *kunb = ku_np ? ku_np + e0 : nullptr;
            CK(launch_solve_small(d, Eb, nb, ln->wsCf.as<ChanFn>(), ln->wsR.as<double>(), sb, Kb, nob,
                                  omb, ntri, mode == RM_MQDT, f32, deep, 0, ln->stream, kub, kunb));
            ++ctx->launches;
            if (split) {
                CK(cudaStreamWaitEvent(ln->stream, ln->ev_join, 0));
                CK(launch_solve_small(d, Eb, nb, ln->wsCf.as<ChanFn>(), ln->wsR.as<double>(), sb, Kb, nob,
                                      omb, ntri, mode == RM_MQDT, f32, deep, 1, ln->stream, kub, kunb));
                ++ctx->launches;
            }
        }
        CK(prof_end(ctx, RM_PH_SOLVE, ln->stream));
    }
    return RM_SUCCESS;
}

}  // namespace

namespace {

int lane_of(rm_ctx *ctx, int lane, Lane **ln)
{
    if (!ctx) return RM_EINVAL;
    if (lane < 0 || lane >= (int)ctx->lanes.size())
        return fail(ctx, RM_EINVAL, "lane %d out of range [0, %d)", lane, (int)ctx->lanes.size());
    *ln = &ctx->lanes[lane];
    return RM_SUCCESS;
}

int solve_on_lane(rm_ctx *ctx, int lane, int pw, int n_E, const double *E, int mode, double *K_out,
                  int *n_open_out, int *status_out)
{
    Lane *ln = nullptr;
    int rc = lane_of(ctx, lane, &ln);
    if (rc) return rc;
    rc = check_pw(ctx, pw, true);
    if (rc) return rc;
    if (n_E <= 0 || !E) return fail(ctx, RM_EINVAL, "n_E=%d must be > 0 with non-NULL E", n_E);
    if (mode != RM_DIRECT && mode != RM_MQDT) return fail(ctx, RM_EINVAL, "mode %d", mode);
    PwHost &P = ctx->pw[pw];
    const bool large = use_large(ctx, P);
    if (!large && P.n > solve_small_max_n())
        return fail(ctx, RM_EUNSUPPORTED, "n_ch=%d above the shared-memory solver limit %d", P.n,
                    solve_small_max_n());
    rc = check_precision(ctx, P);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->opts.device));
    const bool dev_in = is_device_ptr(E);
    rc = register_grid(ctx, ln, P, n_E, E, dev_in);
    if (rc) return rc;
    const double *dE;
    rc = device_energies(ctx, ln, n_E, E, &dE);
    if (rc) return rc;
    if (ctx->opts.autotune && ctx->opts.precision != RM_FP64 && ctx->opts.formulation == RM_FORM_AUTO && !P.tuned) {
        rc = tune_wave(ctx, ln, P, dE, n_E);
        if (rc) return rc;
    }
    int *dstatus = status_out;
    if (!dstatus) {
        CK(ln->wsStatus.reserve((size_t)n_E * sizeof(int)));
        dstatus = ln->wsStatus.as<int>();
    }
    CK(cudaMemsetAsync(dstatus, 0, (size_t)n_E * sizeof(int), ln->stream));
    rc = solve_blocks(ctx, ln, P, dE, n_E, mode, K_out, n_open_out, dstatus, ln->omega.as<double>());
    if (rc) return rc;
    CK(cudaEventRecord(ln->ev_done, ln->stream));
    return RM_SUCCESS;
}

}  // namespace

extern "C" int rm_solve_energies(rm_ctx *ctx, int pw, int n_E, const double *E, int mode,
                                 double *K_out, int *n_open_out, int *status_out)
{
    return solve_on_lane(ctx, 0, pw, n_E, E, mode, K_out, n_open_out, status_out);
}

extern "C" int rm_lane_solve_energies(rm_ctx *ctx, int lane, int pw, int n_E, const double *E, int mode,
                                      double *K_out, int *n_open_out, int *status_out)
{
    return solve_on_lane(ctx, lane, pw, n_E, E, mode, K_out, n_open_out, status_out);
}

extern "C" int rm_solve_energies_qdt(rm_ctx *ctx, int pw, int n_E, const double *E, int ieq, double qetest,
                                     int iqdt, int *n_open_out, int *status_out)
{
    int rc = check_pw(ctx, pw, true);
    if (rc) return rc;
    if (n_E <= 0 || !E) return fail(ctx, RM_EINVAL, "n_E=%d must be > 0 with non-NULL E", n_E);
    if (is_device_ptr(E)) return fail(ctx, RM_EINVAL, "E must be a host array (the mesh is planned on the host)");
    if (iqdt != 1 && iqdt != 2) return fail(ctx, RM_EINVAL, "iqdt %d (1: S matrices, 2: K matrices)", iqdt);
    if (ieq == 0) return fail(ctx, RM_EINVAL, "ieq = 0");
    if (!std::isfinite(qetest)) return fail(ctx, RM_EINVAL, "qetest not finite");
    PwHost &P = ctx->pw[pw];
    Lane *ln = &ctx->lanes[0];
    if (P.n > solve_small_max_n() || use_large(ctx, P))
        return fail(ctx, RM_EUNSUPPORTED, "coarse-mesh interpolation takes at most %d channels (n_ch=%d)",
                    solve_small_max_n(), P.n);
    rc = check_precision(ctx, P);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->opts.device));
    QdtChannels ch;
    ch.n = P.n;
    ch.N = P.N;
    ch.e_thr = P.h_e_thr.data();
    ch.l = P.h_l.data();
    ch.E_k = P.h_Ek.data();
    ch.z = P.z;
    ch.a = P.a_match();
    ch.eps_thr = ctx->opts.eps_thr;
    ch.nu_margin = ctx->opts.nu_margin;
    ch.fnumin = ctx->opts.fnumin;
    ch.kappa_a_max = ctx->opts.mqdt_kappa_a_max;
    for (int m = 1; m < n_E; ++m)
        if (!(E[m] > E[m - 1])) return fail(ctx, RM_EINVAL, "energies must be strictly ascending");
    rc = register_grid(ctx, ln, P, n_E, E, false);
    if (rc) return rc;
    const double *dE;
    rc = device_energies(ctx, ln, n_E, E, &dE);
    if (rc) return rc;
    // channel classes of every fine energy on the device, then the plan
    std::vector<signed char> hcls((size_t)n_E * P.n);
    CK(ln->wsQc.reserve(hcls.size()));
    CK(launch_qdt_classes(P.dev_match(), dE, n_E, make_opts(ctx->opts), ln->wsQc.as<signed char>(), ln->stream));
    ctx->launches++;
    CK(cudaMemcpyAsync(hcls.data(), ln->wsQc.p, hcls.size(), cudaMemcpyDeviceToHost, ln->stream));
    CK(cudaStreamSynchronize(ln->stream));
    QdtPlan pl;
    if (qdt_plan(ch, E, n_E, hcls.data(), ieq, qetest, pl) != RM_SUCCESS)
        return fail(ctx, RM_EINVAL, "energies must be strictly ascending");
    // coarse nodes: K_u (and S_u) through the ordinary pipeline
    const int nn = (int)pl.node_x.size();
    const size_t n2 = (size_t)P.n * P.n;
    std::vector<int> hst(nn), hnp(nn);
    if (nn > 0) {
        CK(ln->wsQn.reserve((size_t)nn * sizeof(double)));
        CK(ln->wsQst.reserve((size_t)nn * 2 * sizeof(int)));
        CK(ln->wsQk.reserve((size_t)nn * n2 * sizeof(double)));
        CK(cudaMemcpyAsync(ln->wsQn.p, pl.node_x.data(), (size_t)nn * sizeof(double), cudaMemcpyHostToDevice,
                           ln->stream));
        int *nst = ln->wsQst.as<int>(), *nnp = nst + nn;
        CK(cudaMemsetAsync(nst, 0, (size_t)nn * 2 * sizeof(int), ln->stream));
        rc = solve_blocks(ctx, ln, P, ln->wsQn.as<double>(), nn, RM_MQDT, nullptr, nullptr, nst, nullptr,
                          ln->wsQk.as<double>(), nnp);
        if (rc) return rc;
        if (iqdt == 1) {
            CK(ln->wsQs.reserve((size_t)nn * n2 * sizeof(double2)));
            CK(launch_qdt_s_from_k(P.n, nn, ln->wsQk.as<double>(), nnp, nst, ln->wsQs.as<double2>(),
                                   ln->stream));
            ctx->launches++;
        }
        CK(cudaMemcpyAsync(hst.data(), nst, (size_t)nn * sizeof(int), cudaMemcpyDeviceToHost, ln->stream));
        CK(cudaMemcpyAsync(hnp.data(), nnp, (size_t)nn * sizeof(int), cudaMemcpyDeviceToHost, ln->stream));
        CK(cudaStreamSynchronize(ln->stream));
    }
    std::vector<int> ok(nn);
    for (int k = 0; k < nn; ++k) {
        int np = 0;
        for (signed char c : pl.cls[pl.node_seg[k]]) np += (c != QDT_DECAY);
        ok[k] = hst[k] == RM_OK && hnp[k] == np;
    }
    std::vector<QdtFine> fine;
    qdt_weights(pl, ok, n_E, fine);
    CK(ln->wsQf.reserve((size_t)n_E * sizeof(QdtFine)));
    CK(cudaMemcpyAsync(ln->wsQf.p, fine.data(), (size_t)n_E * sizeof(QdtFine), cudaMemcpyHostToDevice,
                       ln->stream));
    int *dstatus = status_out;
    if (!dstatus) {
        CK(ln->wsStatus.reserve((size_t)n_E * sizeof(int)));
        dstatus = ln->wsStatus.as<int>();
    }
    CK(cudaMemsetAsync(dstatus, 0, (size_t)n_E * sizeof(int), ln->stream));
    const int ntri = P.n_levels * (P.n_levels + 1) / 2;
    CK(launch_qdt_fine(iqdt, P.dev_match(), dE, n_E, make_opts(ctx->opts), ln->wsQf.as<QdtFine>(),
                       ln->wsQk.as<double>(), ln->wsQs.as<double2>(), ln->wsQst.as<int>(), dstatus,
                       n_open_out, ln->omega.as<double>(), ntri, ln->stream));
    ctx->launches++;
    return RM_SUCCESS;
}

namespace {

int collision_strengths_lane(rm_ctx *ctx, Lane *ln, double *omega_out, int reset)
{
    CK(cudaSetDevice(ctx->opts.device));
    if (ln->grid_nE == 0) {
        if (reset) return RM_SUCCESS;
        return fail(ctx, RM_EINVAL, "no energy grid registered yet");
    }
    const size_t bytes = (size_t)ln->grid_nE * ln->grid_ntri * sizeof(double);
    if (omega_out)
        CK(cudaMemcpyAsync(omega_out, ln->omega.p, bytes, cudaMemcpyDeviceToHost, ln->stream));
    CK(cudaStreamSynchronize(ln->stream));
    int rc = check_device_flag(ctx, ln);
    if (rc) return rc;
    if (reset) {
        ln->grid_nE = ln->grid_nlev = ln->grid_ntri = 0;
        ln->grid_host.clear();
    }
    return RM_SUCCESS;
}

}  // namespace

extern "C" int rm_collision_strengths(rm_ctx *ctx, double *omega_out, int reset)
{
    if (!ctx) return RM_EINVAL;
    return collision_strengths_lane(ctx, &ctx->lanes[0], omega_out, reset);
}

extern "C" int rm_lane_collision_strengths(rm_ctx *ctx, int lane, double *omega_out, int reset)
{
    Lane *ln = nullptr;
    int rc = lane_of(ctx, lane, &ln);
    if (rc) return rc;
    return collision_strengths_lane(ctx, ln, omega_out, reset);
}

extern "C" int rm_lane_query(rm_ctx *ctx, int lane)
{
    Lane *ln = nullptr;
    int rc = lane_of(ctx, lane, &ln);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->opts.device));
    const cudaError_t e = cudaEventQuery(ln->ev_done);
    if (e == cudaSuccess) return 1;
    if (e == cudaErrorNotReady) {
        cudaGetLastError();
        return 0;
    }
    CK(e);
    return 0;
}

extern "C" int rm_lane_sync(rm_ctx *ctx, int lane)
{
    Lane *ln = nullptr;
    int rc = lane_of(ctx, lane, &ln);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->opts.device));
    CK(cudaStreamSynchronize(ln->stream));
    return check_device_flag(ctx, ln);
}

extern "C" void *rm_lane_stream(rm_ctx *ctx, int lane)
{
    if (!ctx || lane < 0 || lane >= (int)ctx->lanes.size()) return nullptr;
    return ctx->lanes[lane].stream;
}

extern "C" int rm_collision_strengths_async(rm_ctx *ctx, double *omega_out, int reset)
{
    if (!ctx) return RM_EINVAL;
    Lane *ln = &ctx->lanes[0];
    if (!omega_out) return fail(ctx, RM_EINVAL, "omega_out is NULL");
    if (ln->grid_nE == 0) return fail(ctx, RM_EINVAL, "no energy grid registered yet");
    CK(cudaSetDevice(ctx->opts.device));
    if (!ln->copy) {
        CK(cudaStreamCreateWithFlags(&ln->copy, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&ln->ev_solved, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ln->ev_copied[0], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ln->ev_copied[1], cudaEventDisableTiming));
    }
    const size_t bytes = (size_t)ln->grid_nE * ln->grid_ntri * sizeof(double);
    const int cur = ln->omega_cur;
    CK(cudaEventRecord(ln->ev_solved, ln->stream));
    CK(cudaStreamWaitEvent(ln->copy, ln->ev_solved, 0));
    CK(cudaMemcpyAsync(omega_out, ln->omega.p, bytes, cudaMemcpyDeviceToHost, ln->copy));
    CK(cudaEventRecord(ln->ev_copied[cur], ln->copy));
    ln->copied[cur] = true;
    if (reset) {
        // later solves accumulate into the other buffer once its own last
        // copy is done; this one drains on the copy stream meanwhile
        std::swap(ln->omega, ln->omega_alt);
        ln->omega_cur = cur ^ 1;
        if (ln->copied[cur ^ 1]) CK(cudaStreamWaitEvent(ln->stream, ln->ev_copied[cur ^ 1], 0));
        ln->grid_nE = ln->grid_nlev = ln->grid_ntri = 0;
        ln->grid_host.clear();
    } else {
        // the accumulator keeps growing: nothing may touch it before the copy
        CK(cudaStreamWaitEvent(ln->stream, ln->ev_copied[cur], 0));
    }
    return RM_SUCCESS;
}

extern "C" int rm_reset_omega(rm_ctx *ctx)
{
    if (!ctx) return RM_EINVAL;
    Lane *ln = &ctx->lanes[0];
    if (ln->grid_nE == 0) return fail(ctx, RM_EINVAL, "no energy grid registered yet");
    CK(cudaSetDevice(ctx->opts.device));
    CK(cudaMemsetAsync(ln->omega.p, 0, (size_t)ln->grid_nE * ln->grid_ntri * sizeof(double),
                       ln->stream));
    return RM_SUCCESS;
}

extern "C" int rm_profile_enable(rm_ctx *ctx, int enable)
{
    if (!ctx) return RM_EINVAL;
    for (Lane &l : ctx->lanes) CK(cudaStreamSynchronize(l.stream));
    ctx->prof = enable != 0;
    for (int p = 0; p < RM_PH_COUNT; ++p) ctx->ev_used[p] = 0;
    return RM_SUCCESS;
}

extern "C" int rm_profile_get(rm_ctx *ctx, int phase, int *launches, double *ms)
{
    if (!ctx || phase < 0 || phase >= RM_PH_COUNT) return RM_EINVAL;
    for (Lane &l : ctx->lanes) CK(cudaStreamSynchronize(l.stream));
    double tot = 0.0;
    for (size_t i = 0; i < ctx->ev_used[phase]; ++i) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, ctx->ev[phase][i].first, ctx->ev[phase][i].second));
        tot += t;
    }
    if (launches) *launches = (int)ctx->ev_used[phase];
    if (ms) *ms = tot;
    return RM_SUCCESS;
}

extern "C" int rm_grid_shape(rm_ctx *ctx, int *n_E, int *n_tri)
{
    if (!ctx) return RM_EINVAL;
    const Lane *ln = &ctx->lanes[0];
    if (n_E) *n_E = ln->grid_nE;
    if (n_tri) *n_tri = ln->grid_ntri;
    return RM_SUCCESS;
}

extern "C" int rm_channel_functions(rm_ctx *ctx, int pw, int n_E, const double *E, double *out,
                                    int *status)
{
    int rc = check_pw(ctx, pw, true);
    if (rc) return rc;
    if (n_E <= 0 || !E || !out) return fail(ctx, RM_EINVAL, "bad arguments");
    if (!is_device_ptr(E) || !is_device_ptr(out) || (status && !is_device_ptr(status)))
        return fail(ctx, RM_EINVAL, "E, out and status must be device pointers");
    CK(cudaSetDevice(ctx->opts.device));
    Lane *ln = &ctx->lanes[0];
    const PwHost &P = ctx->pw[pw];
    CK(ln->wsCf.reserve((size_t)n_E * P.n * sizeof(ChanFn)));
    int *st = status;
    if (!st) {
        CK(ln->wsStatus.reserve((size_t)n_E * sizeof(int)));
        st = ln->wsStatus.as<int>();
    }
    CK(cudaMemsetAsync(st, 0, (size_t)n_E * sizeof(int), ln->stream));
    const PwDev d = P.dev_match();
    CK(launch_chanfn(d, E, n_E, make_opts(ctx->opts), 0, ln->wsCf.as<ChanFn>(), st, nullptr, ln->stream));
    CK(launch_chanfn_export(d, E, n_E, ln->wsCf.as<ChanFn>(), out, ln->stream));
    ctx->launches += 2;
    return RM_SUCCESS;
}

extern "C" int rm_channel_work(rm_ctx *ctx, int pw, int n_E, const double *E, int *work)
{
    int rc = check_pw(ctx, pw, true);
    if (rc) return rc;
    if (n_E <= 0 || !E || !work) return fail(ctx, RM_EINVAL, "bad arguments");
    if (!is_device_ptr(E) || !is_device_ptr(work))
        return fail(ctx, RM_EINVAL, "E and work must be device pointers");
    CK(cudaSetDevice(ctx->opts.device));
    Lane *ln = &ctx->lanes[0];
    const PwDev d = ctx->pw[pw].dev_match();
    CK(launch_chanfn_work(d, E, n_E, make_opts(ctx->opts), reinterpret_cast<int4 *>(work), ln->stream));
    ctx->launches++;
    return RM_SUCCESS;
}

extern "C" int rm_form_r(rm_ctx *ctx, int pw, int n_E, const double *E, double *R_out)
{
    int rc = check_pw(ctx, pw, false);
    if (rc) return rc;
    if (n_E <= 0 || !E || !R_out) return fail(ctx, RM_EINVAL, "bad arguments");
    if (!is_device_ptr(E) || !is_device_ptr(R_out))
        return fail(ctx, RM_EINVAL, "E and R_out must be device pointers");
    CK(cudaSetDevice(ctx->opts.device));
    Lane *ln = &ctx->lanes[0];
    PwHost &P = ctx->pw[pw];
    rc = check_precision(ctx, P);
    if (rc) return rc;
    const int B = std::min(n_E, block_energies(ctx, P));
    CK(ln->wsR.reserve((size_t)B * tri_ld(P.n) * sizeof(double)));
    for (int e0 = 0; e0 < n_E; e0 += B) {
        const int nb = std::min(B, n_E - e0);
        rc = form_r_block(ctx, ln, P, E + e0, nb, ln->wsR.as<double>());
        if (rc) return rc;
        CK(launch_unpack_r(P.n, nb, ln->wsR.as<double>(), R_out + (size_t)e0 * P.n * P.n,
                           ln->stream));
        ctx->launches++;
    }
    return RM_SUCCESS;
}

extern "C" int rm_lane_reserve(rm_ctx *ctx, int lane, int pw, int n_E, size_t *bytes)
{
    Lane *ln = nullptr;
    int rc = lane_of(ctx, lane, &ln);
    if (rc) return rc;
    rc = check_pw(ctx, pw, true);
    if (rc) return rc;
    if (n_E <= 0) return fail(ctx, RM_EINVAL, "n_E=%d must be > 0", n_E);
    PwHost &P = ctx->pw[pw];
    if (!use_large(ctx, P) && P.n > solve_small_max_n())
        return fail(ctx, RM_EUNSUPPORTED, "n_ch=%d above the shared-memory solver limit %d", P.n,
                    solve_small_max_n());
    rc = check_precision(ctx, P);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->opts.device));
    rc = reserve_solve(ctx, ln, P, n_E);
    if (rc) return rc;
    if (bytes) *bytes = ln->ws_bytes() + ln->omega.bytes + ln->omega_alt.bytes;
    return RM_SUCCESS;
}

extern "C" int rm_pw_bytes(rm_ctx *ctx, int pw, size_t *bytes)
{
    const int rc = check_pw(ctx, pw, false);
    if (rc) return rc;
    if (bytes) *bytes = ctx->pw[pw].bytes();
    return RM_SUCCESS;
}

extern "C" int rm_unload_pw(rm_ctx *ctx, int pw)
{
    const int rc = check_pw(ctx, pw, false);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->opts.device));
    ctx->pw[pw].release();
    return RM_SUCCESS;
}

namespace {

struct OmegaSrc {
    const double *p[MAX_LANES];
};

// dst += src[0] + src[1] + ... (in lane order: the same rounding every call)
__global__ void omega_sum_kernel(double *dst, OmegaSrc src, int n_src, size_t count)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        double v = dst[i];
        for (int l = 0; l < n_src; ++l) v += src.p[l][i];
        dst[i] = v;
    }
}

// The launch sequence of one batch: lanes 1.. fork from lane 0, zero their
// accumulators, solve their waves in order, and join; lane 0 adds their
// Omega to its own.
int enqueue_batch(rm_ctx *ctx, const std::vector<std::vector<int>> &assign, const double *dE, int n_E, int mode,
                  int ntri)
{
    Lane *l0 = &ctx->lanes[0];
    const int L = (int)assign.size();
    const size_t count = (size_t)n_E * ntri;
    CK(cudaEventRecord(ctx->ev_batch, l0->stream));
    for (int l = 1; l < L; ++l) {
        Lane *ln = &ctx->lanes[l];
        CK(cudaStreamWaitEvent(ln->stream, ctx->ev_batch, 0));
        CK(cudaMemsetAsync(ln->omega.p, 0, count * sizeof(double), ln->stream));
    }
    for (int l = 0; l < L; ++l) {
        Lane *ln = &ctx->lanes[l];
        for (int w : assign[l]) {
            CK(cudaMemsetAsync(ln->wsStatus.p, 0, (size_t)n_E * sizeof(int), ln->stream));
            const int rc = solve_blocks(ctx, ln, ctx->pw[w], dE, n_E, mode, nullptr, nullptr, ln->wsStatus.as<int>(),
                                        ln->omega.as<double>());
            if (rc) return rc;
        }
    }
    if (L > 1) {
        OmegaSrc src = {};
        for (int l = 1; l < L; ++l) {
            Lane *ln = &ctx->lanes[l];
            CK(cudaEventRecord(ln->ev_done, ln->stream));
            CK(cudaStreamWaitEvent(l0->stream, ln->ev_done, 0));
            src.p[l - 1] = ln->omega.as<double>();
        }
        const unsigned grid = (unsigned)std::min<size_t>((count + 255) / 256, 4096);
        omega_sum_kernel<<<grid, 256, 0, l0->stream>>>(l0->omega.as<double>(), src, L - 1, count);
        CK(cudaGetLastError());
        ctx->launches++;
    }
    return RM_SUCCESS;
}

}  // namespace

extern "C" int rm_solve_batch(rm_ctx *ctx, int n_pw, const int *pws, int n_E, const double *E, int mode,
                              int use_graph)
{
    if (!ctx) return RM_EINVAL;
    if (n_pw <= 0 || !pws || n_E <= 0 || !E)
        return fail(ctx, RM_EINVAL, "n_pw=%d, n_E=%d must be > 0 with non-NULL arrays", n_pw, n_E);
    if (mode != RM_DIRECT && mode != RM_MQDT) return fail(ctx, RM_EINVAL, "mode %d", mode);
    for (int i = 0; i < n_pw; ++i) {
        int rc = check_pw(ctx, pws[i], true);
        if (rc) return rc;
        for (int j = 0; j < i; ++j)
            if (pws[j] == pws[i]) return fail(ctx, RM_EINVAL, "partial wave %d listed twice", pws[i]);
        PwHost &P = ctx->pw[pws[i]];
        if (P.n_levels != ctx->pw[pws[0]].n_levels)
            return fail(ctx, RM_EINVAL, "partial waves %d and %d have different level counts", pws[0], pws[i]);
        if (!use_large(ctx, P) && P.n > solve_small_max_n())
            return fail(ctx, RM_EUNSUPPORTED, "n_ch=%d above the shared-memory solver limit %d", P.n,
                        solve_small_max_n());
        rc = check_precision(ctx, P);
        if (rc) return rc;
    }
    CK(cudaSetDevice(ctx->opts.device));
    Lane *l0 = &ctx->lanes[0];
    PwHost &P0 = ctx->pw[pws[0]];
    const bool dev_in = is_device_ptr(E);
    int rc = register_grid(ctx, l0, P0, n_E, E, dev_in);
    if (rc) return rc;
    const double *dE = E;
    if (!dev_in) {
        if (!finite_all(E, n_E)) return fail(ctx, RM_EINVAL, "non-finite energy");
        CK(ctx->batchE.reserve((size_t)n_E * sizeof(double)));
        CK(cudaMemcpyAsync(ctx->batchE.p, E, (size_t)n_E * sizeof(double), cudaMemcpyHostToDevice, l0->stream));
        dE = ctx->batchE.as<double>();
    }
    const int ntri = P0.n_levels * (P0.n_levels + 1) / 2;
    // the formation of every wave is chosen before anything is captured
    if (ctx->opts.autotune && ctx->opts.precision != RM_FP64 && ctx->opts.formulation == RM_FORM_AUTO)
        for (int i = 0; i < n_pw; ++i)
            if (!ctx->pw[pws[i]].tuned) {
                rc = tune_wave(ctx, l0, ctx->pw[pws[i]], dE, n_E);
                if (rc) return rc;
            }
    // longest processing time first: each wave (cost ~ formation n^2 N plus
    // matching n^3) goes to the lane with the least work so far
    const int L = std::min((int)ctx->lanes.size(), n_pw);
    std::vector<int> order(n_pw);
    std::iota(order.begin(), order.end(), 0);
    auto cost = [&](int i) {
        const PwHost &P = ctx->pw[pws[i]];
        return (double)P.n * P.n * ((double)P.N + 4.0 * P.n);
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
    std::vector<std::vector<int>> assign(L);
    std::vector<double> load(L, 0.0);
    for (int i : order) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        assign[l].push_back(pws[i]);
        load[l] += cost(i);
    }
    for (int l = 0; l < L; ++l) {
        Lane *ln = &ctx->lanes[l];
        for (int w : assign[l]) {
            rc = reserve_solve(ctx, ln, ctx->pw[w], n_E);
            if (rc) return rc;
        }
        CK(ln->wsStatus.reserve((size_t)n_E * sizeof(int)));
        CK(ln->omega.reserve((size_t)n_E * ntri * sizeof(double)));
    }
    const bool graphs = use_graph && !ctx->prof && l0->stream != nullptr && l0->stream != cudaStreamLegacy &&
                        l0->stream != cudaStreamPerThread;
    const std::vector<int> key(pws, pws + n_pw);
    if (graphs) {
        const unsigned long long gen = g_buf_gen.load();
        for (size_t g = 0; g < ctx->graphs.size(); ++g) {
            BatchGraph &bg = ctx->graphs[g];
            const bool same = bg.pws == key && bg.n_E == n_E && bg.mode == mode && bg.E == dE &&
                              bg.omega == l0->omega.p && bg.lanes == L;
            if (!same) continue;
            if (bg.gen == gen) {
                CK(cudaGraphLaunch(bg.exec, l0->stream));
                ctx->launches += bg.launches;
                CK(cudaEventRecord(l0->ev_done, l0->stream));
                return RM_SUCCESS;
            }
            cudaGraphExecDestroy(bg.exec);   // captured under buffers since freed or moved
            ctx->graphs.erase(ctx->graphs.begin() + g);
            break;
        }
    }
    const long long before = ctx->launches;
    rc = enqueue_batch(ctx, assign, dE, n_E, mode, ntri);
    if (rc) return rc;
    CK(cudaEventRecord(l0->ev_done, l0->stream));
    const long long nl = ctx->launches - before;
    if (graphs) {
        // the same sequence captured (not run) for later calls with these arguments
        const unsigned long long gen = g_buf_gen.load();
        CK(cudaStreamBeginCapture(l0->stream, cudaStreamCaptureModeRelaxed));
        const int crc = enqueue_batch(ctx, assign, dE, n_E, mode, ntri);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(l0->stream, &g);
        ctx->launches = before + nl;
        if (crc == RM_SUCCESS && ce == cudaSuccess && g && g_buf_gen.load() == gen) {
            cudaGraphExec_t ex = nullptr;
            if (cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
                BatchGraph bg;
                bg.pws = key;
                bg.n_E = n_E;
                bg.mode = mode;
                bg.lanes = L;
                bg.E = dE;
                bg.omega = l0->omega.p;
                bg.gen = gen;
                bg.exec = ex;
                bg.launches = nl;
                ctx->graphs.push_back(bg);
            }
        }
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
    }
    return RM_SUCCESS;
}

extern "C" int rm_autotune_info(rm_ctx *ctx, int pw, int *formulation, int *tile_n, int *stages, double *ms4)
{
    const int rc = check_pw(ctx, pw, false);
    if (rc) return rc;
    const PwHost &P = ctx->pw[pw];
    if (!P.tuned) return fail(ctx, RM_EINVAL, "partial wave %d has not been tuned", pw);
    int tn = 0, st = 0;
    if (P.tune_form == RM_FORM_PAIRS) tc_pair_variant_shape(P.tune_var, &tn, &st);
    if (formulation) *formulation = P.tune_form;
    if (tile_n) *tile_n = tn;
    if (stages) *stages = st;
    if (ms4)
        for (int i = 0; i < 4; ++i) ms4[i] = P.tune_ms[i];
    return RM_SUCCESS;
}

extern "C" int rm_set_wait_probe(rm_ctx *ctx, unsigned long long limit_ns)
{
    if (!ctx) return RM_EINVAL;
    if (limit_ns > 10000000000ull) return fail(ctx, RM_EINVAL, "probe limit %llu ns above 10 s", limit_ns);
    ctx->wait_probe_ns = limit_ns;
    return RM_SUCCESS;
}

extern "C" int rm_sync(rm_ctx *ctx)
{
    if (!ctx) return RM_EINVAL;
    CK(cudaSetDevice(ctx->opts.device));
    for (Lane &l : ctx->lanes) {
        CK(cudaStreamSynchronize(l.stream));
        if (l.copy) CK(cudaStreamSynchronize(l.copy));
    }
    for (Lane &l : ctx->lanes) {
        const int rc = check_device_flag(ctx, &l);
        if (rc) return rc;
    }
    return RM_SUCCESS;
}

extern "C" long long rm_launch_count(rm_ctx *ctx) { return ctx ? ctx->launches : 0; }

extern "C" const char *rm_strerror(int code)
{
    switch (code) {
    case RM_SUCCESS: return "success";
    case RM_EINVAL: return "invalid argument";
    case RM_ENOMEM: return "out of memory";
    case RM_ECUDA: return "CUDA runtime error";
    case RM_EGRID: return "energy grid differs from the registered grid";
    case RM_ENOTLOADED: return "partial wave not loaded";
    case RM_EUNSUPPORTED: return "unsupported option for this size or mode";
    case RM_ETIMEOUT: return "bounded device wait timed out";
    case RM_ETHRESHOLD: return "energy on a channel threshold";
    case RM_ENEAR_POLE: return "energy on an R-matrix pole";
    case RM_ESINGULAR: return "matching system singular";
    case RM_ECF_NOCONV: return "Coulomb continued fraction did not converge";
    default: return "unknown code";
    }
}

extern "C" const char *rm_last_error(rm_ctx *ctx) { return ctx ? ctx->err : "NULL context"; }
