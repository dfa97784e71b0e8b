// Allocation-free K-matrix entry point (rm_k_matrices_noalloc, include/rmgb.h).
//
// The regular entry points keep their workspace in device memory the context
// allocates with cudaMalloc. Some callers cannot allow that: code whose GPU
// memory is owned entirely by another allocator (a framework's memory pool
// that must see every byte), and latency-bound loops for which the implicit
// device-wide synchronisation of cudaMalloc/cudaFree is not acceptable. This
// file gives them one call that allocates nothing: its workspace is the
// file-scope array below, which every GPU that loads the library holds until
// the process exits.
#include <mutex>
#include <stdio.h>

#include "rm_internal.cuh"

using namespace rmgb;

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)32 << 20;   // 32 MiB per device

// Workspace of rm_k_matrices_noalloc. In host code this name is only a
// stand-in for the device array; its device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[MAX_DEVICES];   // device address of the array, per device

int say(char *buf, size_t len, int code, const char *msg, long a = 0, long b = 0)
{
    if (buf && len) snprintf(buf, len, msg, a, b);
    return code;
}

size_t round_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Puts the caller's current device back on every return path: the call
// switches to `device` for its own work only.
struct DeviceRestore {
    int prev = -1;
    DeviceRestore()
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
    }
    ~DeviceRestore()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" int rm_k_matrices_noalloc(int device, int n_ch, int n_poles, int n_E,
                                     const double *E_k, const double *W, const double *e_thr,
                                     const int *l, double z, double a, double b, const double *E,
                                     double eps_thr, double *K_out, int *n_open_out,
                                     int *status_out, void *stream, char *errbuf, size_t errlen)
{
    if (n_ch <= 0 || n_poles <= 0 || n_E <= 0)
        return say(errbuf, errlen, RM_EINVAL, "n_ch=%ld, n_poles and n_E must be > 0", n_ch);
    if (n_ch > solve_small_max_n())
        return say(errbuf, errlen, RM_EUNSUPPORTED,
                   "n_ch=%ld exceeds the allocation-free limit of %ld channels", n_ch,
                   solve_small_max_n());
    if (!E_k || !W || !e_thr || !l || !E || !status_out)
        return say(errbuf, errlen, RM_EINVAL, "NULL input or status pointer");
    if (!(a > 0) || !(z >= 0) || !(eps_thr >= 0))
        return say(errbuf, errlen, RM_EINVAL, "need a > 0, z >= 0, eps_thr >= 0");
    if (device < 0 || device >= MAX_DEVICES)
        return say(errbuf, errlen, RM_EINVAL, "device %ld out of range", device);
    const size_t per_energy = (size_t)n_ch * sizeof(ChanFn) + (size_t)tri_ld(n_ch) * sizeof(double);
    if (round_up(per_energy) + 512 > NOALLOC_SCRATCH_BYTES)
        return say(errbuf, errlen, RM_EUNSUPPORTED,
                   "one energy needs %ld bytes of workspace, more than the %ld-byte static array",
                   (long)per_energy, (long)NOALLOC_SCRATCH_BYTES);
    DeviceRestore restore;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return say(errbuf, errlen, RM_ECUDA, "cudaSetDevice(%ld) failed", device);
    }
    // One-time set-up per device, with that device current: the device
    // address of the static workspace. The address is kept for the life of
    // the process, so it is stale after a cudaDeviceReset of that device
    // (documented in the header).
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_addr[device]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return say(errbuf, errlen, RM_ECUDA,
                           "cudaGetSymbolAddress of the static workspace failed on device %ld",
                           device);
            }
            g_scratch_addr[device] = p;
        }
        scratch = g_scratch_addr[device];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // Energies per chunk that fit the workspace: [ChanFn x chunk x n][packed R x chunk].
    size_t chunk = (NOALLOC_SCRATCH_BYTES - 512) / (per_energy + 1);
    while (chunk > 1 && round_up(chunk * n_ch * sizeof(ChanFn)) +
                            chunk * (size_t)tri_ld(n_ch) * sizeof(double) > NOALLOC_SCRATCH_BYTES)
        --chunk;
    if (chunk > 32768) chunk = 32768;
    ChanFn *cf = static_cast<ChanFn *>(scratch);
    double *R = reinterpret_cast<double *>(static_cast<unsigned char *>(scratch) +
                                           round_up(chunk * n_ch * sizeof(ChanFn)));
    PwDev d = {};
    d.n = n_ch;
    d.N = n_poles;
    d.a = a;
    d.b = b;
    d.z = z;
    d.Ek = E_k;
    d.W = W;
    d.e_thr = e_thr;
    d.l = l;
    Opts o = {eps_thr, 0.0, 0.0, 0.1, 5.0};
    // status must start at zero (kernels only record the first failure)
    cudaError_t err = cudaMemsetAsync(status_out, 0, (size_t)n_E * sizeof(int), s);
    for (int e0 = 0; err == cudaSuccess && e0 < n_E; e0 += (int)chunk) {
        const int nb = (int)((size_t)(n_E - e0) < chunk ? (size_t)(n_E - e0) : chunk);
        const double *Eb = E + e0;
        int *sb = status_out + e0;
        err = launch_nearpole(d, Eb, nb, sb, s);
        if (err == cudaSuccess) err = launch_chanfn(d, Eb, nb, o, 0, cf, sb, nullptr, s);
        if (err == cudaSuccess) err = launch_form_r_fp64(d, Eb, nb, R, s);
        if (err == cudaSuccess)
            err = launch_solve_small(d, Eb, nb, cf, R, sb,
                                     K_out ? K_out + (size_t)e0 * n_ch * n_ch : nullptr,
                                     n_open_out ? n_open_out + e0 : nullptr, nullptr, 0, 0, 0, nullptr, 0, s);
    }
    if (err != cudaSuccess) {
        if (errbuf && errlen) snprintf(errbuf, errlen, "CUDA error: %s", cudaGetErrorString(err));
        return RM_ECUDA;
    }
    return RM_SUCCESS;
}
