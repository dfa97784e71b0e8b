// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/rmgb.h"

namespace rmgb {

// Boundary data of one channel at one energy (step (b)).
//   open (CH_OPEN):        (gh, ghp) = (c, c'),  (s, sp) = (s, s')   energy-normalised Coulomb
//   closed (CH_CLOSED):    (gh, ghp) = (theta, theta') with theta^2 + (a theta')^2 = 1, s = sp = 0
//   MQDT-eliminated closed (CH_MQDT): (gh, ghp) = (g, g'), (s, sp) = (f, f'),
//                          tanb = tan(pi nu)
enum ChanKind { CH_OPEN = 0, CH_CLOSED = 1, CH_MQDT = 2 };
struct __align__(16) ChanFn {
    double gh, ghp, s, sp;
    double tanb;
    int kind;
    int pad;
};

// R is stored per energy as its upper triangle, row-wise:
//   R_ij (i <= j) at tri_idx(i, j, n) = i n - i(i-1)/2 + (j - i),
// with the per-energy stride rounded up to a multiple of 4 doubles.
__host__ __device__ __forceinline__ int tri_count(int n) { return n * (n + 1) / 2; }
__host__ __device__ __forceinline__ int tri_ld(int n) { return (tri_count(n) + 3) & ~3; }
__host__ __device__ __forceinline__ int tri_idx(int i, int j, int n)
{
    return i * n - (i * (i - 1)) / 2 + (j - i);
}

// Near-threshold interpolation table of one channel (step (b)). At fixed
// r = a the pair f = s / sqrt(A), g~ = c sqrt(A) (open side, A(eps, l) =
// prod_{p=1..l} (1 + p^2 eps / z^2)) continues analytically into the closed
// side, where f is the energy-analytic regular solution and g~ the g of the
// quantum-defect pair at half-integer nu; the decaying solution is then
// theta ~ A f cos(pi nu) - g~ sin(pi nu). Values at THR_NODES energies
// straddling the threshold (half on each side, ascending in x) give every
// channel quantity for |eps| < zone by barycentric interpolation instead of
// continued fractions whose depth grows as 1/|eps|. zone = 0: not covered.
constexpr int THR_NODES = 16;
struct ThrNodes {
    double x[THR_NODES];        // eps of the nodes
    double w[THR_NODES];        // barycentric weights
    double y[4][THR_NODES];     // f, f', g~, g~'
    double zone;
    double h;                   // node spacing in energy
};

// Device-side description of one partial wave.
struct PwDev {
    int n;             // channels
    int N;             // poles
    double a, b, z, g;
    int n_levels;
    const double *Ek;  // [N] sorted ascending
    const double *W;   // [n][N] row-major FP64
    const double *e_thr;  // [n]
    const int *l;      // [n]
    const int *level;  // [n]
    const int *lev_start;  // [n_levels+1] CSR of channels per level
    const int *lev_chan;   // [n]
    const double *lev_thr; // [n_levels] threshold of each level (+inf if unused)
    const ThrNodes *thr = nullptr;  // [n] near-threshold tables (nullptr: none)
    const float2 *Ek_hl = nullptr;  // [N] E_k as hi + lo floats (mixed-precision formation)
    // open-side tables: Chebyshev coefficients of f = s / sqrt(A), f' = s' /
    // sqrt(A), g~ = c sqrt(A), g~' = c' sqrt(A) in k = sqrt(eps) on segments
    // [q dk, (q + 1) dk), q < otab_nseg: otab[((i nseg + q) 4 + f) OTAB_M + m];
    // otab_bad[i] != 0: channel i's table failed its check (nullptr: none)
    const double *otab = nullptr;
    const int *otab_bad = nullptr;
    double otab_dk = 0.0;
    int otab_nseg = 0;
    // closed-side tables: Chebyshev coefficients of the direction
    // (theta, a theta') (unnormalised, continuous in energy) in
    // nu = z / sqrt(-eps) on cells [nu_lo + q dnu, nu_lo + (q + 1) dnu),
    // q < ctab_nseg, each split into ctab_nsub[i nseg + q] (1, 2, 4, 8 or 16)
    // equal sub-segments (0: the cell has no coefficients):
    // ctab[(((i nseg + q) CTAB_SUB + s) 2 + f) OTAB_M + m]
    const double *ctab = nullptr;
    const unsigned char *ctab_nsub = nullptr;
    double ctab_nu_lo = 0.0, ctab_dnu = 0.0;
    int ctab_nseg = 0;
};

constexpr int OTAB_M = 12;            // Chebyshev nodes per open-side segment
constexpr double OTAB_C = 0.9;        // segment width in k: OTAB_C / a
constexpr double OTAB_EPS_MAX = 16.0; // Ry above threshold covered by the open-side tables
constexpr double CTAB_DNU = 0.25;     // closed-side cell width in nu
constexpr int CTAB_SUB = 16;          // at most this many sub-segments per cell
constexpr double CTAB_EPS_MIN = -16.0; // Ry below threshold covered by the closed-side tables
constexpr int CTAB_MAX_SEG = 4096;    // at most this many closed-side segments per channel
constexpr double CTAB_KA_MIN = 6.0;   // closed-side tables only where kappa a >= this

struct Opts {
    double eps_thr, delta_pole, fnumin, nu_margin, kappa_a_max;
};

// ---- launchers (each returns cudaGetLastError() of its launch) ----------

// Outer-region propagation (see propagate.cu): R(a) in Rp (packed, stride
// tri_ld(n)) replaced by R(r1) for every energy with status RM_OK; pw carries
// the inner radius a; A = [lmax][n][n] coefficients on the device.
constexpr int PROP_MAXN = 64;
constexpr int PROP_MAX_LAMBDA = 4;
size_t propagate_smem(int n, int lmax);
// The state and the coefficients fit one CTA's shared memory (above 32
// channels at most (4 + lmax) n^2 doubles: lmax <= 3 at 64 channels).
bool propagate_fits(int n, int lmax);
cudaError_t launch_propagate(const PwDev &pw, const double *E, int nE, const double *A, int lmax, double r1,
                             int steps, double *Rp, int *status, cudaStream_t s);
// FP32 matching and T step (direct mode, n <= solve_small_max_n()),
// register-tiled; launch_solve_small forwards f32 launches here.
cudaError_t launch_solve_f32(const PwDev &pw, const double *E, int nE, const ChanFn *cf, const double *R,
                             int *status, double *K_out, int *n_open_out, double *omega, int n_tri,
                             const int *deep_ws, int pass, cudaStream_t s);
// mqdt != 0: closed channels in the quantum-defect set get CH_MQDT data.
// deep_ws (or nullptr): the list written by launch_chanfn_deep_mark; the
// listed deep pairs are then left to launch_chanfn_deep.
cudaError_t launch_chanfn(const PwDev &pw, const double *E, int nE, const Opts &o, int mqdt,
                          ChanFn *cf, int *status, const int *deep_ws, cudaStream_t s);
// Near-threshold tables of the n channels (z > 0): computes tab[0..n) on the
// stream; pw.thr is not read.
cudaError_t launch_thr_nodes(const PwDev &pw, ThrNodes *tab, cudaStream_t s);
// Open-side tables of the n channels (z > 0) for pw.otab_dk / pw.otab_nseg:
// coefficients into coef, failures into bad[n] (zeroed here).
cudaError_t launch_open_table(const PwDev &pw, double *coef, int *bad, cudaStream_t s);
// Closed-side tables of the n channels (z > 0) for pw.ctab_nu_lo / ctab_dnu /
// ctab_nseg: coefficients into coef, sub-segment counts into nsub (0 for a
// cell that failed its check).
cudaError_t launch_closed_table(const PwDev &pw, double *coef, unsigned char *nsub, cudaStream_t s);
// Largest nu any channel's closed-side table reaches (its near-threshold
// zone edge, or kappa a = CTAB_KA_MIN if that comes first), for the cell
// count.
double closed_table_nu_hi(double z, double a, int l_max);
// Near-threshold (deep) pairs: deep_ws = [count][list of CAP pair indices][nE
// energy marks], chanfn_deep_ws_bytes(nE) bytes. The mark launch zeroes it
// and fills it; the deep launch evaluates the listed pairs. If the list
// overflowed (count > chanfn_deep_cap()), nothing is left out and nothing is
// deferred.
size_t chanfn_deep_ws_bytes(int nE);
// |eps| below which a pair not covered by its channel's table is deep.
double chanfn_deep_eps(double z);
int chanfn_deep_cap();
cudaError_t launch_chanfn_deep_mark(const PwDev &pw, const double *E, int nE, const Opts &o, int *deep_ws,
                                    cudaStream_t s);
cudaError_t launch_chanfn_deep(const PwDev &pw, const double *E, int nE, const Opts &o, int mqdt, ChanFn *cf,
                               int *status, const int *deep_ws, cudaStream_t s);
cudaError_t launch_nearpole(const PwDev &pw, const double *E, int nE, int *status,
                            cudaStream_t s);
// Iteration counts of step (b) (direct mode), [nE][n] int4 {kind, CF1
// iterations, CF2 forward iterations, recurrence steps in l}.
cudaError_t launch_chanfn_work(const PwDev &pw, const double *E, int nE, const Opts &o, int4 *work,
                               cudaStream_t s);
cudaError_t launch_form_r_fp64(const PwDev &pw, const double *E, int nE, double *R,
                               cudaStream_t s);
// mqdt != 0: the channel data may hold MQDT-eliminated channels (larger
// shared-memory layout). f32 != 0 (direct mode only): the matching system is
// eliminated in FP32.
// deep_ws (or nullptr): pass 0 leaves out the energies marked by
// launch_chanfn_deep_mark, pass 1 solves only those. ku_out (or nullptr,
// FP64 matching): instead of K, T and Omega, write the unphysical K_u of the
// P channels (open and MQDT-eliminated, channel order) to ku_out [nE][n][n]
// (row stride n) and its order to ku_np [nE].
cudaError_t launch_solve_small(const PwDev &pw, const double *E, int nE, const ChanFn *cf,
                               const double *R, int *status, double *K_out, int *n_open_out,
                               double *omega, int n_tri, int mqdt, int f32, const int *deep_ws, int pass,
                               cudaStream_t s, double *ku_out = nullptr, int *ku_np = nullptr);
// Mixed-precision formation (tensor cores). Operand kinds:
enum TcKind { TC_BF16X3 = 0, TC_TF32X3 = 1 };
// Split of P_pk = w_ik w_jk / (2a) into hi/lo operands, [n_pairs][Kpad] K-major.
cudaError_t launch_split_p(const PwDev &pw, int kind, int Kpad, void *P_hi, void *P_lo,
                           cudaStream_t s);
// Split of D_ek = 1/(E_k - E_e) (0 when |E_k - E_e| < delta) into hi/lo, [nE][Kpad].
// pw.Ek_hl must be set; e_hl: nE float2 of scratch (E as hi + lo floats).
cudaError_t launch_split_d(const PwDev &pw, const double *E, int nE, double delta, int kind, int Kpad,
                           void *D_hi, void *D_lo, float2 *e_hl, cudaStream_t s);
// R_packed[e][p] = sum_k D[e][k] P[p][k] over the three hi/lo products;
// variant: tile of 128 energies x tile_n pairs with a ring of `stages`
// (tc_pair_variant_shape), 0 <= variant < tc_pair_variants().
int tc_pair_variants();
void tc_pair_variant_shape(int variant, int *tile_n, int *stages);
cudaError_t launch_form_r_tc(int kind, const void *D_hi, const void *D_lo, const void *P_hi,
                             const void *P_lo, int nE, int n_pairs, int Kpad, double *Rp, int ldR,
                             int *err_flag, cudaStream_t s, int variant = 0, unsigned long long probe_ns = 0);
// R_packed[e][p] += (1/2a) w_ik w_jk / (E_k - E_e) over poles with |E_k - E_e| < delta (FP64),
// the near/far decision taken exactly as launch_split_d takes it (pw.Ek_hl).
// ws: near_pole_ws_bytes(nE) bytes of device scratch (list of the energies
// with poles within delta, and their pole ranges).
size_t near_pole_ws_bytes(int nE);
cudaError_t launch_near_pole_fixup(const PwDev &pw, const double *E, int nE, double delta, double *Rp, void *ws,
                                   cudaStream_t s);
// Per-energy formulation (formation_tc_energy.cu): R(E) = W diag(d(E)) W^T / 2a.
int pe_max_n();
// Workspace per energy: FP32 partial tiles of every K segment + d(E) in FP32
// (D32 holds [nE][Kpad] floats followed by nE int2 near-pole ranges).
size_t pe_bytes_per_energy(int n, int N, int kind);
// W in FP32 plus w split hi/lo, [n][Kpad] each.
size_t pe_operand_bytes(int n, int N, int kind);
cudaError_t launch_pe_prep_w(const PwDev &pw, int kind, int Kpad, float *W32, void *Wh, void *Wl,
                             cudaStream_t s);
cudaError_t launch_pe_d32(const PwDev &pw, const double *E, int nE, double delta, int Kpad, float *D32,
                          cudaStream_t s);
// probe_ns != 0 (both tensor-core formations): the bounded-wait self-test
// (rm_set_wait_probe) instead of the formation.
cudaError_t launch_form_r_pe(int kind, int n, int Kpad, const float *W32, const void *Wh, const void *Wl,
                             const float *D32, int nE, float *part, int *err_flag, cudaStream_t s,
                             unsigned long long probe_ns = 0);
// Sums the segments in FP64, adds the near-pole terms, scales by 1/2a -> packed R.
cudaError_t launch_pe_reduce(const PwDev &pw, int kind, int Kpad, const double *E, int nE, double delta,
                             const float *D32, const float *part, double *Rp, int ldR, cudaStream_t s);
// Packed -> full symmetric [nE][n][n] (inspection only).
cudaError_t launch_unpack_r(int n, int nE, const double *Rp, double *R, cudaStream_t s);
int tc_kpad(int N, int kind);

cudaError_t launch_chanfn_export(const PwDev &pw, const double *E, int nE, const ChanFn *cf,
                                 double *out, cudaStream_t s);

// Largest channel count the shared-memory solver takes.
int solve_small_max_n();

// Global-memory solver for any channel count (steps (c) and (d)).
// f32 != 0: matching system, T step in FP32 (MQDT elimination, K and Omega
// FP64), for channel counts where solve_large_f32_supported holds.
size_t solve_large_bytes_per_energy(int n);
bool solve_large_f32_supported(int n);
cudaError_t launch_solve_large(const PwDev &pw, const double *E, int nE, const ChanFn *cf,
                               const double *R, int *status, double *K_out, int *n_open_out,
                               double *omega, int n_tri, void *ws, int *launches, cudaStream_t s,
                               int f32 = 0);

// ---- MQDT coarse-mesh interpolation (qdt.cu) ------------------------------------
enum QdtClass : signed char { QDT_OPEN = 0, QDT_ELIM = 1, QDT_DECAY = 2, QDT_THRESHOLD = 3 };
enum QdtFlag { QDT_FLAG_OK = 0, QDT_FLAG_THRESHOLD = 1, QDT_FLAG_NONODE = 2 };

// Host view of one partial wave's channels and the MQDT options.
struct QdtChannels {
    int n, N;
    const double *e_thr;   // [n]
    const int *l;          // [n]
    const double *E_k;     // [N] sorted
    double z, a, eps_thr, nu_margin, fnumin, kappa_a_max;
};

// Segments of fine energies with equal channel classes, their valid nodes,
// and the energy at which each fine energy is interpolated (qetest).
struct QdtPlan {
    std::vector<int> seg;                      // [n_E] segment or -1 (on a threshold)
    std::vector<int> i0, i1;                   // fine index range per segment
    std::vector<std::vector<signed char>> cls; // classes per segment
    std::vector<double> e_int;                 // [n_E]
    std::vector<double> node_x;                // valid nodes, segment by segment
    std::vector<int> node_seg, seg_node0, seg_nnodes;
};

// Interpolation of one fine energy: K_u or S_u = (1 - t) node a + t node b.
struct QdtFine {
    int a, b;
    double t;
    int flag;
};

// Classes of every (energy, channel) on the device, [nE][n] (QDT_THRESHOLD in
// the first entry of an energy on a threshold).
cudaError_t launch_qdt_classes(const PwDev &pw, const double *E, int nE, const Opts &o, signed char *cls,
                               cudaStream_t s);
// From those classes (host copy): RM_EINVAL if ieq == 0 or E is not strictly
// ascending.
int qdt_plan(const QdtChannels &c, const double *E, int n_E, const signed char *cls_all, int ieq,
             double qetest, QdtPlan &pl);
// Weights over the nodes with node_ok != 0 (failed nodes left out).
void qdt_weights(const QdtPlan &pl, const std::vector<int> &node_ok, int n_E, std::vector<QdtFine> &fine);
// Node K_u [nn][n][n] -> S_u = 2 (1 - i K_u)^{-1} - 1 (complex, same layout).
cudaError_t launch_qdt_s_from_k(int n, int n_nodes, const double *Ku, const int *np_node, int *status,
                                double2 *Su, cudaStream_t s);
// Fine energies: interpolation, elimination at the fine energy, Omega.
cudaError_t launch_qdt_fine(int iqdt, const PwDev &pw, const double *E, int nE, const Opts &o,
                            const QdtFine *fine, const double *Ku, const double2 *Su, const int *node_status,
                            int *status, int *n_open_out, double *omega, int n_tri, cudaStream_t s);

}  // namespace rmgb
