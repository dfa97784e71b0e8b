/*
 * rmgb — GB300-native outer-region R-matrix hot path: R -> K -> Omega.
 *
 * For every (partial wave, incident energy) pair the library
 *   (a) forms the channel R-matrix (Section "Overview", Eq. rmatrix)
 *         R_ij(E) = (1/2a) sum_k w_ik w_jk / (E_k - E),
 *   (b) evaluates the asymptotic channel functions at r = a: energy-normalised
 *       Coulomb functions s = F/sqrt(k), c = G/sqrt(k) for open channels and
 *       the decaying Whittaker function for closed channels (Section
 *       "Overview", Eq. radial with U = 0; Section "Glossary of terms", open
 *       and closed channels),
 *   (c) solves the matching condition (Eq. match)
 *         psi(a) = R (a psi'(a) - b psi(a))
 *       for the open-channel K-matrix, eliminating closed channels by their
 *       decaying boundary condition or, in MQDT mode, through the unphysical
 *       K-matrix (Section "namelist stgf MQDT variables", iqdt),
 *   (d) forms T = 2iK(1 - iK)^{-1} and accumulates g |T|^2 into collision
 *       strengths Omega_IJ(E) (Section "Glossary of terms").
 *
 * Units: energies in Rydberg, radii in Bohr. Channels keep their input order;
 * K rows and columns are the open channels in ascending channel index.
 *
 * Conventions for every call:
 *  - Return value 0 on success, a negative RM_E* code on error; no call aborts,
 *    traps or exits. rm_last_error(ctx) gives a one-line reason.
 *  - Host pointers are read during the call and not retained (except the
 *    output of rm_collision_strengths_async, written until rm_sync). Pointers marked
 *    "device" must be device memory of the context's GPU (e.g. torch tensors).
 *  - A context is not thread-safe: use one context per host thread.
 *  - Work is enqueued on the context's stream; only rm_collision_strengths,
 *    rm_sync and the calls documented as synchronous wait for it.
 */
#ifndef RMGB_H
#define RMGB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
/* Call return codes (negative). */
#define RM_SUCCESS        0
#define RM_EINVAL        -1   /* bad argument (size, pointer, non-finite value) */
#define RM_ENOMEM        -2   /* device or host allocation failed; no partial state */
#define RM_ECUDA         -3   /* a CUDA runtime call failed */
#define RM_EGRID         -4   /* energy grid differs from the one Omega accumulates on */
#define RM_ENOTLOADED    -5   /* partial wave has no poles or no channels */
#define RM_EUNSUPPORTED  -6   /* option not supported for this size or mode */
#define RM_ETIMEOUT      -7   /* a bounded device wait gave up */

/* Per-energy status codes (written to status_out, non-negative). An energy
 * whose status is not RM_OK contributes nothing to Omega. */
#define RM_OK             0
#define RM_ETHRESHOLD     1   /* |E - e_i| < eps_thr for some channel i */
#define RM_ENEAR_POLE     2   /* |E - E_k| < 1e-12 max(1,|E|) for some pole k */
#define RM_ESINGULAR      3   /* matching system (or MQDT elimination) singular */
#define RM_ECF_NOCONV     4   /* a Coulomb continued fraction did not converge */

/* Precision of the R-matrix formation (step (a)). Channel functions are
 * always FP64; the matching solve and T follow rm_opts.solve_precision, and
 * Omega is always accumulated in FP64. */
#define RM_FP64           0   /* FP64 formation */
#define RM_FP32           1   /* tensor cores: tf32 hi/lo split, 3 products, FP32
                                 accumulate; near-pole terms in FP64 */
#define RM_BF16X3         2   /* tensor cores: bf16 hi/lo split, 3 products, FP32
                                 accumulate; near-pole terms in FP64 */

/* Matching modes. */
#define RM_DIRECT         0   /* closed channels by their decaying boundary condition */
#define RM_MQDT           1   /* closed channels through the unphysical K-matrix */

typedef struct rm_ctx rm_ctx;

typedef struct rm_opts {
    int precision;          /* RM_FP64 (default), RM_FP32, RM_BF16X3 */
    double delta_pole;      /* mixed precision: poles with |E_k - E| < delta_pole
                               are summed in FP64 (default 1e-3 Ry) */
    double eps_thr;         /* |E - e_i| below this is RM_ETHRESHOLD (default 1e-10 Ry) */
    double fnumin;          /* MQDT: closed channels with nu < fnumin are not
                               quantum-defect eliminated (default 0) */
    double nu_margin;       /* MQDT: ... nor those with nu < l + nu_margin (default 0.1) */
    int device;             /* CUDA device ordinal (default 0) */
    void *stream;           /* cudaStream_t to enqueue on (cudaStreamLegacy for
                               the legacy default stream); NULL = a non-blocking
                               stream the context creates and owns */
    size_t mem_budget;      /* bytes of per-call device workspace of each lane (0 =
                               32 GiB, at most half the free device memory); it sets
                               the energies per block, and a block of fewer energies
                               than the GPU has SMs leaves the one-CTA-per-energy
                               solvers part of the GPU */
    double mqdt_kappa_a_max;/* MQDT: closed channels with kappa a above this keep the
                               decaying condition (default 5; eliminating them costs
                               ~exp(2 kappa a) in precision) */
    int solver;             /* matching solver: RM_SOLVER_AUTO (default: shared
                               memory up to 96 channels, global memory above),
                               RM_SOLVER_SMALL, RM_SOLVER_LARGE */
    int formulation;        /* mixed-precision formation (Eq. rmatrix on tensor cores):
                               RM_FORM_AUTO (default: pair operand while it is small,
                               per-energy GEMM above), RM_FORM_PAIRS, RM_FORM_ENERGY */
    int solve_precision;    /* steps (c)-(d): RM_FP64 (default) or RM_FP32: the
                               matching system is eliminated in FP32 (partial
                               pivoting) and T = 2(1 - iK)^{-1} - 2 comes from an
                               FP32 complex inversion of 1 - iK, whose error is that
                               of a perturbation of 1 - iK of Frobenius norm
                               <= n_open 2^-24 ||1 - iK||_F; Omega is accumulated in
                               FP64. Shared-memory solver: direct mode only (MQDT
                               runs in FP64). Global-memory solver: direct and MQDT
                               mode (K_u in FP32, the quantum-defect elimination in
                               FP64), up to about 3000 channels (above: FP64) */
    int channel_tables;     /* step (b): 1 builds the per-channel tables
                               (near-threshold interpolation, open- and closed-side
                               Chebyshev expansions; see rm_set_channels) and
                               evaluates pairs from them (to ~1e-12); 0 evaluates
                               every pair by its continued fractions, as
                               rm_k_matrices_noalloc does; -1 (default): 1 with a
                               mixed-precision formation, 0 with FP64 (whose K is
                               meant to match to 1e-9 even where the matching
                               amplifies channel-function errors 1e4-fold) */
    int lanes;              /* number of lanes (default 1, 0 = 1, at most 64): independent
                               streams of work in one context, each with its own
                               workspace and Omega accumulator, sharing the
                               context's partial waves (see rm_lane_solve_energies) */
    int autotune;           /* 1: the mixed-precision formation of each partial wave
                               (pair operand with tiles of 128 energies x 256 pairs
                               and a 2-stage ring, 128 x 128 with 3 or 2 stages, or
                               the per-energy GEMM) is chosen by timing every
                               applicable candidate on the wave's first solve; the
                               choice is kept per (operand type, channels, padded
                               poles, energy-block size) for the whole process, so
                               every context forms R of a wave shape the same way
                               (rm_autotune_info reports it). 0 (default): fixed
                               rules (pair operand up to 192 channels) */
    int pair_tile;          /* pair-operand formation tile: 0 (default) the 128 x 256,
                               2-stage tile or the autotuner's choice; 1, 2, 3 force
                               128 x 256 with 2 stages, 128 x 128 with 3, 128 x 128
                               with 2 */
} rm_opts;

#define RM_SOLVER_AUTO    0
#define RM_SOLVER_SMALL   1
#define RM_SOLVER_LARGE   2

/* Mixed-precision formulations of the formation:
 *   RM_FORM_PAIRS:  one GEMM per block of energies, R_packed[e][ij] =
 *                   sum_k d_k(E_e) (w_ik w_jk / 2a); the pair operand takes
 *                   n(n+1)/2 x N hi/lo elements (at most 4 GB), so it serves
 *                   up to a few hundred channels;
 *   RM_FORM_ENERGY: one GEMM per energy, R(E) = W diag(d(E)) W^T / 2a, with
 *                   the scaled operand formed on the fly; any n up to 8192;
 *                   FP32 accumulation is cut every 4096 poles and the
 *                   segments are summed in FP64. */
#define RM_FORM_AUTO      0
#define RM_FORM_PAIRS     1
#define RM_FORM_ENERGY    2

/* Fills *opts with the defaults above. */
void rm_default_opts(rm_opts *opts);

/* Creates a context on opts->device (opts may be NULL for defaults).
 * Errors: RM_EINVAL (out NULL, bad option), RM_ECUDA. */
int rm_create(rm_ctx **out, const rm_opts *opts);

/* Frees every device buffer the context owns. NULL is a no-op. */
void rm_destroy(rm_ctx *ctx);

/* Loads the inner-region data of partial wave `pw` (0 <= pw < 4096):
 * n_poles pole energies E_k (host, [n_poles]) and surface amplitudes w_ik
 * (Eq. wnk) as W (host, row-major [n_ch][n_poles], W[i*n_poles + k] = w_ik),
 * boundary radius a > 0 and log-derivative b (Eq. match, usually 0).
 * The data are copied to the device (the caller keeps its buffers); poles are
 * stored sorted, which does not change R. Replacing a loaded pw frees its old
 * buffers. Synchronous. Errors: RM_EINVAL (n <= 0, a <= 0, non-finite input),
 * RM_ENOMEM, RM_ECUDA. */
int rm_load_poles(rm_ctx *ctx, int pw, int n_ch, int n_poles, const double *E_k,
                  const double *W, double a, double b);

/* Sets the channels of partial wave `pw`: thresholds e_thr (host, [n_ch], Ry),
 * orbital angular momenta l (host, [n_ch], 0 <= l <= 64), ion charge z >= 0,
 * target level of each channel level (host, [n_ch], 0 <= level < n_levels;
 * channels of one level must share its threshold), and the statistical weight
 * g of the partial wave (e.g. (2J+1)/2). n_ch must equal the loaded n_ch.
 * Closed channels with z = 0 are supported; open channels need z >= 0.
 * For z > 0 the call also computes each channel's near-threshold table: the
 * energy-analytic channel quantities at 16 energies straddling its
 * threshold, from which step (b) interpolates pairs within a few node
 * spacings of the threshold instead of running continued fractions whose
 * length grows as 1/|E - e_i|, and its open-side table: Chebyshev expansions
 * (12 terms) of the channel quantities in k = sqrt(E - e_i) on segments of
 * width 0.9 / a from there to 16 Ry above threshold, and its closed-side
 * table: expansions of the direction of (theta, a theta') in nu on cells of
 * 0.25 (split into up to 16 sub-segments) from 16 Ry below threshold to the
 * near-threshold zone; each is checked against direct values, and pairs are
 * evaluated from a table only where it passed (elsewhere the continued
 * fractions run). rm_opts.channel_tables decides whether any of this is done.
 * rm_load_poles recomputes the tables when the channels are already set.
 * Synchronous. Errors: RM_EINVAL, RM_ENOTLOADED, RM_ENOMEM, RM_ECUDA. */
int rm_set_channels(rm_ctx *ctx, int pw, const double *e_thr, const int *l, double z,
                    const int *level, int n_levels, double g_weight);

/* Outer-region propagation with the long-range multipole potential (Section
 * "Overview": the coupled radial functions are carried by Numerov's method
 * from the inner-region boundary r0 = a to an asymptotic radius r1, where the
 * matching is done; namelist variables ipert and mzpts). In Rydberg units
 * the equations are
 *   u_i'' = sum_j [ (l_i(l_i+1)/r^2 - 2z/r - (E - e_i)) delta_ij + U_ij(r) ] u_j,
 *   U(r) = sum_{lambda=1..lambda_max} A^lambda / r^(lambda+1),
 * A (host, [lambda_max][n_ch][n_ch] row-major, A[((lam-1)*n + i)*n + j] =
 * A^lam_ij, each A^lam exactly symmetric; any unit factor is absorbed into A).
 * The solution matrix Psi with Psi(a) = R(a), a Psi'(a) - b Psi(a) = 1 is
 * carried to r1 >= a by Numerov's method on n_steps equal steps (FP64, one
 * CTA per energy; the first step is started by four Runge-Kutta steps of a
 * quarter step, Psi'(r1) comes from an O(h^4) central formula, and every
 * 1/kappa_max of radius the solution basis is renormalised so that strongly
 * closed channels do not swamp the others), and
 * R(r1) = Psi (r1 Psi' - b Psi)^-1 replaces R in the matching of
 * rm_solve_energies and rm_solve_energies_qdt, whose channel functions (and
 * channel tables) are then taken at r1. The error is O(h^4), h = (r1 - a) /
 * n_steps; the coupling beyond r1 is not included. lambda_max = 0 switches
 * propagation off (A, r1, n_steps ignored). rm_load_poles clears it.
 * rm_form_r still returns R at a. At most 64 channels, 1 <= lambda_max <= 4,
 * and above 16 channels the state (4 n_ch^2 doubles) and A (lambda_max n_ch^2
 * doubles) must fit one CTA's shared memory (227 KB: lambda_max <= 3 at 64
 * channels).
 * An energy whose r1 Psi' - b Psi (or a renormalisation) is singular gets
 * RM_ESINGULAR. Synchronous when the channels are set (their tables are
 * rebuilt for r1). Errors: RM_EINVAL (lambda_max out of range, A NULL,
 * non-finite or not symmetric, r1 < a, n_steps < 2), RM_EUNSUPPORTED
 * (n_ch > 64, or the shared-memory limit above), RM_ENOTLOADED, RM_ENOMEM,
 * RM_ECUDA. */
int rm_set_multipoles(rm_ctx *ctx, int pw, int lambda_max, const double *A, double r1, int n_steps);

/* Solves n_E energies E (host or device, [n_E], Ry) of partial wave `pw` in
 * `mode` (RM_DIRECT or RM_MQDT) and adds g |T|^2 into the context's Omega
 * accumulator. The first call after creation or a reset registers the grid;
 * later calls must pass the same n_E, the same energies and the same n_levels
 * (RM_EGRID otherwise). Optional outputs (NULL to skip), all device:
 *   K_out      [n_E][n_ch*n_ch]: K_ab at K_out[e*n_ch*n_ch + a*n_ch + b],
 *              a, b < n_open[e] (open channels in ascending order)
 *   n_open_out [n_E] number of channels with E > e_i (every energy)
 *   status_out [n_E] per-energy RM_OK / RM_E* (non-negative) codes
 * Asynchronous on the context stream. Errors: RM_EINVAL, RM_ENOTLOADED,
 * RM_EGRID, RM_EUNSUPPORTED, RM_ENOMEM, RM_ECUDA. */
int rm_solve_energies(rm_ctx *ctx, int pw, int n_E, const double *E, int mode,
                      double *K_out, int *n_open_out, int *status_out);

/* MQDT coarse-mesh interpolation (Section "namelist stgf MQDT variables":
 * imode = -1, ieq, qetest, iqdt). Accumulates g |T|^2 into Omega for the
 * n_E fine energies E (HOST array, strictly ascending; registered as the
 * grid like rm_solve_energies) without solving the matching system at each:
 *   1. the fine mesh is cut into segments of consecutive energies with the
 *      same channel classes (open; closed and eliminated by MQDT: nu >=
 *      max(l + nu_margin, fnumin), kappa a <= mqdt_kappa_a_max; other closed);
 *   2. nodes per segment: its first and last energies, plus every |ieq|-th
 *      fine energy (ieq < 0) or the points of the ieq-point grid spanning
 *      [E_0, E_{n_E - 1}] that fall inside it (ieq > 0); nodes where an
 *      eliminated channel has |sin pi nu| < 1e-3, nodes on a pole and nodes
 *      whose solve fails are left out;
 *   3. at every node the unphysical K_u (RM_MQDT channel functions, the
 *      context's formation precision, FP64 matching) is solved, and for
 *      iqdt = 1 turned into S_u = (1 + i K_u)(1 - i K_u)^{-1};
 *   4. at every fine energy K_u (iqdt = 2) or S_u (iqdt = 1) is interpolated
 *      linearly in energy between the nearest nodes of its segment (linearly
 *      extrapolated beyond its outer nodes, constant with one node), at the
 *      last energy that moved more than qetest Ry since the previous
 *      re-interpolation (qetest <= 0: at the energy itself), and the closed
 *      channels are eliminated with nu of the fine energy:
 *        K = K_oo - K_oc (K_cc + tan pi nu)^{-1} K_co, or
 *        S = S_oo - S_oc (S_cc - exp(-2 i pi nu))^{-1} S_co, T = S - 1.
 * n_open_out (device, [n_E], nullable), status_out (device, [n_E], nullable):
 * RM_ETHRESHOLD on a threshold, RM_ESINGULAR where a segment has no usable
 * node or the elimination is singular. At most 96 channels. Synchronises
 * the context stream once (after the node solves).
 * Errors: RM_EINVAL (E on the device, not ascending, ieq = 0, iqdt not 1 or
 * 2), RM_ENOTLOADED, RM_EGRID, RM_EUNSUPPORTED, RM_ENOMEM, RM_ECUDA. */
int rm_solve_energies_qdt(rm_ctx *ctx, int pw, int n_E, const double *E, int ieq, double qetest,
                          int iqdt, int *n_open_out, int *status_out);

/* Inspection of the host planning of rm_solve_energies_qdt (no device work;
 * runs without a GPU): for n_E fine energies E (host, strictly ascending)
 * with channel classes cls (host, [n_E][n_ch] signed char: 0 open, 1
 * eliminated by MQDT, 2 other closed, 3 in every slot of an energy on a
 * threshold), thresholds e_thr (host, [n_ch]), charge z and the sorted pole
 * energies E_k (host, [n_poles]), cuts the segments and places the nodes as
 * rm_solve_energies_qdt does (ieq, qetest; nodes dropped on a pole, within
 * 2.5e-5 max(z^2, 1) Ry of a threshold, or where an eliminated channel has
 * |sin pi nu| < 1e-3) and the interpolation of each fine energy, taking the
 * solve of node k as failed where node_ok[k] == 0 (node_ok: host, [node
 * count], NULL: every node solved; the count is the *n_nodes of a call with
 * NULL). Outputs (host): seg [n_E] (segment, -1
 * on a threshold), e_int [n_E] (interpolation energy, qetest), node_x and
 * node_seg [node_cap] (valid nodes, segment by segment), *n_nodes, node_a,
 * node_b [n_E] (K_u at the energy = (1 - t) node a + t node b; a = b with
 * one node; -1 where the energy has none) and t [n_E]. Errors: RM_EINVAL
 * (NULL or bad sizes, energies not ascending, ieq = 0, more nodes than
 * node_cap). */
int rm_qdt_plan_inspect(int n_ch, const double *e_thr, double z, int n_poles, const double *E_k,
                        int n_E, const double *E, const signed char *cls, int ieq, double qetest,
                        const int *node_ok, int node_cap, int *seg, double *e_int, int *n_nodes,
                        double *node_x, int *node_seg, int *node_a, int *node_b, double *t);

/* Copies the accumulated collision strengths to omega_out (host,
 * [n_E][n_levels*(n_levels+1)/2], upper triangle row-wise: (I, J), I <= J,
 * at I*n_levels - I*(I-1)/2 + (J - I)); entries of levels closed at E are 0.
 * Synchronises the stream. reset != 0 zeroes the accumulator and forgets the
 * grid. omega_out may be NULL (reset only). Errors: RM_EINVAL (no grid yet),
 * RM_ECUDA. */
int rm_collision_strengths(rm_ctx *ctx, double *omega_out, int reset);

/* As rm_collision_strengths, without waiting: the copy of the accumulated
 * collision strengths to omega_out (host, same layout; page-locked memory for
 * the copy to overlap) is enqueued on the context's copy stream after the
 * work already enqueued, and the call returns. omega_out is written
 * asynchronously: the caller must not read or free it before rm_sync.
 * reset != 0 forgets the grid as rm_collision_strengths does, and the next
 * solves accumulate into a second device buffer while this one drains, so
 * that a loop of solve + read-out keeps the GPU busy during the copies; with
 * reset = 0 the next work on the context stream waits for the copy.
 * Errors: RM_EINVAL (no grid yet, omega_out NULL), RM_ECUDA. */
int rm_collision_strengths_async(rm_ctx *ctx, double *omega_out, int reset);

/* Zeroes the Omega accumulator, keeping the registered grid. Asynchronous.
 * Errors: RM_EINVAL (no grid yet), RM_ECUDA. */
int rm_reset_omega(rm_ctx *ctx);

/* Number of energies and of Omega entries per energy of the registered grid
 * (both 0 before the first solve). */
int rm_grid_shape(rm_ctx *ctx, int *n_E, int *n_tri);

/* Inspection of step (b), for tests: channel functions of `pw` at n_E
 * energies E (device). Writes out (device, [n_E][n_ch][4] doubles): open
 * channel {s, s', c, c'}; closed channel {theta, theta', 0, 0} scaled so that
 * theta^2 + (a theta')^2 = 1; and status (device, [n_E], may be NULL).
 * Asynchronous. Errors: RM_EINVAL, RM_ENOTLOADED, RM_ECUDA. */
int rm_channel_functions(rm_ctx *ctx, int pw, int n_E, const double *E, double *out,
                         int *status);

/* Inspection of step (b)'s arithmetic (no counterpart in the paper: it lets
 * a caller account for the work of the continued fractions): for `pw` at
 * n_E energies E (device) in direct mode, writes work (device,
 * [n_E][n_ch][4] ints): {kind, CF1 iterations, CF2 forward iterations n2, l
 * steps}, kind 0 = open (CF1 at l, CF2 at l = 0, l downward and upward
 * recurrence steps), 1 = closed (its CF2 at L0, then l - L0 ladder steps),
 * 3 = near the threshold, interpolated from the channel's node table, 4 =
 * open, from the channel's Chebyshev table, 5 = closed, from the channel's
 * direction table (none of these runs a continued fraction; the l field
 * holds l), -1 = on a threshold. Kinds 3-5 occur only in contexts with
 * channel tables (rm_opts.channel_tables). A CF2 with n2 > 32 is re-evaluated backwards from
 * depth 2 n2 + 20; one with n2 <= 32 is taken from its forward value.
 * Asynchronous. Errors: RM_EINVAL, RM_ENOTLOADED, RM_ECUDA. */
int rm_channel_work(rm_ctx *ctx, int pw, int n_E, const double *E, int *work);

/* Inspection of step (a), for tests: R-matrices of `pw` at n_E energies E
 * (device) at r = a (before any propagation), with the context's formation
 * precision, written to R_out
 * (device, [n_E][n_ch][n_ch], full symmetric matrix). Asynchronous.
 * Errors: RM_EINVAL, RM_ENOTLOADED, RM_ENOMEM, RM_ECUDA. */
int rm_form_r(rm_ctx *ctx, int pw, int n_E, const double *E, double *R_out);

/* Per-phase device timing (tracing). With enable != 0 the context records a
 * CUDA event pair on its stream around every kernel of every phase;
 * rm_profile_get synchronises and returns, for phase p, the number of
 * launches and their summed device time in milliseconds since the last
 * enable. Phases: */
#define RM_PH_NEARPOLE    0   /* near-pole check */
#define RM_PH_CHANFN      1   /* step (b) channel functions */
#define RM_PH_FORM        2   /* step (a) R formation kernel (all precisions) */
#define RM_PH_FIXUP       3   /* step (a) near-pole FP64 terms (mixed precision) */
#define RM_PH_SOLVE       4   /* steps (c)+(d) matching, T, Omega */
#define RM_PH_SPLIT       5   /* step (a) operand split of 1/(E_k - E) (mixed precision) */
#define RM_PH_PROPAGATE   6   /* outer-region propagation a -> r1 (rm_set_multipoles) */
#define RM_PH_COUNT       7
int rm_profile_enable(rm_ctx *ctx, int enable);
int rm_profile_get(rm_ctx *ctx, int phase, int *launches, double *ms);

/* Allocation-free K-matrices (no counterpart in the paper: a deployment
 * convenience). For callers that cannot let the library call cudaMalloc --
 * code whose GPU memory belongs entirely to another allocator, or a
 * latency-bound loop that cannot take the device-wide synchronisation of
 * cudaMalloc/cudaFree. Needs no context; computes, like rm_solve_energies in
 * RM_DIRECT mode with RM_FP64 formation, the open-channel K-matrices of one
 * partial wave at n_E energies, and writes no Omega.
 * Inputs, all device memory of `device`: E_k [n_poles] sorted ascending (the
 * near-pole check assumes it), W [n_ch][n_poles] row-major, e_thr [n_ch],
 * l [n_ch], E [n_E]; scalars z, a, b, eps_thr as in rm_set_channels /
 * rm_load_poles / rm_opts. Outputs (device): K_out [n_E][n_ch*n_ch] (NULL to
 * skip), n_open_out [n_E] (NULL to skip), status_out [n_E] (required).
 * Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default stream).
 * The library allocates nothing for it: its workspace is one static 32 MiB
 * device array per GPU, held from library load until process exit. The
 * first call on a device looks up that array's device address and keeps it
 * for the rest of the process; make that first call before any stream
 * capture, and do not call this entry point on a device after a
 * cudaDeviceReset of it (the kept address belongs to the old context). The
 * call makes `device` current for its own work and restores the caller's
 * current device before it returns. Every call shares the array, so
 * calls whose work overlaps on the GPU (different streams, threads or
 * processes sharing a context) race and must be serialised by the caller.
 * Limits: n_ch <= 96 (RM_EUNSUPPORTED beyond). errbuf (may be NULL) receives
 * a one-line reason on error. Returns RM_SUCCESS, RM_EINVAL,
 * RM_EUNSUPPORTED or RM_ECUDA. */
int rm_k_matrices_noalloc(int device, int n_ch, int n_poles, int n_E, const double *E_k,
                          const double *W, const double *e_thr, const int *l, double z,
                          double a, double b, const double *E, double eps_thr, double *K_out,
                          int *n_open_out, int *status_out, void *stream, char *errbuf,
                          size_t errlen);

/* ---- lanes (no counterpart in the paper: concurrent use of one context) ----
 * A context with rm_opts.lanes = L > 1 has L lanes. Each lane has its own
 * CUDA stream (lane 0's is the context's stream), its own workspace and its
 * own Omega accumulator and registered grid; all lanes share the context's
 * partial waves (poles, amplitudes, channel tables and the tensor-core
 * operands, each built once). Work enqueued on different lanes may overlap on
 * the device. The calls without a lane argument act on lane 0. Loading,
 * replacing or unloading a partial wave while another lane has work on it
 * enqueued is the caller's error. */

/* rm_solve_energies on lane `lane` (0 <= lane < lanes): accumulates into that
 * lane's Omega, on that lane's grid. Asynchronous on the lane's stream.
 * Errors: as rm_solve_energies, RM_EINVAL for a bad lane. */
int rm_lane_solve_energies(rm_ctx *ctx, int lane, int pw, int n_E, const double *E, int mode,
                           double *K_out, int *n_open_out, int *status_out);

/* rm_collision_strengths on lane `lane` (synchronises that lane only). */
int rm_lane_collision_strengths(rm_ctx *ctx, int lane, double *omega_out, int reset);

/* 1 when all work enqueued on the lane by rm_lane_solve_energies /
 * rm_solve_energies has completed, 0 while some is pending (no waiting),
 * negative on error. */
int rm_lane_query(rm_ctx *ctx, int lane);

/* Waits for the lane's stream. */
int rm_lane_sync(rm_ctx *ctx, int lane);

/* The lane's cudaStream_t (NULL for a bad lane or context). */
void *rm_lane_stream(rm_ctx *ctx, int lane);

/* Sizes lane `lane`'s workspace and Omega accumulator for a solve of n_E
 * energies of partial wave `pw` (and builds the wave's tensor-core operands
 * if the context's precision uses them), so that such a solve allocates no
 * device memory; *bytes (may be NULL) receives the lane's device bytes after
 * it. Synchronous. Errors: RM_EINVAL, RM_ENOTLOADED, RM_EUNSUPPORTED,
 * RM_ENOMEM, RM_ECUDA. */
int rm_lane_reserve(rm_ctx *ctx, int lane, int pw, int n_E, size_t *bytes);

/* Device bytes held for partial wave `pw` (poles, amplitudes, channel tables,
 * operands). Errors: RM_EINVAL, RM_ENOTLOADED. */
int rm_pw_bytes(rm_ctx *ctx, int pw, size_t *bytes);

/* Frees the device buffers of partial wave `pw` (it must be loaded again
 * before use). Work already enqueued that reads it completes first
 * (cudaFree synchronises the device). Errors: RM_EINVAL, RM_ENOTLOADED. */
int rm_unload_pw(rm_ctx *ctx, int pw);

/* Batched solve of n_pw partial waves pws (host, [n_pw], distinct, all with
 * the same n_levels) on one energy grid E (host or device, [n_E]) in `mode`,
 * accumulating the sum over the waves of g |T|^2 into the context's Omega
 * (lane 0's accumulator and grid, as rm_solve_energies). Partial waves are
 * independent (Section "Computational details": the energy and partial-wave
 * loops are the parallel ones), so the waves are spread over the context's
 * lanes, largest first to the least-loaded lane (cost ~ n^2 (n_poles + 4 n):
 * formation plus matching), each lane solving its waves one after another
 * while the lanes overlap on the device; the other lanes' accumulators are
 * then added into lane 0's in lane order, so the result is the same every
 * call for a fixed lane count (it differs from one call per wave by the order
 * of the additions only). With use_graph != 0 the whole launch sequence of
 * the call (every lane, their fork and join) is also captured into a CUDA
 * graph, and a later call with the same waves, energies, mode and
 * accumulator replays it with one cudaGraphLaunch; a graph is dropped once
 * any device buffer of the library has been freed or moved since it was
 * captured. With rm_opts.autotune the formation of every wave is chosen
 * before any capture. Lanes other than 0 have their accumulators overwritten.
 * Per-energy statuses are not returned (an energy that fails in a wave adds
 * nothing to Omega). Asynchronous on lane 0's stream. Errors: RM_EINVAL,
 * RM_ENOTLOADED, RM_EGRID, RM_EUNSUPPORTED, RM_ENOMEM, RM_ECUDA. */
int rm_solve_batch(rm_ctx *ctx, int n_pw, const int *pws, int n_E, const double *E, int mode, int use_graph);

/* What the autotuner (rm_opts.autotune) chose for partial wave `pw`:
 * formulation RM_FORM_PAIRS (tile of 128 energies x tile_n pairs, a ring of
 * `stages`) or RM_FORM_ENERGY (tile_n = stages = 0), and ms4 (host, [4],
 * nullable) the measured ms per energy of the candidates: pair 256 x 2, pair
 * 128 x 3, pair 128 x 2, per-energy (-1 where not applicable or taken from
 * an earlier choice for the same shape). Errors: RM_EINVAL (not tuned),
 * RM_ENOTLOADED. */
int rm_autotune_info(rm_ctx *ctx, int pw, int *formulation, int *tile_n, int *stages, double *ms4);

/* Self-test of the bounded device waits (no counterpart in the paper). Every
 * wait of the tensor-core formation kernels on an mbarrier gives up after
 * about 2 s, sets the context's error flag and lets the kernel exit, so that
 * a fault of the pipeline reports RM_ETIMEOUT instead of hanging the GPU.
 * With limit_ns > 0 (at most 10 s), each CTA of those kernels instead first
 * waits, before it allocates tensor memory or issues any copy or MMA, on a
 * barrier that nothing arrives at: the wait gives up after limit_ns, sets the
 * flag and the CTA exits, so no R is formed and the next rm_sync or
 * rm_collision_strengths returns RM_ETIMEOUT (the flag is then cleared).
 * limit_ns = 0 (the default) restores normal operation; the context stays
 * usable. Errors: RM_EINVAL. */
int rm_set_wait_probe(rm_ctx *ctx, unsigned long long limit_ns);

/* Waits for all work enqueued on every lane of the context and for the
 * copies of rm_collision_strengths_async. */
int rm_sync(rm_ctx *ctx);

/* Number of kernels this context has launched since creation. */
long long rm_launch_count(rm_ctx *ctx);

/* Static description of a code (never NULL). */
const char *rm_strerror(int code);

/* One-line description of the last error on ctx (never NULL). */
const char *rm_last_error(rm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* RMGB_H */
