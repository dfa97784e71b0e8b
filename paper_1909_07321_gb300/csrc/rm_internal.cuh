// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rmgb.h"

namespace rmgb {

// Boundary data of one channel at one energy (step (b)).
//   open:   (gh, ghp) = (c, c'),  (s, sp) = (s, s')   energy-normalised Coulomb
//   closed: (gh, ghp) = (theta, theta') with theta^2 + (a theta')^2 = 1, s = sp = 0
struct __align__(16) ChanFn {
    double gh, ghp, s, sp;
};

// MQDT extra data of a closed channel (only filled in MQDT mode):
//   q != 0 marks a channel eliminated by quantum-defect theory; then
//   (f, fp) replaces (s, s'), (g, gp) replaces (theta, theta'), tanb = tan(pi nu).
struct __align__(16) MqdtFn {
    double f, fp, g, gp, tanb;
    int q;
    int pad;
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
};

struct Opts {
    double eps_thr, delta_pole, fnumin, nu_margin;
};

// ---- launchers (each returns cudaGetLastError() of its launch) ----------

cudaError_t launch_chanfn(const PwDev &pw, const double *E, int nE, const Opts &o, int mqdt,
                          ChanFn *cf, MqdtFn *mq, int *status, cudaStream_t s);
cudaError_t launch_nearpole(const PwDev &pw, const double *E, int nE, int *status,
                            cudaStream_t s);
cudaError_t launch_form_r_fp64(const PwDev &pw, const double *E, int nE, double *R,
                               cudaStream_t s);
cudaError_t launch_solve_small(const PwDev &pw, const double *E, int nE, const ChanFn *cf,
                               const MqdtFn *mq, const double *R, int mqdt, int *status,
                               double *K_out, int *n_open_out, double *omega, int n_tri,
                               cudaStream_t s);
cudaError_t launch_chanfn_export(const PwDev &pw, const double *E, int nE, const ChanFn *cf,
                                 double *out, cudaStream_t s);

// Largest channel count the shared-memory solver takes.
int solve_small_max_n();

}  // namespace rmgb
