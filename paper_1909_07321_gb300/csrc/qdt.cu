// MQDT coarse-mesh interpolation (Section "namelist stgf MQDT variables":
// imode = -1, a full solution on a coarse mesh and an interpolative
// solution on the fine mesh; ieq, qetest; iqdt = 1 unphysical S matrices,
// iqdt = 2 unphysical K matrices).
//
// The unphysical K_u (open channels and the closed channels of the MQDT set
// carried with the energy-analytic pair f, g) has no closed-channel
// resonances. It is solved at coarse nodes (the ordinary pipeline, stopped
// at K_u), converted to S_u = (1 + i K_u)(1 - i K_u)^{-1} = 2 (1 - i K_u)^{-1}
// - 1 for iqdt = 1, interpolated linearly to each fine energy, and the
// closed channels are eliminated with nu of that energy:
//   iqdt = 1:  S = S_oo - S_oc (S_cc - diag(exp(-2 i pi nu)))^{-1} S_co,
//              |T_ab|^2 = |S_ab - delta_ab|^2;
//   iqdt = 2:  K = K_oo - K_oc (K_cc + diag(tan pi nu))^{-1} K_co, then T.
// Omega_IJ += g sum_{a in I, b in J} |T_ab|^2, one thread per level pair.
//
// The host side here plans segments (runs of fine energies with the same
// channel classes: open / eliminated / decaying), their nodes, and the
// re-interpolation energies (qetest); the weights are set after the node
// solves so that failed nodes are left out.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <set>

#include "dense_smem.cuh"
#include "rm_internal.cuh"

namespace rmgb {

// ---- host planning -------------------------------------------------------------

namespace {

constexpr double QDT_SIN_MIN = 1e-3;
// A node keeps this far (x max(z^2, 1) Ry) from every threshold: nearer, the
// Coulomb continued fractions are so deep that one node would cost more than
// the rest of the mesh (its segment end is extrapolated instead).
constexpr double QDT_NODE_MIN_EPS = 2.5e-5;

double sin_pi(double nu)
{
    const double m = std::nearbyint(nu);
    const double f = nu - m;
    const double s = std::sin(M_PI * f);
    return (std::fmod(std::fabs(m), 2.0) == 0.0) ? s : -s;
}

}  // namespace

int qdt_plan(const QdtChannels &c, const double *E, int n_E, const signed char *cls_all, int ieq,
             double qetest, QdtPlan &pl)
{
    if (ieq == 0 || n_E <= 0) return RM_EINVAL;
    for (int m = 1; m < n_E; ++m)
        if (!(E[m] > E[m - 1])) return RM_EINVAL;
    pl = QdtPlan();
    pl.seg.assign(n_E, -1);
    pl.e_int.assign(E, E + n_E);
    const size_t n = (size_t)c.n;
    int prev = -1;   // previous fine energy off a threshold, if adjacent
    for (int m = 0; m < n_E; ++m) {
        const signed char *cur = cls_all + (size_t)m * n;
        if (cur[0] == QDT_THRESHOLD) {
            prev = -1;
            continue;
        }
        if (prev >= 0 && std::equal(cur, cur + n, cls_all + (size_t)prev * n)) {
            pl.i1.back() = m;
        } else {
            pl.i0.push_back(m);
            pl.i1.push_back(m);
            pl.cls.emplace_back(cur, cur + n);
        }
        pl.seg[m] = (int)pl.i0.size() - 1;
        prev = m;
    }
    // nodes (candidates) and validity
    const double step = (ieq >= 2) ? (E[n_E - 1] - E[0]) / (ieq - 1) : 0.0;
    for (size_t s = 0; s < pl.i0.size(); ++s) {
        const int i0 = pl.i0[s], i1 = pl.i1[s];
        std::set<double> pts = {E[i0], E[i1]};
        if (ieq < 0) {
            for (int m = i0; m <= i1; m += -ieq) pts.insert(E[m]);
        } else {
            for (int j = 0; j < ieq; ++j) {
                const double g = (ieq >= 2) ? E[0] + (double)j * step : E[0];
                if (g > E[i0] && g < E[i1]) pts.insert(g);
            }
        }
        pl.seg_node0.push_back((int)pl.node_x.size());
        const std::vector<signed char> &cx = pl.cls[s];
        for (double x : pts) {
            // between two fine energies of equal classes every energy has those
            // classes (each channel goes decaying -> eliminated -> open as E rises)
            bool bad = false;
            // pole (sorted E_k): the nearest two
            const double *it = std::lower_bound(c.E_k, c.E_k + c.N, x);
            const double tol = 1e-12 * std::fmax(1.0, std::fabs(x));
            if (it != c.E_k + c.N && std::fabs(*it - x) < tol) bad = true;
            if (it != c.E_k && std::fabs(*(it - 1) - x) < tol) bad = true;
            const double near = QDT_NODE_MIN_EPS * std::fmax(c.z * c.z, 1.0);
            for (int i = 0; i < c.n && !bad; ++i)
                if (std::fabs(x - c.e_thr[i]) < near) bad = true;
            // |sin pi nu| of every eliminated channel (with a relative margin, so
            // that the device's own test cannot disagree)
            for (int i = 0; i < c.n && !bad; ++i)
                if (cx[i] == QDT_ELIM) {
                    const double nu = c.z / std::sqrt(c.e_thr[i] - x);
                    if (std::fabs(sin_pi(nu)) < QDT_SIN_MIN * (1.0 + 1e-9)) bad = true;
                }
            if (bad) continue;
            pl.node_x.push_back(x);
            pl.node_seg.push_back((int)s);
        }
        pl.seg_nnodes.push_back((int)pl.node_x.size() - pl.seg_node0.back());
    }
    // re-interpolation energies
    for (size_t s = 0; s < pl.i0.size(); ++s) {
        double last = E[pl.i0[s]];
        for (int m = pl.i0[s]; m <= pl.i1[s]; ++m) {
            if (m == pl.i0[s] || qetest <= 0.0 || E[m] - last > qetest) last = E[m];
            pl.e_int[m] = last;
        }
    }
    return RM_SUCCESS;
}

void qdt_weights(const QdtPlan &pl, const std::vector<int> &node_ok, int n_E, std::vector<QdtFine> &fine)
{
    fine.assign(n_E, QdtFine{0, 0, 0.0, QDT_FLAG_THRESHOLD});
    for (size_t s = 0; s < pl.i0.size(); ++s) {
        std::vector<int> idx;
        for (int k = 0; k < pl.seg_nnodes[s]; ++k)
            if (node_ok[pl.seg_node0[s] + k]) idx.push_back(pl.seg_node0[s] + k);
        for (int m = pl.i0[s]; m <= pl.i1[s]; ++m) {
            QdtFine f{0, 0, 0.0, QDT_FLAG_OK};
            if (idx.empty()) {
                f.flag = QDT_FLAG_NONODE;
            } else if (idx.size() == 1) {
                f.a = f.b = idx[0];
            } else {
                const double x = pl.e_int[m];
                int j = 0;
                while (j + 1 < (int)idx.size() && pl.node_x[idx[j + 1]] <= x) ++j;
                j = std::min(std::max(j, 0), (int)idx.size() - 2);
                f.a = idx[j];
                f.b = idx[j + 1];
                f.t = (x - pl.node_x[f.a]) / (pl.node_x[f.b] - pl.node_x[f.a]);
            }
            fine[m] = f;
        }
    }
}

}  // namespace rmgb

// Inspection of the host planning (no device work): see rmgb.h.
extern "C" int rm_qdt_plan_inspect(int n_ch, const double *e_thr, double z, int n_poles, const double *E_k, int n_E,
                                   const double *E, const signed char *cls, int ieq, double qetest,
                                   const int *node_ok, int node_cap, int *seg, double *e_int, int *n_nodes,
                                   double *node_x, int *node_seg, int *node_a, int *node_b, double *t)
{
    using namespace rmgb;
    if (n_ch <= 0 || n_E <= 0 || n_poles < 0 || node_cap < 0 || !e_thr || !E || !cls || (n_poles > 0 && !E_k) ||
        !seg || !e_int || !n_nodes || (node_cap > 0 && (!node_x || !node_seg)) || !node_a || !node_b || !t)
        return RM_EINVAL;
    if (!std::isfinite(z) || z < 0.0) return RM_EINVAL;
    QdtChannels ch{};
    ch.n = n_ch;
    ch.N = n_poles;
    ch.e_thr = e_thr;
    ch.l = nullptr;
    ch.E_k = E_k;
    ch.z = z;
    QdtPlan pl;
    if (qdt_plan(ch, E, n_E, cls, ieq, qetest, pl) != RM_SUCCESS) return RM_EINVAL;
    const int nn = (int)pl.node_x.size();
    if (nn > node_cap) return RM_EINVAL;
    std::vector<int> ok(nn, 1);
    if (node_ok)
        for (int k = 0; k < nn; ++k) ok[k] = node_ok[k] != 0;
    std::vector<QdtFine> fine;
    qdt_weights(pl, ok, n_E, fine);
    for (int m = 0; m < n_E; ++m) {
        seg[m] = pl.seg[m];
        e_int[m] = pl.e_int[m];
        const bool has = fine[m].flag == QDT_FLAG_OK;
        node_a[m] = has ? fine[m].a : -1;
        node_b[m] = has ? fine[m].b : -1;
        t[m] = has ? fine[m].t : 0.0;
    }
    for (int k = 0; k < nn; ++k) {
        node_x[k] = pl.node_x[k];
        node_seg[k] = pl.node_seg[k];
    }
    *n_nodes = nn;
    return RM_SUCCESS;
}

namespace rmgb {

// ---- device ---------------------------------------------------------------------

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a - b c
__device__ __forceinline__ double2 cfms(double2 a, double2 b, double2 c)
{
    return make_double2(a.x - fma(b.x, c.x, -b.y * c.y), a.y - fma(b.x, c.y, b.y * c.x));
}
__device__ __forceinline__ double2 crcp(double2 a)
{
    const double d = 1.0 / fma(a.x, a.x, a.y * a.y);
    return make_double2(a.x * d, -a.y * d);
}

// Complex Gaussian elimination with partial pivoting of the first `rows`
// columns of the rows x w matrix M (row stride ld). Sets sh->bad on a zero
// or non-finite pivot.
__device__ void cblock_eliminate(double2 *M, int ld, int rows, int w, ElimShared *sh, double2 *pinv_s)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int c = 0; c < rows; ++c) {
        if (warp == 0) {
            double best = -1.0;
            int bi = c;
            for (int r = c + lane; r < rows; r += 32) {
                const double2 v = M[r * ld + c];
                const double a = fma(v.x, v.x, v.y * v.y);
                if (a > best) { best = a; bi = r; }
            }
            for (int off = 16; off > 0; off >>= 1) {
                const double ob = __shfl_down_sync(0xffffffffu, best, off);
                const int oi = __shfl_down_sync(0xffffffffu, bi, off);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (lane == 0) {
                sh->piv = bi;
                const double2 pv = M[bi * ld + c];
                if (!(best > 0.0) || !isfinite(pv.x) || !isfinite(pv.y)) sh->bad = 1;
                *pinv_s = crcp(pv);
            }
        }
        __syncthreads();
        if (sh->bad) return;
        const int p = sh->piv;
        if (p != c) {
            for (int q = c + tid; q < w; q += NT) {
                const double2 t = M[c * ld + q];
                M[c * ld + q] = M[p * ld + q];
                M[p * ld + q] = t;
            }
            __syncthreads();
        }
        constexpr int G = 4;
        const double2 pinv = *pinv_s;
        const int nr = rows - c - 1;
        const double2 *prow = M + c * ld;
        for (int q = tid; q < nr * G; q += NT) {
            const int r = c + 1 + q / G, j = q - (q / G) * G;
            double2 *row = M + r * ld;
            const double2 f = cmul(row[c], pinv);
            for (int cc = c + 1 + j; cc < w; cc += G) row[cc] = cfms(row[cc], f, prow[cc]);
        }
        __syncthreads();
    }
}

__device__ void cblock_backsub(double2 *M, int ld, int rows, int rhs0, int n_rhs)
{
    for (int qq = threadIdx.x; qq < n_rhs; qq += NT) {
        const int cq = rhs0 + qq;
        for (int t = rows - 1; t >= 0; --t) {
            double2 s = M[t * ld + cq];
            for (int u = t + 1; u < rows; ++u) s = cfms(s, M[t * ld + u], M[u * ld + cq]);
            M[t * ld + cq] = cmul(s, crcp(M[t * ld + t]));
        }
    }
    __syncthreads();
}

// Node K_u -> S_u = 2 (1 - i K_u)^{-1} - 1: one CTA per node, [A | I] eliminated.
__global__ void __launch_bounds__(NT) qdt_s_from_k_kernel(int n, const double *__restrict__ Ku,
                                                         const int *__restrict__ np_node,
                                                         int *__restrict__ status,
                                                         double2 *__restrict__ Su)
{
    extern __shared__ double2 smc[];
    __shared__ ElimShared esh;
    __shared__ double2 pinv_s;
    const int k = blockIdx.x, tid = threadIdx.x;
    if (status[k] != RM_OK) return;
    const int m = np_node[k];
    const int w = 2 * m, ld = w + 1;
    const double *K = Ku + (size_t)k * n * n;
    if (tid == 0) esh.bad = 0;
    for (int q = tid; q < m * w; q += NT) {
        const int r = q / w, c = q - (q / w) * w;
        double2 v;
        if (c < m) v = make_double2(r == c ? 1.0 : 0.0, -K[(size_t)r * n + c]);
        else v = make_double2(r == c - m ? 1.0 : 0.0, 0.0);
        smc[r * ld + c] = v;
    }
    __syncthreads();
    cblock_eliminate(smc, ld, m, w, &esh, &pinv_s);
    if (esh.bad) {   // an unusable node: left out through its status
        if (tid == 0) status[k] = RM_ESINGULAR;
        return;
    }
    cblock_backsub(smc, ld, m, m, m);
    double2 *S = Su + (size_t)k * n * n;
    for (int q = tid; q < m * m; q += NT) {
        const int r = q / m, c = q - (q / m) * m;
        const double2 v = smc[r * ld + m + c];
        S[(size_t)r * n + c] = make_double2(2.0 * v.x - (r == c ? 1.0 : 0.0), 2.0 * v.y);
    }
}

// Fine energies: one CTA each.
template <int IQDT>
__global__ void __launch_bounds__(NT) qdt_fine_kernel(PwDev pw, const double *__restrict__ E, Opts o,
                                                      const QdtFine *__restrict__ fine,
                                                      const double *__restrict__ Ku,
                                                      const double2 *__restrict__ Su,
                                                      const int *__restrict__ node_status,
                                                      int *__restrict__ status, int *__restrict__ n_open_out,
                                                      double *__restrict__ omega, int n_tri)
{
    extern __shared__ double sm[];
    __shared__ int pch[SOLVE_SMALL_MAXN];       // P position -> channel
    __shared__ int open_pos[SOLVE_SMALL_MAXN];  // channel -> open position (-1 otherwise)
    __shared__ int qpos[SOLVE_SMALL_MAXN], opos[SOLVE_SMALL_MAXN];
    __shared__ double vtan[SOLVE_SMALL_MAXN];
    __shared__ double2 dq[SOLVE_SMALL_MAXN];
    __shared__ int s_np, s_no, s_nq, s_flag;
    __shared__ ElimShared esh;
    __shared__ double2 pinv_s;
    const int e = blockIdx.x, tid = threadIdx.x;
    const int n = pw.n;
    const double x = E[e];
    const QdtFine f = fine[e];
    if (tid == 0) {
        int no_all = 0;
        for (int i = 0; i < n; ++i) no_all += (x - pw.e_thr[i] > 0.0);
        if (n_open_out) n_open_out[e] = no_all;
        int flag = f.flag;
        if (flag == QDT_FLAG_OK && (node_status[f.a] != RM_OK || node_status[f.b] != RM_OK))
            flag = QDT_FLAG_NONODE;
        int np = 0, no = 0, nq = 0;
        for (int i = 0; i < n && flag == QDT_FLAG_OK; ++i) {
            const double eps = x - pw.e_thr[i];
            open_pos[i] = -1;
            if (eps > 0.0) {
                open_pos[i] = no;
                opos[no++] = np;
                pch[np++] = i;
            } else if (pw.z > 0.0) {
                const double kap = sqrt(-eps);
                const double nu = pw.z / kap;
                if (nu >= fmax(pw.l[i] + o.nu_margin, o.fnumin) && kap * pw.a <= o.kappa_a_max) {
                    double sb, cb;
                    sincospi(nu, &sb, &cb);
                    vtan[nq] = sb / cb;
                    dq[nq] = make_double2(cb * cb - sb * sb, -2.0 * sb * cb);   // exp(-2 i pi nu)
                    qpos[nq++] = np;
                    pch[np++] = i;
                }
            }
        }
        s_np = np;
        s_no = no;
        s_nq = nq;
        s_flag = flag;
        esh.bad = 0;
        if (flag == QDT_FLAG_THRESHOLD) status[e] = RM_ETHRESHOLD;
        if (flag == QDT_FLAG_NONODE) status[e] = RM_ESINGULAR;
    }
    __syncthreads();
    if (s_flag != QDT_FLAG_OK || s_no == 0) return;
    const int np = s_np, no = s_no, nq = s_nq;
    const double t = f.t, u = 1.0 - t;
    const size_t nn = (size_t)n * n;
    const double g = pw.g;
    const int nl = pw.n_levels;
    const int npair = nl * (nl + 1) / 2;
    double *om = omega + (size_t)e * n_tri;
    if (IQDT == 2) {
        // K_u(E) in region B, then the real elimination and the T step
        const int lu = np + 1;
        double *Kb = sm + (size_t)2 * n * (n + 1);
        const double *KA = Ku + f.a * nn, *KB = Ku + f.b * nn;
        for (int q = tid; q < np * np; q += NT) {
            const int p = q / np, r = q - (q / np) * np;
            Kb[p * lu + r] = u * KA[(size_t)p * n + r] + t * KB[(size_t)p * n + r];
        }
        __syncthreads();
        const int lk = no + 1;
        if (nq == 0) {
            for (int q = tid; q < no * no; q += NT) {   // np = no: symmetrise into stride lk
                const int p = q / no, r = q - (q / no) * no;
                sm[p * lk + r] = 0.5 * (Kb[p * lu + r] + Kb[r * lu + p]);
            }
            __syncthreads();
            for (int q = tid; q < no * no; q += NT) {
                const int p = q / no, r = q - (q / no) * no;
                Kb[p * lk + r] = sm[p * lk + r];
            }
            __syncthreads();
        } else if (!mqdt_eliminate(Kb, lu, no, nq, qpos, opos, vtan, sm, Kb, nullptr, 0, &esh)) {
            if (tid == 0) status[e] = RM_ESINGULAR;
            return;
        }
        if (!t_omega(pw, x, Kb, lk, sm, lk, no, open_pos, vtan, om, &esh)) {
            if (tid == 0) status[e] = RM_ESINGULAR;
            return;
        }
        return;
    }
    // iqdt = 1: S-form elimination; S_ab formed where it is summed
    const double2 *SA = Su + f.a * nn, *SB = Su + f.b * nn;
    auto su = [&](int p, int r) {
        const double2 a = SA[(size_t)p * n + r], b = SB[(size_t)p * n + r];
        return make_double2(u * a.x + t * b.x, u * a.y + t * b.y);
    };
    const int w2 = nq + no, ld2 = w2 + 1;
    double2 *C = reinterpret_cast<double2 *>(sm);
    if (nq > 0) {
        for (int q = tid; q < nq * w2; q += NT) {
            const int i = q / w2, j = q - (q / w2) * w2;
            double2 v;
            if (j < nq) {
                v = su(qpos[i], qpos[j]);
                if (i == j) v = make_double2(v.x - dq[i].x, v.y - dq[i].y);
            } else {
                v = su(qpos[i], opos[j - nq]);
            }
            C[i * ld2 + j] = v;
        }
        __syncthreads();
        cblock_eliminate(C, ld2, nq, w2, &esh, &pinv_s);
        if (esh.bad) {
            if (tid == 0) status[e] = RM_ESINGULAR;
            return;
        }
        cblock_backsub(C, ld2, nq, nq, no);   // Y = (S_cc - D)^{-1} S_co
    }
    for (int q = tid; q < npair; q += NT) {
        int I, J;
        tri_pair(q, nl, I, J);
        if (!(x - pw.lev_thr[I] > 0.0) || !(x - pw.lev_thr[J] > 0.0)) continue;
        double s = 0.0;
        for (int ia = pw.lev_start[I]; ia < pw.lev_start[I + 1]; ++ia) {
            const int a = open_pos[pw.lev_chan[ia]];
            for (int ib = pw.lev_start[J]; ib < pw.lev_start[J + 1]; ++ib) {
                const int b = open_pos[pw.lev_chan[ib]];
                double2 v = su(opos[a], opos[b]);
                for (int i = 0; i < nq; ++i) v = cfms(v, su(opos[a], qpos[i]), C[i * ld2 + nq + b]);
                if (a == b) v.x -= 1.0;
                s += fma(v.x, v.x, v.y * v.y);
            }
        }
        om[q] += g * s;
    }
}

// Channel classes of every (energy, channel): QDT_OPEN, QDT_ELIM (the
// channel kernel's MQDT rules without its |sin pi nu| guard), QDT_DECAY; an
// energy on a threshold gets QDT_THRESHOLD in its first entry.
__global__ void qdt_class_kernel(PwDev pw, const double *__restrict__ E, int nE, Opts o,
                                 signed char *__restrict__ cls)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nE) return;
    const double x = E[e];
    signed char *row = cls + (size_t)e * pw.n;
    bool thr = false;
    for (int i = 0; i < pw.n; ++i) {
        const double eps = x - pw.e_thr[i];
        signed char c = QDT_DECAY;
        if (fabs(eps) < o.eps_thr) thr = true;
        if (eps > 0.0) {
            c = QDT_OPEN;
        } else if (pw.z > 0.0) {
            const double kap = sqrt(-eps);
            const double nu = pw.z / kap;
            if (nu >= fmax(pw.l[i] + o.nu_margin, o.fnumin) && kap * pw.a <= o.kappa_a_max) c = QDT_ELIM;
        }
        row[i] = c;
    }
    if (thr) row[0] = QDT_THRESHOLD;
}

}  // namespace

cudaError_t launch_qdt_classes(const PwDev &pw, const double *E, int nE, const Opts &o, signed char *cls,
                               cudaStream_t s)
{
    if (nE == 0) return cudaSuccess;
    qdt_class_kernel<<<(nE + 127) / 128, 128, 0, s>>>(pw, E, nE, o, cls);
    return cudaGetLastError();
}

size_t qdt_s_smem(int n) { return (size_t)n * (2 * n + 1) * sizeof(double2); }

cudaError_t launch_qdt_s_from_k(int n, int n_nodes, const double *Ku, const int *np_node, int *status,
                                double2 *Su, cudaStream_t s)
{
    if (n_nodes == 0) return cudaSuccess;
    const size_t smem = qdt_s_smem(n);
    cudaError_t e = cudaFuncSetAttribute(qdt_s_from_k_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    qdt_s_from_k_kernel<<<n_nodes, NT, smem, s>>>(n, Ku, np_node, status, Su);
    return cudaGetLastError();
}

cudaError_t launch_qdt_fine(int iqdt, const PwDev &pw, const double *E, int nE, const Opts &o,
                            const QdtFine *fine, const double *Ku, const double2 *Su, const int *node_status,
                            int *status, int *n_open_out, double *omega, int n_tri, cudaStream_t s)
{
    if (nE == 0) return cudaSuccess;
    if (pw.n > SOLVE_SMALL_MAXN) return cudaErrorInvalidValue;
    cudaError_t e;
    if (iqdt == 2) {
        const size_t smem = (size_t)3 * pw.n * (pw.n + 1) * sizeof(double);
        e = cudaFuncSetAttribute(qdt_fine_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        qdt_fine_kernel<2><<<nE, NT, smem, s>>>(pw, E, o, fine, Ku, Su, node_status, status, n_open_out, omega,
                                                n_tri);
    } else {
        const size_t smem = (size_t)pw.n * (pw.n + 1) * sizeof(double2);
        e = cudaFuncSetAttribute(qdt_fine_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        qdt_fine_kernel<1><<<nE, NT, smem, s>>>(pw, E, o, fine, Ku, Su, node_status, status, n_open_out, omega,
                                                n_tri);
    }
    return cudaGetLastError();
}

}  // namespace rmgb
