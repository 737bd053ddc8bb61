/*
 * ORACLE -- test infrastructure only.  Only tests/, __graft_entry__.smoke()
 * and bench.py's CPU-baseline leg may load this code; the product path never
 * does.  It shares no source with the CUDA library.
 *
 * One kinetic step of source iteration for the steady gray RTE: for every
 * discrete ordinate, the cell-centred finite-volume transport equation with
 * first-order upwind face values is solved exactly by visiting cells in
 * upwind order, then the angular moments are summed in direction-index order.
 *
 *   Eq. (RTE_d) with 1/(c dt) = 0 (steady) and the right-hand side written as
 *   sigma_t I - S, S = (sigma_s rho^m + q)/(4 pi)  (Eq. (RTE_SI), Sec. 2.2):
 *       sigma_t I_i + (1/V_i) sum_j I_ij (Omega . A_ij) = S_i
 *   Eq. (Iij) with psi = 0: I_ij = I_i if Omega.n_ij >= 0, else I_j
 *   (or the boundary inflow, Eq. (micro_bc) with alpha_w = 0).
 *   Moments, Eqs. (def_rho), (def_F), (RTE_M0): rho = sum w I,
 *   F = sum w Omega I, P = sum w Omega Omega I (Sec. 4.1 quadrature sum).
 *   Boundary kinetic flux F_iw . n = sum_k w_k (Omega_k . n) I_iw,k
 *   (Sec. 4.4, F_iw^init).
 *
 * With a pseudo-time shift (Sec. 4.3) the step is the paper's delta form:
 * the UW1 residual at the stored I^m (Eq. (RTE_d_res)), then the lower-
 * triangular increment system with the shifted diagonal (Eqs. (RTE_d_mtx),
 * (elem_main_shifted)) solved in upwind order, and I^{m+1/2} = I^m + dI.
 *
 * Plain FP64, plain loops, no blocking.  Built twice from this one file: plain
 * (the oracle the tests use) and with -fopenmp (the same arithmetic in the
 * same order, the ordinates on all host cores; only for timing the oracle).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* boundary face numbering: W j, E ny+j, S 2ny+i, N 2ny+nx+i */

/* neighbour across face f (0 W, 1 E, 2 S, 3 N) of cell (i,j), or -1 */
static int neighbour(int nx, int ny, int i, int j, int f)
{
    const int c = i + nx * j;
    if (f == 0) return i > 0 ? c - 1 : -1;
    if (f == 1) return i < nx - 1 ? c + 1 : -1;
    if (f == 2) return j > 0 ? c - nx : -1;
    return j < ny - 1 ? c + nx : -1;
}

/* boundary face number across face f of cell (i,j) (only on the boundary) */
static int bface(int nx, int ny, int i, int j, int f)
{
    if (f == 0) return j;
    if (f == 1) return ny + j;
    if (f == 2) return 2 * ny + i;
    return 2 * ny + nx + i;
}

/* upwind value across face f: the neighbour's intensity, or the inflow
   (Eq. (micro_bc) with alpha_w = 0; vacuum when inflow is NULL) */
static double upwind(const double* Ik, const double* inflow, int nx, int ny, int K, int k,
                     int i, int j, int f)
{
    const int nb = neighbour(nx, ny, i, j, f);
    if (nb >= 0) return Ik[nb];
    return inflow ? inflow[(size_t)bface(nx, ny, i, j, f) * K + k] : 0.0;
}

/* The intensities of ordinate k (I, [N]) by one exact upwind sweep, or in
   the delta form when shift is given (dI: [N] scratch). */
static void sweep_ordinate(int nx, int ny, const double* dx, const double* dy, int K, int k,
                           double m, double e, const double* sigma_t, const double* S,
                           const double* inflow, const double* shift, const double* I_prev,
                           double* I, double* dI)
{
    const int N = nx * ny;
    /* upwind visiting order: a cell is visited after the neighbours whose
       shared face has Omega.n < 0 seen from this cell */
    const int i0 = (m >= 0.0) ? 0 : nx - 1, di = (m >= 0.0) ? 1 : -1;
    const int j0 = (e >= 0.0) ? 0 : ny - 1, dj = (e >= 0.0) ? 1 : -1;
    for (int jj = 0; jj < ny; ++jj) {
        const int j = j0 + dj * jj;
        for (int ii = 0; ii < nx; ++ii) {
            const int i = i0 + di * ii;
            const int c = i + nx * j;
            const double V = dx[i] * dy[j];
            /* the four faces: outward normal and area */
            const double An[4] = {dy[j], dy[j], dx[i], dx[i]};   /* W E S N */
            const double on[4] = {-m, m, -e, e};                 /* Omega . n */
            if (!shift) {
                /* exact solve of the cell equation given the upwind values */
                double diag = sigma_t[c];
                double rhs = S[c];
                for (int f = 0; f < 4; ++f) {
                    const double oa = on[f] * An[f];   /* Omega . A_ij */
                    if (on[f] >= 0.0) {
                        diag += oa / V;                 /* outflow: I_ij = I_i */
                    } else {
                        rhs -= oa / V * upwind(I, inflow, nx, ny, K, k, i, j, f);
                    }
                }
                I[c] = rhs / diag;
            } else {
                /* delta form with the pseudo-time shift (Eqs. (RTE_d_increment),
                   (delta_Iij), (RTE_d_res), (RTE_d_mtx), (elem_main_shifted)):
                   residual of the UW1 equation at I^m, then
                   d_ii dI_i + sum_{inflow j} d_ij dI_j = r_i, I^{m+1/2} = I^m + dI */
                const double* Im = I_prev + (size_t)k * N;
                double r = S[c] - sigma_t[c] * Im[c];
                double dii = shift[c] + sigma_t[c];
                double lower = 0.0;
                for (int f = 0; f < 4; ++f) {
                    const double oa = on[f] * An[f];
                    if (on[f] >= 0.0) {
                        r -= oa / V * Im[c];
                        dii += oa / V;
                    } else {
                        r -= oa / V * upwind(Im, inflow, nx, ny, K, k, i, j, f);
                        /* d_ij dI_j with dI on an inflow boundary face = 0 */
                        const int nb = neighbour(nx, ny, i, j, f);
                        if (nb >= 0) lower += oa / V * dI[nb];
                    }
                }
                dI[c] = (r - lower) / dii;
                I[c] = Im[c] + dI[c];
            }
        }
    }
}

/*
 * The ordinates are independent: with -fopenmp they are swept in parallel
 * (one ordinate per task), and every moment and boundary-flux sum then runs
 * per cell / per face over the ordinates in index order, so the results do
 * not depend on the thread count (and equal the single-threaded build's).
 */
int oracle_sweep(int nx, int ny, const double* dx, const double* dy, int K,
                 const double* mu, const double* eta, const double* w,
                 const double* sigma_t, const double* S, const double* inflow,
                 const double* shift, const double* I_prev,
                 double* I_out, double* rho, double* Fx, double* Fy,
                 double* Pxx, double* Pxy, double* Pyy, double* fb)
{
    const int N = nx * ny;
    const int nbf = 2 * (nx + ny);
    /* every ordinate's intensities: the caller's I_out, else scratch */
    double* Iall = I_out ? I_out : (double*)malloc(sizeof(double) * (size_t)K * (size_t)N);
    if (!Iall) return -1;
    int failed = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < K; ++k) {
        double* dI = shift ? (double*)malloc(sizeof(double) * (size_t)N) : NULL;
        if (shift && !dI) {
#pragma omp atomic write
            failed = 1;
            continue;
        }
        sweep_ordinate(nx, ny, dx, dy, K, k, mu[k], eta[k], sigma_t, S, inflow, shift, I_prev,
                       Iall + (size_t)k * N, dI);
        free(dI);
    }
    if (failed) {
        if (!I_out) free(Iall);
        return -1;
    }
#pragma omp parallel for
    for (int c = 0; c < N; ++c) {
        double r = 0.0, fx = 0.0, fy = 0.0, pxx = 0.0, pxy = 0.0, pyy = 0.0;
        for (int k = 0; k < K; ++k) {
            const double m = mu[k], e = eta[k], I = Iall[(size_t)k * N + c];
            r += w[k] * I;
            fx += w[k] * m * I;
            fy += w[k] * e * I;
            pxx += w[k] * m * m * I;
            pxy += w[k] * m * e * I;
            pyy += w[k] * e * e * I;
        }
        rho[c] = r; Fx[c] = fx; Fy[c] = fy;
        Pxx[c] = pxx; Pxy[c] = pxy; Pyy[c] = pyy;
    }
    /* boundary faces: outgoing uses the boundary cell, incoming the inflow */
#pragma omp parallel for
    for (int f = 0; f < nbf; ++f) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k) {
            const double m = mu[k], e = eta[k];
            const double* I = Iall + (size_t)k * N;
            int c; double on;
            if (f < ny) { c = nx * f; on = -m; }
            else if (f < 2 * ny) { c = (nx - 1) + nx * (f - ny); on = m; }
            else if (f < 2 * ny + nx) { c = f - 2 * ny; on = -e; }
            else { c = (f - 2 * ny - nx) + nx * (ny - 1); on = e; }
            const double Iface = (on >= 0.0) ? I[c] : (inflow ? inflow[(size_t)f * K + k] : 0.0);
            acc += w[k] * on * Iface;
        }
        fb[f] = acc;
    }
    if (!I_out) free(Iall);
    return 0;
}

/* Threads the OpenMP build uses (1 without OpenMP). */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Transposed kinetic operator (adjoint of the kinetic step).  The sweep above
 * solves, for each ordinate k, the lower-triangular system A_k I_k = S with
 *   (A_k)_cc = sigma_t,c + sum_{faces f of c, Omega.n >= 0} (Omega.n A_f)/V_c,
 *   (A_k)_cn = (Omega.n_f A_f)/V_c  for the inflow faces f (Omega.n < 0) of c,
 *   n the neighbour across f.
 * This routine solves A_k^T phi_k = psi_k: row n of A_k^T couples n to the
 * cells c that take n as an upwind neighbour, i.e. the neighbours across the
 * faces of n with Omega.n_f > 0, with the coefficient -(Omega.n_f A_f)/V_c
 * seen from n.  Those cells come after n in upwind order, so the system is
 * solved by visiting the cells in reverse upwind order.  psi and phi are
 * [K][N]; there is no boundary term (inflow enters the forward problem as a
 * source, not through A_k).
 */
int oracle_sweep_transposed(int nx, int ny, const double* dx, const double* dy, int K,
                            const double* mu, const double* eta, const double* sigma_t,
                            const double* psi, double* phi)
{
    const int N = nx * ny;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < K; ++k) {
        const double m = mu[k], e = eta[k];
        const double* pk = psi + (size_t)k * N;
        double* fk = phi + (size_t)k * N;
        const int i0 = (m >= 0.0) ? 0 : nx - 1, di = (m >= 0.0) ? 1 : -1;
        const int j0 = (e >= 0.0) ? 0 : ny - 1, dj = (e >= 0.0) ? 1 : -1;
        for (int jj = ny - 1; jj >= 0; --jj) {
            const int j = j0 + dj * jj;
            for (int ii = nx - 1; ii >= 0; --ii) {
                const int i = i0 + di * ii;
                const int n = i + nx * j;
                const double V = dx[i] * dy[j];
                const double An[4] = {dy[j], dy[j], dx[i], dx[i]};   /* W E S N */
                const double on[4] = {-m, m, -e, e};                 /* Omega . n */
                double diag = sigma_t[n];
                double rhs = pk[n];
                for (int f = 0; f < 4; ++f) {
                    if (on[f] >= 0.0) diag += on[f] * An[f] / V;
                    if (on[f] > 0.0) {
                        const int c = neighbour(nx, ny, i, j, f);
                        if (c >= 0) {
                            const int ic = c % nx, jc = c / nx;
                            rhs += on[f] * An[f] / (dx[ic] * dy[jc]) * fk[c];
                        }
                    }
                }
                fk[n] = rhs / diag;
            }
        }
    }
    return 0;
}

/*
 * Increment system of the delta form (Sec. 4.1, Eqs. (RTE_d_increment),
 * (delta_Iij), (RTE_d_mtx), (elem_mtx); Sec. 4.3, Eq. (elem_main_shifted)):
 * for every ordinate k,
 *   d_ii dI_i + sum_{faces f of i with Omega.n < 0, neighbour j} d_ij dI_j = R_i,
 *   d_ii = shift_i + sigma_t,i + sum_{Omega.n >= 0} (Omega.n A_f)/V_i,
 *   d_ij = (Omega.n_f A_f)/V_i,
 * first-order upwind increments with dI = 0 on inflow faces (the inflow is
 * fixed), solved by visiting the cells in upwind order.  R and dI are [K][N]
 * (R per unit volume); shift may be NULL.
 */
int oracle_sweep_delta(int nx, int ny, const double* dx, const double* dy, int K,
                       const double* mu, const double* eta, const double* sigma_t,
                       const double* shift, const double* R, double* dI)
{
    const int N = nx * ny;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < K; ++k) {
        const double m = mu[k], e = eta[k];
        const double* Rk = R + (size_t)k * N;
        double* dk = dI + (size_t)k * N;
        const int i0 = (m >= 0.0) ? 0 : nx - 1, di = (m >= 0.0) ? 1 : -1;
        const int j0 = (e >= 0.0) ? 0 : ny - 1, dj = (e >= 0.0) ? 1 : -1;
        for (int jj = 0; jj < ny; ++jj) {
            const int j = j0 + dj * jj;
            for (int ii = 0; ii < nx; ++ii) {
                const int i = i0 + di * ii;
                const int c = i + nx * j;
                const double V = dx[i] * dy[j];
                const double An[4] = {dy[j], dy[j], dx[i], dx[i]};   /* W E S N */
                const double on[4] = {-m, m, -e, e};                 /* Omega . n */
                double dii = sigma_t[c] + (shift ? shift[c] : 0.0);
                double lower = 0.0;
                for (int f = 0; f < 4; ++f) {
                    const double oa = on[f] * An[f];
                    if (on[f] >= 0.0) {
                        dii += oa / V;
                    } else {
                        const int nb = neighbour(nx, ny, i, j, f);
                        if (nb >= 0) lower += oa / V * dk[nb];
                    }
                }
                dk[c] = (Rk[c] - lower) / dii;
            }
        }
    }
    return 0;
}
