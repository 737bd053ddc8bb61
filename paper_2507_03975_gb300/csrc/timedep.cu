// Time-dependent gray radiation-material problem (gsis_td_solve): backward
// Euler in time (Sec. 4.1, Eq. (RTE_d)), emission phi = a c T^4 (Sec. 2.1,
// Eqs. (RTE_g), (Tm_g)), inner iterations by GSIS or by SI with the
// Fleck-Cummings linearisation.
//
// Kinetic step (Eqs. (RTE_g_semi), (RTE_d_res)): the steady sweep in its
// delta form with the diagonal shift 1/(c dt) and the stored intensities
// I^n of the previous step as I_old:
//   (1/(c dt) + sigma_t) I^{m+1/2} + upwind = S + I^n/(c dt),
// I^n = In + cn (the isotropic correction of Eq. (GSIS_update) of the last
// iterate is kept per cell and enters the source as cn/(c dt)).
//
// GSIS (Eqs. (GSIS_dse), (MSE_d), (Tm_d), (MSE_d1), (MSE_d2)): per iteration
// one Newton step of the macroscopic rho-T system about T^m, T eliminated
// cell by cell: kappa = 4 a c T^3, D2 = C_v/dt + kappa sigma_a, f = (C_v/dt)/D2,
//   [D_steady + V (1/(c dt) + f sigma_a - sigma_a)] rho^{m+1} = b_steady with
//   q -> q + rho^n/(c dt) + f sigma_a (phi^m + kappa (T^n - T^m)),
//   T^{m+1} = T^n + sigma_a (rho^{m+1} - phi^m + kappa (T^m - T^n)) / D2.
// SI (Eqs. (Tm_semi_linear), (RTE_SI), (arti_sigmaT), (SI_update)):
//   S = ((sigma_s + (1 - f_n) sigma_a) rho^m + f_n sigma_a phi^n + q)/4pi,
//   at the end of the step T^{n+1} = ((1 - f_n) rho + f_n phi^n + 3 phi^n)/kappa_n.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "gsis.h"
#include "gsis_internal.cuh"
#include "host.h"

using namespace gsis;

namespace {

constexpr double kInvFourPi = 0.079577471545947667884441881686257;   // 1 / (4 pi)

struct TdArgs {
    int nx, ny, N;
    const double* dx; const double* dy;
    const double* sigma_a; const double* sigma_s; const double* q;
    double* rho_m;                // rho^m -> rho^{m+1}
    const double* rho_h;          // rho^{m+1/2}
    const double* x;              // synthetic solution (GSIS)
    double* T; double* T_n; double* rho_n;
    double* cn; double* cnext;
    double* qeff; double* diag; const double* diag0;
    double* src; float* src_f;
    double inv_cdt, ac, cv_dt;    // 1/(c dt), a c, C_v / dt
    int gsis;
    double* partials; double* hist; Status* status;
    double tol; int fixed_iters, max_iter;
};

int grid_for(long long n, int block, int cap)
{
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

__device__ __forceinline__ double pow4(double t)
{
    const double t2 = t * t;
    return t2 * t2;
}

// Angular source of the kinetic step from (rho, T) and the correction cn.
__device__ __forceinline__ double td_source(const TdArgs& a, int c, double rho, double T)
{
    const double sa = a.sigma_a[c];
    double s;
    if (a.gsis) {
        s = fma(a.sigma_s[c], rho, fma(sa, a.ac * pow4(T), a.q[c]));
    } else {   // Fleck-Cummings about T^n
        const double Tn = a.T_n[c];
        const double kap = 4.0 * a.ac * Tn * Tn * Tn;
        const double f = a.cv_dt / (a.cv_dt + kap * sa);
        s = fma(a.sigma_s[c] + (1.0 - f) * sa, rho, fma(f * sa, a.ac * pow4(Tn), a.q[c]));
    }
    return fma(s, kInvFourPi, a.inv_cdt * a.cn[c]);
}

__device__ __forceinline__ void put_source(const TdArgs& a, int c, double s)
{
    a.src[c] = s;
    if (a.src_f) a.src_f[c] = (float)s;
}

// Initial state: rho^0, T^0 (checked), I^0 = rho^0/4pi is filled by fill_iso_kernel.
__global__ void td_init_kernel(TdArgs a, const double* __restrict__ rho0, const double* __restrict__ T0)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.N; c += gridDim.x * blockDim.x) {
        const double r = rho0[c], t = T0[c];
        if (!(r >= 0.0) || !isfinite(r) || !(t > 0.0) || !isfinite(t)) atomicOr(&a.status->error, kErrBadInput);
        a.rho_m[c] = r;
        a.T[c] = t;
        a.cn[c] = 0.0;
        a.cnext[c] = 0.0;
    }
}

template <typename T>
__global__ void fill_iso_kernel(T* I, int K, int N, const double* __restrict__ rho)
{
    const size_t tot = (size_t)K * N;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x)
        I[t] = (T)(rho[t % N] * kInvFourPi);
}

// Start of a time step: rho^n, T^n, I^n correction; the first source.
__global__ void td_begin_kernel(TdArgs a)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.N; c += gridDim.x * blockDim.x) {
        const double r = a.rho_m[c], t = a.T[c];
        a.rho_n[c] = r;
        a.T_n[c] = t;
        a.cn[c] = a.cnext[c];
        a.cnext[c] = 0.0;
    }
}

__global__ void td_source_kernel(TdArgs a)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.N; c += gridDim.x * blockDim.x)
        put_source(a, c, td_source(a, c, a.rho_m[c], a.T[c]));
}

// GSIS: diagonal and volume source of the Newton-eliminated synthetic
// equation about the current T^m (volume-multiplied, as D_steady).
__global__ void td_coef_kernel(TdArgs a)
{
    if (ld_volatile_int(&a.status->done)) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.N; c += gridDim.x * blockDim.x) {
        const int j = c / a.nx, i = c - j * a.nx;
        const double V = a.dx[i] * a.dy[j];
        const double sa = a.sigma_a[c], t = a.T[c];
        const double kap = 4.0 * a.ac * t * t * t;
        const double f = a.cv_dt / fma(kap, sa, a.cv_dt);
        const double phi = a.ac * pow4(t);
        a.qeff[c] = fma(a.rho_n[c], a.inv_cdt, fma(f * sa, fma(kap, a.T_n[c] - t, phi), a.q[c]));
        a.diag[c] = fma(V, a.inv_cdt + fma(f, sa, -sa), a.diag0[c]);
    }
}

// Err(rho), rho^m <- rho^{m+1}, T^{m+1} (GSIS), the correction of I and the
// next source.
__global__ void __launch_bounds__(kRedBlock) td_update_kernel(TdArgs a)
{
    __shared__ double sm[33];
    __shared__ int am_last;
    if (ld_volatile_int(&a.status->done)) return;
    double num = 0.0, den = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.N; c += gridDim.x * blockDim.x) {
        const int j = c / a.nx, i = c - j * a.nx;
        const double V = a.dx[i] * a.dy[j];
        const double od = a.rho_m[c];
        double nw, t = a.T[c];
        if (a.gsis) {
            nw = a.x[c];
            const double sa = a.sigma_a[c];
            const double kap = 4.0 * a.ac * t * t * t;
            const double D2 = fma(kap, sa, a.cv_dt);
            const double phi = a.ac * pow4(t);
            const double tn = a.T_n[c];
            t = tn + sa * fma(kap, t - tn, nw - phi) / D2;
            a.T[c] = t;
            a.cnext[c] = (nw - a.rho_h[c]) * kInvFourPi;
        } else {
            nw = a.rho_h[c];
        }
        const double d = nw - od;
        num = fma(d * d, V, num);
        den = fma(nw * nw, V, den);
        a.rho_m[c] = nw;
        put_source(a, c, td_source(a, c, nw, t));
    }
    num = block_sum(num, sm);
    den = block_sum(den, sm);
    err_reduce_decide(num, den, a.partials, a.hist, a.status, a.tol, a.fixed_iters, a.max_iter, blockIdx.x,
                      gridDim.x, &am_last);
}

// SI: material temperature at the end of the step from the Fleck-Cummings
// emission phi^{n+1} = (1 - f) rho + f phi^n.
__global__ void td_end_si_kernel(TdArgs a)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.N; c += gridDim.x * blockDim.x) {
        const double sa = a.sigma_a[c], tn = a.T_n[c];
        const double kap = 4.0 * a.ac * tn * tn * tn;
        const double f = a.cv_dt / fma(kap, sa, a.cv_dt);
        const double phin = a.ac * pow4(tn);
        const double phi = fma(1.0 - f, a.rho_m[c], f * phin);
        a.T[c] = (phi + 3.0 * phin) / kap;
    }
}

cudaError_t launch_td_coef_hot_rhs(const Plan& P, const TdArgs& a, int g, cudaStream_t st)
{
    td_coef_kernel<<<g, kRedBlock, 0, st>>>(a);
    const cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : launch_hot_rhs(P, P.rho_h, P.Fx, P.Fy, P.fb, P.rho_m, st);
}

cudaError_t launch_td_update(const Plan& P, const TdArgs& a, cudaStream_t st)
{
    td_update_kernel<<<P.red_grid, kRedBlock, 0, st>>>(a);
    return cudaGetLastError();
}

TdArgs td_args(const Plan& P, const gsis_time_params* tp, int gsis)
{
    TdArgs a{};
    a.nx = P.nx; a.ny = P.ny; a.N = P.N;
    a.dx = P.dx; a.dy = P.dy;
    a.sigma_a = P.sigma_a; a.sigma_s = P.sigma_s; a.q = P.q;
    a.rho_m = P.rho_m; a.rho_h = P.rho_h; a.x = P.x;
    a.T = P.td.T; a.T_n = P.td.T_n; a.rho_n = P.td.rho_n;
    a.cn = P.td.cn; a.cnext = P.td.cnext;
    a.qeff = P.td.qeff; a.diag = P.diag; a.diag0 = P.td.diag0;
    a.src = P.src; a.src_f = P.fp32 ? P.src_f : nullptr;
    a.inv_cdt = 1.0 / (tp->c * tp->dt);
    a.ac = tp->a * tp->c;
    a.cv_dt = tp->cv / tp->dt;
    a.gsis = gsis;
    a.partials = P.partials + (size_t)9 * kMaxCgBlocks;
    a.hist = P.hist;
    a.status = P.status;
    a.tol = P.tol; a.fixed_iters = P.fixed_iters; a.max_iter = P.max_iter;
    return a;
}

Sizes td_sizes(const gsis_mesh* m, const gsis_quadrature* q, const gsis_options* o)
{
    Sizes z = sizes_of(m, q, o);
    z.td = 1;
    return z;
}

int check_tp(const gsis_time_params* tp, const gsis_options* opt)
{
    if (!tp) return fail(GSIS_ERR_ARG, "time parameters are NULL");
    for (double v : {tp->dt, tp->c, tp->a, tp->cv})
        if (!(v > 0.0) || !std::isfinite(v)) return fail(GSIS_ERR_ARG, "dt, c, a and cv must be finite and > 0");
    if (tp->nsteps < 1 || tp->nsteps > 100000000) return fail(GSIS_ERR_ARG, "nsteps out of range");
    if (opt->cfl_p > 0.0 || opt->beta > 0.0)
        return fail(GSIS_ERR_ARG, "the time-dependent solve takes no pseudo-time (cfl_p, beta <= 0)");
    if (opt->spatial_order != 1) return fail(GSIS_ERR_ARG, "the time-dependent solve runs first-order upwind face values");
    return GSIS_OK;
}

}  // namespace

extern "C" {

int gsis_td_workspace_bytes(const gsis_mesh* mesh, const gsis_quadrature* quad, const gsis_options* opt,
                            size_t* bytes)
{
    int rc;
    if ((rc = check_mesh(mesh)) || (rc = check_quad(quad)) || (rc = check_opt(opt))) return rc;
    if (!bytes) return fail(GSIS_ERR_ARG, "bytes is NULL");
    *bytes = layout(td_sizes(mesh, quad, opt), nullptr, nullptr);
    return GSIS_OK;
}

int gsis_td_solve(const gsis_mesh* mesh, const gsis_quadrature* quad, const gsis_options* opt,
                  const gsis_time_params* tp, const double* sigma_a, const double* sigma_s, const double* q,
                  const double* inflow, const double* rho0, const double* T0, double* rho, double* T, double* F,
                  int* step_iters, double* step_err, void* workspace, size_t workspace_bytes, void* stream)
{
    int rc;
    if ((rc = check_mesh(mesh)) || (rc = check_quad(quad)) || (rc = check_opt(opt)) || (rc = check_tp(tp, opt)))
        return rc;
    if (!sigma_a || !sigma_s || !q || !rho0 || !T0 || !rho || !T)
        return fail(GSIS_ERR_ARG, "a required device pointer is NULL");
    const Sizes z = td_sizes(mesh, quad, opt);
    if ((rc = check_ws(workspace, workspace_bytes, layout(z, nullptr, nullptr)))) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Plan P{};
    layout(z, static_cast<char*>(workspace), &P);
    P.shift0 = 1.0 / (tp->c * tp->dt);
    if ((rc = prepare(P, mesh, quad, opt, sigma_a, sigma_s, q, inflow, st))) return rc;
    const int gsis = opt->scheme == GSIS_SCHEME_GSIS;
    P.pt = 1;                 // the delta-form sweep: shift 1/(c dt), I_old = I^n
    P.q_syn = P.td.qeff;
    const int g = grid_for(P.N, kRedBlock, P.num_sms * 8);
    TdArgs a = td_args(P, tp, gsis);
    CK(cudaMemcpyAsync(P.td.diag0, P.diag, (size_t)P.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    td_init_kernel<<<g, kRedBlock, 0, st>>>(a, rho0, T0);
    CK(cudaGetLastError());
    {
        const size_t n = (size_t)P.K * P.N;
        const int gi = grid_for((long long)n, 256, P.num_sms * 16);
        if (P.fp32) fill_iso_kernel<float><<<gi, 256, 0, st>>>(static_cast<float*>(P.In), P.K, P.N, rho0);
        else fill_iso_kernel<double><<<gi, 256, 0, st>>>(static_cast<double*>(P.In), P.K, P.N, rho0);
        CK(cudaGetLastError());
    }
    Status S{};
    if ((rc = read_status(S, P, st))) return rc;

    const int nmax = opt->fixed_iters > 0 ? opt->fixed_iters : opt->max_iter;
    int result = GSIS_OK;
    for (int n = 0; n < tp->nsteps; ++n) {
        if (n > 0) std::swap(P.I, P.In);   // I^n = the last sweep's intensities (+ cn)
        a = td_args(P, tp, gsis);
        CK(cudaMemsetAsync(P.status, 0, sizeof(Status), st));
        td_begin_kernel<<<g, kRedBlock, 0, st>>>(a);
        CK(cudaGetLastError());
        if (gsis) {   // multigrid hierarchy of the step's operator (coupling at T^n)
            td_coef_kernel<<<g, kRedBlock, 0, st>>>(a);
            CK(cudaGetLastError());
            CK(launch_mg_setup(P, st));
        }
        td_source_kernel<<<g, kRedBlock, 0, st>>>(a);
        CK(cudaGetLastError());
        int launched = 0;
        while (launched < nmax) {
            const int batch = std::min(opt->check_every, nmax - launched);
            for (int b = 0; b < batch; ++b) {
                TIMED(GSIS_KCLASS_SWEEP, 1, launch_sweep(P, st));
                TIMED(GSIS_KCLASS_MOMENTS, 2,
                      launch_moments_to(P, gsis, false, P.rho_h, nullptr, nullptr, false, P.fb, false, st));
                if (gsis) {
                    TIMED(GSIS_KCLASS_HOT_RHS, 3, launch_td_coef_hot_rhs(P, a, g, st));
                    TIMED(GSIS_KCLASS_SYNTH, 1, launch_synthetic_solve(P, P.rho_m, P.x, st));
                }
                TIMED(GSIS_KCLASS_UPDATE, 1, launch_td_update(P, a, st));
            }
            launched += batch;
            if ((rc = read_status(S, P, st))) return rc;
            if (S.done) break;
        }
        if (!gsis) {
            td_end_si_kernel<<<g, kRedBlock, 0, st>>>(a);
            CK(cudaGetLastError());
        }
        if (step_iters) step_iters[n] = S.iter;
        if (step_err) step_err[n] = S.err;
        if (S.reason == kDiverged) {
            result = fail(GSIS_ERR_DIVERGED, "step %d: Err = %g after %d iterations", n, S.err, S.iter);
            break;
        }
        if (S.reason != kConverged && S.reason != kFixedDone) {
            result = fail(GSIS_ERR_MAXITER, "step %d: Err = %g after %d iterations", n, S.err, S.iter);
            break;
        }
    }
    if (F) CK(launch_moments_to(P, true, false, P.rho_h, F, nullptr, false, P.fb, true, st));
    CK(cudaMemcpyAsync(rho, P.rho_m, (size_t)P.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(T, P.td.T, (size_t)P.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    return result;
}

}  // extern "C"
