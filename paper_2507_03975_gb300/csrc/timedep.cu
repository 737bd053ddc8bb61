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
    double* hr1; double* hr2; double* ht1; double* ht2;   // predictor history (null: none kept)
    double* ckap; double* cphi; double* cf;               // GSIS: kappa, phi, f of td_coef_kernel at T^m
    int pred;                                             // this step's extrapolation order
    double* src; float* src_f;
    double inv_cdt, ac, cv_dt, dt_cv;   // 1/(c dt), a c, C_v / dt, dt / C_v
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
        if (a.hr1 && a.pred == 0) {   // the history's first entry (step 0)
            a.hr1[c] = r;
            a.hr2[c] = r;
            a.ht1[c] = t;
            a.ht2[c] = t;
        } else if (a.hr1) {   // first iterate extrapolated from the last steps' results
            const double r1 = a.hr1[c], t1 = a.ht1[c];
            double rp, tq;
            if (a.pred == 1) {
                rp = r + (r - r1);
                tq = t + (t - t1);
            } else {
                rp = fma(3.0, r - r1, a.hr2[c]);
                tq = fma(3.0, t - t1, a.ht2[c]);
            }
            a.rho_m[c] = fmax(rp, 0.5 * r);
            a.T[c] = fmax(tq, 0.5 * t);
            a.hr2[c] = r1;
            a.ht2[c] = t1;
            a.hr1[c] = r;
            a.ht1[c] = t;
        }
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
        // the material update of this iteration linearises about the same T^m
        a.ckap[c] = kap;
        a.cphi[c] = phi;
        a.cf[c] = f;
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
            // kappa, phi and 1/(C_v/dt + kappa sigma_a) = f dt/C_v at T^m, as
            // td_coef_kernel formed them in this iteration (no FP64 division here)
            const double kap = a.ckap[c], phi = a.cphi[c];
            const double tn = a.T_n[c];
            t = tn + sa * fma(kap, t - tn, nw - phi) * (a.cf[c] * a.dt_cv);
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

// coef = false: the coefficients already hold this T^m (the step's first
// iteration, right after the step operator formed them at the same T^m)
cudaError_t launch_td_coef_hot_rhs(const Plan& P, const TdArgs& a, int g, cudaStream_t st, bool coef)
{
    if (coef) {
        td_coef_kernel<<<g, kRedBlock, 0, st>>>(a);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return launch_hot_rhs(P, P.rho_h, P.Fx, P.Fy, P.fb, P.rho_m, st);
}

cudaError_t launch_td_update(const Plan& P, const TdArgs& a, cudaStream_t st)
{
    td_update_kernel<<<P.red_grid, kRedBlock, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_td_begin(const TdArgs& a, int g, cudaStream_t st)
{
    td_begin_kernel<<<g, kRedBlock, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_td_step_operator(const Plan& P, const TdArgs& a, int g, cudaStream_t st)
{
    td_coef_kernel<<<g, kRedBlock, 0, st>>>(a);
    const cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : launch_mg_setup(P, st);
}

cudaError_t launch_td_source(const TdArgs& a, int g, cudaStream_t st)
{
    td_source_kernel<<<g, kRedBlock, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_td_end_si(const TdArgs& a, int g, cudaStream_t st)
{
    td_end_si_kernel<<<g, kRedBlock, 0, st>>>(a);
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
    a.dt_cv = tp->dt / tp->cv;
    a.ckap = P.td.ckap; a.cphi = P.td.cphi; a.cf = P.td.cf;
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
    z.ordsrc = 1;   // the sweep's source src + I^n/(c dt) per ordinate
    return z;
}

int check_tp(const gsis_time_params* tp, const gsis_options* opt)
{
    if (!tp) return fail(GSIS_ERR_ARG, "time parameters are NULL");
    for (double v : {tp->dt, tp->c, tp->a, tp->cv})
        if (!(v > 0.0) || !std::isfinite(v)) return fail(GSIS_ERR_ARG, "dt, c, a and cv must be finite and > 0");
    if (tp->nsteps < 1 || tp->nsteps > 100000000) return fail(GSIS_ERR_ARG, "nsteps out of range");
    if (tp->predictor < 0 || tp->predictor > 2) return fail(GSIS_ERR_ARG, "predictor must be 0, 1 or 2");
    if (opt->cfl_p > 0.0 || opt->beta > 0.0)
        return fail(GSIS_ERR_ARG, "the time-dependent solve takes no pseudo-time (cfl_p, beta <= 0)");
    if (opt->spatial_order != 1) return fail(GSIS_ERR_ARG, "the time-dependent solve runs first-order upwind face values");
    return GSIS_OK;
}

// One backward-Euler step from the state held in the plan (rho_m, T, the
// correction cnext and In: I^n = In + cn); leaves the step's last iterate
// (I = I^{m+1/2}, rho_h, rho_m, T, cnext) and its status in S.  With
// opt->stall_window > 0 (and no fixed iteration count) the step also ends
// when Err has not reached a new minimum for that many checks; *stalled
// says so (the FP32 kinetic step has a floor of Err near 1e-8).  pred >= 0
// keeps the last steps' results and starts the step from their
// extrapolation of order pred (gsis_time_params::predictor); -1 keeps none.
int run_step(Plan& P, const gsis_time_params* tp, const gsis_options* opt, int gsis, Status& S, cudaStream_t st,
             bool* stalled = nullptr, int pred = -1)
{
    int rc;
    const int g = grid_for(P.N, kRedBlock, P.num_sms * 8);
    const int nmax = opt->fixed_iters > 0 ? opt->fixed_iters : opt->max_iter;
    TdArgs a = td_args(P, tp, gsis);
    if (pred >= 0) {   // keep the predictor's history; extrapolate with order pred
        a.hr1 = P.td.hr1; a.hr2 = P.td.hr2; a.ht1 = P.td.ht1; a.ht2 = P.td.ht2;
        a.pred = pred;
    }
    CK(cudaMemsetAsync(P.status, 0, sizeof(Status), st));
    TIMED(GSIS_KCLASS_SETUP, 1, launch_td_begin(a, g, st));
    if (gsis)   // multigrid hierarchy of the step's operator (coupling at T^n): 1 + nl kernels
        TIMED(GSIS_KCLASS_SETUP, 1 + mg_setup_launches(P), launch_td_step_operator(P, a, g, st));
    TIMED(GSIS_KCLASS_SETUP, 1, launch_td_source(a, g, st));
    if (P.X || P.X_f) TIMED(GSIS_KCLASS_SETUP, 1, launch_ordinate_source(P, st));
    if (stalled) *stalled = false;
    double best = INFINITY;
    int since_best = 0;
    int launched = 0;
    while (launched < nmax) {
        const int batch = std::min(opt->check_every, nmax - launched);
        for (int b = 0; b < batch; ++b) {
            TIMED(GSIS_KCLASS_SWEEP, 1, launch_sweep(P, st));
            TIMED(GSIS_KCLASS_MOMENTS, P.order == 2 ? 2 : 1,
                  launch_moments_to(P, gsis, false, P.rho_h, nullptr, nullptr, false, P.fb, false, st));
            if (gsis) {
                const bool coef = launched + b > 0;
                TIMED(GSIS_KCLASS_HOT_RHS, coef ? 3 : 2, launch_td_coef_hot_rhs(P, a, g, st, coef));
                TIMED(GSIS_KCLASS_SYNTH, 1, launch_synthetic_solve(P, P.rho_m, P.x, st));
            }
            TIMED(GSIS_KCLASS_UPDATE, 1, launch_td_update(P, a, st));
            if (P.X || P.X_f) TIMED(GSIS_KCLASS_UPDATE, 1, launch_ordinate_source(P, st));
        }
        launched += batch;
        if ((rc = read_status(S, P, st))) return rc;
        if (S.done) break;
        if (opt->stall_window > 0 && opt->fixed_iters <= 0) {
            if (S.err < best) {
                best = S.err;
                since_best = 0;
            } else if (++since_best >= opt->stall_window) {
                if (stalled) *stalled = true;
                break;
            }
        }
    }
    if (!gsis) TIMED(GSIS_KCLASS_SETUP, 1, launch_td_end_si(a, g, st));
    return GSIS_OK;
}

int step_result(const Status& S, int n)
{
    if (S.reason == kDiverged) return fail(GSIS_ERR_DIVERGED, "step %d: Err = %g after %d iterations", n, S.err, S.iter);
    if (S.reason != kConverged && S.reason != kFixedDone)
        return fail(GSIS_ERR_MAXITER, "step %d: Err = %g after %d iterations", n, S.err, S.iter);
    return GSIS_OK;
}

cudaError_t launch_td_init(const Plan& P, const TdArgs& a, int g, const double* rho0, const double* T0,
                           cudaStream_t st)
{
    td_init_kernel<<<g, kRedBlock, 0, st>>>(a, rho0, T0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t n = (size_t)P.K * P.N;
    const int gi = grid_for((long long)n, 256, P.num_sms * 16);
    if (P.fp32) fill_iso_kernel<float><<<gi, 256, 0, st>>>(static_cast<float*>(P.In), P.K, P.N, rho0);
    else fill_iso_kernel<double><<<gi, 256, 0, st>>>(static_cast<double*>(P.In), P.K, P.N, rho0);
    return cudaGetLastError();
}

// Start of a run: the step-independent synthetic diagonal, rho^0, T^0 and
// I^0 = rho^0/4pi in In.
int td_start(Plan& P, const gsis_time_params* tp, int gsis, const double* rho0, const double* T0, cudaStream_t st)
{
    const int g = grid_for(P.N, kRedBlock, P.num_sms * 8);
    const TdArgs a = td_args(P, tp, gsis);
    CK(cudaMemcpyAsync(P.td.diag0, P.diag, (size_t)P.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    TIMED(GSIS_KCLASS_SETUP, 2, launch_td_init(P, a, g, rho0, T0, st));
    return GSIS_OK;
}

__global__ void add_f_kernel(float* out, const float* __restrict__ a, const float* __restrict__ b, int n)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) out[c] = a[c] + b[c];
}

// Storage of the time-step adjoint after the solve layout: the transposed
// solve of the carried intensities (chi) and the carry (phi), a zero source,
// the FP32 transposed-sweep diagonal, six per-cell vectors, the checkpoints
// (every C-th step's input state: In, cnext, rho, T and the predictor's
// history of the last two steps' rho and T) and the records of one
// segment of C steps (each step's I^{m+1/2}, rho^{m+1/2}, rho, T).
struct AdjStore {
    void* chi; void* carry; void* zero;
    float* sigt_shift_f;
    double* sig_eff; double* c0; double* rb_extra; double* ybar_rho; double* ybar_T; double* sphi;
    std::vector<void*> ck_I, rec_I;
    std::vector<double*> ck_v, rec_v;   // 7 N (checkpoint) and 3 N (record) doubles each
};

size_t adj_store(const Sizes& z, int nck, int seg, char* base, AdjStore* A)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off += (bytes + kAlign - 1) / kAlign * kAlign;
        return p;
    };
    const size_t N = (size_t)z.nx * z.ny, K = (size_t)z.K;
    const size_t Ts = z.fp32 ? sizeof(float) : sizeof(double);
    AdjStore tmp;
    AdjStore& a = A ? *A : tmp;
    a.chi = take(K * N * Ts);
    a.carry = take(K * N * Ts);
    a.zero = take(N * Ts);
    a.sigt_shift_f = z.fp32 ? reinterpret_cast<float*>(take(N * sizeof(float))) : nullptr;
    double** v[] = {&a.sig_eff, &a.c0, &a.rb_extra, &a.ybar_rho, &a.ybar_T, &a.sphi};
    for (double** d : v) *d = reinterpret_cast<double*>(take(N * sizeof(double)));
    a.ck_I.assign(nck, nullptr);
    a.ck_v.assign(nck, nullptr);
    for (int i = 0; i < nck; ++i) {
        a.ck_I[i] = take(K * N * Ts);
        a.ck_v[i] = reinterpret_cast<double*>(take(7 * N * sizeof(double)));
    }
    a.rec_I.assign(seg, nullptr);
    a.rec_v.assign(seg, nullptr);
    for (int i = 0; i < seg; ++i) {
        a.rec_I[i] = take(K * N * Ts);
        a.rec_v[i] = reinterpret_cast<double*>(take(3 * N * sizeof(double)));
    }
    return off;
}

Sizes td_adj_sizes(const gsis_mesh* m, const gsis_quadrature* q, const gsis_options* o)
{
    Sizes z = td_sizes(m, q, o);
    z.adjoint = 1;
    return z;
}

int check_td_adjoint(const gsis_mesh* mesh, const gsis_quadrature* quad, const gsis_options* opt,
                     const gsis_time_params* tp, int checkpoint_every, std::vector<int>* refl)
{
    int rc;
    if ((rc = check_mesh(mesh)) || (rc = check_quad(quad)) || (rc = check_opt(opt)) || (rc = check_tp(tp, opt)))
        return rc;
    if (opt->scheme != GSIS_SCHEME_GSIS) return fail(GSIS_ERR_ARG, "the adjoint is that of the GSIS time steps");
    if (checkpoint_every < 1) return fail(GSIS_ERR_ARG, "checkpoint_every must be >= 1");
    if (!uniform_spacing(mesh->dx, mesh->nx) || !uniform_spacing(mesh->dy, mesh->ny))
        return fail(GSIS_ERR_ARG, "the adjoint needs a uniform mesh (transposed sweep = reflected sweep)");
    std::vector<int> r;
    if (!reflection_table(quad, r))
        return fail(GSIS_ERR_ARG, "the adjoint needs a quadrature closed under Omega -> -Omega with equal weights");
    if (refl) *refl = r;
    return GSIS_OK;
}

size_t td_adj_bytes(const Sizes& z, int nsteps, int C)
{
    const int seg = std::min(C, nsteps);
    const int nck = (nsteps + C - 1) / C;
    return layout(z, nullptr, nullptr) + adj_store(z, nck, seg, nullptr, nullptr);
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
    if ((rc = td_start(P, tp, gsis, rho0, T0, st))) return rc;
    Status S{};
    if ((rc = read_status(S, P, st))) return rc;

    int result = GSIS_OK;
    int n_stalled = 0, first_stalled = -1;
    for (int n = 0; n < tp->nsteps; ++n) {
        if (n > 0) std::swap(P.I, P.In);   // I^n = the last sweep's intensities (+ cn)
        bool stalled = false;
        const int pred = tp->predictor > 0 ? std::min(tp->predictor, n) : -1;
        if ((rc = run_step(P, tp, opt, gsis, S, st, &stalled, pred))) return rc;
        if (step_iters) step_iters[n] = S.iter;
        if (step_err) step_err[n] = S.err;
        if (stalled) {   // the step ends at its floor of Err; the run goes on
            if (n_stalled++ == 0) first_stalled = n;
            continue;
        }
        if ((result = step_result(S, n)) != GSIS_OK) break;
    }
    if (result == GSIS_OK && n_stalled > 0)
        result = fail(GSIS_ERR_STALLED, "%d of %d steps ended on a stalled Err (first: step %d)", n_stalled,
                      tp->nsteps, first_stalled);
    if (F) CK(launch_moments_to(P, true, false, P.rho_h, F, nullptr, false, P.fb, true, st));
    CK(cudaMemcpyAsync(rho, P.rho_m, (size_t)P.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(T, P.td.T, (size_t)P.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    return result;
}

int gsis_td_adjoint_workspace_bytes(const gsis_mesh* mesh, const gsis_quadrature* quad, const gsis_options* opt,
                                    const gsis_time_params* tp, int checkpoint_every, size_t* bytes)
{
    int rc;
    if ((rc = check_td_adjoint(mesh, quad, opt, tp, checkpoint_every, nullptr))) return rc;
    if (!bytes) return fail(GSIS_ERR_ARG, "bytes is NULL");
    *bytes = td_adj_bytes(td_adj_sizes(mesh, quad, opt), tp->nsteps, checkpoint_every);
    return GSIS_OK;
}

int gsis_td_adjoint(const gsis_mesh* mesh, const gsis_quadrature* quad, const gsis_options* opt,
                    const gsis_time_params* tp, int checkpoint_every, const double* sigma_a, const double* sigma_s,
                    const double* q, const double* inflow, const double* rho0, const double* T0,
                    const double* dJ_drho, const double* dJ_dT, double* rho, double* T, double* grad_sigma_a,
                    double* grad_sigma_s, double* grad_rho0, double* grad_T0, int* adj_iters, void* workspace,
                    size_t workspace_bytes, void* stream)
{
    int rc;
    std::vector<int> refl;
    if ((rc = check_td_adjoint(mesh, quad, opt, tp, checkpoint_every, &refl))) return rc;
    if (!sigma_a || !sigma_s || !q || !rho0 || !T0 || !grad_sigma_a || !grad_sigma_s)
        return fail(GSIS_ERR_ARG, "a required device pointer is NULL");
    const Sizes z = td_adj_sizes(mesh, quad, opt);
    const int nsteps = tp->nsteps, C = std::min(checkpoint_every, nsteps);
    const int nck = (nsteps + C - 1) / C;
    if ((rc = check_ws(workspace, workspace_bytes, td_adj_bytes(z, nsteps, C)))) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Plan P{};
    const size_t main = layout(z, static_cast<char*>(workspace), &P);
    AdjStore A;
    adj_store(z, nck, C, static_cast<char*>(workspace) + main, &A);
    P.shift0 = 1.0 / (tp->c * tp->dt);
    if ((rc = prepare(P, mesh, quad, opt, sigma_a, sigma_s, q, inflow, st))) return rc;
    P.pt = 1;
    P.q_syn = P.td.qeff;
    const size_t N = (size_t)P.N, KN = (size_t)P.K * P.N;
    const size_t Ts = P.fp32 ? sizeof(float) : sizeof(double), Nd = N * sizeof(double);
    CK(cudaMemcpyAsync(P.refl, refl.data(), refl.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    if ((rc = td_start(P, tp, 1, rho0, T0, st))) return rc;
    CK(cudaMemsetAsync(A.zero, 0, N * Ts, st));
    if (P.fp32) {
        add_f_kernel<<<grid_for(P.N, 256, P.num_sms * 8), 256, 0, st>>>(A.sigt_shift_f, P.sigt_f, P.shift_f, P.N);
        CK(cudaGetLastError());
    }
    Status S{};
    if ((rc = read_status(S, P, st))) return rc;

    // forward run, keeping the input state of every C-th step
    void* const I0 = P.I;
    void* const In0 = P.In;
    double* const rho_m0 = P.rho_m;
    double* const rho_h0 = P.rho_h;
    double* const T0d = P.td.T;
    auto save_state = [&](double* v) -> int {
        CK(cudaMemcpyAsync(v, P.td.cnext, Nd, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(v + N, P.rho_m, Nd, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(v + 2 * N, P.td.T, Nd, cudaMemcpyDeviceToDevice, st));
        if (tp->predictor > 0) {   // the history the next step extrapolates from
            double* const h[] = {P.td.hr1, P.td.hr2, P.td.ht1, P.td.ht2};
            for (int k = 0; k < 4; ++k)
                CK(cudaMemcpyAsync(v + (3 + k) * N, h[k], Nd, cudaMemcpyDeviceToDevice, st));
        }
        return GSIS_OK;
    };
    auto step_pred = [&](int n) { return tp->predictor > 0 ? std::min(tp->predictor, n) : -1; };
    for (int n = 0; n < nsteps; ++n) {
        if (n > 0) std::swap(P.I, P.In);
        if (n % C == 0) {
            CK(cudaMemcpyAsync(A.ck_I[n / C], P.In, KN * Ts, cudaMemcpyDeviceToDevice, st));
            if ((rc = save_state(A.ck_v[n / C]))) return rc;
        }
        bool stalled = false;   // a stalled step ends at its floor, as in gsis_td_solve
        if ((rc = run_step(P, tp, opt, 1, S, st, &stalled, step_pred(n)))) return rc;
        if (!stalled && (rc = step_result(S, n))) return rc;
    }
    if (rho) CK(cudaMemcpyAsync(rho, P.rho_m, Nd, cudaMemcpyDeviceToDevice, st));
    if (T) CK(cudaMemcpyAsync(T, P.td.T, Nd, cudaMemcpyDeviceToDevice, st));

    // reverse sweep over the segments: recompute the segment's steps from its
    // checkpoint, then the step adjoints last to first
    TdAdjVecs v{};
    v.diag0 = P.td.diag0;
    v.sig_eff = A.sig_eff; v.c0 = A.c0; v.rb_extra = A.rb_extra;
    v.ybar_rho = A.ybar_rho; v.ybar_T = A.ybar_T; v.sphi = A.sphi;
    v.carry = A.carry;
    v.inv_cdt = 1.0 / (tp->c * tp->dt);
    v.ac = tp->a * tp->c;
    v.cv_dt = tp->cv / tp->dt;
    if (dJ_drho) CK(cudaMemcpyAsync(A.ybar_rho, dJ_drho, Nd, cudaMemcpyDeviceToDevice, st));
    else CK(cudaMemsetAsync(A.ybar_rho, 0, Nd, st));
    if (dJ_dT) CK(cudaMemcpyAsync(A.ybar_T, dJ_dT, Nd, cudaMemcpyDeviceToDevice, st));
    else CK(cudaMemsetAsync(A.ybar_T, 0, Nd, st));
    CK(cudaMemsetAsync(A.sphi, 0, Nd, st));
    CK(cudaMemsetAsync(grad_sigma_a, 0, Nd, st));
    CK(cudaMemsetAsync(grad_sigma_s, 0, Nd, st));
    CK(cudaMemsetAsync(P.nu, 0, Nd, st));
    const int nmax = opt->fixed_iters > 0 ? opt->fixed_iters : opt->max_iter;
    bool have_carry = false;
    int result = GSIS_OK;
    for (int sg = nck - 1; sg >= 0; --sg) {
        const int n0 = sg * C, n1 = std::min(n0 + C, nsteps);
        // the segment's input state
        P.I = I0; P.In = In0; P.rho_m = rho_m0; P.rho_h = rho_h0; P.td.T = T0d;
        CK(cudaMemcpyAsync(P.td.cnext, A.ck_v[sg], Nd, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(P.rho_m, A.ck_v[sg] + N, Nd, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(P.td.T, A.ck_v[sg] + 2 * N, Nd, cudaMemcpyDeviceToDevice, st));
        if (tp->predictor > 0) {
            double* const h[] = {P.td.hr1, P.td.hr2, P.td.ht1, P.td.ht2};
            for (int k = 0; k < 4; ++k)
                CK(cudaMemcpyAsync(h[k], A.ck_v[sg] + (3 + k) * N, Nd, cudaMemcpyDeviceToDevice, st));
        }
        for (int r = 0; r < n1 - n0; ++r) {
            P.In = r == 0 ? A.ck_I[sg] : A.rec_I[r - 1];
            P.I = A.rec_I[r];
            bool stalled = false;
            if ((rc = run_step(P, tp, opt, 1, S, st, &stalled, step_pred(n0 + r)))) return rc;
            if (!stalled && (rc = step_result(S, n0 + r))) return rc;
            double* rv = A.rec_v[r];
            CK(cudaMemcpyAsync(rv, P.rho_h, Nd, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(rv + N, P.rho_m, Nd, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(rv + 2 * N, P.td.T, Nd, cudaMemcpyDeviceToDevice, st));
        }
        for (int r = n1 - n0 - 1; r >= 0; --r) {
            const int n = n0 + r;
            // the step's fixed point
            P.I = A.rec_I[r];
            P.rho_h = A.rec_v[r];
            P.rho_m = A.rec_v[r] + N;
            v.T = A.rec_v[r] + 2 * N;
            v.chi = have_carry ? A.chi : nullptr;
            P.g = A.c0;
            P.adj_sig = A.sig_eff;
            P.adj_rb_extra = A.rb_extra;
            P.adj_sigt_f = A.sigt_shift_f;
            CK(cudaMemsetAsync(P.status, 0, sizeof(Status), st));
            TIMED(GSIS_KCLASS_SETUP, 1, launch_td_adjoint_setup(P, v, st));
            CK(launch_mg_setup(P, st));
            if (have_carry) TIMED(GSIS_KCLASS_SWEEP, 1, launch_sweep_pt_into(P, A.zero, A.carry, A.chi, st));
            TIMED(GSIS_KCLASS_SETUP, 1, launch_td_adjoint_start(P, v, st));
            // transposed GSIS iteration of the step: lam = c + (sig_eff/4pi) sum_k phi_A,k(D'^{-1} lam)
            auto pass = [&](bool update) -> int {
                TIMED(GSIS_KCLASS_HOT_RHS, 1, launch_synth_resid(P, P.b, P.nu, st));
                TIMED(GSIS_KCLASS_SYNTH, 1, launch_synthetic_solve(P, P.nu, P.x, st));
                TIMED(GSIS_KCLASS_HOT_RHS, 2, launch_adjoint_rhs(P, P.x, st));
                TIMED(GSIS_KCLASS_SWEEP, 1, launch_adjoint_sweep(P, st));
                if (update) TIMED(GSIS_KCLASS_UPDATE, 1, launch_adjoint_update(P, st));
                return GSIS_OK;
            };
            int launched = 0;
            while (launched < nmax) {
                const int batch = std::min(opt->check_every, nmax - launched);
                for (int b = 0; b < batch; ++b)
                    if ((rc = pass(true))) return rc;
                launched += batch;
                if ((rc = read_status(S, P, st))) return rc;
                if (S.done) break;
            }
            if (adj_iters) adj_iters[n] = S.iter;
            if (S.reason == kDiverged) {
                result = fail(GSIS_ERR_DIVERGED, "adjoint of step %d: Err = %g after %d iterations", n, S.err, S.iter);
            } else if (S.reason != kConverged && S.reason != kFixedDone && result == GSIS_OK) {
                result = fail(GSIS_ERR_MAXITER, "adjoint of step %d: Err = %g after %d iterations", n, S.err, S.iter);
            }
            // nu and phi at the final lam, the step's gradient terms and its carry
            CK(cudaMemsetAsync(&P.status->done, 0, sizeof(int), st));
            if ((rc = pass(false))) return rc;
            TIMED(GSIS_KCLASS_UPDATE, 1, launch_td_adjoint_gradient(P, v, grad_sigma_a, grad_sigma_s, st));
            if ((rc = read_status(S, P, st))) return rc;
            have_carry = true;
            if (result == GSIS_ERR_DIVERGED) break;
        }
        if (result == GSIS_ERR_DIVERGED) break;
    }
    P.I = I0; P.In = In0; P.rho_m = rho_m0; P.rho_h = rho_h0; P.td.T = T0d;
    if (grad_rho0) CK(cudaMemcpyAsync(grad_rho0, A.ybar_rho, Nd, cudaMemcpyDeviceToDevice, st));
    if (grad_T0) CK(cudaMemcpyAsync(grad_T0, A.ybar_T, Nd, cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    return result;
}

}  // extern "C"
