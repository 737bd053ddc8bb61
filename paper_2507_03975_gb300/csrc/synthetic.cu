// Synthetic (macroscopic) step of GSIS and the per-iteration update.
//
//  * Adaptive least-squares gradient (Sec. 5.2, Eqs. (shifted_j),
//    (new_vector), (LSF_mdf)).  On a Cartesian mesh the shifted displacement
//    to neighbour j is axis-aligned, x'_j - x_i = +-(h_i/2 + (sigma_j/sigma_i) h_j/2),
//    so the 2x2 normal equations (Eq. (LSM_mtx)) are diagonal and
//    G_x = sum_{E,W} d_j (U_j - U_i) / sum d_j^2 (interior neighbours only).
//  * High-order terms HoT = F^{m+1/2} + G/(3 sigma_t) (Eq. (GSIS_HoT)).
//  * Right-hand side (times V_i) of the finite-volume synthetic equation,
//    face-averaged HoT on interior faces (Eq. (Fij_d)) and the boundary flux
//    F_iw^init + beta (rho_i - rho_i^{m+1/2}) (Eqs. (macro_bc_delta_flux),
//    (macro_bc_delta_flux2)):
//      b_i = V_i q_i - sum_int A (HoT_i + HoT_j)/2 . n - sum_bnd A (F_iw.n - beta rho_i^{m+1/2}).
//  * (the solve of D rho = b is in mg.cu)
//  * Err(rho) (Eq. (Err_W)), convergence decision, next angular source.
#include <cuda_runtime.h>

#include "gsis_internal.cuh"

namespace gsis {

namespace {

constexpr double kFourPi = 12.566370614359172953850573533118;

int grid_for(long long n, int block, int cap)
{
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

__global__ void hot_kernel(int nx, int ny, const double* __restrict__ dx, const double* __restrict__ dy,
                           const double* __restrict__ sigt, const double* __restrict__ rho,
                           const double* __restrict__ Fx, const double* __restrict__ Fy,
                           double* hotx, double* hoty, const int* done)
{
    if (ld_volatile_int(done)) return;
    const int N = nx * ny;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const int j = c / nx, i = c - j * nx;
        const double si = sigt[c], ri = rho[c];
        double num = 0.0, den = 0.0;
        if (i + 1 < nx) {
            const double d = 0.5 * dx[i] + (sigt[c + 1] / si) * 0.5 * dx[i + 1];
            num += d * (rho[c + 1] - ri);
            den += d * d;
        }
        if (i > 0) {
            const double d = -(0.5 * dx[i] + (sigt[c - 1] / si) * 0.5 * dx[i - 1]);
            num += d * (rho[c - 1] - ri);
            den += d * d;
        }
        const double gx = den > 0.0 ? num / den : 0.0;
        num = 0.0;
        den = 0.0;
        if (j + 1 < ny) {
            const double d = 0.5 * dy[j] + (sigt[c + nx] / si) * 0.5 * dy[j + 1];
            num += d * (rho[c + nx] - ri);
            den += d * d;
        }
        if (j > 0) {
            const double d = -(0.5 * dy[j] + (sigt[c - nx] / si) * 0.5 * dy[j - 1]);
            num += d * (rho[c - nx] - ri);
            den += d * d;
        }
        const double gy = den > 0.0 ? num / den : 0.0;
        hotx[c] = Fx[c] + gx / (3.0 * si);
        hoty[c] = Fy[c] + gy / (3.0 * si);
    }
}

__global__ void rhs_kernel(int nx, int ny, const double* __restrict__ dx, const double* __restrict__ dy,
                           const double* __restrict__ sigt, const double* __restrict__ q,
                           const double* __restrict__ rho_h, const double* __restrict__ hotx,
                           const double* __restrict__ hoty, const double* __restrict__ fb, double* b,
                           const int* done)
{
    if (ld_volatile_int(done)) return;
    const int N = nx * ny;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const int j = c / nx, i = c - j * nx;
        const double hx = dx[i], hy = dy[j];
        double v = hx * hy * q[c];
        if (i + 1 < nx) v -= hy * 0.5 * (hotx[c] + hotx[c + 1]);
        if (i > 0) v += hy * 0.5 * (hotx[c] + hotx[c - 1]);
        if (j + 1 < ny) v -= hx * 0.5 * (hoty[c] + hoty[c + nx]);
        if (j > 0) v += hx * 0.5 * (hoty[c] + hoty[c - nx]);
        const double st = sigt[c], rh = rho_h[c];
        const double bx = 2.0 / (3.0 * st * hx) + 0.25, by = 2.0 / (3.0 * st * hy) + 0.25;
        if (i == 0) v -= hy * (fb[j] - bx * rh);
        if (i == nx - 1) v -= hy * (fb[ny + j] - bx * rh);
        if (j == 0) v -= hx * (fb[2 * ny + i] - by * rh);
        if (j == ny - 1) v -= hx * (fb[2 * ny + nx + i] - by * rh);
        b[c] = v;
    }
}

struct UpdArgs {
    int nx, ny, N;
    const double* dx; const double* dy;
    const double* sigma_s; const double* q; const double* shift;
    const double* rho_new; double* rho_m; const double* rho_h;
    double* src; float* src_f;
    int pt;
    double tol;
    int fixed_iters, max_iter;
    double* partials;   // [2][gridDim]
    double* hist;
    Status* status;
};

// Err(rho^{m+1}) against rho^m, rho^m <- rho^{m+1}, next angular source
// (with the pseudo-time delta form the stored I^m is the GSIS-corrected
// intensity I^{m+1/2} + (rho^{m+1} - rho^{m+1/2})/4pi (Eq. (GSIS_update));
// the sweep keeps I^{m+1/2}, so the correction enters the source:
// src = (sigma_s rho + q)/4pi + shift (rho - rho^{m+1/2})/4pi).
__global__ void __launch_bounds__(kRedBlock) update_kernel(const UpdArgs a)
{
    __shared__ double sm[33];
    __shared__ int am_last;
    if (ld_volatile_int(&a.status->done)) return;
    double num = 0.0, den = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.N; c += gridDim.x * blockDim.x) {
        const int j = c / a.nx, i = c - j * a.nx;
        const double V = a.dx[i] * a.dy[j];
        const double nw = a.rho_new[c], od = a.rho_m[c];
        num += (nw - od) * (nw - od) * V;
        den += nw * nw * V;
        a.rho_m[c] = nw;
        double s = (a.sigma_s[c] * nw + a.q[c]) / kFourPi;
        if (a.pt) s += a.shift[c] * (nw - a.rho_h[c]) / kFourPi;
        a.src[c] = s;
        if (a.src_f) a.src_f[c] = (float)s;
    }
    num = block_sum(num, sm);
    den = block_sum(den, sm);
    if (threadIdx.x == 0) {
        a.partials[blockIdx.x] = num;
        a.partials[gridDim.x + blockIdx.x] = den;
        __threadfence();
        const unsigned t = atomicAdd(&a.status->ticket, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    if (threadIdx.x < 32) {
        __threadfence();
        const double sn = warp_sum_array(a.partials, gridDim.x);
        const double sd = warp_sum_array(a.partials + gridDim.x, gridDim.x);
        if (threadIdx.x == 0) {
            double err;
            if (sd > 0.0) err = sqrt(sn / sd);
            else err = (sn == 0.0) ? 0.0 : INFINITY;
            Status* S = a.status;
            const int it = S->iter;
            a.hist[it] = err;
            S->iter = it + 1;
            S->err = err;
            int reason = kRunning;
            if (!isfinite(err) || err > 1e6) reason = kDiverged;
            else if (a.fixed_iters > 0) { if (it + 1 >= a.fixed_iters) reason = kFixedDone; }
            else if (err < a.tol) reason = kConverged;
            else if (it + 1 >= a.max_iter) reason = kMaxIter;
            if (reason != kRunning) {
                S->reason = reason;
                S->done = 1;
            }
            S->ticket = 0u;
        }
    }
}

}  // namespace

cudaError_t launch_hot_rhs(const Plan& P, const double* rho_h, const double* Fx, const double* Fy,
                           const double* fb, cudaStream_t st)
{
    const int g = grid_for(P.N, 256, P.num_sms * 8);
    hot_kernel<<<g, 256, 0, st>>>(P.nx, P.ny, P.dx, P.dy, P.sigt, rho_h, Fx, Fy, P.hotx, P.hoty,
                                  &P.status->done);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    rhs_kernel<<<g, 256, 0, st>>>(P.nx, P.ny, P.dx, P.dy, P.sigt, P.q, rho_h, P.hotx, P.hoty, fb, P.b,
                                  &P.status->done);
    return cudaGetLastError();
}

cudaError_t launch_update(const Plan& P, const double* rho_new, cudaStream_t st)
{
    UpdArgs a{};
    a.nx = P.nx; a.ny = P.ny; a.N = P.N; a.dx = P.dx; a.dy = P.dy;
    a.sigma_s = P.sigma_s; a.q = P.q; a.shift = P.shift;
    a.rho_new = rho_new; a.rho_m = P.rho_m; a.rho_h = P.rho_h;
    a.src = P.src; a.src_f = P.fp32 ? P.src_f : nullptr;
    a.pt = P.pt; a.tol = P.tol; a.fixed_iters = P.fixed_iters; a.max_iter = P.max_iter;
    a.partials = P.partials + (size_t)9 * kMaxCgBlocks;
    a.hist = P.hist;
    a.status = P.status;
    update_kernel<<<P.red_grid, kRedBlock, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gsis
