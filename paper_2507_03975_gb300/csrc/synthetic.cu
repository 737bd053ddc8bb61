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

constexpr double kInvFourPi = 0.079577471545947667884441881686257;   // 1 / (4 pi)

int grid_for(long long n, int block, int cap)
{
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// HoT = F + G / (3 sigma_t) with the gradient weights of the cell set-up.
__global__ void hot_kernel(int nx, int ny, const double* __restrict__ hw, const double* __restrict__ rho,
                           const double* __restrict__ Fx, const double* __restrict__ Fy, double* hotx,
                           double* hoty, const int* done)
{
    if (ld_volatile_int(done)) return;
    const int N = nx * ny;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const int j = c / nx, i = c - j * nx;
        const double ri = rho[c];
        double gx = 0.0, gy = 0.0;
        if (i + 1 < nx) gx = fma(hw[c], rho[c + 1] - ri, gx);
        if (i > 0) gx = fma(hw[N + c], rho[c - 1] - ri, gx);
        if (j + 1 < ny) gy = fma(hw[2 * N + c], rho[c + nx] - ri, gy);
        if (j > 0) gy = fma(hw[3 * N + c], rho[c - nx] - ri, gy);
        hotx[c] = Fx[c] + gx;
        hoty[c] = Fy[c] + gy;
    }
}

struct RhsArgs {
    int nx, ny;
    const double* dx; const double* dy;
    const double* sigt; const double* q; const double* rho_h;
    const double* hotx; const double* hoty; const double* fb; const double* bface;
    double* b;
    // first residual of the synthetic solve, r0 = b - D guess
    const double* diag; const double* cx; const double* cy; const double* guess;
    float* r0;          // FP32 copy for the inner iteration
    double* partials;   // [2][gridDim]
    double* norms;      // out: [0] = r0.r0, [1] = b.b
    Status* status;
};

// b, then r0 = b - D guess (five-point D) and the fixed-order sums r0.r0, b.b
// (last-block ticket).
__global__ void __launch_bounds__(kRedBlock) rhs_kernel(const RhsArgs a)
{
    __shared__ double sm[33];
    __shared__ int am_last;
    if (ld_volatile_int(&a.status->done)) return;
    const int nx = a.nx, ny = a.ny, N = nx * ny;
    const double* dx = a.dx; const double* dy = a.dy;
    const double* hotx = a.hotx; const double* hoty = a.hoty; const double* fb = a.fb;
    double lrr = 0.0, lbb = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const int j = c / nx, i = c - j * nx;
        const double hx = dx[i], hy = dy[j];
        double v = hx * hy * a.q[c];
        if (i + 1 < nx) v -= hy * 0.5 * (hotx[c] + hotx[c + 1]);
        if (i > 0) v += hy * 0.5 * (hotx[c] + hotx[c - 1]);
        if (j + 1 < ny) v -= hx * 0.5 * (hoty[c] + hoty[c + nx]);
        if (j > 0) v += hx * 0.5 * (hoty[c] + hoty[c - nx]);
        const double rh = a.rho_h[c];
        const double* bf = a.bface;
        if (i == 0) v -= hy * fb[j] - bf[j] * rh;
        if (i == nx - 1) v -= hy * fb[ny + j] - bf[ny + j] * rh;
        if (j == 0) v -= hx * fb[2 * ny + i] - bf[2 * ny + i] * rh;
        if (j == ny - 1) v -= hx * fb[2 * ny + nx + i] - bf[2 * ny + nx + i] * rh;
        a.b[c] = v;
        const double* g = a.guess;
        double dg = a.diag[c] * g[c];
        if (i + 1 < nx) dg -= a.cx[c] * g[c + 1];
        if (i > 0) dg -= a.cx[c - 1] * g[c - 1];
        if (j + 1 < ny) dg -= a.cy[c] * g[c + nx];
        if (j > 0) dg -= a.cy[c - nx] * g[c - nx];
        const double rv = v - dg;
        a.r0[c] = (float)rv;
        lrr += rv * rv;
        lbb += v * v;
    }
    lrr = block_sum(lrr, sm);
    lbb = block_sum(lbb, sm);
    if (threadIdx.x == 0) {
        a.partials[blockIdx.x] = lrr;
        a.partials[gridDim.x + blockIdx.x] = lbb;
        __threadfence();
        const unsigned t = atomicAdd(&a.status->ticket, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    if (threadIdx.x < 32) {
        __threadfence();
        const double srr = warp_sum_array(a.partials, gridDim.x);
        const double sbb = warp_sum_array(a.partials + gridDim.x, gridDim.x);
        if (threadIdx.x == 0) {
            a.norms[0] = srr;
            a.norms[1] = sbb;
            a.status->ticket = 0u;
        }
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
        double s = (a.sigma_s[c] * nw + a.q[c]) * kInvFourPi;
        if (a.pt) s += a.shift[c] * (nw - a.rho_h[c]) * kInvFourPi;
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
                           const double* fb, const double* guess, cudaStream_t st)
{
    const int g = grid_for(P.N, 256, P.num_sms * 8);
    hot_kernel<<<g, 256, 0, st>>>(P.nx, P.ny, P.hw, rho_h, Fx, Fy, P.hotx, P.hoty, &P.status->done);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    RhsArgs a{};
    a.nx = P.nx; a.ny = P.ny; a.dx = P.dx; a.dy = P.dy;
    a.sigt = P.sigt; a.q = P.q; a.rho_h = rho_h; a.hotx = P.hotx; a.hoty = P.hoty; a.fb = fb; a.b = P.b;
    a.bface = P.bface;
    a.diag = P.diag; a.cx = P.cx; a.cy = P.cy; a.guess = guess;
    a.r0 = P.mg.r0;
    a.partials = P.partials;
    a.norms = P.partials + (size_t)4 * kMaxCgBlocks;
    a.status = P.status;
    rhs_kernel<<<P.red_grid, kRedBlock, 0, st>>>(a);
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
