// Adjoint of the steady GSIS solution with respect to the per-cell
// opacities (reverse mode).
//
// The converged solution rho* and the kinetic intensities I_k taken at it
// satisfy A_k(sigma) I_k = s(sigma, rho*) (Sec. 4.1, Eqs. (RTE_d), (RTE_SI))
// and D(sigma) rho* = b(sigma; rho_1/2, F, F_b) (Sec. 4.2, Eqs. (MSE_d1),
// (Fij_d), (macro_bc_delta_flux)).  For J with dJ/drho = g the Lagrangian
//   L = J + sum_k phi_k.(s - A_k I_k) + nu.(b - D rho)
// is stationary when A_k^T phi_k = (db/dI_k)^T nu and D nu = g +
// (sigma_s/4pi) sum_k phi_k; with lam = D nu this is the transposed GSIS
// iteration lam = M^T lam + g, run here step by step:
//   1. nu = D^{-1} lam              (the synthetic solver: D is symmetric)
//   2. (rho_bar_1/2, F_bar, F_bar_b) = (db/d(rho_1/2, F, F_b))^T nu
//   3. psi_k = w_k (rho_bar + mu_k F_bar_x + eta_k F_bar_y) + boundary terms;
//      phi_k = A_k^{-T} psi_k, which on a uniform mesh is the sweep of the
//      reflected direction -Omega_k with that source and the boundary terms
//      as its inflow (csrc/sweep.cu, adjoint source mode)
//   4. lam = g + (sigma_s/4pi) sum_k phi_k
// and dJ/dsigma = dL/dsigma at the converged (rho*, I, phi, nu).
#include <cuda_runtime.h>

#include "gsis_internal.cuh"

namespace gsis {

namespace {

constexpr double kInvFourPi = 0.079577471545947667884441881686257;   // 1 / (4 pi)

// r0 = b - D guess (FP32 copy) and the fixed-order sums r0.r0, b.b
// (last-block ticket): the first residual of the synthetic solver for a
// general right-hand side.
__global__ void __launch_bounds__(kRedBlock) resid_kernel(int nx, int ny, const double* __restrict__ b,
                                                          const double* __restrict__ guess,
                                                          const double* __restrict__ diag,
                                                          const double* __restrict__ cx,
                                                          const double* __restrict__ cy, float* r0, double* partials,
                                                          double* norms, Status* status)
{
    __shared__ double sm[33];
    __shared__ int am_last;
    if (ld_volatile_int(&status->done)) return;
    const int N = nx * ny;
    double lrr = 0.0, lbb = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const int j = c / nx, i = c - j * nx;
        double dg = diag[c] * guess[c];
        if (i + 1 < nx) dg -= cx[c] * guess[c + 1];
        if (i > 0) dg -= cx[c - 1] * guess[c - 1];
        if (j + 1 < ny) dg -= cy[c] * guess[c + nx];
        if (j > 0) dg -= cy[c - nx] * guess[c - nx];
        const double bv = b[c], rv = bv - dg;
        r0[c] = (float)rv;
        lrr += rv * rv;
        lbb += bv * bv;
    }
    lrr = block_sum(lrr, sm);
    lbb = block_sum(lbb, sm);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = lrr;
        partials[gridDim.x + blockIdx.x] = lbb;
        __threadfence();
        const unsigned t = atomicAdd(&status->ticket, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    if (threadIdx.x < 32) {
        __threadfence();
        const double srr = warp_sum_array(partials, gridDim.x);
        const double sbb = warp_sum_array(partials + gridDim.x, gridDim.x);
        if (threadIdx.x == 0) {
            norms[0] = srr;
            norms[1] = sbb;
            status->ticket = 0u;
        }
    }
}

// Adjoint of the face-averaged high-order flux of the right-hand side
// (b_c -= A (HoT_c + HoT_nb)/2 . n on every interior face):
//   hx_c = dy_j/2 (nu_E - nu_c) [E exists] + dy_j/2 (nu_c - nu_W) [W exists], same in y;
// also keeps nu for the next solve's initial guess.
__global__ void hbar_kernel(int nx, int ny, const double* __restrict__ dx, const double* __restrict__ dy,
                            const double* __restrict__ nu_new, double* nu_keep, double* hx, double* hy,
                            const int* done)
{
    if (ld_volatile_int(done)) return;
    const int N = nx * ny;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const int j = c / nx, i = c - j * nx;
        const double n0 = nu_new[c];
        double vx = 0.0, vy = 0.0;
        if (i + 1 < nx) vx += 0.5 * dy[j] * (nu_new[c + 1] - n0);
        if (i > 0) vx += 0.5 * dy[j] * (n0 - nu_new[c - 1]);
        if (j + 1 < ny) vy += 0.5 * dx[i] * (nu_new[c + nx] - n0);
        if (j > 0) vy += 0.5 * dx[i] * (n0 - nu_new[c - nx]);
        nu_keep[c] = n0;
        hx[c] = vx;
        hy[c] = vy;
    }
}

// rho_bar_1/2 = sum over boundary faces of A beta nu_c  +  (ALSM gradient)^T h_bar
// with the owner-cell weights hw (HoT_c = F_c + sum_nb hw_c,nb (rho_nb - rho_c)):
//   rb_c = -(hwE_c + hwW_c) hx_c - (hwN_c + hwS_c) hy_c
//          + hwE_W hx_W + hwW_E hx_E + hwN_S hy_S + hwS_N hy_N;
// the adjoint of the kinetic boundary flux, F_bar_b = -A nu_c, enters the
// transposed sweep as the inflow -w_k V_c nu_c of every boundary face.
__global__ void rbar_kernel(int nx, int ny, int K, const double* __restrict__ dx, const double* __restrict__ dy,
                            const double* __restrict__ hw, const double* __restrict__ bface,
                            const double* __restrict__ ow, const double* __restrict__ nu,
                            const double* __restrict__ hx, const double* __restrict__ hy,
                            const double* __restrict__ extra, double* rb, float* rb_f, float* hx_f, float* hy_f,
                            double* inflow_adj, const int* done)
{
    if (ld_volatile_int(done)) return;
    const int N = nx * ny;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const int j = c / nx, i = c - j * nx;
        double v = -(hw[c] + hw[N + c]) * hx[c] - (hw[2 * N + c] + hw[3 * N + c]) * hy[c];
        if (i > 0) v += hw[c - 1] * hx[c - 1];                    // W's east weight
        if (i + 1 < nx) v += hw[N + c + 1] * hx[c + 1];           // E's west weight
        if (j > 0) v += hw[2 * N + c - nx] * hy[c - nx];          // S's north weight
        if (j + 1 < ny) v += hw[3 * N + c + nx] * hy[c + nx];     // N's south weight
        const double n0 = nu[c];
        if (i == 0) v += bface[j] * n0;
        if (i == nx - 1) v += bface[ny + j] * n0;
        if (j == 0) v += bface[2 * ny + i] * n0;
        if (j == ny - 1) v += bface[2 * ny + nx + i] * n0;
        if (extra) v += extra[c];
        rb[c] = v;
        if (rb_f) {
            rb_f[c] = (float)v;
            hx_f[c] = (float)hx[c];
            hy_f[c] = (float)hy[c];
        }
    }
    // boundary faces (W j, E ny+j, S 2ny+i, N 2ny+nx+i) x directions
    const int nbf = 2 * (nx + ny);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nbf * K; t += gridDim.x * blockDim.x) {
        const int f = t / K, k = t - f * K;
        int c;
        if (f < ny) c = nx * f;
        else if (f < 2 * ny) c = nx - 1 + nx * (f - ny);
        else if (f < 2 * ny + nx) c = f - 2 * ny;
        else c = (f - 2 * ny - nx) + nx * (ny - 1);
        const int jc = c / nx, ic = c - jc * nx;
        inflow_adj[t] = -ow[k] * dx[ic] * dy[jc] * nu[c];
    }
}

// lam_new = g + (sigma_s/4pi) sum_s phi_s (directions in sorted order), Err of
// lam (Eq. (Err_W) applied to lam), iteration control; lam_new also becomes
// the right-hand side of the next synthetic solve.
template <typename T>
struct AdjUpdArgs {
    int nx, ny, N, K;
    const double* dx; const double* dy;
    const double* sigma_s; const double* g;
    const T* phi;
    double* lam; double* b;
    double tol;
    int fixed_iters, max_iter;
    double* partials;
    double* hist;
    Status* status;
};

template <typename T>
__global__ void __launch_bounds__(kRedBlock) adj_update_kernel(const AdjUpdArgs<T> a)
{
    __shared__ double sm[33];
    __shared__ int am_last;
    if (ld_volatile_int(&a.status->done)) return;
    double num = 0.0, den = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.N; c += gridDim.x * blockDim.x) {
        const int j = c / a.nx, i = c - j * a.nx;
        double sp = 0.0;
        for (int s = 0; s < a.K; ++s) sp += (double)a.phi[(size_t)s * a.N + c];
        const double nw = a.g[c] + a.sigma_s[c] * kInvFourPi * sp;
        const double od = a.lam[c];
        const double V = a.dx[i] * a.dy[j];
        num += (nw - od) * (nw - od) * V;
        den += nw * nw * V;
        a.lam[c] = nw;
        a.b[c] = nw;
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

// d(HoT contribution N / (3 sigma_i S)) of owner cell i along one axis with
// respect to sigma_t of i (dself), of its + neighbour (dplus) and of its -
// neighbour (dminus).  N = dP (rho_P - rho_i) + dM (rho_M - rho_i),
// S = dP^2 + dM^2, dP = h_i/2 + (sig_P/sig_i) h_P/2, dM = -(h_i/2 + (sig_M/sig_i) h_M/2)
// (Eqs. (shifted_j), (new_vector), (LSF_mdf) on the Cartesian mesh).
struct HotDeriv {
    double dself, dplus, dminus;
};

__device__ HotDeriv hot_deriv(double sig, double rho, double h, bool hasP, double sigP, double rhoP, double hP,
                              bool hasM, double sigM, double rhoM, double hM)
{
    HotDeriv r{0.0, 0.0, 0.0};
    const double dP = hasP ? 0.5 * h + (sigP / sig) * 0.5 * hP : 0.0;
    const double dM = hasM ? -(0.5 * h + (sigM / sig) * 0.5 * hM) : 0.0;
    const double S = dP * dP + dM * dM;
    if (S <= 0.0) return r;
    const double DP = hasP ? rhoP - rho : 0.0, DM = hasM ? rhoM - rho : 0.0;
    const double Nn = dP * DP + dM * DM;
    const double c3 = 1.0 / (3.0 * sig * S);
    // with respect to sigma_i
    const double dPs = hasP ? -sigP * hP / (2.0 * sig * sig) : 0.0;
    const double dMs = hasM ? sigM * hM / (2.0 * sig * sig) : 0.0;
    const double Ns = dPs * DP + dMs * DM, Ss = 2.0 * (dP * dPs + dM * dMs);
    r.dself = Ns * c3 - Nn * Ss * c3 / S - Nn * c3 / sig;
    if (hasP) {
        const double d = hP / (2.0 * sig);
        r.dplus = d * DP * c3 - Nn * 2.0 * dP * d * c3 / S;
    }
    if (hasM) {
        const double d = -hM / (2.0 * sig);
        r.dminus = d * DM * c3 - Nn * 2.0 * dM * d * c3 / S;
    }
    return r;
}

template <typename T>
struct GradArgs {
    int nx, ny, N, K;
    const double* dx; const double* dy;
    const double* sigt;
    const double* rho;      // rho*
    const double* rho_h;    // rho_1/2 of the kinetic step at rho*
    const double* nu; const double* hx; const double* hy;
    const T* phi; const T* I;
    const int* refl;
    double* grad_sa; double* grad_ss;
};

// dJ/dsigma_a, dJ/dsigma_s of cell c = explicit derivative of the Lagrangian:
//   kinetic:    sum_k phi_k (ds/dsigma - I_k dd/dsigma_t)   (ds_c/dsigma_s,c = rho*_c / 4pi)
//   synthetic:  nu.(db/dsigma) - nu.(dD/dsigma) rho*
// with b depending on sigma_t through the HoT weights and the boundary beta,
// D through Gamma_f = 2/(3 (sig_c h_c + sig_n h_n)) (Eq. (Gamma_ij_com2)),
// beta_f = 2/(3 sig_c h) + 1/4 and V sigma_a on the diagonal.
// nu.(db/dsigma_c) - nu.(dD/dsigma_c) rho* of cell c: b depends on sigma_t
// through the HoT weights and the boundary beta, D through
// Gamma_f = 2/(3 (sig_c h_c + sig_n h_n)) (Eq. (Gamma_ij_com2)) and
// beta_f = 2/(3 sig_c h) + 1/4 (V sigma_a on the diagonal is left to the caller).
template <typename T>
__device__ double synthetic_sigma_terms(const GradArgs<T>& a, int c)
{
    const int nx = a.nx, ny = a.ny;
    const int j = c / nx, i = c - j * nx;
    const double st = a.sigt[c], r0 = a.rho[c], n0 = a.nu[c], hxc = a.dx[i], hyc = a.dy[j];
    double E = 0.0;
    // -nu.(dD/dsigma_c) rho*: interior faces
    auto face = [&](int nb, double hc, double hn, double A) {
        const double den = st * hc + a.sigt[nb] * hn;
        const double dG = -2.0 * hc / (3.0 * den * den);
        E -= A * dG * (n0 - a.nu[nb]) * (r0 - a.rho[nb]);
    };
    if (i + 1 < nx) face(c + 1, hxc, a.dx[i + 1], hyc);
    if (i > 0) face(c - 1, hxc, a.dx[i - 1], hyc);
    if (j + 1 < ny) face(c + nx, hyc, a.dy[j + 1], hxc);
    if (j > 0) face(c - nx, hyc, a.dy[j - 1], hxc);
    // boundary faces: beta in D (-) and in b (+ A beta rho_1/2)
    auto bnd = [&](double h, double A) {
        const double dB = -2.0 / (3.0 * st * st * h);
        E += A * dB * n0 * (a.rho_h[c] - r0);
    };
    if (i == 0) bnd(hxc, hyc);
    if (i == nx - 1) bnd(hxc, hyc);
    if (j == 0) bnd(hyc, hxc);
    if (j == ny - 1) bnd(hyc, hxc);
    // nu.(db/dsigma) through the HoT weights of c and of its neighbours
    auto hotx = [&](int ci) {
        const int jj = ci / nx, ii = ci - jj * nx;
        const bool P = ii + 1 < nx, M = ii > 0;
        return hot_deriv(a.sigt[ci], a.rho_h[ci], a.dx[ii], P, P ? a.sigt[ci + 1] : 1.0,
                         P ? a.rho_h[ci + 1] : 0.0, P ? a.dx[ii + 1] : 0.0, M, M ? a.sigt[ci - 1] : 1.0,
                         M ? a.rho_h[ci - 1] : 0.0, M ? a.dx[ii - 1] : 0.0);
    };
    auto hoty = [&](int ci) {
        const int jj = ci / nx;
        const bool P = jj + 1 < ny, M = jj > 0;
        return hot_deriv(a.sigt[ci], a.rho_h[ci], a.dy[jj], P, P ? a.sigt[ci + nx] : 1.0,
                         P ? a.rho_h[ci + nx] : 0.0, P ? a.dy[jj + 1] : 0.0, M, M ? a.sigt[ci - nx] : 1.0,
                         M ? a.rho_h[ci - nx] : 0.0, M ? a.dy[jj - 1] : 0.0);
    };
    E += a.hx[c] * hotx(c).dself + a.hy[c] * hoty(c).dself;
    if (i > 0) E += a.hx[c - 1] * hotx(c - 1).dplus;        // c is the + neighbour of W
    if (i + 1 < nx) E += a.hx[c + 1] * hotx(c + 1).dminus;  // c is the - neighbour of E
    if (j > 0) E += a.hy[c - nx] * hoty(c - nx).dplus;
    if (j + 1 < ny) E += a.hy[c + nx] * hoty(c + nx).dminus;
    return E;
}

// dJ/dsigma_a, dJ/dsigma_s of cell c = explicit derivative of the Lagrangian:
//   kinetic:    sum_k phi_k (ds/dsigma - I_k dd/dsigma_t)   (ds_c/dsigma_s,c = rho*_c / 4pi)
//   synthetic:  nu.(db/dsigma) - nu.(dD/dsigma) rho*  (synthetic_sigma_terms, and
//               -V nu rho* from V sigma_a on the diagonal)
template <typename T>
__global__ void adj_grad_kernel(const GradArgs<T> a)
{
    const int nx = a.nx, N = a.N;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const int j = c / nx, i = c - j * nx;
        double sphi = 0.0, sphiI = 0.0;
        for (int s = 0; s < a.K; ++s) {
            const double ph = (double)a.phi[(size_t)s * N + c];
            sphi += ph;
            sphiI += ph * (double)a.I[(size_t)a.refl[s] * N + c];
        }
        const double r0 = a.rho[c], n0 = a.nu[c];
        const double V = a.dx[i] * a.dy[j];
        const double E = synthetic_sigma_terms(a, c);
        a.grad_ss[c] = r0 * kInvFourPi * sphi - sphiI + E;
        a.grad_sa[c] = -sphiI + E - V * n0 * r0;
    }
}

// ---------------------------------------------------- time-step adjoint
// Step n of a backward-Euler GSIS run at its fixed point (I^h, rho, T), with
// kappa = 4 a c T^3, D2 = C_v/dt + kappa sigma_a, f = (C_v/dt)/D2 and the
// adjoints (I', rho', T') of its output state, carried as phi' (I' = phi'/(c dt)):
//   A_k^T phi_k = y_I,k + (db/dI_k)^T nu,  y_I,k = (phi'_k - w_k sum_j phi'_j/4pi)/(c dt),
//   D' nu = y_rho + sigma_a y_T/D2 + ((sigma_s + (1 - f) sigma_a)/4pi) sum_k phi_k,
//   D' = D_steady + diag(V (1/(c dt) + f sigma_a - sigma_a)),
//   tau = (y_T + (sigma_a kappa/4pi) sum_k phi_k + V sigma_a kappa nu)/D2.
// The part of phi from the carried intensities, chi_k = A_k^{-T}(phi'_k/(c dt)),
// is one transposed sweep per step; the isotropic part of y_I joins rho_bar.
struct TdAdjArgs {
    int nx, ny, N;
    const double* dx; const double* dy;
    const double* sigma_a; const double* sigma_s;
    TdAdjVecs v;
    double* diag;
};

__global__ void td_adj_setup_kernel(const TdAdjArgs a)
{
    const TdAdjVecs& v = a.v;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.N; c += gridDim.x * blockDim.x) {
        const int j = c / a.nx, i = c - j * a.nx;
        const double V = a.dx[i] * a.dy[j];
        const double sa = a.sigma_a[c], t = v.T[c];
        const double kap = 4.0 * v.ac * t * t * t;
        const double D2 = fma(kap, sa, v.cv_dt);
        const double f = v.cv_dt / D2;
        a.diag[c] = fma(V, v.inv_cdt + fma(f, sa, -sa), v.diag0[c]);
        v.sig_eff[c] = fma(1.0 - f, sa, a.sigma_s[c]);
        v.c0[c] = v.ybar_rho[c] + sa * v.ybar_T[c] / D2;
        v.rb_extra[c] = -v.inv_cdt * v.sphi[c] * kInvFourPi;
    }
}

// c = c0 + (sig_eff/4pi) sum_k chi_k; the first lam and right-hand side.
template <typename T>
__global__ void td_adj_start_kernel(const TdAdjArgs a, int K, double* lam, double* b)
{
    const TdAdjVecs& v = a.v;
    const T* chi = static_cast<const T*>(v.chi);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.N; c += gridDim.x * blockDim.x) {
        double sx = 0.0;
        if (chi)
            for (int s = 0; s < K; ++s) sx += (double)chi[(size_t)s * a.N + c];
        const double cv = fma(v.sig_eff[c] * kInvFourPi, sx, v.c0[c]);
        v.c0[c] = cv;
        lam[c] = cv;
        b[c] = cv;
    }
}

// phi = phi_A + chi (carried to the previous step), tau, the step's explicit
// terms added to the gradient, and the adjoints of the step's input state:
//   y_rho' = (V nu + sum_k phi_k/4pi)/(c dt),  y_T' = tau C_v/dt.
// Explicit terms beyond the steady ones (sigma_a only): the emission in the
// kinetic source (phi(T)/4pi) sum_k phi_k, in the synthetic balance
// V nu phi(T), and the material equation tau (rho - phi(T)).
template <typename T>
__global__ void td_adj_grad_kernel(const GradArgs<T> a, const TdAdjArgs t)
{
    const TdAdjVecs& v = t.v;
    const T* chi = static_cast<const T*>(v.chi);
    T* carry = static_cast<T*>(v.carry);
    const int nx = a.nx, N = a.N;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const int j = c / nx, i = c - j * nx;
        double sphi = 0.0, sphiI = 0.0;
        for (int s = 0; s < a.K; ++s) {
            const size_t o = (size_t)s * N + c;
            T ph = a.phi[o];
            if (chi) ph += chi[o];
            carry[o] = ph;
            sphi += (double)ph;
            sphiI += (double)ph * (double)a.I[(size_t)a.refl[s] * N + c];
        }
        const double r0 = a.rho[c], n0 = a.nu[c];
        const double V = a.dx[i] * a.dy[j];
        const double sa = t.sigma_a[c], tc = v.T[c];
        const double kap = 4.0 * v.ac * tc * tc * tc;
        const double D2 = fma(kap, sa, v.cv_dt);
        const double emis = v.ac * tc * tc * tc * tc;
        const double tau = (v.ybar_T[c] + sa * kap * (kInvFourPi * sphi + V * n0)) / D2;
        const double E = synthetic_sigma_terms(a, c);
        a.grad_ss[c] += r0 * kInvFourPi * sphi - sphiI + E;
        a.grad_sa[c] += -sphiI + E - V * n0 * r0 + emis * kInvFourPi * sphi + V * n0 * emis + tau * (r0 - emis);
        v.ybar_rho[c] = v.inv_cdt * fma(V, n0, kInvFourPi * sphi);
        v.ybar_T[c] = tau * v.cv_dt;
        v.sphi[c] = sphi;
    }
}

int grid_for(long long n, int block, int cap)
{
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

template <typename T>
cudaError_t launch_adj_update_t(const Plan& P, cudaStream_t st)
{
    AdjUpdArgs<T> a{};
    a.nx = P.nx; a.ny = P.ny; a.N = P.N; a.K = P.K;
    a.dx = P.dx; a.dy = P.dy;
    a.sigma_s = P.adj_sig ? P.adj_sig : P.sigma_s; a.g = P.g;
    a.phi = static_cast<const T*>(P.Iadj);
    a.lam = P.lam; a.b = P.b;
    a.tol = P.tol; a.fixed_iters = P.fixed_iters; a.max_iter = P.max_iter;
    a.partials = P.partials + (size_t)9 * kMaxCgBlocks;
    a.hist = P.hist;
    a.status = P.status;
    adj_update_kernel<T><<<P.red_grid, kRedBlock, 0, st>>>(a);
    return cudaGetLastError();
}


TdAdjArgs td_adj_args(const Plan& P, const TdAdjVecs& v)
{
    TdAdjArgs a{};
    a.nx = P.nx; a.ny = P.ny; a.N = P.N;
    a.dx = P.dx; a.dy = P.dy;
    a.sigma_a = P.sigma_a; a.sigma_s = P.sigma_s;
    a.v = v;
    a.diag = P.diag;
    return a;
}

template <typename T>
GradArgs<T> grad_args(const Plan& P, double* gsa, double* gss)
{
    GradArgs<T> a{};
    a.nx = P.nx; a.ny = P.ny; a.N = P.N; a.K = P.K;
    a.dx = P.dx; a.dy = P.dy; a.sigt = P.sigt; a.rho = P.rho_m; a.rho_h = P.rho_h;
    a.nu = P.nu; a.hx = P.adj_x; a.hy = P.adj_y;
    a.phi = static_cast<const T*>(P.Iadj);
    a.I = static_cast<const T*>(P.I);
    a.refl = P.refl;
    a.grad_sa = gsa; a.grad_ss = gss;
    return a;
}

}  // namespace

cudaError_t launch_td_adjoint_setup(const Plan& P, const TdAdjVecs& v, cudaStream_t st)
{
    td_adj_setup_kernel<<<grid_for(P.N, 256, P.num_sms * 8), 256, 0, st>>>(td_adj_args(P, v));
    return cudaGetLastError();
}

cudaError_t launch_td_adjoint_start(const Plan& P, const TdAdjVecs& v, cudaStream_t st)
{
    const int g = grid_for(P.N, 256, P.num_sms * 8);
    if (P.fp32) td_adj_start_kernel<float><<<g, 256, 0, st>>>(td_adj_args(P, v), P.K, P.lam, P.b);
    else td_adj_start_kernel<double><<<g, 256, 0, st>>>(td_adj_args(P, v), P.K, P.lam, P.b);
    return cudaGetLastError();
}

cudaError_t launch_td_adjoint_gradient(const Plan& P, const TdAdjVecs& v, double* grad_sa, double* grad_ss,
                                       cudaStream_t st)
{
    const int g = grid_for(P.N, 128, P.num_sms * 8);
    if (P.fp32) td_adj_grad_kernel<float><<<g, 128, 0, st>>>(grad_args<float>(P, grad_sa, grad_ss), td_adj_args(P, v));
    else td_adj_grad_kernel<double><<<g, 128, 0, st>>>(grad_args<double>(P, grad_sa, grad_ss), td_adj_args(P, v));
    return cudaGetLastError();
}

cudaError_t launch_synth_resid(const Plan& P, const double* b, const double* guess, cudaStream_t st)
{
    resid_kernel<<<P.red_grid, kRedBlock, 0, st>>>(P.nx, P.ny, b, guess, P.diag, P.cx, P.cy, P.mg.r0, P.partials,
                                                   P.partials + (size_t)4 * kMaxCgBlocks, P.status);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_rhs(const Plan& P, const double* nu_new, cudaStream_t st)
{
    const int g = grid_for(P.N, 256, P.num_sms * 8);
    hbar_kernel<<<g, 256, 0, st>>>(P.nx, P.ny, P.dx, P.dy, nu_new, P.nu, P.adj_x, P.adj_y, &P.status->done);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    rbar_kernel<<<g, 256, 0, st>>>(P.nx, P.ny, P.K, P.dx, P.dy, P.hw, P.bface, P.ow, P.nu, P.adj_x, P.adj_y,
                                   P.adj_rb_extra, P.adj_a, P.fp32 ? P.adj_a_f : nullptr, P.adj_x_f, P.adj_y_f,
                                   P.adj_inflow, &P.status->done);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_update(const Plan& P, cudaStream_t st)
{
    return P.fp32 ? launch_adj_update_t<float>(P, st) : launch_adj_update_t<double>(P, st);
}

template <typename T>
cudaError_t launch_adj_grad_t(const Plan& P, double* gsa, double* gss, cudaStream_t st)
{
    adj_grad_kernel<T><<<grid_for(P.N, 128, P.num_sms * 8), 128, 0, st>>>(grad_args<T>(P, gsa, gss));
    return cudaGetLastError();
}

cudaError_t launch_adjoint_gradient(const Plan& P, double* grad_sa, double* grad_ss, cudaStream_t st)
{
    return P.fp32 ? launch_adj_grad_t<float>(P, grad_sa, grad_ss, st) : launch_adj_grad_t<double>(P, grad_sa, grad_ss, st);
}

}  // namespace gsis
