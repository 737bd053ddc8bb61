// Second-order upwind (UW2) kinetic step in the paper's delta form (Sec. 4.1):
// the residual of the UW2 equations at the stored intensities, and the
// boundary kinetic flux with reconstructed outgoing face values.  The
// increment sweep itself is the sweep kernel's delta mode (csrc/sweep.cu).
//
// Per ordinate s and cell i (sorted direction index, I^m = I + corr):
//  * least-squares gradient with the adaptive shifted neighbour positions
//    (Sec. 5.2, Eqs. (shifted_j), (new_vector), (LSF_mdf)); on the Cartesian
//    mesh G_x = sum_{E,W} g_j (I_j - I_i) with the set-up weights g_j;
//  * Barth-Jespersen limiter psi (or none): the unlimited change to each face
//    Delta_f = G . (x_f - x_i) is scaled so that no face value leaves
//    [min, max] of the cell and its face neighbours;
//  * face values I_i + psi G . (x_f - x_i) (Eq. (Ii,k)) from the upwind side
//    (Eq. (Iij)), the inflow on incoming boundary faces;
//  * R = S - sigma_t I_i - mu (I_E - I_W)/dx - eta (I_N - I_S)/dy
//    (Eq. (RTE_d_res), steady, per unit volume).
// One thread per (ordinate, cell); it reconstructs its own cell and its two
// upwind neighbours (the neighbours' values come through L1/L2).
#include <cuda_runtime.h>

#include "gsis_internal.cuh"

namespace gsis {

namespace {

template <typename T>
struct Uw2Args {
    int nx, ny, N, K;
    const T* I;                 // [K][N] stored intensities
    const T* corr;              // [N] isotropic correction (I^m = I + corr), or null
    const T* gw;                // [4][N] gradient weights E, W, N, S
    const double* dx; const double* dy;
    const T* src; const T* sigt;
    const double* qmu; const double* qeta; const int* perm;
    const double* inflow;       // [nbf][K] original direction index, or null
    T* R;                       // [K][N] out
    int limiter;                // 0 Barth-Jespersen, 1 none
    const int* done;
};

template <typename T>
__device__ __forceinline__ T value(const Uw2Args<T>& a, const T* Is, int c)
{
    return a.corr ? Is[c] + a.corr[c] : Is[c];
}

// Limited gradient (psi G_x, psi G_y) of ordinate Is at cell (i, j).
template <typename T>
__device__ __forceinline__ void limited_gradient(const Uw2Args<T>& a, const T* Is, int i, int j, T& gx, T& gy)
{
    const int nx = a.nx, ny = a.ny, N = a.N;
    const int c = i + nx * j;
    const T Ic = value(a, Is, c);
    T lo = Ic, hi = Ic;
    gx = T(0);
    gy = T(0);
    if (i + 1 < nx) {
        const T v = value(a, Is, c + 1);
        gx = fma(a.gw[c], v - Ic, gx);
        lo = fmin(lo, v); hi = fmax(hi, v);
    }
    if (i > 0) {
        const T v = value(a, Is, c - 1);
        gx = fma(a.gw[N + c], v - Ic, gx);
        lo = fmin(lo, v); hi = fmax(hi, v);
    }
    if (j + 1 < ny) {
        const T v = value(a, Is, c + nx);
        gy = fma(a.gw[2 * (size_t)N + c], v - Ic, gy);
        lo = fmin(lo, v); hi = fmax(hi, v);
    }
    if (j > 0) {
        const T v = value(a, Is, c - nx);
        gy = fma(a.gw[3 * (size_t)N + c], v - Ic, gy);
        lo = fmin(lo, v); hi = fmax(hi, v);
    }
    if (a.limiter != 0) return;
    const T hx2 = (T)(0.5 * a.dx[i]), hy2 = (T)(0.5 * a.dy[j]);
    const T dfx = hx2 * gx, dfy = hy2 * gy;   // change to the E and N faces (W, S: the negatives)
    T psi = T(1);
    const T deltas[4] = {-dfx, dfx, -dfy, dfy};
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const T d = deltas[f];
        if (d > T(0)) psi = fmin(psi, (hi - Ic) / d);
        else if (d < T(0)) psi = fmin(psi, (lo - Ic) / d);
    }
    gx *= psi;
    gy *= psi;
}

template <typename T>
__global__ void __launch_bounds__(256) uw2_residual_kernel(const Uw2Args<T> a)
{
    if (a.done && ld_volatile_int(a.done)) return;
    const int nx = a.nx, ny = a.ny, N = a.N, K = a.K;
    const size_t tot = (size_t)K * N;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(t / N), c = (int)(t - (size_t)s * N);
        const int j = c / nx, i = c - j * nx;
        const T* Is = a.I + (size_t)s * N;
        const double mu = a.qmu[s], eta = a.qeta[s];
        const int k = a.perm[s];
        const T hx = (T)a.dx[i], hy = (T)a.dy[j];
        const T Ic = value(a, Is, c);
        T gx, gy;
        limited_gradient(a, Is, i, j, gx, gy);
        T fE, fW, fN, fS;   // face values
        if (mu >= 0.0) {
            fE = fma(T(0.5) * hx, gx, Ic);
            if (i > 0) {
                T ux, uy;
                limited_gradient(a, Is, i - 1, j, ux, uy);
                fW = fma(T(0.5) * (T)a.dx[i - 1], ux, value(a, Is, c - 1));
            } else {
                fW = a.inflow ? (T)a.inflow[(size_t)j * K + k] : T(0);
            }
        } else {
            fW = fma(T(-0.5) * hx, gx, Ic);
            if (i + 1 < nx) {
                T ux, uy;
                limited_gradient(a, Is, i + 1, j, ux, uy);
                fE = fma(T(-0.5) * (T)a.dx[i + 1], ux, value(a, Is, c + 1));
            } else {
                fE = a.inflow ? (T)a.inflow[(size_t)(ny + j) * K + k] : T(0);
            }
        }
        if (eta >= 0.0) {
            fN = fma(T(0.5) * hy, gy, Ic);
            if (j > 0) {
                T ux, uy;
                limited_gradient(a, Is, i, j - 1, ux, uy);
                fS = fma(T(0.5) * (T)a.dy[j - 1], uy, value(a, Is, c - nx));
            } else {
                fS = a.inflow ? (T)a.inflow[(size_t)(2 * ny + i) * K + k] : T(0);
            }
        } else {
            fS = fma(T(-0.5) * hy, gy, Ic);
            if (j + 1 < ny) {
                T ux, uy;
                limited_gradient(a, Is, i, j + 1, ux, uy);
                fN = fma(T(-0.5) * (T)a.dy[j + 1], uy, value(a, Is, c + nx));
            } else {
                fN = a.inflow ? (T)a.inflow[(size_t)(2 * ny + nx + i) * K + k] : T(0);
            }
        }
        T r = a.src[c] - a.sigt[c] * Ic;
        r -= (T)mu * (fE - fW) / hx;
        r -= (T)eta * (fN - fS) / hy;
        a.R[t] = r;
    }
}

// Kinetic net flux through every boundary face with UW2 face values of the
// stored intensities (outgoing: reconstructed boundary cell, incoming: inflow);
// one warp per face, lanes over the original direction index.
template <typename T>
__global__ void __launch_bounds__(256) uw2_bflux_kernel(const Uw2Args<T> a, const int* __restrict__ sidx,
                                                        const double* __restrict__ mu, const double* __restrict__ eta,
                                                        const double* __restrict__ w, double* fb)
{
    if (a.done && ld_volatile_int(a.done)) return;
    const int nx = a.nx, ny = a.ny, K = a.K, N = a.N;
    const int nbf = 2 * (nx + ny);
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int f = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; f < nbf; f += warps) {
        int i, j, axis;
        double sgn;
        if (f < ny) { i = 0; j = f; axis = 0; sgn = -1.0; }
        else if (f < 2 * ny) { i = nx - 1; j = f - ny; axis = 0; sgn = 1.0; }
        else if (f < 2 * ny + nx) { i = f - 2 * ny; j = 0; axis = 1; sgn = -1.0; }
        else { i = f - 2 * ny - nx; j = ny - 1; axis = 1; sgn = 1.0; }
        const int c = i + nx * j;
        T acc = T(0);
        for (int k = lane; k < K; k += 32) {
            const double on = sgn * (axis == 0 ? mu[k] : eta[k]);
            T Iface;
            if (on >= 0.0) {
                const T* Is = a.I + (size_t)sidx[k] * N;
                T gx, gy;
                limited_gradient(a, Is, i, j, gx, gy);
                const T h = (T)(axis == 0 ? a.dx[i] : a.dy[j]);
                Iface = fma((T)sgn * T(0.5) * h, axis == 0 ? gx : gy, value(a, Is, c));
            } else {
                Iface = a.inflow ? (T)a.inflow[(size_t)f * K + k] : T(0);
            }
            acc = fma((T)(w[k] * on), Iface, acc);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (lane == 0) fb[f] = (double)acc;
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
Uw2Args<T> uw2_args(const Plan& P, bool with_corr, const int* done)
{
    Uw2Args<T> a{};
    a.nx = P.nx; a.ny = P.ny; a.N = P.N; a.K = P.K;
    a.I = static_cast<const T*>(P.I);
    a.dx = P.dx; a.dy = P.dy;
    a.qmu = P.qmu; a.qeta = P.qeta; a.perm = P.perm;
    a.inflow = P.inflow;
    a.R = static_cast<T*>(P.R);
    a.limiter = P.limiter;
    a.done = done;
    if constexpr (sizeof(T) == 8) {
        a.corr = with_corr ? P.corr : nullptr;
        a.gw = P.gw; a.src = P.src; a.sigt = P.sigt;
    } else {
        a.corr = with_corr ? P.corr_f : nullptr;
        a.gw = P.gw_f; a.src = P.src_f; a.sigt = P.sigt_f;
    }
    return a;
}

}  // namespace

cudaError_t launch_uw2_residual(const Plan& P, cudaStream_t st)
{
    const long long tot = (long long)P.K * P.N;
    const int g = grid_for(tot, 256, P.num_sms * 16);
    if (P.fp32) uw2_residual_kernel<float><<<g, 256, 0, st>>>(uw2_args<float>(P, true, &P.status->done));
    else uw2_residual_kernel<double><<<g, 256, 0, st>>>(uw2_args<double>(P, true, &P.status->done));
    return cudaGetLastError();
}

cudaError_t launch_uw2_bflux(const Plan& P, double* fb_out, const int* done, cudaStream_t st)
{
    const int g = grid_for((long long)P.nbf * 32, 256, P.num_sms * 4);
    if (P.fp32)
        uw2_bflux_kernel<float><<<g, 256, 0, st>>>(uw2_args<float>(P, false, done), P.sidx, P.omu, P.oeta, P.ow,
                                                   fb_out);
    else
        uw2_bflux_kernel<double><<<g, 256, 0, st>>>(uw2_args<double>(P, false, done), P.sidx, P.omu, P.oeta,
                                                    P.ow, fb_out);
    return cudaGetLastError();
}

}  // namespace gsis
