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
// The residual kernel is tiled (a cell tile plus halo per CTA, each limited
// gradient computed once); the boundary flux reads global memory.
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

// Limited gradient from the cell value, the existing face neighbours' values
// and the least-squares weights.  The Barth-Jespersen factor uses that the
// four face changes are +-dfx, +-dfy: min over faces of the admissible ratio
// = min(hi - Ic, Ic - lo) / max(|dfx|, |dfy|) (one division, and none when no
// face needs limiting; correctly rounded division is monotone, so this is
// the per-face minimum exactly).
template <typename T>
__device__ __forceinline__ void limited_gradient_vals(T Ic, bool hE, T vE, bool hW, T vW, bool hN, T vN, bool hS,
                                                      T vS, T wE, T wW, T wN, T wS, T hx, T hy, int limiter, T& gx,
                                                      T& gy)
{
    T lo = Ic, hi = Ic;
    gx = T(0);
    gy = T(0);
    if (hE) { gx = fma(wE, vE - Ic, gx); lo = fmin(lo, vE); hi = fmax(hi, vE); }
    if (hW) { gx = fma(wW, vW - Ic, gx); lo = fmin(lo, vW); hi = fmax(hi, vW); }
    if (hN) { gy = fma(wN, vN - Ic, gy); lo = fmin(lo, vN); hi = fmax(hi, vN); }
    if (hS) { gy = fma(wS, vS - Ic, gy); lo = fmin(lo, vS); hi = fmax(hi, vS); }
    if (limiter != 0) return;
    const T dm = fmax(fabs(T(0.5) * hx * gx), fabs(T(0.5) * hy * gy));
    const T room = fmin(hi - Ic, Ic - lo);
    if (dm > T(0) && room < dm) {
        const T psi = room / dm;
        gx *= psi;
        gy *= psi;
    }
}

// Limited gradient of ordinate Is at cell (i, j), values from global memory.
template <typename T>
__device__ __forceinline__ void limited_gradient(const Uw2Args<T>& a, const T* Is, int i, int j, T& gx, T& gy)
{
    const int nx = a.nx, ny = a.ny, N = a.N;
    const int c = i + nx * j;
    const bool hE = i + 1 < nx, hW = i > 0, hN = j + 1 < ny, hS = j > 0;
    limited_gradient_vals(value(a, Is, c), hE, hE ? value(a, Is, c + 1) : T(0), hW, hW ? value(a, Is, c - 1) : T(0),
                          hN, hN ? value(a, Is, c + nx) : T(0), hS, hS ? value(a, Is, c - nx) : T(0), a.gw[c],
                          a.gw[N + c], a.gw[2 * (size_t)N + c], a.gw[3 * (size_t)N + c], (T)a.dx[i], (T)a.dy[j],
                          a.limiter, gx, gy);
}

// Tiled residual: a CTA takes a TX x TY tile of cells and DPB ordinates; per
// ordinate the intensities of the tile and a two-cell halo go to shared
// memory, the limited gradients of the tile and a one-cell halo are computed
// once, then every tile cell assembles its residual from its own and its
// upwind neighbours' reconstructions.
constexpr int kTX = 32, kTY = 8, kLX = kTX + 4, kLY = kTY + 4, kGX = kTX + 2, kGY = kTY + 2;
constexpr int kDPB = 8;

template <typename T>
__global__ void __launch_bounds__(256) uw2_residual_kernel(const Uw2Args<T> a)
{
    __shared__ T sI[kLY][kLX];
    __shared__ T sgx[kGY][kGX], sgy[kGY][kGX];
    if (a.done && ld_volatile_int(a.done)) return;
    const int nx = a.nx, ny = a.ny, N = a.N, K = a.K;
    const int i0 = blockIdx.x * kTX, j0 = blockIdx.y * kTY;
    const int s0 = blockIdx.z * kDPB, s1 = min(K, s0 + kDPB);
    const int tid = threadIdx.x;
    // gradient-region cells of this thread (fixed across ordinates): weights in registers
    constexpr int kG = (kGX * kGY + 255) / 256;
    int gcell[kG];
    T w4[kG][4], ghx[kG], ghy[kG];
#pragma unroll
    for (int u = 0; u < kG; ++u) {
        const int q = tid + 256 * u;
        gcell[u] = -1;
        if (q < kGX * kGY) {
            const int gr = q / kGX, gc = q - gr * kGX;
            const int i = i0 - 1 + gc, j = j0 - 1 + gr;
            if (i >= 0 && i < nx && j >= 0 && j < ny) {
                const int c = i + nx * j;
                gcell[u] = q;
                w4[u][0] = a.gw[c];
                w4[u][1] = a.gw[N + c];
                w4[u][2] = a.gw[2 * (size_t)N + c];
                w4[u][3] = a.gw[3 * (size_t)N + c];
                ghx[u] = (T)a.dx[i];
                ghy[u] = (T)a.dy[j];
            }
        }
    }
    // this thread's tile cell
    const int tx = tid % kTX, ty = tid / kTX;
    const int ic = i0 + tx, jc = j0 + ty;
    const bool mine = ic < nx && jc < ny;
    const int cc = mine ? ic + nx * jc : 0;
    T srcc = T(0), sigc = T(0), hxc = T(1), hyc = T(1), hxW = T(1), hxE = T(1), hyS = T(1), hyN = T(1);
    if (mine) {
        srcc = a.src[cc];
        sigc = a.sigt[cc];
        hxc = (T)a.dx[ic];
        hyc = (T)a.dy[jc];
        if (ic > 0) hxW = (T)a.dx[ic - 1];
        if (ic + 1 < nx) hxE = (T)a.dx[ic + 1];
        if (jc > 0) hyS = (T)a.dy[jc - 1];
        if (jc + 1 < ny) hyN = (T)a.dy[jc + 1];
    }
    for (int s = s0; s < s1; ++s) {
        const T* Is = a.I + (size_t)s * N;
        for (int q = tid; q < kLX * kLY; q += 256) {
            const int r = q / kLX, c = q - r * kLX;
            const int i = i0 - 2 + c, j = j0 - 2 + r;
            T v = T(0);
            if (i >= 0 && i < nx && j >= 0 && j < ny) v = value(a, Is, i + nx * j);
            sI[r][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kG; ++u) {
            if (gcell[u] < 0) continue;
            const int q = gcell[u];
            const int gr = q / kGX, gc = q - gr * kGX;
            const int i = i0 - 1 + gc, j = j0 - 1 + gr;
            const int r = gr + 1, c = gc + 1;   // position in sI
            T gx, gy;
            limited_gradient_vals(sI[r][c], i + 1 < nx, sI[r][c + 1], i > 0, sI[r][c - 1], j + 1 < ny, sI[r + 1][c],
                                  j > 0, sI[r - 1][c], w4[u][0], w4[u][1], w4[u][2], w4[u][3], ghx[u], ghy[u],
                                  a.limiter, gx, gy);
            sgx[gr][gc] = gx;
            sgy[gr][gc] = gy;
        }
        __syncthreads();
        if (mine) {
            const double mu = a.qmu[s], eta = a.qeta[s];
            const int k = a.perm[s];
            const int gr = ty + 1, gc = tx + 1, r = ty + 2, c = tx + 2;
            const T Ic = sI[r][c], gx = sgx[gr][gc], gy = sgy[gr][gc];
            T fE, fW, fN, fS;
            if (mu >= 0.0) {
                fE = fma(T(0.5) * hxc, gx, Ic);
                fW = ic > 0 ? fma(T(0.5) * hxW, sgx[gr][gc - 1], sI[r][c - 1])
                            : (a.inflow ? (T)a.inflow[(size_t)jc * K + k] : T(0));
            } else {
                fW = fma(T(-0.5) * hxc, gx, Ic);
                fE = ic + 1 < nx ? fma(T(-0.5) * hxE, sgx[gr][gc + 1], sI[r][c + 1])
                                 : (a.inflow ? (T)a.inflow[(size_t)(ny + jc) * K + k] : T(0));
            }
            if (eta >= 0.0) {
                fN = fma(T(0.5) * hyc, gy, Ic);
                fS = jc > 0 ? fma(T(0.5) * hyS, sgy[gr - 1][gc], sI[r - 1][c])
                            : (a.inflow ? (T)a.inflow[(size_t)(2 * ny + ic) * K + k] : T(0));
            } else {
                fS = fma(T(-0.5) * hyc, gy, Ic);
                fN = jc + 1 < ny ? fma(T(-0.5) * hyN, sgy[gr + 1][gc], sI[r + 1][c])
                                 : (a.inflow ? (T)a.inflow[(size_t)(2 * ny + nx + ic) * K + k] : T(0));
            }
            T rr = srcc - sigc * Ic;
            rr -= (T)mu * (fE - fW) / hxc;
            rr -= (T)eta * (fN - fS) / hyc;
            a.R[(size_t)s * N + cc] = rr;
        }
        __syncthreads();
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
    const dim3 grid((P.nx + kTX - 1) / kTX, (P.ny + kTY - 1) / kTY, (P.K + kDPB - 1) / kDPB);
    if (P.fp32) uw2_residual_kernel<float><<<grid, 256, 0, st>>>(uw2_args<float>(P, true, &P.status->done));
    else uw2_residual_kernel<double><<<grid, 256, 0, st>>>(uw2_args<double>(P, true, &P.status->done));
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
