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

#include <algorithm>

#include <cstring>

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

struct HotArgs {
    int nx, ny;
    const double* hw; const double* rho; const double* Fx; const double* Fy;
    double* hotx; double* hoty;
    const int* done;
};

// HoT = F + G / (3 sigma_t) with the gradient weights of the cell set-up.
// HoT of cell c = (i, j) (Eq. (GSIS_HoT)): F + the least-squares gradient of
// rho with 1/(3 sigma_t) folded into the weights hw; one operation sequence
// for every kernel that forms it, so stored and recomputed values agree bit
// for bit.
__device__ __forceinline__ double hot_x(const double* hw, const double* rho, const double* Fx, int N, int nx,
                                        int c, int i)
{
    const double ri = rho[c];
    double gx = 0.0;
    if (i + 1 < nx) gx = fma(hw[c], rho[c + 1] - ri, gx);
    if (i > 0) gx = fma(hw[N + c], rho[c - 1] - ri, gx);
    return Fx[c] + gx;
}

__device__ __forceinline__ double hot_y(const double* hw, const double* rho, const double* Fy, int N, int nx,
                                        int ny, int c, int j)
{
    const double ri = rho[c];
    double gy = 0.0;
    if (j + 1 < ny) gy = fma(hw[2 * N + c], rho[c + nx] - ri, gy);
    if (j > 0) gy = fma(hw[3 * N + c], rho[c - nx] - ri, gy);
    return Fy[c] + gy;
}

__device__ __forceinline__ void hot_body(const HotArgs& a, int bid, int nblk)
{
    if (ld_volatile_int(a.done)) return;
    const int nx = a.nx, ny = a.ny, N = nx * ny;
    for (int c = bid * blockDim.x + threadIdx.x; c < N; c += nblk * blockDim.x) {
        const int j = c / nx, i = c - j * nx;
        a.hotx[c] = hot_x(a.hw, a.rho, a.Fx, N, nx, c, i);
        a.hoty[c] = hot_y(a.hw, a.rho, a.Fy, N, nx, ny, c, j);
    }
}

__global__ void hot_kernel(const HotArgs a) { hot_body(a, blockIdx.x, gridDim.x); }

struct RhsArgs {
    int nx, ny;
    const double* dx; const double* dy;
    const double* sigt; const double* q; const double* rho_h;
    const double* hotx; const double* hoty; const double* fb; const double* bface;
    const double* hw; const double* Fx; const double* Fy;   // FUSE: HoT recomputed from rho_h, Fx, Fy
    double* b;
    // first residual of the synthetic solve, r0 = b - D guess
    const double* diag; const double* cx; const double* cy; const double* guess;
    float* r0;          // FP32 copy for the inner iteration
    double* partials;   // [2][gridDim]
    double* norms;      // out: [0] = r0.r0, [1] = b.b
    Status* status;
    int resid;          // 0: b only (the planned synthetic solver forms its own first residual)
};

// b, then r0 = b - D guess (five-point D) and the fixed-order sums r0.r0, b.b
// (last-block ticket).  Block bid of the problem's nblk blocks.
// FUSE: HoT formed here at the cell and its neighbours (the same operations
// as hot_body, so the same b) instead of read from hotx / hoty.
template <bool FUSE = false>
__device__ __forceinline__ void rhs_body(const RhsArgs& a, int bid, int nblk)
{
    __shared__ double sm[33];
    __shared__ int am_last;
    if (ld_volatile_int(&a.status->done)) return;
    const int nx = a.nx, ny = a.ny, N = nx * ny;
    const double* dx = a.dx; const double* dy = a.dy;
    const double* hotx = a.hotx; const double* hoty = a.hoty; const double* fb = a.fb;
    double lrr = 0.0, lbb = 0.0;
    for (int c = bid * blockDim.x + threadIdx.x; c < N; c += nblk * blockDim.x) {
        const int j = c / nx, i = c - j * nx;
        const double hx = dx[i], hy = dy[j];
        // explicit fma: the single-problem and batched kernels that inline
        // this body then round identically
        auto HX = [&](int cc, int ii) {
            if constexpr (FUSE) return hot_x(a.hw, a.rho_h, a.Fx, N, nx, cc, ii);
            else return hotx[cc];
        };
        auto HY = [&](int cc, int jj) {
            if constexpr (FUSE) return hot_y(a.hw, a.rho_h, a.Fy, N, nx, ny, cc, jj);
            else return hoty[cc];
        };
        const double hxc = HX(c, i), hyc = HY(c, j);
        double v = hx * hy * a.q[c];
        if (i + 1 < nx) v = fma(-0.5 * hy, hxc + HX(c + 1, i + 1), v);
        if (i > 0) v = fma(0.5 * hy, hxc + HX(c - 1, i - 1), v);
        if (j + 1 < ny) v = fma(-0.5 * hx, hyc + HY(c + nx, j + 1), v);
        if (j > 0) v = fma(0.5 * hx, hyc + HY(c - nx, j - 1), v);
        const double rh = a.rho_h[c];
        const double* bf = a.bface;
        if (i == 0) v -= fma(hy, fb[j], -(bf[j] * rh));
        if (i == nx - 1) v -= fma(hy, fb[ny + j], -(bf[ny + j] * rh));
        if (j == 0) v -= fma(hx, fb[2 * ny + i], -(bf[2 * ny + i] * rh));
        if (j == ny - 1) v -= fma(hx, fb[2 * ny + nx + i], -(bf[2 * ny + nx + i] * rh));
        a.b[c] = v;
        if (!a.resid) continue;
        const double* g = a.guess;
        double dg = a.diag[c] * g[c];
        if (i + 1 < nx) dg = fma(-a.cx[c], g[c + 1], dg);
        if (i > 0) dg = fma(-a.cx[c - 1], g[c - 1], dg);
        if (j + 1 < ny) dg = fma(-a.cy[c], g[c + nx], dg);
        if (j > 0) dg = fma(-a.cy[c - nx], g[c - nx], dg);
        const double rv = v - dg;
        a.r0[c] = (float)rv;
        lrr = fma(rv, rv, lrr);
        lbb = fma(v, v, lbb);
    }
    if (!a.resid) return;   // uniform over the launch
    lrr = block_sum(lrr, sm);
    lbb = block_sum(lbb, sm);
    if (threadIdx.x == 0) {
        a.partials[bid] = lrr;
        a.partials[nblk + bid] = lbb;
        __threadfence();
        const unsigned t = atomicAdd(&a.status->ticket, 1u);
        am_last = (t == (unsigned)nblk - 1u);
    }
    __syncthreads();
    if (!am_last) return;
    if (threadIdx.x < 32) {
        __threadfence();
        const double srr = warp_sum_array(a.partials, nblk);
        const double sbb = warp_sum_array(a.partials + nblk, nblk);
        if (threadIdx.x == 0) {
            a.norms[0] = srr;
            a.norms[1] = sbb;
            a.status->ticket = 0u;
        }
    }
}

template <bool FUSE>
__global__ void __launch_bounds__(kRedBlock) rhs_kernel(const RhsArgs a) { rhs_body<FUSE>(a, blockIdx.x, gridDim.x); }

struct UpdArgs {
    int nx, ny, N;
    const double* dx; const double* dy;
    const double* sigma_s; const double* q; const double* shift;
    const double* rho_new; double* rho_m; const double* rho_h;
    double* src; float* src_f;
    double* corr; float* corr_f;   // second-order delta form: isotropic correction of I (or null)
    // FP64 steady pseudo-time: the next sweep's per-ordinate source
    // X[k][c] = src_c + shift_c I^m[k][c] (null: not formed here)
    int K;
    const double* I;
    double* X;
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
// X[k][c] = fma(sh, I[k][c], s) for every ordinate of cell c; the loads of a
// slab of ordinates are all issued before its stores.
__device__ __forceinline__ void ordinate_row(int K, int N, int c, double sh, double s,
                                             const double* __restrict__ I, double* __restrict__ X)
{
    constexpr int kSlab = 8;
    for (int k0 = 0; k0 < K; k0 += kSlab) {
        double v[kSlab];
#pragma unroll
        for (int kk = 0; kk < kSlab; ++kk) v[kk] = k0 + kk < K ? I[(size_t)(k0 + kk) * N + c] : 0.0;
#pragma unroll
        for (int kk = 0; kk < kSlab; ++kk)
            if (k0 + kk < K) X[(size_t)(k0 + kk) * N + c] = fma(sh, v[kk], s);
    }
}

__device__ __forceinline__ void update_body(const UpdArgs& a, int bid, int nblk)
{
    __shared__ double sm[33];
    __shared__ int am_last;
    if (ld_volatile_int(&a.status->done)) return;
    double num = 0.0, den = 0.0;
    for (int c = bid * blockDim.x + threadIdx.x; c < a.N; c += nblk * blockDim.x) {
        const int j = c / a.nx, i = c - j * a.nx;
        const double V = a.dx[i] * a.dy[j];
        const double nw = a.rho_new[c], od = a.rho_m[c];
        const double d = nw - od;
        // explicit fma (identical rounding in every kernel inlining this body)
        num = fma(d * d, V, num);
        den = fma(nw * nw, V, den);
        a.rho_m[c] = nw;
        double s = fma(a.sigma_s[c], nw, a.q[c]) * kInvFourPi;
        if (a.pt) s = fma(a.shift[c] * (nw - a.rho_h[c]), kInvFourPi, s);
        a.src[c] = s;
        if (a.src_f) a.src_f[c] = (float)s;
        // the same FMA as ordinate_source_kernel: the same bits
        if (a.X) ordinate_row(a.K, a.N, c, a.shift[c], s, a.I, a.X);

        if (a.corr) {   // I^{m+1} = I^{m+1/2} + (rho^{m+1} - rho^{m+1/2})/4pi, kept per cell
            const double cc = (nw - a.rho_h[c]) * kInvFourPi;
            a.corr[c] = cc;
            if (a.corr_f) a.corr_f[c] = (float)cc;
        }
    }
    num = block_sum(num, sm);
    den = block_sum(den, sm);
    err_reduce_decide(num, den, a.partials, a.hist, a.status, a.tol, a.fixed_iters, a.max_iter, bid, nblk, &am_last);
}

__global__ void __launch_bounds__(kRedBlock) update_kernel(const UpdArgs a) { update_body(a, blockIdx.x, gridDim.x); }

// Batched launches: problem p owns blocks [bstart[p], bstart[p + 1]).
template <typename A, void (*BODY)(const A&, int, int)>
__global__ void __launch_bounds__(kRedBlock) batch_kernel(const A* __restrict__ tab, const int* __restrict__ bstart,
                                                          int B)
{
    const int p = batch_find(bstart, B, blockIdx.x);
    const int b0 = __ldg(bstart + p);
    const A a = tab[p];
    BODY(a, blockIdx.x - b0, __ldg(bstart + p + 1) - b0);
}

HotArgs hot_args(const Plan& P, const double* rho_h, const double* Fx, const double* Fy)
{
    HotArgs h{};
    h.nx = P.nx; h.ny = P.ny; h.hw = P.hw; h.rho = rho_h; h.Fx = Fx; h.Fy = Fy;
    h.hotx = P.hotx; h.hoty = P.hoty; h.done = &P.status->done;
    return h;
}

RhsArgs rhs_args(const Plan& P, const double* rho_h, const double* fb, const double* guess)
{
    RhsArgs a{};
    a.nx = P.nx; a.ny = P.ny; a.dx = P.dx; a.dy = P.dy;
    a.sigt = P.sigt; a.q = P.q_syn ? P.q_syn : P.q; a.rho_h = rho_h; a.hotx = P.hotx; a.hoty = P.hoty; a.fb = fb; a.b = P.b;
    a.bface = P.bface;
    a.diag = P.diag; a.cx = P.cx; a.cy = P.cy; a.guess = guess;
    a.r0 = P.mg.r0;
    a.partials = P.partials;
    a.norms = P.partials + (size_t)4 * kMaxCgBlocks;
    a.status = P.status;
    // only the cluster solver reads r0 and the norms; the tiled grid solver
    // (planned: P.synth_tiled) forms its first residual itself
    a.resid = P.synth_grid > 0 && P.synth_tiled ? 0 : 1;
    return a;
}

UpdArgs upd_args(const Plan& P, const double* rho_new)
{
    UpdArgs a{};
    a.nx = P.nx; a.ny = P.ny; a.N = P.N; a.dx = P.dx; a.dy = P.dy;
    a.sigma_s = P.sigma_s; a.q = P.q; a.shift = P.shift;
    a.rho_new = rho_new; a.rho_m = P.rho_m; a.rho_h = P.rho_h;
    a.src = P.src; a.src_f = P.fp32 ? P.src_f : nullptr;
    a.pt = P.pt && P.order == 1;   // second order: the correction is carried explicitly
    a.corr = P.order == 2 ? P.corr : nullptr;
    a.corr_f = P.order == 2 && P.fp32 ? P.corr_f : nullptr;
    // FP64 steady pseudo-time: the next sweeps' sources too (FP32 ones come from
    // ordinate_source_kernel / ord_body, faster there than inside this kernel)
    if (P.order == 1 && !P.In && P.X && !P.fp32) {
        a.K = P.K; a.I = static_cast<const double*>(P.I); a.X = P.X;
    }

    a.tol = P.tol; a.fixed_iters = P.fixed_iters; a.max_iter = P.max_iter;
    a.partials = P.partials + (size_t)9 * kMaxCgBlocks;
    a.hist = P.hist;
    a.status = P.status;
    return a;
}

}  // namespace

cudaError_t launch_hot_rhs(const Plan& P, const double* rho_h, const double* Fx, const double* Fy,
                           const double* fb, const double* guess, cudaStream_t st, bool fuse)
{
    if (fuse) {   // one launch, HoT formed where the right-hand side needs it; hotx / hoty not written
        RhsArgs a = rhs_args(P, rho_h, fb, guess);
        a.hw = P.hw; a.Fx = Fx; a.Fy = Fy;
        rhs_kernel<true><<<P.red_grid, kRedBlock, 0, st>>>(a);
        return cudaGetLastError();
    }
    const int g = grid_for(P.N, 256, P.num_sms * 8);
    hot_kernel<<<g, 256, 0, st>>>(hot_args(P, rho_h, Fx, Fy));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    rhs_kernel<false><<<P.red_grid, kRedBlock, 0, st>>>(rhs_args(P, rho_h, fb, guess));
    return cudaGetLastError();
}

// Ordinates per thread in the per-ordinate source kernels: all their loads
// are in flight before the stores.
template <typename T>
__host__ __device__ constexpr int ord_slab() { return sizeof(T) == 4 ? 16 : 8; }

// X[k][c] = fma(shift_c, I[k][c], src_c) over tiles of (blockDim.x cells) x
// (ord_slab ordinates), tile t = bid, bid + nblk, ...: coalesced rows, no
// per-element division.
template <typename T>
__device__ __forceinline__ void ord_tiles(int N, int K, const T* __restrict__ shift, const T* __restrict__ I,
                                          const T* __restrict__ src, T* __restrict__ X, int bid, int nblk)
{
    constexpr int S = ord_slab<T>();
    const int cb = (N + (int)blockDim.x - 1) / (int)blockDim.x;
    const int ntiles = cb * ((K + S - 1) / S);
    for (int tile = bid; tile < ntiles; tile += nblk) {
        const int slab = tile / cb;
        const int c = (tile - slab * cb) * (int)blockDim.x + (int)threadIdx.x;
        if (c >= N) continue;
        const int k0 = slab * S;
        const T sh = shift[c], sv = src[c];
        const T* Ik = I + (size_t)k0 * N + c;
        T* Xk = X + (size_t)k0 * N + c;
        T v[S];
#pragma unroll
        for (int kk = 0; kk < S; ++kk) v[kk] = k0 + kk < K ? Ik[(size_t)kk * N] : T(0);
#pragma unroll
        for (int kk = 0; kk < S; ++kk)
            if (k0 + kk < K) Xk[(size_t)kk * N] = fma(sh, v[kk], sv);   // float: the FP32 overload
    }
}

int ord_tile_count(int N, int K, int fp32)
{
    const int S = fp32 ? ord_slab<float>() : ord_slab<double>();
    return ((N + kRedBlock - 1) / kRedBlock) * ((K + S - 1) / S);
}

// The pseudo-time / time-step sweep's source per ordinate, formed as that
// sweep would form it: X[k][c] = fma(shift_c, I[k][c], src_c) (FP64 or FP32).
template <typename T>
__global__ void __launch_bounds__(kRedBlock) ordinate_source_kernel(int N, int K, const T* __restrict__ shift,
                                                                    const T* __restrict__ I,
                                                                    const T* __restrict__ src, T* X,
                                                                    const int* done)
{
    if (ld_volatile_int(done)) return;
    ord_tiles<T>(N, K, shift, I, src, X, blockIdx.x, gridDim.x);
}

cudaError_t launch_ordinate_source(const Plan& P, cudaStream_t st)
{
    const int grid = std::max(1, std::min(ord_tile_count(P.N, P.K, P.fp32), P.num_sms * 8));
    // the stored intensities the pseudo-time sweep reads: I^m in place, or a
    // time step's I^n
    const void* iold = P.In ? P.In : P.I;
    if (P.fp32)
        ordinate_source_kernel<float><<<grid, kRedBlock, 0, st>>>(
            P.N, P.K, P.shift_f, static_cast<const float*>(iold), P.src_f, P.X_f, &P.status->done);
    else
        ordinate_source_kernel<double><<<grid, kRedBlock, 0, st>>>(
            P.N, P.K, P.shift, static_cast<const double*>(iold), P.src, P.X, &P.status->done);
    return cudaGetLastError();
}

cudaError_t launch_update(const Plan& P, const double* rho_new, cudaStream_t st)
{
    update_kernel<<<P.red_grid, kRedBlock, 0, st>>>(upd_args(P, rho_new));
    return cudaGetLastError();
}

// Batched records of one GSIS / SI iteration (the arrays the per-problem
// iteration passes); each returns the problem's blocks.
size_t hot_batch_rec_bytes() { return sizeof(HotArgs); }
size_t rhs_batch_rec_bytes() { return sizeof(RhsArgs); }
size_t upd_batch_rec_bytes() { return sizeof(UpdArgs); }

int hot_batch_rec(const Plan& P, void* out)
{
    const HotArgs h = hot_args(P, P.rho_h, P.Fx, P.Fy);
    std::memcpy(out, &h, sizeof(h));
    return grid_for(P.N, kRedBlock, P.num_sms * 8);
}

int rhs_batch_rec(const Plan& P, void* out)
{
    const RhsArgs a = rhs_args(P, P.rho_h, P.fb, P.rho_m);
    std::memcpy(out, &a, sizeof(a));
    return P.red_grid;
}

int upd_batch_rec(const Plan& P, bool gsis, void* out)
{
    const UpdArgs a = upd_args(P, gsis ? P.x : P.rho_h);
    std::memcpy(out, &a, sizeof(a));
    return P.red_grid;
}

cudaError_t launch_hot_rhs_batch(const BatchTables& bt, cudaStream_t st)
{
    batch_kernel<HotArgs, hot_body><<<bt.hot_blocks, kRedBlock, 0, st>>>(
        static_cast<const HotArgs*>(bt.hot), bt.hot_bstart, bt.B);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    batch_kernel<RhsArgs, rhs_body<false>><<<bt.rhs_blocks, kRedBlock, 0, st>>>(
        static_cast<const RhsArgs*>(bt.rhs), bt.rhs_bstart, bt.B);
    return cudaGetLastError();
}

// Batched FP32 per-ordinate source: X[k][c] = fma(shift_c, I[k][c], src_c),
// the same operation as the single problem's ordinate_source_kernel.
struct OrdArgs {
    int N, K;
    const float* shift; const float* I; const float* src;
    float* X;
    const int* done;
};

__device__ __forceinline__ void ord_body(const OrdArgs& a, int bid, int nblk)
{
    if (ld_volatile_int(a.done)) return;
    ord_tiles<float>(a.N, a.K, a.shift, a.I, a.src, a.X, bid, nblk);
}

size_t ord_batch_rec_bytes() { return sizeof(OrdArgs); }

int ord_batch_rec(const Plan& P, void* out)
{
    OrdArgs a{};
    a.N = P.N; a.K = P.K;
    a.shift = P.shift_f; a.I = static_cast<const float*>(P.I); a.src = P.src_f;
    a.X = P.X_f;
    a.done = &P.status->done;
    std::memcpy(out, &a, sizeof(a));
    return std::min(ord_tile_count(P.N, P.K, 1), P.num_sms * 8);
}

cudaError_t launch_ordsrc_batch(const BatchTables& bt, cudaStream_t st)
{
    batch_kernel<OrdArgs, ord_body><<<bt.ord_blocks, kRedBlock, 0, st>>>(static_cast<const OrdArgs*>(bt.ord),
                                                                           bt.ord_bstart, bt.B);
    return cudaGetLastError();
}

cudaError_t launch_update_batch(const BatchTables& bt, cudaStream_t st)
{
    batch_kernel<UpdArgs, update_body><<<bt.upd_blocks, kRedBlock, 0, st>>>(
        static_cast<const UpdArgs*>(bt.upd), bt.upd_bstart, bt.B);
    return cudaGetLastError();
}

}  // namespace gsis
