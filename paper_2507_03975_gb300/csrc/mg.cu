// Synthetic solve D rho = b (Eqs. (MSE_d1), (elem_mtx_M): symmetric positive
// definite 5-point finite-volume operator) on one thread-block cluster.
//
// Outer loop (FP64 iterative refinement): r = b - D x in FP64; stop when
// ||r|| <= rtol ||b|| or when the inner-iteration budget is spent; otherwise
// solve D d = r approximately in FP32 and set x <- x + d.
// Inner solver (FP32): conjugate gradients preconditioned by one multigrid
// V-cycle: 2x2 cell aggregation with piecewise-constant transfer, Galerkin
// coarse operators (again 5-point), damped Jacobi smoothing (nu steps before
// and after, weight omega), coarse correction scaled by alpha, down to one
// cell.  Pre- and post-smoothing are the same symmetric operator, so the
// V-cycle is a symmetric positive definite preconditioner for alpha < 2.
// Levels with few cells run inside CTA 0 (block barriers only); the others
// are spread over the whole cluster (cluster barriers).  All reductions are
// fixed-order sums, identical in every CTA, so every CTA takes the same
// branches and the result is bit-reproducible.
//
// Warm start x0 = previous rho: the correction vanishes with the residual,
// so a capped number of inner iterations (the paper's capped LU-SGS/SOR
// sub-iterations of Sec. 4.2) leaves the GSIS fixed point unchanged.
#include <algorithm>
#include <cooperative_groups.h>
#include <cstring>
#include <map>
#include <mutex>
#include <cuda_runtime.h>

#include "gsis_internal.cuh"

namespace cg = cooperative_groups;

namespace gsis {

namespace {

int grid_for(long long n, int block, int cap)
{
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// Quiet NaN written into a synthetic solution whose residual is not finite.
__device__ constexpr double kNaN = __builtin_nan("");

// ------------------------------------------------------------ set-up
__global__ void mg_copy_fine_kernel(int N, const double* __restrict__ d, const double* __restrict__ cx,
                                    const double* __restrict__ cy, double* d64, double* cx64, double* cy64,
                                    float* d32, float* cx32, float* cy32)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        d64[c] = d[c];
        cx64[c] = cx[c];
        cy64[c] = cy[c];
        d32[c] = (float)d[c];
        cx32[c] = (float)cx[c];
        cy32[c] = (float)cy[c];
    }
}

// Galerkin operator P^T A P for piecewise-constant 2x2 aggregation: the
// coarse diagonal is the sum of the children's diagonals minus twice the
// couplings inside the aggregate; a coarse face coefficient is the sum of the
// fine face coefficients across the aggregate's face.
__global__ void mg_coarsen_kernel(int nx, int ny, const double* __restrict__ d, const double* __restrict__ cx,
                                  const double* __restrict__ cy, int cnx, int cny, double* dc, double* cxc,
                                  double* cyc, float* dcf, float* cxcf, float* cycf)
{
    const int Nc = cnx * cny;
    for (int C = blockIdx.x * blockDim.x + threadIdx.x; C < Nc; C += gridDim.x * blockDim.x) {
        const int J = C / cnx, I = C - J * cnx;
        const int i0 = 2 * I, j0 = 2 * J;
        const bool hx = i0 + 1 < nx, hy = j0 + 1 < ny;
        double sd = 0.0, se = 0.0, sn = 0.0;
        for (int dj = 0; dj < (hy ? 2 : 1); ++dj)
            for (int di = 0; di < (hx ? 2 : 1); ++di) sd += d[(j0 + dj) * nx + i0 + di];
        for (int dj = 0; dj < (hy ? 2 : 1); ++dj) {
            if (hx) sd -= 2.0 * cx[(j0 + dj) * nx + i0];
            se += cx[(j0 + dj) * nx + i0 + (hx ? 1 : 0)];
        }
        for (int di = 0; di < (hx ? 2 : 1); ++di) {
            if (hy) sd -= 2.0 * cy[j0 * nx + i0 + di];
            sn += cy[(j0 + (hy ? 1 : 0)) * nx + i0 + di];
        }
        dc[C] = sd;
        cxc[C] = se;
        cyc[C] = sn;
        dcf[C] = (float)sd;
        cxcf[C] = (float)se;
        cycf[C] = (float)sn;
    }
}

// Inverse of one coarse level's operator A (n = nx ny <= kDirectMax cells;
// A = diag d, -cx between horizontal neighbours, -cy between vertical ones:
// symmetric positive definite) by Gauss-Jordan elimination in place,
// without pivoting (every pivot of an SPD matrix is positive), in FP32 like
// the V-cycle it serves; stored as (A^-1 + A^-T) / 2, so the stored matrix
// is exactly symmetric.  One CTA of 512 threads: thread (i0, j) holds the
// elements (i0 + 8 m, j), m = 0..7; per pivot one barrier after the reads
// of the pivot row and column, one after the update.  Once per operator.
constexpr int kInvThreads = 512;
__global__ void __launch_bounds__(kInvThreads) mg_direct_inverse_kernel(int nx, int ny, const double* __restrict__ d,
                                                                        const double* __restrict__ cx,
                                                                        const double* __restrict__ cy, float* inv)
{
    __shared__ float A[kDirectMax][kDirectMax];
    const int n = nx * ny, j = threadIdx.x & (kDirectMax - 1), i0 = threadIdx.x / kDirectMax;
    constexpr int kRows = kDirectMax / (kInvThreads / kDirectMax);
    for (int m = 0; m < kRows; ++m) {
        const int r = i0 + 8 * m;
        if (r >= n || j >= n) continue;
        const int ir = r % nx, jr = r / nx;
        double v = 0.0;
        if (j == r) v = d[r];
        else if (j == r + 1 && ir + 1 < nx) v = -cx[r];
        else if (j == r - 1 && ir > 0) v = -cx[j];
        else if (j == r + nx && jr + 1 < ny) v = -cy[r];
        else if (j == r - nx && jr > 0) v = -cy[j];
        A[r][j] = (float)v;
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        const float p = 1.f / A[k][k];
        float aik[kRows];
#pragma unroll
        for (int m = 0; m < kRows; ++m) aik[m] = i0 + 8 * m < n ? A[i0 + 8 * m][k] : 0.f;
        const float rkj = j == k ? p : (j < n ? A[k][j] * p : 0.f);
        __syncthreads();
        if (j < n) {
#pragma unroll
            for (int m = 0; m < kRows; ++m) {
                const int r = i0 + 8 * m;
                if (r >= n) continue;
                if (r == k) A[r][j] = rkj;
                else A[r][j] = j == k ? -aik[m] * p : __fmaf_rn(-aik[m], rkj, A[r][j]);
            }
        }
        __syncthreads();
    }
    for (int m = 0; m < kRows; ++m) {
        const int r = i0 + 8 * m;
        if (r < n && j < n) inv[r * n + j] = 0.5f * (A[r][j] + A[j][r]);
    }
}

// ------------------------------------------------------------ solve
struct MgLevelDev {
    int nx, ny;
    const float* d; const float* cx; const float* cy;
    float* x; float* t; float* r;
};

struct MgArgs {
    int nl, local_from;
    MgLevelDev lv[kMaxLevels];
    int loff[kMaxLevels];   // float offsets of the local levels in dynamic shared memory
    int nx, ny, N;
    const double* diag; const double* cx; const double* cy;
    const double* b; const double* guess; double* x;
    float* r0; float* dl; float* s; float* p; float* q;
    double rtol;
    int max_iter, nu;
    float inner_rtol, omega, alpha;
    Status* status;
    // grid-wide form: reduction slots [3][2][gridDim] and the barrier words
    double* gslots_d; float* gslots_f;
    unsigned* gbar;                 // [0]: the grid barrier word (top bit flips per barrier)
    long long wait_cycles;
    const float* cinv;              // inverse of level `direct`'s operator (tiled form)
    int direct;
};

// Work distribution of one level: the whole cluster, or CTA 0 alone.
struct Range {
    int start, step;
    bool active;
};

__device__ __forceinline__ float ld(const float* p) { return __ldcg(p); }

__device__ __forceinline__ float apply_A(const MgLevelDev& L, const float* v, int c)
{
    const int j = c / L.nx, i = c - j * L.nx;
    float y = L.d[c] * ld(v + c);
    if (i + 1 < L.nx) y -= L.cx[c] * ld(v + c + 1);
    if (i > 0) y -= L.cx[c - 1] * ld(v + c - 1);
    if (j + 1 < L.ny) y -= L.cy[c] * ld(v + c + L.nx);
    if (j > 0) y -= L.cy[c - L.nx] * ld(v + c - L.nx);
    return y;
}

// For every cell of the range: v = f(c) for up to U cells first (all loads in
// flight together), then store(c, v).  f must only read, store only write.
template <int U, class F, class S>
__device__ __forceinline__ void for_cells(const Range& R, int n, F f, S store)
{
    if (!R.active) return;
    for (int c0 = R.start; c0 < n; c0 += R.step * U) {
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c = c0 + u * R.step;
            v[u] = c < n ? f(c) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c = c0 + u * R.step;
            if (c < n) store(c, v[u]);
        }
    }
}

class ClusterCtx {
  public:
    __device__ ClusterCtx(int local_from) : cl_(cg::this_cluster())
    {
        rank_ = (int)cl_.block_rank();
        nblk_ = (int)cl_.num_blocks();
        (void)local_from;
    }
    __device__ void sync() { cl_.sync(); }
    __device__ int rank() const { return rank_; }
    __device__ Range range(bool local) const
    {
        if (local) return Range{(int)threadIdx.x, (int)blockDim.x, rank_ == 0};
        return Range{rank_ * (int)blockDim.x + (int)threadIdx.x, nblk_ * (int)blockDim.x, true};
    }
    // Fixed-order cluster-wide sums of two floats / two doubles; every CTA
    // gets the same bits.  Slots rotate so that no second barrier is needed.
    __device__ void sum2f(float a, float b, float out[2], float* slots, int& rot)
    {
        a = blockf(a);
        b = blockf(b);
        float* mine = slots + 2 * rot;
        if (threadIdx.x == 0) {
            mine[0] = a;
            mine[1] = b;
        }
        cl_.sync();
        float s0 = 0.f, s1 = 0.f;
        for (int r = 0; r < nblk_; ++r) {
            const float* o = cl_.map_shared_rank(mine, r);
            s0 += o[0];
            s1 += o[1];
        }
        out[0] = s0;
        out[1] = s1;
        rot = (rot + 1) % 3;
    }
    __device__ void sum2d(double a, double b, double out[2], double* slots, int& rot)
    {
        a = blockd(a);
        b = blockd(b);
        double* mine = slots + 2 * rot;
        if (threadIdx.x == 0) {
            mine[0] = a;
            mine[1] = b;
        }
        cl_.sync();
        double s0 = 0.0, s1 = 0.0;
        for (int r = 0; r < nblk_; ++r) {
            const double* o = cl_.map_shared_rank(mine, r);
            s0 += o[0];
            s1 += o[1];
        }
        out[0] = s0;
        out[1] = s1;
        rot = (rot + 1) % 3;
    }

  private:
    __device__ float blockf(float v)
    {
        __shared__ float w[32];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        __syncthreads();
        if (lane == 0) w[wid] = v;
        __syncthreads();
        float t = lane < nw ? w[lane] : 0.f;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
        return t;
    }
    __device__ double blockd(double v)
    {
        __shared__ double w[32];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        __syncthreads();
        if (lane == 0) w[wid] = v;
        __syncthreads();
        double t = lane < nw ? w[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
        return t;
    }
    cg::cluster_group cl_;
    int rank_, nblk_;
};

// The same interface over a whole cooperative grid (one CTA per SM): the
// fine levels spread over every SM.  The barrier is one word in global
// memory whose top bit flips once per completed barrier: CTA 0 adds
// 2^31 - (G - 1), every other CTA adds 1, so the bit changes with the last
// arrival whatever the order and the low bits return to zero.  Each CTA
// reads the bit once at the start (no barrier of this launch can complete
// before its own first arrival) and afterwards knows the value to wait for,
// so an arrival is a release reduction without a reply and the wait polls
// with acquire loads.  Every wait is bounded; after a time-out (the status's
// timeout bit) later barriers return at once so that every CTA finishes,
// and the word is valid again after the next status reset.  Sums: each
// CTA's partial in a rotating global table, then every warp adds the table
// in a fixed order (same bits everywhere).
class GridCtx {
  public:
    __device__ GridCtx(const MgArgs& a) : a_(a)
    {
        if (threadIdx.x == 0) phase_ = ld_acquire_u32(a_.gbar) & kFlip;
    }
    __device__ void sync()
    {
        __syncthreads();
        if (threadIdx.x == 0 && !ld_volatile_int(&a_.status->error)) {
            const unsigned inc = blockIdx.x == 0 ? kFlip - (gridDim.x - 1u) : 1u;
            asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(a_.gbar), "r"(inc) : "memory");
            phase_ ^= kFlip;
            const long long t0 = clock64();
            while ((ld_acquire_u32(a_.gbar) & kFlip) != phase_) {
                if (clock64() - t0 > a_.wait_cycles) {
                    atomicOr(&a_.status->error, kErrTimeout);
                    break;
                }
            }
        }
        __syncthreads();
    }
    __device__ int rank() const { return blockIdx.x; }
    __device__ Range range(bool local) const
    {
        if (local) return Range{(int)threadIdx.x, (int)blockDim.x, blockIdx.x == 0};
        return Range{(int)(blockIdx.x * blockDim.x + threadIdx.x), (int)(gridDim.x * blockDim.x), true};
    }
    __device__ void sum2f(float a, float b, float out[2], float*, int& rot)
    {
        a = blockf(a);
        b = blockf(b);
        float* tab = a_.gslots_f + (size_t)rot * 2 * gridDim.x;
        if (threadIdx.x == 0) {
            tab[2 * blockIdx.x] = a;
            tab[2 * blockIdx.x + 1] = b;
        }
        sync();
        float s0 = 0.f, s1 = 0.f;
        table_sum(tab, s0, s1);
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(kFull, s0, o);
            s1 += __shfl_xor_sync(kFull, s1, o);
        }
        out[0] = s0;
        out[1] = s1;
        rot = (rot + 1) % 3;
    }
    __device__ void sum2d(double a, double b, double out[2], double*, int& rot)
    {
        a = blockd(a);
        b = blockd(b);
        double* tab = a_.gslots_d + (size_t)rot * 2 * gridDim.x;
        if (threadIdx.x == 0) {
            tab[2 * blockIdx.x] = a;
            tab[2 * blockIdx.x + 1] = b;
        }
        sync();
        double s0 = 0.0, s1 = 0.0;
        table_sum(tab, s0, s1);
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(kFull, s0, o);
            s1 += __shfl_xor_sync(kFull, s1, o);
        }
        out[0] = s0;
        out[1] = s1;
        rot = (rot + 1) % 3;
    }

  private:
    static constexpr unsigned kFlip = 0x80000000u;
    __device__ static unsigned ld_acquire_u32(const unsigned* p)
    {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
        return v;
    }
    // Lane l adds the table's pairs l, l + 32, l + 64, ... in that order;
    // each group of eight is loaded before any is added, so the L2 reads
    // overlap instead of one round trip per pair.
    template <typename T>
    __device__ void table_sum(const T* tab, T& s0, T& s1)
    {
        constexpr int kG = 8;
        const int lane = threadIdx.x & 31, n = gridDim.x;
        for (int r0 = 0; r0 < n; r0 += 32 * kG) {
            T v0[kG], v1[kG];
#pragma unroll
            for (int g = 0; g < kG; ++g) {
                const int r = r0 + lane + 32 * g;
                v0[g] = r < n ? __ldcg(tab + 2 * r) : T(0);
                v1[g] = r < n ? __ldcg(tab + 2 * r + 1) : T(0);
            }
#pragma unroll
            for (int g = 0; g < kG; ++g)
                if (r0 + lane + 32 * g < n) {
                    s0 += v0[g];
                    s1 += v1[g];
                }
        }
    }
    __device__ float blockf(float v)
    {
        __shared__ float w[32];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        __syncthreads();
        if (lane == 0) w[wid] = v;
        __syncthreads();
        float t = lane < nw ? w[lane] : 0.f;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
        return t;
    }
    __device__ double blockd(double v)
    {
        __shared__ double w[32];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        __syncthreads();
        if (lane == 0) w[wid] = v;
        __syncthreads();
        double t = lane < nw ? w[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
        return t;
    }
    const MgArgs& a_;
    unsigned phase_ = 0;   // thread 0: the barrier word's top bit after the last completed barrier
};

__device__ __forceinline__ float apply_S(const MgLevelDev& L, const float* v, int c)
{
    const int j = c / L.nx, i = c - j * L.nx;
    float y = L.d[c] * v[c];
    if (i + 1 < L.nx) y -= L.cx[c] * v[c + 1];
    if (i > 0) y -= L.cx[c - 1] * v[c - 1];
    if (j + 1 < L.ny) y -= L.cy[c] * v[c + L.nx];
    if (j > 0) y -= L.cy[c - L.nx] * v[c - L.nx];
    return y;
}

// V-cycle over levels [l0, nl) inside one CTA, all data in its shared memory
// (S[l] point into it): input S[l0].r, output S[l0].t.
__device__ void vcycle_local(const MgLevelDev* S, int l0, int nl, int nu, float om, float alpha)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int l = l0; l < nl - 1; ++l) {
        const MgLevelDev& L = S[l];
        const int n = L.nx * L.ny;
        float* cur = L.x;
        float* oth = L.t;
        for (int c = tid; c < n; c += nt) cur[c] = om * L.r[c] / L.d[c];
        for (int k = 1; k < nu; ++k) {
            __syncthreads();
            for (int c = tid; c < n; c += nt) oth[c] = cur[c] + om * (L.r[c] - apply_S(L, cur, c)) / L.d[c];
            float* tmp = cur;
            cur = oth;
            oth = tmp;
        }
        __syncthreads();
        const MgLevelDev& C = S[l + 1];
        const int nc = C.nx * C.ny;
        for (int cc = tid; cc < nc; cc += nt) {
            const int J = cc / C.nx, I = cc - J * C.nx;
            float sum = 0.f;
            for (int q = 0; q < 4; ++q) {
                const int i = 2 * I + (q & 1), j = 2 * J + (q >> 1);
                if (i < L.nx && j < L.ny) {
                    const int c = j * L.nx + i;
                    sum += L.r[c] - apply_S(L, cur, c);
                }
            }
            C.r[cc] = sum;
        }
        __syncthreads();
    }
    {
        const MgLevelDev& L = S[nl - 1];
        for (int c = tid; c < L.nx * L.ny; c += nt) L.t[c] = L.r[c] / L.d[c];
        __syncthreads();
    }
    for (int l = nl - 2; l >= l0; --l) {
        const MgLevelDev& L = S[l];
        const MgLevelDev& C = S[l + 1];
        const int n = L.nx * L.ny;
        float* cur = (nu % 2) ? L.x : L.t;
        float* oth = (nu % 2) ? L.t : L.x;
        for (int c = tid; c < n; c += nt) {
            const int j = c / L.nx, i = c - j * L.nx;
            cur[c] += alpha * C.t[(j / 2) * C.nx + i / 2];
        }
        for (int k = 0; k < nu; ++k) {
            __syncthreads();
            for (int c = tid; c < n; c += nt) oth[c] = cur[c] + om * (L.r[c] - apply_S(L, cur, c)) / L.d[c];
            float* tmp = cur;
            cur = oth;
            oth = tmp;
        }
        __syncthreads();
    }
}

// z = M^{-1} s: one V-cycle; input in lv[0].r, output in lv[0].t.  Levels
// above local_from are spread over the cluster (L2 data, cluster barriers);
// the rest run in CTA 0 on its shared-memory copy S.
template <class Ctx>
__device__ void vcycle(const MgArgs& a, const MgLevelDev* S, Ctx& cx)
{
    constexpr int U = 4;
    const int nl = a.nl, lf = a.local_from;
    const float om = a.omega;
    const Range R = cx.range(false);
    // ---- down over the distributed levels
    for (int l = 0; l < lf; ++l) {
        const MgLevelDev& L = a.lv[l];
        const int n = L.nx * L.ny;
        float* cur = L.x;
        float* oth = L.t;
        for_cells<U>(R, n, [&](int c) { return om * ld(L.r + c) / L.d[c]; },
                     [&](int c, float v) { cur[c] = v; });
        for (int k = 1; k < a.nu; ++k) {
            cx.sync();
            float* src = cur;
            for_cells<U>(R, n,
                         [&](int c) { return ld(src + c) + om * (ld(L.r + c) - apply_A(L, src, c)) / L.d[c]; },
                         [&](int c, float v) { oth[c] = v; });
            float* tmp = cur;
            cur = oth;
            oth = tmp;
        }
        cx.sync();
        const MgLevelDev& C = a.lv[l + 1];
        const float* fin = cur;
        for_cells<U>(R, C.nx * C.ny,
                     [&](int cc) {
                         const int J = cc / C.nx, I = cc - J * C.nx;
                         float sum = 0.f;
#pragma unroll
                         for (int q = 0; q < 4; ++q) {
                             const int i = 2 * I + (q & 1), j = 2 * J + (q >> 1);
                             if (i < L.nx && j < L.ny) {
                                 const int c = j * L.nx + i;
                                 sum += ld(L.r + c) - apply_A(L, fin, c);
                             }
                         }
                         return sum;
                     },
                     [&](int cc, float v) { C.r[cc] = v; });
        cx.sync();   // the coarse residual is read by other threads next
    }
    if (lf == 0) cx.sync();   // level 0 itself is local: make the input visible to CTA 0
    // ---- local levels in CTA 0's shared memory
    if (cx.rank() == 0) {
        const MgLevelDev& G = a.lv[lf];
        const MgLevelDev& L = S[lf];
        const int n = G.nx * G.ny;
        for (int c = threadIdx.x; c < n; c += blockDim.x) L.r[c] = ld(G.r + c);
        __syncthreads();
        vcycle_local(S, lf, nl, a.nu, om, a.alpha);
        for (int c = threadIdx.x; c < n; c += blockDim.x) G.t[c] = L.t[c];
    }
    cx.sync();
    // ---- up over the distributed levels
    for (int l = lf - 1; l >= 0; --l) {
        const MgLevelDev& L = a.lv[l];
        const MgLevelDev& C = a.lv[l + 1];
        const int n = L.nx * L.ny;
        float* cur = (a.nu % 2) ? L.x : L.t;   // buffer holding the pre-smoothed iterate
        float* oth = (a.nu % 2) ? L.t : L.x;
        {
            float* dst = cur;
            for_cells<U>(R, n,
                         [&](int c) {
                             const int j = c / L.nx, i = c - j * L.nx;
                             return ld(dst + c) + a.alpha * ld(C.t + (j / 2) * C.nx + i / 2);
                         },
                         [&](int c, float v) { dst[c] = v; });
        }
        for (int k = 0; k < a.nu; ++k) {
            cx.sync();
            float* src = cur;
            float* dst = oth;
            for_cells<U>(R, n,
                         [&](int c) { return ld(src + c) + om * (ld(L.r + c) - apply_A(L, src, c)) / L.d[c]; },
                         [&](int c, float v) { dst[c] = v; });
            float* tmp = cur;
            cur = oth;
            oth = tmp;
        }
        cx.sync();
    }
}

template <class Ctx>
__device__ __forceinline__ void mg_solve_body(const MgArgs& a, Ctx& cx)
{
    constexpr int U = 4;   // cells per thread whose loads are in flight together
    __shared__ float slots_f[6];
    __shared__ double slots_d[6];
    extern __shared__ __align__(16) float mg_smem[];
    if (ld_volatile_int(&a.status->done)) return;   // same value in every CTA (set by an earlier kernel)
    // shared-memory copy of the local levels (used by CTA 0 only)
    __shared__ MgLevelDev S[kMaxLevels];
    if (threadIdx.x == 0)
        for (int l = a.local_from; l < a.nl; ++l) {
            const int n = a.lv[l].nx * a.lv[l].ny;
            float* base = mg_smem + a.loff[l];
            S[l] = MgLevelDev{a.lv[l].nx, a.lv[l].ny, base, base + n, base + 2 * n, base + 3 * n, base + 4 * n,
                              base + 5 * n};
        }
    if (cx.rank() == 0)
        for (int l = a.local_from; l < a.nl; ++l) {
            const int n = a.lv[l].nx * a.lv[l].ny;
            float* base = mg_smem + a.loff[l];
            for (int c = threadIdx.x; c < n; c += blockDim.x) {
                base[c] = a.lv[l].d[c];
                base[n + c] = a.lv[l].cx[c];
                base[2 * n + c] = a.lv[l].cy[c];
            }
        }
    __syncthreads();
    int rotf = 0, rotd = 0;
    const Range G = cx.range(false);
    const int N = a.N, nx = a.nx, ny = a.ny;
    const int stride = G.step;
    for (int c = G.start; c < N; c += stride) a.x[c] = a.guess[c];
    double bb_rr[2];
    {
        double loc = 0.0;
        for (int c = G.start; c < N; c += stride) loc += a.b[c] * a.b[c];
        cx.sum2d(loc, 0.0, bb_rr, slots_d, rotd);
    }
    const double bb = bb_rr[0];
    const double stop2 = a.rtol * a.rtol * bb;
    int total = 0;
    double relres = 0.0;
    const MgLevelDev& L0 = a.lv[0];
    for (;;) {
        // FP64 residual of the current x
        cx.sync();
        double loc = 0.0;
        for (int c0 = G.start; c0 < N; c0 += stride * U) {
            double y[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int c = c0 + u * stride;
                y[u] = 0.0;
                if (c < N) {
                    const int j = c / nx, i = c - j * nx;
                    double v = a.diag[c] * __ldcg(a.x + c);
                    if (i + 1 < nx) v -= a.cx[c] * __ldcg(a.x + c + 1);
                    if (i > 0) v -= a.cx[c - 1] * __ldcg(a.x + c - 1);
                    if (j + 1 < ny) v -= a.cy[c] * __ldcg(a.x + c + nx);
                    if (j > 0) v -= a.cy[c - nx] * __ldcg(a.x + c - nx);
                    y[u] = a.b[c] - v;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int c = c0 + u * stride;
                if (c < N) {
                    a.r0[c] = (float)y[u];
                    loc += y[u] * y[u];
                }
            }
        }
        double rr[2];
        cx.sum2d(loc, 0.0, rr, slots_d, rotd);
        relres = bb > 0.0 ? sqrt(rr[0] / bb) : 0.0;
        if (rr[0] <= stop2 || total >= a.max_iter) break;
        // FP32 MG-PCG for D d = r0, d = 0 to start: s = r0, z = M s, p = z
        for (int c = G.start; c < N; c += stride) {
            const float r = a.r0[c];
            a.dl[c] = 0.f;
            a.s[c] = r;
            L0.r[c] = r;
        }
        vcycle(a, S, cx);
        float f2[2];
        {
            float l0 = 0.f, l1 = 0.f;
            for (int c = G.start; c < N; c += stride) {
                const float z = ld(L0.t + c), sv = a.s[c];
                a.p[c] = z;
                l0 += sv * z;
                l1 += sv * sv;
            }
            cx.sum2f(l0, l1, f2, slots_f, rotf);
        }
        float rz = f2[0];
        if (!(rz > 0.f) || !(rz < INFINITY) || !isfinite(rr[0])) {
            // No usable FP32 search direction, so the inner loop could not
            // advance `total` and nothing else would end the refinement: a
            // residual beyond the FP32 range or not finite (a diverging GSIS
            // iteration), or one that vanished in FP32.  Leave; a non-finite
            // one poisons x so that Err(rho) reports the divergence.  rz and
            // rr are the same in every CTA, so all leave together.
            const bool bad = !(rz == 0.f) || !isfinite(rr[0]);
            if (bad) {
                for (int c = G.start; c < N; c += stride) a.x[c] = kNaN;
                relres = kNaN;
            }
            break;
        }
        const float s00 = f2[1];
        const float istop = a.inner_rtol * a.inner_rtol * s00;
        while (total < a.max_iter && rz > 0.f) {
            // q = D p, p.q   (p of every CTA visible after the previous barrier)
            float lpq = 0.f;
            for (int c0 = G.start; c0 < N; c0 += stride * U) {
                float qv[U], pv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int c = c0 + u * stride;
                    qv[u] = 0.f;
                    pv[u] = 0.f;
                    if (c < N) {
                        qv[u] = apply_A(L0, a.p, c);
                        pv[u] = ld(a.p + c);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int c = c0 + u * stride;
                    if (c < N) {
                        a.q[c] = qv[u];
                        lpq += pv[u] * qv[u];
                    }
                }
            }
            cx.sum2f(lpq, 0.f, f2, slots_f, rotf);
            const float alpha = rz / f2[0];
            float lss = 0.f;
            for (int c = G.start; c < N; c += stride) {
                a.dl[c] += alpha * ld(a.p + c);
                const float sc = a.s[c] - alpha * a.q[c];
                a.s[c] = sc;
                L0.r[c] = sc;
                lss += sc * sc;
            }
            ++total;
            cx.sum2f(lss, 0.f, f2, slots_f, rotf);
            if (f2[0] <= istop || total >= a.max_iter) break;
            vcycle(a, S, cx);
            float lrz = 0.f;
            for (int c = G.start; c < N; c += stride) lrz += a.s[c] * ld(L0.t + c);
            cx.sum2f(lrz, 0.f, f2, slots_f, rotf);
            const float beta = f2[0] / rz;
            rz = f2[0];
            for (int c = G.start; c < N; c += stride) a.p[c] = ld(L0.t + c) + beta * a.p[c];
            cx.sync();   // the next product reads the neighbours' p
        }
        for (int c = G.start; c < N; c += stride) a.x[c] += (double)a.dl[c];
        if (total >= a.max_iter) {   // budget spent: no further residual evaluation
            relres = -1.0;
            break;
        }
    }
    if (cx.range(false).start == 0) {
        a.status->synth_iters = total;
        a.status->synth_iters_total += total;
        a.status->synth_relres = relres;
    }
    // No CTA may exit while another can still read its shared-memory slots
    // (the last cluster reduction reads every CTA's slot after its barrier).
    cx.sync();
}

__global__ void __launch_bounds__(kMgBlock) mg_solve_kernel(const MgArgs a)
{
    ClusterCtx cx(a.local_from);
    mg_solve_body(a, cx);
}

// The same solver over a cooperative grid of one CTA per SM (meshes whose
// strip plan does not fit a cluster's shared memory).
__global__ void __launch_bounds__(kMgBlock) mg_solve_grid_kernel(const MgArgs a)
{
    GridCtx cx(a);
    mg_solve_body(a, cx);
}

// ------------------------------------------------------------ tiled grid solver
// The same iteration (FP64 refinement around FP32 MG-PCG, V-cycle with two
// damped-Jacobi steps before and after, coarse correction x alpha) over a
// cooperative grid, arranged so that each phase costs one grid barrier:
//
//  * CTAs 1..px*py own one rectangle of every distributed level (levels
//    0..local_from-1): the level-0 rectangles of a px x py block grid, with
//    boundaries at multiples of 2^(local_from-1), divided by 2^l on level l,
//    so a rectangle's 2x2 restriction is the next level's rectangle.  CTA 0
//    owns no rectangle; it runs the levels from local_from down to the
//    first level of at most kDirectMax cells in its shared memory and
//    solves that level with its inverse (`mg_direct_inverse_kernel`).
//  * Barrier: one word whose top bit flips per completed barrier (see
//    GridCtx); reductions read their per-CTA table eight slots per lane.
//  * Down phase of level l, per sub-tile of the rectangle (one sub-tile on
//    the workloads' meshes): the sub-tile and a two-cell halo of r and of the
//    level's coefficients go to shared memory, x1 = omega r / d and x2 = one
//    Jacobi step are formed on all of it (a zero ring of ghost cells keeps
//    the stencil branch-free; values near the halo's outer edge are wrong
//    and never used), then on the own cells x2 is stored and the residual
//    r - A x2 is restricted into the next level (on the last distributed
//    level it is stored for CTA 0 to restrict).
//  * Up phase: x2 + alpha P t_coarse and two Jacobi steps on the sub-tile
//    with its halo; the own cells' result is the level's correction t.
//  * CG: the level-0 down phase also performs the update s <- s - a q
//    (pointwise, so halo cells repeat the owners' arithmetic bit for bit;
//    s alternates between two buffers) and dl <- dl + a p; the new search
//    direction uses A p = A z + beta (A p_old), so p, q and p.q take one
//    phase.  A V-cycle costs 2 local_from + 1 barriers (old form: ~25).
//  * Loads are issued several per thread before any is used (coefficients,
//    read-only in the kernel, by asynchronous copies; values other CTAs
//    wrote, from L2), so a phase waits on about one memory latency.
constexpr int kTileMaxDim = 160;    // rectangles along one axis
constexpr int kTileArrays = 6;      // shared arrays per sub-tile: r, 1/d, cx, cy, two iterates
constexpr int kLocalArrays = 7;     // per coarse level in CTA 0: d, cx, cy, 1/d, x, t, r
constexpr int kTileU = 2;           // cells per thread whose loads are in flight together
constexpr int kTileBlock = 512;     // threads per CTA (128 registers each: no spills)
constexpr int kTileLoadU = 4;       // the same in the sub-tile loads

struct TileArgs {
    MgArgs m;
    int px, py;
    int bx[kTileMaxDim + 1], by[kTileMaxDim + 1];   // level-0 rectangle boundaries (bx[px] = nx, by[py] = ny)
    int tile_cells;                                 // padded cells of one sub-tile array
};

__device__ __forceinline__ void mg_cp_async4(void* smem, const void* gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}

// 16 bytes, L2 only (data other CTAs wrote earlier in the kernel); both
// addresses 16-byte aligned.
__device__ __forceinline__ void mg_cp_async16_cg(void* smem, const void* gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}

// Cells k = tid, tid + nt, ... of a w-wide row-major block, as (i, j): one
// division per thread, then steps with a carry.
struct CellWalk {
    int i, j, di, dj, w;
    __device__ CellWalk(int w_) : w(w_)
    {
        i = (int)threadIdx.x % w;
        j = (int)threadIdx.x / w;
        di = (int)blockDim.x % w;
        dj = (int)blockDim.x / w;
    }
    __device__ void next()
    {
        i += di;
        j += dj;
        if (i >= w) {
            i -= w;
            ++j;
        }
    }
};

// For the cells of rectangle [i0, i0 + w) x [j0, j0 + h) of a row-major
// array with row length nx: v = f(c, i, j) for U cells first (their
// loads in flight together), then g(c, v).
template <class T, int U = kTileU, class F, class G>
__device__ __forceinline__ void rect_cells(int i0, int j0, int w, int h, int nx, F f, G g)
{
    const int n = w * h;
    if (n <= 0) return;
    CellWalk cw(w);
    for (int k0 = threadIdx.x; k0 < n; k0 += U * blockDim.x) {
        T v[U];
        int cc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            cc[u] = -1;
            if (k0 + u * (int)blockDim.x < n) {
                const int gi = i0 + cw.i, gj = j0 + cw.j;
                cc[u] = gj * nx + gi;
                v[u] = f(cc[u], gi, gj);
            }
            cw.next();
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (cc[u] >= 0) g(cc[u], v[u]);
    }
}

// One sub-tile region of level L in shared memory: cells [gi0, gi0 + rw) x
// [gj0, gj0 + rh) of the level at local (li, lj), padded by a ghost ring.
struct TileView {
    int gi0, gj0, rw, rh, pw;
    float *R, *ID, *CX, *CY, *XA, *XB;
    __device__ int at(int li, int lj) const { return (lj + 1) * pw + li + 1; }
};

__device__ __forceinline__ float tile_nb(const TileView& v, const float* X, int p)
{
    return v.R[p] + v.CX[p] * X[p + 1] + v.CX[p - 1] * X[p - 1] + v.CY[p] * X[p + v.pw] +
           v.CY[p - v.pw] * X[p - v.pw];
}

__device__ __forceinline__ float tile_jacobi(const TileView& v, const float* X, int p, float om, float id)
{
    return (1.f - om) * X[p] + om * tile_nb(v, X, p) * id;
}

// Rectangle of CTA b (1-based among the working CTAs) on level l.
__device__ __forceinline__ void tile_rect(const TileArgs& a, int l, int b, int& i0, int& i1, int& j0, int& j1)
{
    const int bxi = (b - 1) % a.px, byi = (b - 1) / a.px;
    i0 = a.bx[bxi] >> l;
    i1 = bxi + 1 == a.px ? a.m.lv[l].nx : a.bx[bxi + 1] >> l;
    j0 = a.by[byi] >> l;
    j1 = byi + 1 == a.py ? a.m.lv[l].ny : a.by[byi + 1] >> l;
}

// Rows per sub-tile of a rectangle of width w (even, >= 2): what fits.
__device__ __forceinline__ int tile_rows(const TileArgs& a, int w)
{
    int r = a.tile_cells / (w + 6) - 6;
    r &= ~1;
    return r < 2 ? 2 : r;
}

// Loads a sub-tile's region [si0-2, si1+2) x [sj0-2, sj1+2) (clipped to the
// level) into v: d into ID (the first pass inverts it), the couplings (zero
// across the level's edge), R = rin(c) and, if load_x, XA = xin(c, i, j);
// zeroes the ghost ring of the iterates and couplings.
template <class RF, class XF>
__device__ __forceinline__ void tile_load(TileView& v, float* base, int cells, const MgLevelDev& L, int si0,
                                          int si1, int sj0, int sj1, RF rin, bool load_x, XF xin)
{
    v.gi0 = max(si0 - 2, 0);
    v.gj0 = max(sj0 - 2, 0);
    v.rw = min(si1 + 2, L.nx) - v.gi0;
    v.rh = min(sj1 + 2, L.ny) - v.gj0;
    v.pw = v.rw + 2;
    v.R = base;
    v.ID = base + (size_t)cells;
    v.CX = base + 2 * (size_t)cells;
    v.CY = base + 3 * (size_t)cells;
    v.XA = base + 4 * (size_t)cells;
    v.XB = base + 5 * (size_t)cells;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ph = v.rh + 2;
    for (int k = tid; k < 2 * v.pw + 2 * ph; k += nt) {   // ghost ring: rows -1 and rh, columns -1 and rw
        int p;
        if (k < v.pw) p = k;
        else if (k < 2 * v.pw) p = (ph - 1) * v.pw + (k - v.pw);
        else if (k < 2 * v.pw + ph) p = (k - 2 * v.pw) * v.pw;
        else p = (k - 2 * v.pw - ph) * v.pw + v.pw - 1;
        v.XA[p] = 0.f;
        v.XB[p] = 0.f;
        v.CX[p] = 0.f;
        v.CY[p] = 0.f;
    }
    const int n = v.rw * v.rh;
    {   // coefficients: read-only in the kernel, so L1-cached asynchronous copies
        CellWalk cw(v.rw);
        for (int k = tid; k < n; k += nt, cw.next()) {
            const int gi = v.gi0 + cw.i, gj = v.gj0 + cw.j, c = gj * L.nx + gi, p = v.at(cw.i, cw.j);
            mg_cp_async4(v.ID + p, L.d + c);
            if (gi + 1 < L.nx) mg_cp_async4(v.CX + p, L.cx + c);
            else v.CX[p] = 0.f;
            if (gj + 1 < L.ny) mg_cp_async4(v.CY + p, L.cy + c);
            else v.CY[p] = 0.f;
        }
    }
    {   // r (and x): values other CTAs wrote earlier in the kernel, from L2, kTileLoadU in flight per thread
        CellWalk cw(v.rw);
        for (int k0 = tid; k0 < n; k0 += kTileLoadU * nt) {
            float rv[kTileLoadU], xv[kTileLoadU];
            int pp[kTileLoadU];
#pragma unroll
            for (int u = 0; u < kTileLoadU; ++u) {
                pp[u] = -1;
                if (k0 + u * nt < n) {
                    const int gi = v.gi0 + cw.i, gj = v.gj0 + cw.j, c = gj * L.nx + gi;
                    pp[u] = v.at(cw.i, cw.j);
                    rv[u] = rin(c);
                    xv[u] = load_x ? xin(c, gi, gj) : 0.f;
                }
                cw.next();
            }
#pragma unroll
            for (int u = 0; u < kTileLoadU; ++u)
                if (pp[u] >= 0) {
                    v.R[pp[u]] = rv[u];
                    if (load_x) v.XA[pp[u]] = xv[u];
                }
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
}

// The coarse levels in CTA 0's shared memory (tiled grid solver): the same
// smoothing and transfers as vcycle_local (x2 from r in one pass, the
// residual, the 2x2 restriction; x2 + alpha P x_coarse and two Jacobi steps),
// with 1/d precomputed and no division in a loop, but the first level of at
// most kDirectMax cells is solved exactly with its precomputed inverse
// instead of being cycled on down to one cell.  A level is a set
// of float offsets into the dynamic shared memory, passed by value: held in
// registers, its arrays are addressed as shared memory and no store inside a
// loop can make the compiler reload them.
struct LocalLevel {
    int nx, ny;
    int d, cx, cy, id, x, t, r;
};

// One array of a LocalLevel in the dynamic shared memory.
struct LocalArr {
    int off;
    __device__ float& operator[](int c) const
    {
        extern __shared__ __align__(16) float mg_smem[];
        return mg_smem[off + c];
    }
};
struct LocalView {
    int nx, ny;
    LocalArr d, cx, cy, id, x, t, r;
    __device__ explicit LocalView(const LocalLevel& L)
        : nx(L.nx), ny(L.ny), d{L.d}, cx{L.cx}, cy{L.cy}, id{L.id}, x{L.x}, t{L.t}, r{L.r} {}
};

__device__ __forceinline__ void local_down(const LocalLevel Ls, const LocalLevel Cs, float om)
{
    const LocalView L(Ls), C(Cs);
    const int tid = threadIdx.x, nt = blockDim.x;
    auto sync = [] { __syncthreads(); };
    const int nx = L.nx, ny = L.ny, n = nx * ny;
    auto x1 = [&](int c) { return om * L.r[c] * L.id[c]; };
    int i = tid % nx, j = tid / nx;
    const int di = nt % nx, dj = nt / nx;
    auto step = [&] { i += di; j += dj; if (i >= nx) { i -= nx; ++j; } };
    for (int c = tid; c < n; c += nt, step()) {
        float nb = L.r[c];
        if (i + 1 < nx) nb += L.cx[c] * x1(c + 1);
        if (i > 0) nb += L.cx[c - 1] * x1(c - 1);
        if (j + 1 < ny) nb += L.cy[c] * x1(c + nx);
        if (j > 0) nb += L.cy[c - nx] * x1(c - nx);
        L.x[c] = (1.f - om) * x1(c) + om * nb * L.id[c];
    }
    sync();
    i = tid % nx;
    j = tid / nx;
    for (int c = tid; c < n; c += nt, step()) {
        float res = L.r[c] - L.d[c] * L.x[c];
        if (i + 1 < nx) res += L.cx[c] * L.x[c + 1];
        if (i > 0) res += L.cx[c - 1] * L.x[c - 1];
        if (j + 1 < ny) res += L.cy[c] * L.x[c + nx];
        if (j > 0) res += L.cy[c - nx] * L.x[c - nx];
        L.t[c] = res;
    }
    sync();
    const int cnx = C.nx, cn = cnx * C.ny;
    int I = tid % cnx, J = tid / cnx;
    const int dI = nt % cnx, dJ = nt / cnx;
    for (int cc = tid; cc < cn; cc += nt) {
        float sum = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int fi = 2 * I + (q & 1), fj = 2 * J + (q >> 1);
            if (fi < nx && fj < ny) sum += L.t[fj * nx + fi];
        }
        C.r[cc] = sum;
        I += dI;
        J += dJ;
        if (I >= cnx) { I -= cnx; ++J; }
    }
    sync();
}

__device__ __forceinline__ void local_up(const LocalLevel Ls, const LocalLevel Cs, float om, float alpha)
{
    const LocalView L(Ls), C(Cs);
    const int tid = threadIdx.x, nt = blockDim.x;
    auto sync = [] { __syncthreads(); };
    const int nx = L.nx, ny = L.ny, n = nx * ny, cnx = C.nx;
    auto y0 = [&](int c, int i, int j) { return L.x[c] + alpha * C.x[(j >> 1) * cnx + (i >> 1)]; };
    int i = tid % nx, j = tid / nx;
    const int di = nt % nx, dj = nt / nx;
    auto step = [&] { i += di; j += dj; if (i >= nx) { i -= nx; ++j; } };
    for (int c = tid; c < n; c += nt, step()) {   // y1 = Jacobi(y0) into t
        float nb = L.r[c];
        if (i + 1 < nx) nb += L.cx[c] * y0(c + 1, i + 1, j);
        if (i > 0) nb += L.cx[c - 1] * y0(c - 1, i - 1, j);
        if (j + 1 < ny) nb += L.cy[c] * y0(c + nx, i, j + 1);
        if (j > 0) nb += L.cy[c - nx] * y0(c - nx, i, j - 1);
        L.t[c] = (1.f - om) * y0(c, i, j) + om * nb * L.id[c];
    }
    sync();
    i = tid % nx;
    j = tid / nx;
    for (int c = tid; c < n; c += nt, step()) {   // y2 = Jacobi(y1) into x
        float nb = L.r[c];
        if (i + 1 < nx) nb += L.cx[c] * L.t[c + 1];
        if (i > 0) nb += L.cx[c - 1] * L.t[c - 1];
        if (j + 1 < ny) nb += L.cy[c] * L.t[c + nx];
        if (j > 0) nb += L.cy[c - nx] * L.t[c - nx];
        L.x[c] = (1.f - om) * L.t[c] + om * nb * L.id[c];
    }
    sync();
}

// x = A^-1 r on the direct level (n <= kDirectMax cells) from its inverse
// at float offset cinv (row-major n x n): warp w forms rows 4w..4w+3, lane l
// the products of columns l and l + 32, then a butterfly sum.
__device__ __forceinline__ void local_direct(const LocalLevel Bs, int cinv)
{
    extern __shared__ __align__(16) float mg_smem[];
    const LocalView B(Bs);
    const int n = B.nx * B.ny, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const float r0 = lane < n ? B.r[lane] : 0.f, r1 = lane + 32 < n ? B.r[lane + 32] : 0.f;
    for (int c0 = 4 * (int)(threadIdx.x >> 5); c0 < n; c0 += 4 * nw) {
        float acc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int row = cinv + min(c0 + u, n - 1) * n;
            float v = lane < n ? mg_smem[row + lane] * r0 : 0.f;
            if (lane + 32 < n) v = __fmaf_rn(mg_smem[row + lane + 32], r1, v);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
            acc[u] = v;
        }
        if (lane == 0)
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (c0 + u < n) B.x[c0 + u] = acc[u];
    }
    __syncthreads();
}

// V-cycle over the coarse levels [l0, ld] in CTA 0's shared memory: input
// S[l0].r, output S[l0].x; level ld is solved exactly.
__device__ void vcycle_local_direct(const LocalLevel* S, int l0, int ld, int cinv, float om, float alpha)
{
    for (int l = l0; l < ld; ++l) local_down(S[l], S[l + 1], om);
    local_direct(S[ld], cinv);
    for (int l = ld - 1; l >= l0; --l) local_up(S[l], S[l + 1], om, alpha);
}

__global__ void __launch_bounds__(kTileBlock) mg_tile_grid_kernel(const TileArgs ta)
{
    const MgArgs& a = ta.m;
    GridCtx cx(a);
    __shared__ float slots_f[6];
    __shared__ double slots_d[6];
    __shared__ LocalLevel S[kMaxLevels];
    extern __shared__ __align__(16) float mg_smem[];
    if (ld_volatile_int(&a.status->done)) return;   // same value in every CTA (set by an earlier kernel)
    const int lf = a.local_from;
    const float om = a.omega, alpha = a.alpha;
    const int b = blockIdx.x;                         // 0: coarse levels; 1..px*py: rectangles
    const bool worker = b >= 1 && b <= ta.px * ta.py;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ld = a.direct;   // levels lf..ld in CTA 0, ld solved with its inverse
    int cinv = 0;              // float offset of the inverse, after the levels
    for (int l = lf; l <= ld; ++l) cinv += (kLocalArrays * a.lv[l].nx * a.lv[l].ny + 3) & ~3;
    if (b == 0) {   // the coarse levels in shared memory, with 1/d, and the inverse
        if (tid == 0) {
            int off = 0;
            for (int l = lf; l <= ld; ++l) {
                const int n = a.lv[l].nx * a.lv[l].ny;
                const int p = off;
                S[l] = LocalLevel{a.lv[l].nx, a.lv[l].ny, p, p + n, p + 2 * n, p + 3 * n, p + 4 * n, p + 5 * n,
                                  p + 6 * n};
                off += (kLocalArrays * n + 3) & ~3;
            }
        }
        const int nd = a.lv[ld].nx * a.lv[ld].ny;
        for (int e = tid; e < nd * nd; e += nt) mg_smem[cinv + e] = a.cinv[e];
        __syncthreads();
        for (int l = lf; l <= ld; ++l) {
            const int n = a.lv[l].nx * a.lv[l].ny;
            const LocalView V(S[l]);
            for (int c = tid; c < n; c += nt) {
                const float d = a.lv[l].d[c];
                V.d[c] = d;
                V.id[c] = 1.f / d;
                V.cx[c] = a.lv[l].cx[c];
                V.cy[c] = a.lv[l].cy[c];
            }
        }
        __syncthreads();
    }
    int i0 = 0, i1 = 0, j0 = 0, j1 = 0;   // level-0 rectangle
    if (worker) tile_rect(ta, 0, b, i0, i1, j0, j1);
    const int nx = a.nx, ny = a.ny;
    const int w0 = i1 - i0, h0 = j1 - j0;
    const MgLevelDev& L0 = a.lv[0];
    int sc = 0;   // the CG residual alternates between a.s (0) and level 0's r (1)
    auto sbuf = [&](int k) { return k ? L0.r : a.s; };
    float* const z = L0.t;
    int rotf = 0, rotd = 0;

    auto down_level = [&](int l, auto rin) {
        const MgLevelDev& L = a.lv[l];
        int si0, si1, sj0, sj1;
        tile_rect(ta, l, b, si0, si1, sj0, sj1);
        if (si1 <= si0 || sj1 <= sj0) return;
        const int rows = tile_rows(ta, si1 - si0);
        const bool last = l == lf - 1;
        const MgLevelDev& C = a.lv[l + 1];
        for (int t0 = sj0; t0 < sj1; t0 += rows) {
            const int t1 = min(t0 + rows, sj1);
            TileView v;
            tile_load(v, mg_smem, ta.tile_cells, L, si0, si1, t0, t1, rin, false,
                      [](int, int, int) { return 0.f; });
            const int n = v.rw * v.rh;
            {   // x1 = omega r / d (and 1/d in place)
                CellWalk cw(v.rw);
                for (int k = tid; k < n; k += nt, cw.next()) {
                    const int p = v.at(cw.i, cw.j);
                    const float id = 1.f / v.ID[p];
                    v.ID[p] = id;
                    v.XA[p] = om * v.R[p] * id;
                }
            }
            __syncthreads();
            {
                CellWalk cw(v.rw);
                for (int k = tid; k < n; k += nt, cw.next()) {
                    const int p = v.at(cw.i, cw.j);
                    v.XB[p] = tile_jacobi(v, v.XA, p, om, v.ID[p]);
                }
            }
            __syncthreads();
            // own cells: store x2; the residual r - A x2 into XA (its x1 is no longer read)
            const int ow = si1 - si0, oh = t1 - t0;
            {
                CellWalk cw(ow);
                for (int k = tid; k < ow * oh; k += nt, cw.next()) {
                    const int gi = si0 + cw.i, gj = t0 + cw.j, c = gj * L.nx + gi;
                    const int p = v.at(gi - v.gi0, gj - v.gj0);
                    const float res = tile_nb(v, v.XB, p) - __frcp_rn(v.ID[p]) * v.XB[p];
                    L.x[c] = v.XB[p];
                    if (last) L.t[c] = res;   // restricted by CTA 0
                    else v.XA[p] = res;
                }
            }
            __syncthreads();
            if (!last) {   // 2x2 restriction into the next level's rectangle
                const int I0 = si0 >> 1, I1 = (si1 + 1) >> 1, J0 = t0 >> 1, J1 = (t1 + 1) >> 1;
                const int cw_ = I1 - I0;
                CellWalk cw(cw_);
                for (int k = tid; k < cw_ * (J1 - J0); k += nt, cw.next()) {
                    const int I = I0 + cw.i, J = J0 + cw.j;
                    float sum = 0.f;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int gi = 2 * I + (q & 1), gj = 2 * J + (q >> 1);
                        if (gi < si1 && gj < t1) sum += v.XA[v.at(gi - v.gi0, gj - v.gj0)];
                    }
                    C.r[J * C.nx + I] = sum;
                }
            }
            __syncthreads();   // the next sub-tile reuses the arrays
        }
    };
    auto up_level = [&](int l, auto rin, bool level0, float& lrz) {
        const MgLevelDev& L = a.lv[l];
        const MgLevelDev& C = a.lv[l + 1];
        const float* ct = C.t;   // the coarse correction (CTA 0 copies its output there)
        int si0, si1, sj0, sj1;
        tile_rect(ta, l, b, si0, si1, sj0, sj1);
        if (si1 <= si0 || sj1 <= sj0) return;
        const int rows = tile_rows(ta, si1 - si0);
        for (int t0 = sj0; t0 < sj1; t0 += rows) {
            const int t1 = min(t0 + rows, sj1);
            TileView v;
            tile_load(v, mg_smem, ta.tile_cells, L, si0, si1, t0, t1, rin, true,
                      [&](int c, int gi, int gj) {
                          return __ldcg(L.x + c) + alpha * __ldcg(ct + (gj >> 1) * C.nx + (gi >> 1));
                      });
            const int n = v.rw * v.rh;
            {
                CellWalk cw(v.rw);
                for (int k = tid; k < n; k += nt, cw.next()) {
                    const int p = v.at(cw.i, cw.j);
                    const float id = 1.f / v.ID[p];
                    v.ID[p] = id;
                    v.XB[p] = tile_jacobi(v, v.XA, p, om, id);
                }
            }
            __syncthreads();
            const int ow = si1 - si0, oh = t1 - t0;
            {
                CellWalk cw(ow);
                for (int k = tid; k < ow * oh; k += nt, cw.next()) {
                    const int gi = si0 + cw.i, gj = t0 + cw.j, c = gj * L.nx + gi;
                    const int p = v.at(gi - v.gi0, gj - v.gj0);
                    const float y = tile_jacobi(v, v.XB, p, om, v.ID[p]);
                    L.t[c] = y;
                    if (level0) lrz += v.R[p] * y;
                }
            }
            __syncthreads();
        }
    };
    // levels 1 .. lf-1 down, the coarse levels in CTA 0, back up to level 1;
    // every phase ends on a grid barrier
    auto inner_levels = [&]() {
        for (int l = 1; l < lf; ++l) {
            if (worker) {
                const float* rl = a.lv[l].r;
                down_level(l, [&](int c) { return __ldcg(rl + c); });
            }
            cx.sync();
        }
        if (b == 0) {   // restriction of level lf-1's residual, then the coarse V-cycle
            const MgLevelDev& F = a.lv[lf - 1];
            const LocalView Lc(S[lf]);
            const int n = Lc.nx * Lc.ny;
            // stage level lf-1's residual through the coarse level's x and t
            // (free until its V-cycle) in chunks of whole fine-row pairs: one
            // L2 round trip per chunk instead of one per two coarse cells
            const int stage = S[lf].x;                  // float offset; x and t are adjacent
            const int prows = (2 * n / F.nx) & ~1;      // fine rows per chunk
            const bool staged = F.nx % 4 == 0 && stage % 4 == 0 && prows >= 2 &&
                                (reinterpret_cast<size_t>(F.t) & 15) == 0;
            if (staged) {
                extern __shared__ __align__(16) float mg_smem_stage[];
                float* const buf = mg_smem_stage + stage;
                const int q4 = F.nx / 4;                // 16-byte pieces per fine row
                for (int r0 = 0; r0 < F.ny; r0 += prows) {
                    const int nr = min(prows, F.ny - r0);
                    for (int k = tid; k < nr * q4; k += nt)
                        mg_cp_async16_cg(buf + 4 * k, F.t + (size_t)r0 * F.nx + 4 * k);
                    asm volatile("cp.async.wait_all;" ::: "memory");
                    __syncthreads();
                    const int J0 = r0 >> 1, J1 = min(Lc.ny, (r0 + nr + 1) >> 1);
                    for (int k = tid; k < (J1 - J0) * Lc.nx; k += nt) {
                        const int J = J0 + k / Lc.nx, I = k - (J - J0) * Lc.nx;
                        float sum = 0.f;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int gi = 2 * I + (q & 1), gj = 2 * J + (q >> 1);
                            if (gi < F.nx && gj < F.ny) sum += buf[(gj - r0) * F.nx + gi];
                        }
                        Lc.r[J * Lc.nx + I] = sum;
                    }
                    __syncthreads();
                }
            }
            constexpr int kU = 2;   // coarse cells per thread whose 8 loads are in flight together
            for (int c0 = 0; !staged && c0 < n; c0 += kU * nt) {
                float v[kU][4];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int cc = c0 + tid + u * nt;
                    const int J = cc / Lc.nx, I = cc - J * Lc.nx;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int gi = 2 * I + (q & 1), gj = 2 * J + (q >> 1);
                        v[u][q] = cc < n && gi < F.nx && gj < F.ny ? __ldcg(F.t + gj * F.nx + gi) : 0.f;
                    }
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int cc = c0 + tid + u * nt;
                    if (cc >= n) break;
                    const int J = cc / Lc.nx, I = cc - J * Lc.nx;
                    float sum = 0.f;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (2 * I + (q & 1) < F.nx && 2 * J + (q >> 1) < F.ny) sum += v[u][q];
                    Lc.r[cc] = sum;
                }
            }
            __syncthreads();
            vcycle_local_direct(S, lf, ld, cinv, om, alpha);
            for (int c = tid; c < n; c += nt) a.lv[lf].t[c] = Lc.x[c];
        }
        cx.sync();
        for (int l = lf - 1; l >= 1; --l) {
            if (worker) {
                const float* rl = a.lv[l].r;
                float dummy = 0.f;
                up_level(l, [&](int c) { return __ldcg(rl + c); }, false, dummy);
            }
            cx.sync();
        }
    };

    // ---- FP64 refinement
    int total = 0;
    double relres = 0.0, bb = 0.0;
    for (int outer = 0;; ++outer) {
        if (outer > 0) cx.sync();   // every CTA's x update visible
        const double* xs = outer == 0 ? a.guess : a.x;
        double lrr = 0.0, lbb = 0.0;
        float* s = sbuf(sc);
        rect_cells<double2, 2>(i0, j0, w0, h0, nx,
                            [&](int c, int i, int j) {
                                double v = a.diag[c] * __ldcg(xs + c);
                                if (i + 1 < nx) v -= a.cx[c] * __ldcg(xs + c + 1);
                                if (i > 0) v -= a.cx[c - 1] * __ldcg(xs + c - 1);
                                if (j + 1 < ny) v -= a.cy[c] * __ldcg(xs + c + nx);
                                if (j > 0) v -= a.cy[c - nx] * __ldcg(xs + c - nx);
                                const double bc = a.b[c];
                                return make_double2(bc - v, bc);
                            },
                            [&](int c, double2 rb) {
                                if (outer == 0) {
                                    a.x[c] = xs[c];
                                    lbb += rb.y * rb.y;
                                }
                                s[c] = (float)rb.x;
                                a.dl[c] = 0.f;
                                lrr += rb.x * rb.x;
                            });
        double v2[2];
        cx.sum2d(lrr, lbb, v2, slots_d, rotd);
        if (outer == 0) bb = v2[1];
        const double rr = v2[0];
        relres = bb > 0.0 ? sqrt(rr / bb) : 0.0;
        if (rr <= a.rtol * a.rtol * bb || total >= a.max_iter) break;
        // z = M s: level 0 down, the inner levels, level 0 up
        if (worker) {
            const float* sr = s;
            down_level(0, [&](int c) { return __ldcg(sr + c); });
        }
        cx.sync();
        inner_levels();
        float lrz = 0.f, lss = 0.f;
        if (worker) {
            const float* sr = s;
            up_level(0, [&](int c) { return __ldcg(sr + c); }, true, lrz);
            rect_cells<float>(i0, j0, w0, h0, nx, [&](int c, int, int) { return s[c]; },
                              [&](int, float sv) { lss += sv * sv; });
        }
        float f2[2];
        cx.sum2f(lrz, lss, f2, slots_f, rotf);
        float rz = f2[0];
        if (!(rz > 0.f) || !(rz < INFINITY) || !isfinite(rr)) {
            // no usable FP32 search direction (as in mg_solve_body): leave;
            // a non-finite residual poisons x so that Err(rho) reports it
            const bool bad = !(rz == 0.f) || !isfinite(rr);
            if (bad) {
                rect_cells<int>(i0, j0, w0, h0, nx, [](int, int, int) { return 0; },
                                [&](int c, int) { a.x[c] = kNaN; });
                relres = kNaN;
            }
            break;
        }
        const float istop = a.inner_rtol * a.inner_rtol * f2[1];
        float beta = 0.f;
        bool first = true;
        while (total < a.max_iter && rz > 0.f) {
            // p = z + beta p, q = A p = A z + beta q, p.q (first: p = z, q = A z)
            float lpq = 0.f;
            rect_cells<float2, 2>(i0, j0, w0, h0, nx,
                               [&](int c, int i, int j) {
                                   const float zc = __ldcg(z + c);
                                   float az = L0.d[c] * zc;
                                   if (i + 1 < nx) az -= L0.cx[c] * __ldcg(z + c + 1);
                                   if (i > 0) az -= L0.cx[c - 1] * __ldcg(z + c - 1);
                                   if (j + 1 < ny) az -= L0.cy[c] * __ldcg(z + c + nx);
                                   if (j > 0) az -= L0.cy[c - nx] * __ldcg(z + c - nx);
                                   const float pv = first ? zc : __fmaf_rn(beta, a.p[c], zc);
                                   const float qv = first ? az : __fmaf_rn(beta, a.q[c], az);
                                   return make_float2(pv, qv);
                               },
                               [&](int c, float2 pq) {
                                   a.p[c] = pq.x;
                                   a.q[c] = pq.y;
                                   lpq += pq.x * pq.y;
                               });
            cx.sum2f(lpq, 0.f, f2, slots_f, rotf);
            first = false;
            const float al = rz / f2[0];
            ++total;
            const bool more = total < a.max_iter;
            // s <- s - al q, dl <- dl + al p; then level 0 down on the new s
            const float* so = sbuf(sc);
            float* sn = sbuf(sc ^ 1);
            float lss2 = 0.f;
            if (worker) {
                rect_cells<float2>(i0, j0, w0, h0, nx,
                                   [&](int c, int, int) {
                                       return make_float2(__fmaf_rn(-al, __ldcg(a.q + c), __ldcg(so + c)),
                                                          __fmaf_rn(al, a.p[c], a.dl[c]));
                                   },
                                   [&](int c, float2 sd) {
                                       sn[c] = sd.x;
                                       a.dl[c] = sd.y;
                                       lss2 += sd.x * sd.x;
                                   });
                // the same arithmetic as the owners' update above: halo cells get the same bits
                if (more) down_level(0, [&](int c) { return __fmaf_rn(-al, __ldcg(a.q + c), __ldcg(so + c)); });
            }
            sc ^= 1;
            cx.sum2f(lss2, 0.f, f2, slots_f, rotf);
            if (f2[0] <= istop || !more) break;
            inner_levels();
            float lrz2 = 0.f;
            if (worker) {
                const float* sr = sbuf(sc);
                up_level(0, [&](int c) { return __ldcg(sr + c); }, true, lrz2);
            }
            cx.sum2f(lrz2, 0.f, f2, slots_f, rotf);
            beta = f2[0] / rz;
            rz = f2[0];
        }
        rect_cells<float>(i0, j0, w0, h0, nx, [&](int c, int, int) { return a.dl[c]; },
                          [&](int c, float d) { a.x[c] += (double)d; });
        if (total >= a.max_iter) {   // budget spent: no further residual evaluation
            relres = -1.0;
            break;
        }
    }
    if (b == 0 && tid == 0) {
        a.status->synth_iters = total;
        a.status->synth_iters_total += total;
        a.status->synth_relres = relres;
    }
}

// ------------------------------------------------------------ strip solver
// The same iteration (FP64 refinement around FP32 MG-PCG, identical cycle)
// with every level resident in the cluster's shared memory.  Levels 0..ld
// are cut into row strips, one per CTA; the cut is made on level P = ld + 1
// and doubled downwards, so a coarse cell and its children always live in
// the same CTA and the grid transfers stay local.  Each strip array carries
// one halo row above and below; a phase that writes a boundary row also
// stores it into the neighbour's halo row (distributed shared memory) before
// the cluster barrier, so every read after the barrier is local.  Levels P..
// live whole in CTA 0: the other CTAs store their restricted rows of level P
// into CTA 0, and CTA 0 stores level P's correction back into every CTA.
// Reductions store each CTA's partial into every CTA's slot table and sum
// the table in a fixed order: all CTAs get the same bits.
constexpr int kSA_D = 0, kSA_ID = 1, kSA_CX = 2, kSA_CY = 3, kSA_X = 4, kSA_T = 5, kSA_R = 6;
constexpr int kSA_P = 7, kSA_DL = 8;   // level 0 only
constexpr int kMaxCl = 16;
// The grid-wide solver above this many cells: smaller meshes that miss the
// strip plan by a few kilobytes (e.g. 234^2) stay on the cluster form, which
// the batched solve also runs, so both give the same bits.
constexpr long long kGridMinCells = 256 * 256;

struct SLevel {
    int nx, ny;
    int cap;       // floats per array: (largest strip or whole level + 2 halo rows) * nx, 16-byte multiple
    int off;       // float offset of the level's arrays in dynamic shared memory
    const float* gd; const float* gcx; const float* gcy;
};

struct SArgs {
    int nl, ld, cl;
    SLevel lv[kMaxLevels];
    int nx, ny, N;
    const double* diag; const double* cx; const double* cy;
    const double* b; const double* guess; double* x;
    const float* r0;       // b - D guess (FP32), computed with b
    const double* norms;   // [0] = |b - D guess|^2, [1] = |b|^2 (FP64)
    double rtol;
    int max_iter, nu;
    float inner_rtol, omega, alpha;
    Status* status;
};

// This CTA's part of one level: rows [rs, rs + rows); array k at float
// offset off + k * cap, cell (jj, i) at (jj + 1) * nx + i.
struct Strip {
    int nx, ny, rs, rows, cap, off, prev_rows;
    bool prev, next;   // neighbouring strips exist (strip levels only)
};

extern __shared__ __align__(16) float sm_f[];

__device__ __forceinline__ float* sarr(const Strip S, int k) { return sm_f + S.off + k * S.cap; }

__device__ __forceinline__ void strip_rows(const SArgs& a, int l, int r, int& rs, int& re)
{
    const int P = a.ld + 1, nyP = a.lv[P].ny;
    const int s0 = (int)((long long)r * nyP / a.cl), s1 = (int)((long long)(r + 1) * nyP / a.cl);
    const int sh = P - l;
    rs = s0 << sh;
    re = min(s1 << sh, a.lv[l].ny);
}

// Visit this thread's cells of a strip: f(padded index, column, local row);
// thread tid of nt threads takes cells tid, tid + nt, ...
template <class F>
__device__ __forceinline__ void each_cell(const Strip S, F f, int tid, int nt)
{
    const int nx = S.nx, n = S.rows * nx;
    int lc = tid;
    if (lc >= n) return;
    int jj = lc / nx, i = lc - jj * nx;
    const int sj = nt / nx, si = nt - sj * nx;
    for (; lc < n; lc += nt) {
        f(lc + nx, i, jj);
        i += si;
        jj += sj;
        if (i >= nx) {
            i -= nx;
            ++jj;
        }
    }
}

template <class F>
__device__ __forceinline__ void each_cell(const Strip S, F f)
{
    each_cell(S, f, (int)threadIdx.x, (int)blockDim.x);
}

// Visit this thread's cells by padded index only.
template <class F>
__device__ __forceinline__ void each_c(const Strip S, F f, int tid, int nt)
{
    const int end = (S.rows + 1) * S.nx;
    for (int c = S.nx + tid; c < end; c += nt) f(c);
}

// (A v)(cell) with v = array k at padded index c; rows outside the strip come
// from the halos.  No branches: a coupling to a missing neighbour is zero (the
// operator and its Galerkin coarsenings have zero face coefficients on the
// domain boundary, halo rows there stay zero), and every neighbour index stays
// inside the padded array.
__device__ __forceinline__ float strip_Av(const Strip S, int k, int c)
{
    const float* base = sm_f + S.off;
    const float* v = base + k * S.cap;
    const float* cxa = base + kSA_CX * S.cap;
    const float* cya = base + kSA_CY * S.cap;
    const int nx = S.nx;
    float y = base[kSA_D * S.cap + c] * v[c];
    y -= cxa[c] * v[c + 1];
    y -= cxa[c - 1] * v[c - 1];
    y -= cya[c] * v[c + nx];
    y -= cya[c - nx] * v[c - nx];
    return y;
}

class SCluster {
  public:
    __device__ SCluster() : cl_(cg::this_cluster())
    {
        rank_ = (int)cl_.block_rank();
        n_ = (int)cl_.num_blocks();
    }
    __device__ void sync() { cl_.sync(); }
    __device__ int rank() const { return rank_; }
    __device__ int size() const { return n_; }
    template <typename V>
    __device__ V* remote(V* p, int r) { return cl_.map_shared_rank(p, r); }
    // Fixed-order sums over the cluster, identical bits in every thread of
    // every CTA.  slots: [3][kMaxCl][2] rotating tables (a table is written
    // again only after two more barriers, so one barrier per sum suffices).
    template <typename V>
    __device__ void sum2(V a, V b, V out[2], V* slots, int& rot, V* wsm)
    {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(kFull, a, o);
            b += __shfl_xor_sync(kFull, b, o);
        }
        __syncthreads();   // wsm free (previous use complete)
        if (lane == 0) {
            wsm[wid] = a;
            wsm[32 + wid] = b;
        }
        __syncthreads();
        V* table = slots + rot * (2 * kMaxCl);
        if (threadIdx.x < n_) {   // thread q stores this CTA's partial into CTA q's table
            V ta = V(0), tb = V(0);
            for (int w = 0; w < nw; ++w) {
                ta += wsm[w];
                tb += wsm[32 + w];
            }
            V* dst = cl_.map_shared_rank(table, (int)threadIdx.x);
            dst[2 * rank_] = ta;
            dst[2 * rank_ + 1] = tb;
        }
        cl_.sync();
        V s0 = lane < n_ ? table[2 * lane] : V(0), s1 = lane < n_ ? table[2 * lane + 1] : V(0);
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(kFull, s0, o);
            s1 += __shfl_xor_sync(kFull, s1, o);
        }
        out[0] = s0;
        out[1] = s1;
        rot = (rot + 1) % 3;
    }

  private:
    cg::cluster_group cl_;
    int rank_, n_;
};

__device__ __forceinline__ int other_buf(int k) { return k == kSA_X ? kSA_T : kSA_X; }

__device__ __forceinline__ void strip_body(const SArgs& a)
{
    __shared__ float slots_f[3 * 2 * kMaxCl];
    __shared__ double slots_d[3 * 2 * kMaxCl];
    __shared__ float wsm_f[64];
    __shared__ double wsm_d[64];
    __shared__ Strip St[kMaxLevels];
    SCluster cx;
    if (ld_volatile_int(&a.status->done)) return;   // same value in every CTA
    const int r = cx.rank(), ld = a.ld, P = ld + 1, nl = a.nl, nu = a.nu;
    const float om = a.omega, alpha = a.alpha;
    const int down_buf = (nu % 2) ? kSA_X : kSA_T;   // pre-smoothed iterate; post-smoothed: kSA_T
    float* prev_sm = r > 0 ? cx.remote(sm_f, r - 1) : nullptr;
    float* next_sm = r + 1 < cx.size() ? cx.remote(sm_f, r + 1) : nullptr;

    if (threadIdx.x < nl) {
        const int l = threadIdx.x;
        Strip S;
        S.nx = a.lv[l].nx;
        S.ny = a.lv[l].ny;
        S.cap = a.lv[l].cap;
        S.off = a.lv[l].off;
        S.rs = 0;
        S.rows = S.ny;
        S.prev_rows = 0;
        S.prev = false;
        S.next = false;
        if (l <= ld) {
            int rs, re;
            strip_rows(a, l, r, rs, re);
            S.rs = rs;
            S.rows = re - rs;
            if (r > 0) {
                int ps, pe;
                strip_rows(a, l, r - 1, ps, pe);
                S.prev_rows = pe - ps;
                S.prev = true;
            }
            S.next = r + 1 < cx.size();
        }
        St[l] = S;
    }
    // zero every array (halo rows on the domain boundary stay zero)
    {
        const int tot = a.lv[nl - 1].off + 7 * a.lv[nl - 1].cap;
        for (int c = threadIdx.x; c < tot; c += blockDim.x) sm_f[c] = 0.f;
    }
    __syncthreads();
    // coefficients of the levels this CTA holds (and the south coupling of
    // row 0): one flat index over all of them, 4 items' loads in flight per thread
    __shared__ int first[kMaxLevels + 1];
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int l = 0; l < nl; ++l) {
            first[l] = acc;
            if (l <= ld || r == 0) acc += St[l].rows * St[l].nx + (St[l].rs > 0 ? St[l].nx : 0);
        }
        first[nl] = acc;
    }
    __syncthreads();
    {
        const int tot = first[nl];
        constexpr int U = 4;
        for (int e0 = threadIdx.x; e0 < tot; e0 += U * blockDim.x) {
            float dv[U], xv[U], yv[U];
            int lv[U], cc[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * blockDim.x;
                lv[u] = -1;
                if (e < tot) {
                    int l = 0;
                    while (first[l + 1] <= e) ++l;
                    const Strip S = St[l];
                    const SLevel& L = a.lv[l];
                    const int c = e - first[l] - (S.rs > 0 ? S.nx : 0);   // c < 0: south halo row
                    const int g = S.rs * S.nx + c;
                    lv[u] = l;
                    cc[u] = c;
                    yv[u] = L.gcy[g];
                    if (c >= 0) {
                        dv[u] = L.gd[g];
                        xv[u] = L.gcx[g];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (lv[u] < 0) continue;
                const Strip S = St[lv[u]];
                const int c = cc[u] + S.nx;   // padded index
                sarr(S, kSA_CY)[c] = yv[u];
                if (cc[u] >= 0) {
                    sarr(S, kSA_D)[c] = dv[u];
                    sarr(S, kSA_ID)[c] = 1.f / dv[u];
                    sarr(S, kSA_CX)[c] = xv[u];
                }
            }
        }
    }
    __syncthreads();

    // store v into array k of strip S at padded index c, and into the
    // neighbours' halo rows when c lies in the first or last row
    auto put = [&](const Strip S, int k, int c, float v) {
        sarr(S, k)[c] = v;
        if (S.prev && c < 2 * S.nx) prev_sm[S.off + k * S.cap + S.prev_rows * S.nx + c] = v;
        if (S.next && c >= S.rows * S.nx) next_sm[S.off + k * S.cap + c - S.rows * S.nx] = v;
    };
    // `steps` damped-Jacobi steps from buffer cur; returns the buffer of the
    // result.  mode 0: strip level, every thread, cluster barriers; 1: level
    // held whole by CTA 0, every thread, block barriers; 2: the same with the
    // lanes of warp 0 alone and warp barriers (small levels).
    auto jacobi = [&](const Strip S, int cur, int steps, int mode) {
        const float* rr = sarr(S, kSA_R);
        const float* id = sarr(S, kSA_ID);
        const int tid = mode == 2 ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
        const int nt = mode == 2 ? 32 : (int)blockDim.x;
        for (int k = 0; k < steps; ++k) {
            if (mode == 0) cx.sync();
            else if (mode == 1) __syncthreads();
            else __syncwarp();
            const int oth = other_buf(cur), c0 = cur;
            const float* src = sarr(S, cur);
            each_c(S, [&](int c) { put(S, oth, c, src[c] + om * (rr[c] - strip_Av(S, c0, c)) * id[c]); }, tid, nt);
            cur = oth;
        }
        return cur;
    };
    // residual of buffer cur summed over 2x2 children into coarse rows
    // row0.. of the padded coarse array cr (coarse width cnx), thread tid of nt
    auto restrict_to = [&](const Strip S, int cur, float* cr, int cnx, int row0, int tid, int nt) {
        const float* rr = sarr(S, kSA_R);
        const int crows = (S.rows + 1) / 2, nx = S.nx;
        for (int cc = tid; cc < crows * cnx; cc += nt) {
            const int JJ = cc / cnx, I = cc - JJ * cnx;
            float sum = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = 2 * I + (q & 1), jj = 2 * JJ + (q >> 1);
                if (i < nx && jj < S.rows) {
                    const int c = (jj + 1) * nx + i;
                    sum += rr[c] - strip_Av(S, cur, c);
                }
            }
            cr[(row0 + JJ + 1) * cnx + I] = sum;
        }
    };

    // z = M^{-1} s: one V-cycle, input level-0 R, output level-0 T
    auto vcycle = [&]() {
        for (int l = 0; l <= ld; ++l) {   // down over the strips
            const Strip S = St[l];
            {
                const float* rr = sarr(S, kSA_R);
                const float* id = sarr(S, kSA_ID);
                each_c(S, [&](int c) { put(S, kSA_X, c, om * rr[c] * id[c]); }, threadIdx.x, blockDim.x);
            }
            const int cur = jacobi(S, kSA_X, nu - 1, 0);
            cx.sync();
            const Strip C = St[l + 1];
            if (l < ld) {
                restrict_to(S, cur, sarr(C, kSA_R), C.nx, 0, threadIdx.x, blockDim.x);
                __syncthreads();
            } else {   // level P rows go to CTA 0
                restrict_to(S, cur, cx.remote(sarr(C, kSA_R), 0), C.nx, S.rs / 2, threadIdx.x, blockDim.x);
            }
        }
        cx.sync();
        if (r == 0) {   // levels P.. whole in CTA 0: every thread on levels of more
                        // than 64 cells, warp 0 alone below (cheaper barriers)
            int wl = P;
            while (wl < nl - 1 && St[wl].rows * St[wl].nx > 64) ++wl;
            auto down = [&](int l, int mode) {
                const Strip L = St[l];
                const int tid = mode == 2 ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
                const int nt = mode == 2 ? 32 : (int)blockDim.x;
                const float* rr = sarr(L, kSA_R);
                const float* id = sarr(L, kSA_ID);
                float* xv = sarr(L, kSA_X);
                each_c(L, [&](int c) { xv[c] = om * rr[c] * id[c]; }, tid, nt);
                const int cur = jacobi(L, kSA_X, nu - 1, mode);
                if (mode == 2) __syncwarp();
                else __syncthreads();
                const Strip C = St[l + 1];
                restrict_to(L, cur, sarr(C, kSA_R), C.nx, 0, tid, nt);
                if (mode == 2) __syncwarp();
                else __syncthreads();
            };
            auto up = [&](int l, int mode) {
                const Strip L = St[l];
                const Strip C = St[l + 1];
                const int tid = mode == 2 ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
                const int nt = mode == 2 ? 32 : (int)blockDim.x;
                float* xv = sarr(L, down_buf);
                const float* ct = sarr(C, kSA_T);
                each_cell(L, [&](int c, int i, int j) { xv[c] += alpha * ct[(j / 2 + 1) * C.nx + i / 2]; }, tid, nt);
                jacobi(L, down_buf, nu, mode);
                if (mode == 2) __syncwarp();
                else __syncthreads();
            };
            for (int l = P; l < wl; ++l) down(l, 1);
            if (threadIdx.x < 32) {
                for (int l = wl; l < nl - 1; ++l) down(l, 2);
                const Strip L = St[nl - 1];
                const float* rr = sarr(L, kSA_R);
                const float* id = sarr(L, kSA_ID);
                float* tv = sarr(L, kSA_T);
                each_c(L, [&](int c) { tv[c] = rr[c] * id[c]; }, (int)threadIdx.x, 32);
                __syncwarp();
                for (int l = nl - 2; l >= wl; --l) up(l, 2);
            }
            __syncthreads();
            for (int l = wl - 1; l >= P; --l) up(l, 1);
            __syncthreads();
            // level P's correction into every other CTA
            const Strip C = St[P];
            const float* ct = sarr(C, kSA_T) + C.nx;
            const int n = C.rows * C.nx;
            for (int q = 1; q < cx.size(); ++q) {
                float* dst = cx.remote(sarr(C, kSA_T), q) + C.nx;
                for (int c = threadIdx.x; c < n; c += blockDim.x) dst[c] = ct[c];
            }
        }
        cx.sync();
        for (int l = ld; l >= 0; --l) {   // up over the strips
            const Strip S = St[l];
            const Strip C = St[l + 1];
            const float* ct = sarr(C, kSA_T);
            const float* xo = sarr(S, down_buf);
            const int crow0 = l == ld ? S.rs / 2 : 0;   // level P is held whole
            each_cell(S, [&](int c, int i, int jj) {
                put(S, down_buf, c, xo[c] + alpha * ct[(crow0 + jj / 2 + 1) * C.nx + i / 2]);
            });
            jacobi(S, down_buf, nu, 0);
            __syncthreads();
        }
    };

    const Strip S0 = St[0];
    const int nx = a.nx, ny = a.ny;
    const int n0 = S0.rows * nx, g00 = S0.rs * nx;
    float* s_ = sarr(S0, kSA_R) + nx;
    float* dl_ = sarr(S0, kSA_DL) + nx;
    const float* z_ = sarr(S0, kSA_T) + nx;
    const float* p_ = sarr(S0, kSA_P) + nx;
    int rotf = 0, rotd = 0;
    int total = 0;
    double relres = 0.0;
    const double bb = a.norms[1];
    __shared__ int stop_now;
    for (int outer = 0;; ++outer) {
        // residual s = b - D x: from the right-hand-side pass on the first
        // pass (x = guess), else in FP64 here
        double rr;
        if (outer == 0) {
            for (int c = threadIdx.x; c < n0; c += blockDim.x) {
                s_[c] = a.r0[g00 + c];
                dl_[c] = 0.f;
            }
            rr = a.norms[0];
        } else {
            cx.sync();   // every CTA's x update visible
            double lrr = 0.0;
            for (int c0 = threadIdx.x; c0 < n0; c0 += 2 * blockDim.x) {
                double xc[2], xe[2], xw[2], xn[2], xs[2], dg[2], ce[2], cw[2], cn[2], cs[2], bv[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {   // loads only (indices clamped into the strip's rows)
                    const int c = min(c0 + u * blockDim.x, n0 - 1);
                    const int g = g00 + c, jj = c / nx, i = c - jj * nx, j = S0.rs + jj;
                    const int ge = i + 1 < nx ? g + 1 : g, gw = i > 0 ? g - 1 : g;
                    const int gn = j + 1 < ny ? g + nx : g, gs = j > 0 ? g - nx : g;
                    xc[u] = __ldcg(a.x + g);
                    xe[u] = __ldcg(a.x + ge);
                    xw[u] = __ldcg(a.x + gw);
                    xn[u] = __ldcg(a.x + gn);
                    xs[u] = __ldcg(a.x + gs);
                    dg[u] = a.diag[g];
                    ce[u] = i + 1 < nx ? a.cx[g] : 0.0;
                    cw[u] = i > 0 ? a.cx[gw] : 0.0;
                    cn[u] = j + 1 < ny ? a.cy[g] : 0.0;
                    cs[u] = j > 0 ? a.cy[gs] : 0.0;
                    bv[u] = a.b[g];
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int c = c0 + u * blockDim.x;
                    if (c < n0) {
                        const double v = dg[u] * xc[u] - ce[u] * xe[u] - cw[u] * xw[u] - cn[u] * xn[u] - cs[u] * xs[u];
                        const double rv = bv[u] - v;
                        s_[c] = (float)rv;
                        dl_[c] = 0.f;
                        lrr += rv * rv;
                    }
                }
            }
            double v2[2];
            cx.sum2<double>(lrr, 0.0, v2, slots_d, rotd, wsm_d);
            rr = v2[0];
        }
        // stop test in one thread (FP64 is slow here; every thread reads the decision)
        if (threadIdx.x == 0) {
            relres = bb > 0.0 ? sqrt(rr / bb) : 0.0;
            stop_now = (rr <= a.rtol * a.rtol * bb || total >= a.max_iter) ? 1 : 0;
        }
        __syncthreads();
        if (stop_now) {
            if (outer == 0)
                for (int c = threadIdx.x; c < n0; c += blockDim.x) a.x[g00 + c] = a.guess[g00 + c];
            break;
        }
        // FP32 MG-PCG for D d = s, d = 0 to start
        vcycle();
        float f2[2];
        {
            float l0 = 0.f, l1 = 0.f;
            each_c(S0, [&](int c) {
                const float z = z_[c - nx], sv = s_[c - nx];
                put(S0, kSA_P, c, z);
                l0 += sv * z;
                l1 += sv * sv;
            }, threadIdx.x, blockDim.x);
            cx.sum2<float>(l0, l1, f2, slots_f, rotf, wsm_f);
        }
        float rz = f2[0];
        if (!(rz > 0.f) || !(rz < INFINITY) || !isfinite(rr)) {
            // as in mg_solve_body: no usable FP32 search direction, leave the
            // refinement (every CTA holds the same rz and rr); a non-finite
            // residual poisons x, a vanished one keeps the current x
            const bool bad = !(rz == 0.f) || !isfinite(rr);
            const double* xo = outer == 0 ? a.guess : a.x;
            for (int c = threadIdx.x; c < n0; c += blockDim.x) a.x[g00 + c] = bad ? kNaN : xo[g00 + c];
            if (bad) relres = kNaN;
            break;
        }
        const float istop = a.inner_rtol * a.inner_rtol * f2[1];
        while (total < a.max_iter && rz > 0.f) {
            // the previous barrier published p and its halo rows
            float lpq = 0.f;
            each_c(S0, [&](int c) { lpq += p_[c - nx] * strip_Av(S0, kSA_P, c); }, threadIdx.x, blockDim.x);
            cx.sum2<float>(lpq, 0.f, f2, slots_f, rotf, wsm_f);
            const float al = rz / f2[0];
            float lss = 0.f;
            each_c(S0, [&](int c) {   // q = A p again (same bits) instead of storing it
                dl_[c - nx] += al * p_[c - nx];
                const float sc = s_[c - nx] - al * strip_Av(S0, kSA_P, c);
                s_[c - nx] = sc;
                lss += sc * sc;
            }, threadIdx.x, blockDim.x);
            ++total;
            cx.sum2<float>(lss, 0.f, f2, slots_f, rotf, wsm_f);
            if (f2[0] <= istop || total >= a.max_iter) break;
            vcycle();
            float lrz = 0.f;
            for (int c = threadIdx.x; c < n0; c += blockDim.x) lrz += s_[c] * z_[c];
            cx.sum2<float>(lrz, 0.f, f2, slots_f, rotf, wsm_f);
            const float be = f2[0] / rz;
            rz = f2[0];
            each_c(S0, [&](int c) { put(S0, kSA_P, c, z_[c - nx] + be * p_[c - nx]); }, threadIdx.x, blockDim.x);
            cx.sync();   // p and its halo rows visible before the product
        }
        {
            const double* xo = outer == 0 ? a.guess : a.x;
            for (int c = threadIdx.x; c < n0; c += blockDim.x) a.x[g00 + c] = xo[g00 + c] + (double)dl_[c];
        }
        if (total >= a.max_iter) {   // budget spent: no further residual evaluation
            relres = -1.0;
            break;
        }
        __syncthreads();   // stop_now is rewritten by thread 0 on the next pass
    }
    if (r == 0 && threadIdx.x == 0) {
        a.status->synth_iters = total;
        a.status->synth_iters_total += total;
        a.status->synth_relres = relres;
    }
    // no CTA may leave while another can still store into its shared memory
    cx.sync();
}

__global__ void __launch_bounds__(kMgBlock) mg_strip_kernel(const SArgs a) { strip_body(a); }

// One cluster per problem: cluster c solves the problem of tab[c].
__global__ void __launch_bounds__(kMgBlock) mg_strip_batch_kernel(const SArgs* __restrict__ tab)
{
    strip_body(tab[blockIdx.x / cg::this_cluster().num_blocks()]);
}

}  // namespace

// Builds the level hierarchy (once per call; D does not change).
cudaError_t launch_mg_setup(const Plan& P, cudaStream_t st)
{
    const int g0 = grid_for(P.N, 256, P.num_sms * 8);
    mg_copy_fine_kernel<<<g0, 256, 0, st>>>(P.N, P.diag, P.cx, P.cy, P.mg.d64[0], P.mg.cx64[0], P.mg.cy64[0],
                                             P.mg.d[0], P.mg.cx[0], P.mg.cy[0]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int l = 0; l + 1 < P.mg.nl; ++l) {
        const int cn = P.mg.nx[l + 1] * P.mg.ny[l + 1];
        mg_coarsen_kernel<<<grid_for(cn, 256, P.num_sms * 8), 256, 0, st>>>(
            P.mg.nx[l], P.mg.ny[l], P.mg.d64[l], P.mg.cx64[l], P.mg.cy64[l], P.mg.nx[l + 1], P.mg.ny[l + 1],
            P.mg.d64[l + 1], P.mg.cx64[l + 1], P.mg.cy64[l + 1], P.mg.d[l + 1], P.mg.cx[l + 1], P.mg.cy[l + 1]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (mg_setup_launches(P) > P.mg.nl) {
        const int l = P.mg.direct;
        mg_direct_inverse_kernel<<<1, kInvThreads, 0, st>>>(P.mg.nx[l], P.mg.ny[l], P.mg.d64[l], P.mg.cx64[l],
                                                    P.mg.cy64[l], P.mg.cinv);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Kernels launch_mg_setup launches: the fine copy, one coarsening per level,
// and for meshes the grid solver may take the direct level's inverse.
int mg_setup_launches(const Plan& P)
{
    return P.mg.nl + (P.mg.direct >= 1 && (long long)P.N > kGridMinCells ? 1 : 0);
}

namespace {

// Strip plan for cluster size cl: false if level 1 has fewer rows than CTAs
// or the levels do not fit the shared memory of one CTA.
bool strip_plan(const Plan& P, int cl, size_t smem_cap, SArgs& sa, size_t& bytes)
{
    const MgPlan& g = P.mg;
    if (cl < 2 || cl > kMaxCl || g.nl < 2) return false;
    int ld = -1;
    for (int l = 0; l + 1 < g.nl; ++l)
        if (g.ny[l + 1] >= cl) ld = l;
    if (ld < 0) return false;
    const int Pl = ld + 1, nyP = g.ny[Pl];
    size_t off = 0;
    for (int l = 0; l < g.nl; ++l) {
        int rows = g.ny[l];
        if (l <= ld) {
            rows = 0;
            for (int r = 0; r < cl; ++r) {
                const int s0 = (int)((long long)r * nyP / cl), s1 = (int)((long long)(r + 1) * nyP / cl);
                const int rs = s0 << (Pl - l), re = std::min(s1 << (Pl - l), g.ny[l]);
                rows = std::max(rows, re - rs);
            }
        }
        long long cap = (long long)(rows + 2) * g.nx[l];
        cap = (cap + 3) / 4 * 4;   // 16-byte aligned arrays
        const int narr = l == 0 ? 9 : 7;
        sa.lv[l] = SLevel{g.nx[l], g.ny[l], (int)cap, (int)off, g.d[l], g.cx[l], g.cy[l]};
        off += (size_t)narr * (size_t)cap;
        if (off * sizeof(float) > smem_cap) return false;
    }
    sa.nl = g.nl;
    sa.ld = ld;
    sa.cl = cl;
    bytes = off * sizeof(float);
    return true;
}

cudaError_t launch_cluster(const void* fn, void** args, int cl, size_t smem, cudaStream_t st)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(kMgBlock);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

int clusters_fit(const void* fn, int cl, size_t smem)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(kMgBlock);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace

namespace {

// Shared memory one strip-solver CTA may use for its levels.
size_t strip_smem_cap()
{
    static size_t cap = [] {
        int dev = 0, c = 0;
        cudaFuncAttributes fa{}, fb{};
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&c, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, mg_strip_batch_kernel) != cudaSuccess ||
            cudaFuncGetAttributes(&fb, mg_strip_kernel) != cudaSuccess) {
            cudaGetLastError();
            return (size_t)0;
        }
        const size_t stat = std::max(fa.sharedSizeBytes, fb.sharedSizeBytes);
        return (size_t)c > stat ? (size_t)c - stat : (size_t)0;
    }();
    return cap;
}

// Raises a kernel's dynamic shared-memory limit (never lowers it: plans of
// other sizes may launch concurrently).
cudaError_t raise_limit(const void* fn, size_t bytes)
{
    static std::mutex mu;
    static std::map<const void*, size_t> have;
    std::lock_guard<std::mutex> g(mu);
    size_t& h = have[fn];
    if (bytes <= h) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) h = bytes;
    return e;
}

size_t tile_smem_cap()
{
    static size_t cap = [] {
        int dev = 0, c = 0;
        cudaFuncAttributes fa{};
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&c, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, mg_tile_grid_kernel) != cudaSuccess) {
            cudaGetLastError();
            return (size_t)0;
        }
        return (size_t)c > fa.sharedSizeBytes ? (size_t)c - fa.sharedSizeBytes : (size_t)0;
    }();
    return cap;
}

// Rectangle grid of the tiled solver on G CTAs (CTA 0 runs the coarse
// levels): px x py <= G - 1 rectangles whose level-0 boundaries are multiples
// of 2^(local_from - 1), chosen to minimise the largest rectangle with its
// halo; sub-tile arrays sized to the shared memory that is left.  False when
// the mesh has fewer than two distributed levels or a sub-tile of the widest
// rectangle would not fit.
bool tile_plan(const Plan& P, int G, TileArgs& t, size_t& smem)
{
    const int lf = P.mg.local_from, ld = P.mg.direct;
    const size_t cap = tile_smem_cap();
    if (lf < 2 || ld < lf || G < 2) return false;
    // CTA 0's coarse levels lf..ld (kLocalArrays arrays each, 16-byte
    // aligned) and the inverse of level ld's operator
    size_t local_bytes = (size_t)P.mg.nx[ld] * P.mg.ny[ld] * P.mg.nx[ld] * P.mg.ny[ld] * sizeof(float);
    for (int l = lf; l <= ld; ++l)
        local_bytes += (((size_t)kLocalArrays * P.mg.nx[l] * P.mg.ny[l] + 3) & ~(size_t)3) * sizeof(float);
    if (cap < local_bytes) return false;
    const int A = 1 << (lf - 1);
    const int gx = (P.nx + A - 1) / A, gy = (P.ny + A - 1) / A;
    long best = -1;
    int bpx = 0, bpy = 0;
    for (int px = 1; px <= std::min(gx, kTileMaxDim); ++px) {
        const int py = std::min({(G - 1) / px, gy, kTileMaxDim});
        if (py < 1) break;
        const long w = (long)((gx + px - 1) / px) * A, h = (long)((gy + py - 1) / py) * A;
        const long cost = (w + 4) * (h + 4);
        if (best < 0 || cost < best) {
            best = cost;
            bpx = px;
            bpy = py;
        }
    }
    if (best < 0) return false;
    t.px = bpx;
    t.py = bpy;
    int wmax = 0;
    for (int k = 0; k <= bpx; ++k) t.bx[k] = k == bpx ? P.nx : (int)((long)k * gx / bpx) * A;
    for (int k = 0; k <= bpy; ++k) t.by[k] = k == bpy ? P.ny : (int)((long)k * gy / bpy) * A;
    for (int k = 0; k < bpx; ++k) wmax = std::max(wmax, t.bx[k + 1] - t.bx[k]);
    const size_t cells = cap / ((size_t)kTileArrays * sizeof(float));
    if ((size_t)(wmax + 6) * 8 > cells) return false;   // two rows of the widest rectangle
    t.tile_cells = (int)std::min(cells, (size_t)1 << 20);
    smem = std::max(local_bytes, (size_t)kTileArrays * t.tile_cells * sizeof(float));
    return true;
}

void strip_fill(const Plan& P, const double* guess, double* out, SArgs& sa)
{
    sa.nx = P.nx; sa.ny = P.ny; sa.N = P.N;
    sa.diag = P.diag; sa.cx = P.cx; sa.cy = P.cy; sa.b = P.b; sa.guess = guess; sa.x = out;
    sa.r0 = P.mg.r0;
    sa.norms = P.partials + (size_t)4 * kMaxCgBlocks;
    sa.rtol = P.synth_rtol;
    sa.max_iter = P.synth_max_iter;
    sa.nu = 2;
    sa.inner_rtol = 1e-4f;
    sa.omega = 0.8f;
    sa.alpha = 1.8f;
    sa.status = P.status;
}

MgArgs fallback_args(const Plan& P, const double* guess, double* out, size_t& smem)
{
    MgArgs a{};
    a.nl = P.mg.nl;
    a.local_from = P.mg.local_from;
    for (int l = 0; l < P.mg.nl; ++l) {
        a.lv[l] = MgLevelDev{P.mg.nx[l], P.mg.ny[l], P.mg.d[l], P.mg.cx[l], P.mg.cy[l],
                             P.mg.x[l], P.mg.t[l], P.mg.r[l]};
    }
    a.nx = P.nx; a.ny = P.ny; a.N = P.N;
    a.diag = P.diag; a.cx = P.cx; a.cy = P.cy; a.b = P.b; a.guess = guess; a.x = out;
    a.r0 = P.mg.r0; a.dl = P.mg.dl; a.s = P.mg.s; a.p = P.mg.p; a.q = P.mg.q;
    a.rtol = P.synth_rtol;
    a.max_iter = P.synth_max_iter;
    a.nu = 2;
    a.inner_rtol = 1e-4f;
    a.omega = 0.8f;
    a.alpha = 1.8f;
    a.status = P.status;
    a.gslots_d = P.mg_gslots_d;
    a.gslots_f = P.mg_gslots_f;
    a.gbar = P.status->mg_bar;
    a.wait_cycles = P.wait_cycles;
    a.cinv = P.mg.cinv;
    a.direct = P.mg.direct;
    int off = 0;
    for (int l = P.mg.local_from; l < P.mg.nl; ++l) {
        a.loff[l] = off;
        off += 6 * P.mg.nx[l] * P.mg.ny[l];
        off = (off + 3) / 4 * 4;
    }
    smem = (size_t)off * sizeof(float);
    return a;
}

}  // namespace

// Chooses the synthetic solver of P before any launch: the strip solver on
// the largest schedulable cluster (16 or 8 CTAs) whose plan fits, else the
// solver with the fine levels in global memory; sets the kernels' shared
// memory limits, so the launches themselves make no other runtime call (a
// stream capture can record them).
cudaError_t plan_synthetic(Plan& P)
{
    P.synth_cl = 0;
    P.synth_bytes = 0;
    const size_t cap = strip_smem_cap();
    for (int cl = std::min(P.mg.cluster, 16); cap > 0 && cl >= 8; cl /= 2) {
        SArgs sa{};
        size_t bytes = 0;
        if (!strip_plan(P, cl, cap, sa, bytes)) continue;
        const cudaError_t e = raise_limit((const void*)mg_strip_kernel, bytes);
        if (e != cudaSuccess) return e;
        if (clusters_fit((const void*)mg_strip_kernel, cl, bytes) < 1) continue;
        P.synth_cl = cl;
        P.synth_bytes = bytes;
        return cudaSuccess;
    }
    size_t smem = 0;
    (void)fallback_args(P, nullptr, nullptr, smem);
    P.synth_bytes = smem;
    P.synth_grid = 0;
    cudaError_t e = raise_limit((const void*)mg_solve_kernel, smem);
    if (e != cudaSuccess) return e;
    // large meshes: the same solver over a cooperative grid of every SM
    if ((long long)P.N > kGridMinCells && raise_limit((const void*)mg_solve_grid_kernel, smem) == cudaSuccess) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mg_solve_grid_kernel, kMgBlock, smem) ==
                cudaSuccess && per_sm >= 1) {
            P.synth_grid = std::min(kMaxCgBlocks, per_sm * P.num_sms);
        }
        cudaGetLastError();
        // its tiled form: one CTA per SM
        TileArgs t{};
        size_t tsm = 0;
        P.synth_tiled = 0;
        if (P.synth_grid > 0 && tile_plan(P, std::min(kMaxCgBlocks, P.num_sms), t, tsm) &&
            raise_limit((const void*)mg_tile_grid_kernel, tsm) == cudaSuccess) {
            per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mg_tile_grid_kernel, kTileBlock, tsm) ==
                    cudaSuccess && per_sm >= 1) {
                P.synth_tiled = 1;
                P.synth_grid = std::min(kMaxCgBlocks, P.num_sms);
                P.synth_bytes = tsm;
            }
        }
        cudaGetLastError();
    }
    return cudaSuccess;
}

// The solver plan_synthetic chose.
cudaError_t launch_synthetic_solve(const Plan& P, const double* guess, double* out, cudaStream_t st)
{
    if (P.synth_cl > 0) {
        SArgs sa{};
        size_t bytes = 0;
        if (!strip_plan(P, P.synth_cl, (size_t)-1, sa, bytes)) return cudaErrorInvalidConfiguration;
        strip_fill(P, guess, out, sa);
        void* args[] = {&sa};
        return launch_cluster((const void*)mg_strip_kernel, args, P.synth_cl, bytes, st);
    }
    size_t smem = 0;
    MgArgs a = fallback_args(P, guess, out, smem);
    if (P.synth_grid > 0 && P.synth_tiled) {
        TileArgs t{};
        size_t tsm = 0;
        if (!tile_plan(P, P.synth_grid, t, tsm)) return cudaErrorInvalidConfiguration;
        t.m = a;
        void* args[] = {&t};
        return cudaLaunchCooperativeKernel((const void*)mg_tile_grid_kernel, dim3(P.synth_grid), dim3(kTileBlock),
                                           args, tsm, st);
    }
    if (P.synth_grid > 0) {
        void* args[] = {&a};
        return cudaLaunchCooperativeKernel((const void*)mg_solve_grid_kernel, dim3(P.synth_grid), dim3(kMgBlock),
                                           args, smem, st);
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(P.mg.cluster);
    cfg.blockDim = dim3(kMgBlock);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = P.mg.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, mg_solve_kernel, a);
}

size_t strip_batch_rec_bytes() { return sizeof(SArgs); }

// Strip-solver record of P (guess rho^m, solution into x) on clusters of cl
// CTAs; false when its levels do not fit one CTA's shared memory.
bool strip_batch_rec(const Plan& P, int cl, void* out, size_t* bytes)
{
    SArgs sa{};
    size_t b = 0;
    if (!strip_plan(P, cl, strip_smem_cap(), sa, b)) return false;
    strip_fill(P, P.rho_m, P.x, sa);
    std::memcpy(out, &sa, sizeof(sa));
    *bytes = b;
    return true;
}

// Makes clusters of cl CTAs with `bytes` of shared memory launchable by the
// batched strip solver; false if the device cannot schedule one.
bool prepare_strip_batch(int cl, size_t bytes)
{
    if (raise_limit((const void*)mg_strip_batch_kernel, bytes) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return clusters_fit((const void*)mg_strip_batch_kernel, cl, bytes) >= 1;
}

cudaError_t launch_strip_batch(const void* tab, int n, int cl, size_t bytes, cudaStream_t st)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(n * cl);
    cfg.blockDim = dim3(kMgBlock);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, mg_strip_batch_kernel, static_cast<const SArgs*>(tab));
}

// Largest cluster (16, else 8, 4, 2, 1) the device can schedule for the solver
// (queried once per process).
static int mg_cluster_size_query();

int mg_cluster_size()
{
    static const int c = mg_cluster_size_query();
    return c;
}

static int mg_cluster_size_query()
{
    if (cudaFuncSetAttribute(mg_solve_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
    }
    if (cudaFuncSetAttribute(mg_strip_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
    }
    if (cudaFuncSetAttribute(mg_strip_batch_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
    }
    for (int c = 16; c >= 1; c /= 2) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(c);
        cfg.blockDim = dim3(kMgBlock);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = c;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, mg_solve_kernel, &cfg) == cudaSuccess && n >= 1) return c;
        cudaGetLastError();
    }
    return 1;
}

}  // namespace gsis
