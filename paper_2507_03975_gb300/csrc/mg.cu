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
    unsigned* gbar;                 // [0] arrivals, [1] generation
    long long wait_cycles;
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
// fine levels spread over every SM.  The barrier is a counter and a
// generation word in global memory; every wait is bounded, and after a
// time-out (the status's timeout bit) later barriers return at once so that
// every CTA finishes.  Sums: each CTA's partial in a rotating global table,
// then every warp adds the table in a fixed order (same bits everywhere).
class GridCtx {
  public:
    __device__ GridCtx(const MgArgs& a) : a_(a) {}
    __device__ void sync()
    {
        __syncthreads();
        if (threadIdx.x == 0 && !ld_volatile_int(&a_.status->error)) {
            volatile unsigned* gen = a_.gbar + 1;
            const unsigned g = *gen;
            __threadfence();
            if (atomicAdd(a_.gbar, 1u) == gridDim.x - 1) {
                a_.gbar[0] = 0u;
                __threadfence();
                atomicAdd(a_.gbar + 1, 1u);
            } else {
                const long long t0 = clock64();
                while (*gen == g) {
                    if (clock64() - t0 > a_.wait_cycles) {
                        atomicOr(&a_.status->error, kErrTimeout);
                        break;
                    }
                    __nanosleep(32);
                }
            }
            __threadfence();
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
        const int lane = threadIdx.x & 31;
        float s0 = 0.f, s1 = 0.f;
        for (int r = lane; r < (int)gridDim.x; r += 32) {
            s0 += __ldcg(tab + 2 * r);
            s1 += __ldcg(tab + 2 * r + 1);
        }
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
        const int lane = threadIdx.x & 31;
        double s0 = 0.0, s1 = 0.0;
        for (int r = lane; r < (int)gridDim.x; r += 32) {
            s0 += __ldcg(tab + 2 * r);
            s1 += __ldcg(tab + 2 * r + 1);
        }
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(kFull, s0, o);
            s1 += __shfl_xor_sync(kFull, s1, o);
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
    const MgArgs& a_;
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
        // stop test in one thread (FP64 is slow here; every thread reads the verdict)
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
    return cudaSuccess;
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
