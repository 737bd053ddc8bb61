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
#include <cooperative_groups.h>
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
__device__ void vcycle(const MgArgs& a, const MgLevelDev* S, ClusterCtx& cx)
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

__global__ void __launch_bounds__(kMgBlock) mg_solve_kernel(const MgArgs a)
{
    constexpr int U = 4;   // cells per thread whose loads are in flight together
    __shared__ float slots_f[6];
    __shared__ double slots_d[6];
    extern __shared__ __align__(16) float mg_smem[];
    ClusterCtx cx(a.local_from);
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

cudaError_t launch_synthetic_solve(const Plan& P, const double* guess, double* out, cudaStream_t st)
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
    int off = 0;
    for (int l = P.mg.local_from; l < P.mg.nl; ++l) {
        a.loff[l] = off;
        off += 6 * P.mg.nx[l] * P.mg.ny[l];
        off = (off + 3) / 4 * 4;
    }
    const size_t smem = (size_t)off * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(mg_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
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

// Largest cluster (16, else 8, 4, 2, 1) the device can schedule for the solver.
int mg_cluster_size()
{
    if (cudaFuncSetAttribute(mg_solve_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
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
