// Internal declarations of libgsis (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "gsis.h"

namespace gsis {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxK = 4096;            // directions per quadrature (host-side check)
constexpr int kMaxSide = (1 << 20) - 1; // cells per mesh side
constexpr int kSweepMaxPairs = 12;      // (compute, copy) warp pairs per sweep CTA, at most: as many as fit
constexpr size_t kSweepSmemCap = 231424; // dynamic shared memory a sweep CTA may take (the 227 KB opt-in less 1 KB)
constexpr int kRedBlock = 256;          // threads per reduction / stencil block
constexpr int kMaxCgBlocks = 1024;      // partials capacity of the fixed-order grid reductions
constexpr int kMaxLevels = 24;          // multigrid levels (2x2 aggregation down to one cell)
constexpr int kDirectMax = 64;          // cells of the multigrid level solved directly (grid solver)
constexpr int kMgBlock = 1024;          // threads per CTA of the synthetic-solve cluster

// device error bits (Status::error)
constexpr int kErrTimeout = 1;
constexpr int kErrBadInput = 2;

// why the iteration stopped (Status::reason)
constexpr int kRunning = 0;
constexpr int kConverged = 1;
constexpr int kFixedDone = 2;
constexpr int kMaxIter = 3;
constexpr int kDiverged = 4;

// Device-resident control block.
struct Status {
    unsigned int sweep_tasks;         // sweep unit counter (re-armed by each launch's last warp)
    unsigned int sweep_exits;         // sweep warps that have left (same)
    unsigned int sweep_arrived;       // sweep CTAs that have started (same)
    int sweep_mode;                   // sweep unit placement of the running launch (same)
    unsigned int ticket;              // last-block ticket of the Err reduction
    int error;                        // kErr* bits
    int done;                         // != 0: iteration finished, later kernels return at once
    int reason;                       // k* reason code
    int iter;                         // iterations completed
    int synth_iters;                  // synthetic solve iterations (last solve)
    long long synth_iters_total;      // summed over the solve
    double err;                       // last Err(rho)
    double synth_relres;              // last synthetic relative residual
    unsigned int mg_bar[2];           // grid-wide synthetic solver barrier word ([0]; [1] unused)
};

// Multigrid hierarchy of the synthetic operator (level 0 = the mesh).
struct MgPlan {
    int nl, local_from, cluster;
    int nx[kMaxLevels], ny[kMaxLevels];
    double* d64[kMaxLevels]; double* cx64[kMaxLevels]; double* cy64[kMaxLevels];
    float* d[kMaxLevels]; float* cx[kMaxLevels]; float* cy[kMaxLevels];
    float* x[kMaxLevels]; float* t[kMaxLevels]; float* r[kMaxLevels];
    float* r0; float* dl; float* s; float* p; float* q;
    int direct;      // first level of at most kDirectMax cells (-1: none)
    float* cinv;     // its operator's inverse, row-major, FP32 (kDirectMax^2 floats)
};

// Everything a kernel needs, carved from the caller's workspace (device
// pointers) plus the sizes.  Sorted direction index s: quadrant-major
// ((+,+), (-,+), (+,-), (-,-)), original order inside a quadrant.
struct Plan {
    int nx, ny, N, K, nb, nbf;      // nb = ceil(ny/32) row bands
    int fp32;                       // sweep precision
    int pt;                         // pseudo-time shift on
    int scheme;
    double tol;
    int max_iter, fixed_iters;
    double synth_rtol;
    int synth_max_iter;
    long long wait_cycles;
    int num_sms;
    int sweep_grid;                 // persistent sweep CTAs
    int cg_grid;                    // cooperative synthetic CTAs
    int red_grid;                   // per-cell kernels' CTAs (Err reduction partial count)
    double shift0;                  // 1/(c dt) added to the kinetic diagonal (time step; 0 when steady)
    int order;                      // kinetic face values: 1 first-order upwind, 2 second-order (delta form)
    int limiter;                    // order 2: 0 Barth-Jespersen, 1 none
    int synth_cl;                   // synthetic solver: strip-solver cluster size, 0 = global-memory solver
    int synth_grid;                 // global-memory solver over a cooperative grid of this many CTAs (0: one cluster)
    int synth_tiled;                // that grid solver in its tiled form (levels in per-CTA blocks)
    double* mg_gslots_d; float* mg_gslots_f;   // its reduction slots [3][2][kMaxCgBlocks]
    size_t synth_bytes;             // its dynamic shared memory

    // mesh
    const double* dx; const double* dy;
    // quadrature, sorted order
    const double* qmu; const double* qeta; const double* qw;
    const double* omu; const double* oeta; const double* ow;   // original order
    const int* perm;                // s -> original k
    const int* sidx;                // original k -> s
    const int* mpair;               // [K/2][2] original k of the x-reflection pairs (mu, eta), (-mu, eta), equal w
    int has_mpair;                  // the quadrature has such pairs: moments take the paired sums
    // per-direction coefficients |mu_s|/dx_i [K][nx], |eta_s|/dy_j [K][ny]
    const double* acoef; const double* bcoef;
    const float* acoef_f; const float* bcoef_f;
    const double* rsw;              // FP64: 1/d in sweep order [K][nb][nx+31][32]
    void* I;                        // [K][N] T, intensities of the last sweep (sorted s)
    void* In;                       // [K][N] T, intensities of the previous time step (time-dependent only)
    void* edge;                     // [K][nb][nx] T, last row of each band (all-ones bytes = not yet written)
    // cell data
    const double* sigma_a; const double* sigma_s; const double* q; const double* inflow;
    double* sigt; float* sigt_f;
    double* shift; float* shift_f;
    double* src; float* src_f;      // source of the next sweep (with pseudo-time correction)
    double* X;                      // [K][N] FP64 pseudo-time solve: src + shift I^m per ordinate (or null)
    float* X_f;                     // [K][N] FP32 time step: src + I^n/(c dt) per ordinate (or null)
    double* rho_m;                  // rho^m
    double* rho_h;                  // rho^{m+1/2}
    double* Fx; double* Fy; double* fb;
    // synthetic
    double* diag; double* cx; double* cy;
    double* hw;                     // [4][N] HoT gradient weights E, W, N, S (with 1/(3 sigma_t))
    double* bface;                  // [nbf] boundary face area * beta
    double* hotx; double* hoty; double* b;
    double* x; double* r; double* z; double* p; double* qv;
    const double* q_syn;            // volume source of the synthetic equation if not q (time step)
    // second-order upwind (order 2): residual, isotropic correction of the stored I, gradient weights
    void* R;                        // [K][N] T, residual per unit volume of the UW2 equations
    double* corr; float* corr_f;    // I^m = I + corr (per cell; FP32 copy for the FP32 sweep)
    double* gw; float* gw_f;        // [4][N] least-squares weights of I: E, W, N, S
    float* sigt_d;                  // FP32 sweep: sigma_t + pseudo-time shift (increment diagonal)
    double* partials;               // reductions scratch
    double* hist;                   // [max_iter]
    Status* status;
    MgPlan mg;
    // adjoint (allocated by the adjoint layout only)
    void* Iadj;                     // [K][N] T, transposed-sweep solutions (index: the swept, reflected direction)
    double* adj_a; double* adj_x; double* adj_y;      // adjoint moments: rho_bar_1/2, F_bar_x, F_bar_y
    float* adj_a_f; float* adj_x_f; float* adj_y_f;   // FP32 copies (FP32 sweep)
    double* adj_inflow;             // [nbf][K] adjoint of the boundary flux, as an inflow of the transposed sweep
    double* lam;                    // lam = D nu (adjoint of rho)
    double* nu;                     // nu (adjoint of the synthetic equation)
    const double* g;                // dJ/drho (caller's device array)
    int* refl;                      // [K] sorted index of the reflected direction
    const float* adj_sigt_f;        // FP32 transposed sweep: its diagonal sigma_t (+ 1/(c dt)); sigt_f when null
    const double* adj_rb_extra;     // per-cell term added to rho_bar_1/2 (time step adjoint), or null
    const double* adj_sig;          // scattering coefficient of the adjoint update; sigma_s when null
    // time-dependent radiation-material problem (allocated by the time-step layout only)
    struct {
        double* rho_n; double* T_n;     // state at t^n
        double* T;                      // current material temperature T^m
        double* cn;                     // isotropic correction of I^n (I^n = In + cn), per cell
        double* cnext;                  // the correction of the current iterate (becomes cn)
        double* qeff;                   // volume source of the synthetic equation
        double* diag0;                  // synthetic diagonal without the time and coupling terms
        double* hr1; double* hr2;       // rho of the previous two steps (predictor history)
        double* ht1; double* ht2;       // T of the previous two steps
        double* ckap; double* cphi; double* cf;   // kappa, phi, f at T^m (coefficient -> material update)
    } td;
};

// ------------------------------------------------------------ launchers
cudaError_t launch_setup(const Plan& P, cudaStream_t st);          // per-direction coefficients
cudaError_t launch_cell_setup(const Plan& P, double cfl_p, double beta,
                              cudaStream_t st);                    // sigma_t, shift, D, 1/d table, checks
cudaError_t launch_init_state(const Plan& P, cudaStream_t st);     // rho^0 = 0, I^0 = 0, sources
cudaError_t launch_sweep(Plan& P, cudaStream_t st);                // kinetic step (sweep)
cudaError_t launch_moments_to(const Plan& P, bool with_F, bool with_P, double* rho_out, double* Fout,
                              double* Pout, bool gsis_correct, double* fb_out, bool force,
                              cudaStream_t st);                    // rho, F, (P), boundary flux
cudaError_t prepare_kernels(int K, int fp32, int pt);
int sweep_max_active_blocks(int fp32, int pt);
cudaError_t launch_source_from(const Plan& P, const double* rho_in, cudaStream_t st);
// HoT, right-hand side b and the first residual b - D guess of the synthetic
// solve (FP32 copy in mg.r0, norms at partials + 4 * kMaxCgBlocks).
// fuse: one launch that forms HoT inside the right-hand side (hotx / hoty
// are then not written); the two-launch form for the batched, time-dependent
// and single-step paths (faster there, or hotx wanted)
cudaError_t launch_hot_rhs(const Plan& P, const double* rho_h, const double* Fx, const double* Fy,
                           const double* fb, const double* guess, cudaStream_t st, bool fuse = false);
cudaError_t launch_mg_setup(const Plan& P, cudaStream_t st);
int mg_setup_launches(const Plan& P);   // kernels launch_mg_setup launches
cudaError_t plan_synthetic(Plan& P);   // before the first solve launch (no runtime calls in the launch)
cudaError_t launch_synthetic_solve(const Plan& P, const double* guess, double* out, cudaStream_t st);
int mg_cluster_size();
cudaError_t launch_update(const Plan& P, const double* rho_new, cudaStream_t st);
// X = src + shift I per ordinate from the current src and I (after every
// update of the FP64 pseudo-time solve; skipped once the solve has stopped).
cudaError_t launch_ordinate_source(const Plan& P, cudaStream_t st);
// second-order upwind (csrc/uw2.cu, sweep in csrc/sweep.cu)
cudaError_t launch_uw2_residual(const Plan& P, cudaStream_t st);     // R from I + corr and the source
cudaError_t launch_delta_sweep(Plan& P, cudaStream_t st);           // I <- I + corr + dI
cudaError_t launch_uw2_bflux(const Plan& P, double* fb_out, const int* done, cudaStream_t st);
// adjoint (csrc/adjoint.cu, sweep in csrc/sweep.cu)
cudaError_t launch_adjoint_sweep(Plan& P, cudaStream_t st);
cudaError_t launch_synth_resid(const Plan& P, const double* b, const double* guess, cudaStream_t st);
cudaError_t launch_adjoint_rhs(const Plan& P, const double* nu_new, cudaStream_t st);   // nu, h_bar, rho_bar, inflow
cudaError_t launch_adjoint_update(const Plan& P, cudaStream_t st);
cudaError_t launch_adjoint_gradient(const Plan& P, double* grad_sa, double* grad_ss, cudaStream_t st);
// Pseudo-time-form sweep with the given per-cell source, stored intensities
// and output (no inflow): out_s = A_s^{-1}(src + shift iold_s).
cudaError_t launch_sweep_pt_into(Plan& P, const void* src, const void* iold, void* out, cudaStream_t st);

// Adjoint of one backward-Euler step of the time-dependent GSIS run (the
// vectors of the step and of its carry to the previous step).
struct TdAdjVecs {
    const double* T;            // T of the step's fixed point
    const double* diag0;        // synthetic diagonal without time and coupling terms
    double* sig_eff;            // sigma_s + (1 - f) sigma_a
    double* c0;                 // y_bar_rho + sigma_a y_bar_T / D2 (then + sig_eff/4pi sum chi)
    double* rb_extra;           // -(1/(c dt)) sum_k phi'_k / 4pi
    double* ybar_rho; double* ybar_T; double* sphi;   // carry: adjoints of rho^n, T^n; sum_k phi_k
    const void* chi;            // [K][N] T, transposed solve of the carried intensities (null: zero)
    void* carry;                // [K][N] T, phi of the step (out)
    double inv_cdt, ac, cv_dt;
};
cudaError_t launch_td_adjoint_setup(const Plan& P, const TdAdjVecs& v, cudaStream_t st);   // D', sig_eff, c0, rb_extra
cudaError_t launch_td_adjoint_start(const Plan& P, const TdAdjVecs& v, cudaStream_t st);   // c, lam = b = c
cudaError_t launch_td_adjoint_gradient(const Plan& P, const TdAdjVecs& v, double* grad_sa, double* grad_ss,
                                       cudaStream_t st);   // accumulate, carry, next y_bar

// ------------------------------------------------------------ batches
// Device tables of a batched solve (every problem's arguments of one
// iteration, built once); problem p of a per-block table owns blocks
// [bstart[p], bstart[p + 1]).
struct BatchTables {
    int B, fp32, pt, with_F, maxK;
    Status* status;                 // the launch-level sweep counters and error bits
    long long wait_cycles;
    // sweep: SweepArgs<T>[B] and the unit segments (one band of one problem each)
    const void* sweep;
    const int* seg_start; const int* seg_prob; const int* seg_band;
    int nseg, ntasks, sweep_grid;
    int dynamic;                    // 1: units from the counter even when the grid is resident
    // moments and boundary fluxes, HoT, right-hand side, update
    const void* mom; const int* mom_bstart; int mom_blocks;
    const void* hot; const int* hot_bstart; int hot_blocks;
    const void* rhs; const int* rhs_bstart; int rhs_blocks;
    const void* upd; const int* upd_bstart; int upd_blocks;
    // FP32 pseudo-time: the sweeps' per-ordinate sources (or ord_blocks = 0)
    const void* ord; const int* ord_bstart; int ord_blocks;
};

size_t sweep_batch_rec_bytes(int fp32);
void sweep_batch_rec(const Plan& P, void* out);
cudaError_t launch_sweep_batch(const BatchTables& bt, cudaStream_t st);
size_t mom_batch_rec_bytes(int fp32);
int mom_batch_rec(const Plan& P, bool with_F, void* out);
cudaError_t launch_moments_batch(const BatchTables& bt, cudaStream_t st);
size_t hot_batch_rec_bytes();
size_t rhs_batch_rec_bytes();
size_t upd_batch_rec_bytes();
int hot_batch_rec(const Plan& P, void* out);
int rhs_batch_rec(const Plan& P, void* out);
int upd_batch_rec(const Plan& P, bool gsis, void* out);
cudaError_t launch_hot_rhs_batch(const BatchTables& bt, cudaStream_t st);
cudaError_t launch_update_batch(const BatchTables& bt, cudaStream_t st);
size_t ord_batch_rec_bytes();
int ord_batch_rec(const Plan& P, void* out);
cudaError_t launch_ordsrc_batch(const BatchTables& bt, cudaStream_t st);
size_t strip_batch_rec_bytes();
bool strip_batch_rec(const Plan& P, int cl, void* out, size_t* bytes);
bool prepare_strip_batch(int cl, size_t bytes);
cudaError_t launch_strip_batch(const void* tab, int n, int cl, size_t bytes, cudaStream_t st);

int device_sm_count();
void set_last_error(int code, const char* msg);   // message returned by gsis_last_error()

// ------------------------------------------------------------ device helpers
#ifdef __CUDACC__
__device__ __forceinline__ int ld_volatile_int(const int* p)
{
    return *reinterpret_cast<const volatile int*>(p);
}

__device__ __forceinline__ unsigned smem_addr(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

// mbarrier in shared memory (arrive: release, wait: acquire, CTA scope)
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* b)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(b))
                 : "memory");
}

// Arrival on b once every cp.async this thread issued so far has landed
// (the arrival is counted in the barrier's expected count).
__device__ __forceinline__ void cp_async_mbar_arrive(unsigned long long* b)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(b)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_addr(b)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Waits (bounded by `limit` clock cycles) for the phase of parity `parity`
// to complete; false when the bound is hit.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity, long long limit)
{
    if (mbar_try_wait(b, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try_wait(b, parity)) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// Fixed-order block sum of one double per thread (blockDim.x multiple of 32,
// <= 1024).  Result valid in every thread.  `sm` holds >= 33 doubles.
__device__ __forceinline__ double block_sum(double v, double* sm)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    __syncthreads();
    if (lane == 0) sm[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double t = lane < nw ? sm[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
        if (lane == 0) sm[32] = t;
    }
    __syncthreads();
    return sm[32];
}

// Largest i in [0, n) with start[i] <= x (start ascending, start[0] <= x):
// the problem (or segment) of block / unit x in a batched launch.
__device__ __forceinline__ int batch_find(const int* __restrict__ start, int n, int x)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(start + mid) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Fixed-order sum of n doubles by one warp; identical result in all lanes.
__device__ __forceinline__ double warp_sum_array(const double* a, int n);

// Err(rho) = sqrt(sum num / sum den) over the nblk blocks of one problem
// (fixed-order partials, last-block ticket), its history entry and the stop
// decision.  Called by every thread of the block with its block sums.
__device__ __forceinline__ void err_reduce_decide(double num, double den, double* partials, double* hist,
                                                  Status* S, double tol, int fixed_iters, int max_iter, int bid,
                                                  int nblk, int* am_last)
{
    if (threadIdx.x == 0) {
        partials[bid] = num;
        partials[nblk + bid] = den;
        __threadfence();
        const unsigned t = atomicAdd(&S->ticket, 1u);
        *am_last = (t == (unsigned)nblk - 1u);
    }
    __syncthreads();
    if (!*am_last) return;
    if (threadIdx.x < 32) {
        __threadfence();
        const double sn = warp_sum_array(partials, nblk);
        const double sd = warp_sum_array(partials + nblk, nblk);
        if (threadIdx.x == 0) {
            double err;
            if (sd > 0.0) err = sqrt(sn / sd);
            else err = (sn == 0.0) ? 0.0 : INFINITY;
            const int it = S->iter;
            hist[it] = err;
            S->iter = it + 1;
            S->err = err;
            int reason = kRunning;
            if (!isfinite(err) || err > 1e6) reason = kDiverged;
            else if (fixed_iters > 0) { if (it + 1 >= fixed_iters) reason = kFixedDone; }
            else if (err < tol) reason = kConverged;
            else if (it + 1 >= max_iter) reason = kMaxIter;
            if (reason != kRunning) {
                S->reason = reason;
                S->done = 1;
            }
            S->ticket = 0u;
        }
    }
}

__device__ __forceinline__ double warp_sum_array(const double* a, int n)
{
    const int lane = threadIdx.x & 31;
    double t = 0.0;
    for (int i = lane; i < n; i += 32) t += __ldcg(a + i);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
    return t;
}
#endif

}  // namespace gsis
