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
constexpr int kMaxSide = (1 << 20) - 1; // cells per mesh side (edge-flag encoding)
constexpr int kSweepWarps = 4;          // warps per sweep CTA
constexpr int kRedBlock = 256;          // threads per reduction / stencil block
constexpr int kMaxCgBlocks = 1024;      // partials capacity of the fixed-order grid reductions
constexpr int kMaxLevels = 24;          // multigrid levels (2x2 aggregation down to one cell)
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
    unsigned long long sweep_tasks;   // dynamic task counter of the sweep (zeroed after each sweep)
    unsigned int ticket;              // last-block ticket of the Err reduction
    int error;                        // kErr* bits
    int done;                         // != 0: iteration finished, later kernels return at once
    int reason;                       // k* reason code
    int iter;                         // iterations completed
    int synth_iters;                  // synthetic solve iterations (last solve)
    long long synth_iters_total;      // summed over the solve
    double err;                       // last Err(rho)
    double synth_relres;              // last synthetic relative residual
};

// Multigrid hierarchy of the synthetic operator (level 0 = the mesh).
struct MgPlan {
    int nl, local_from, cluster;
    int nx[kMaxLevels], ny[kMaxLevels];
    double* d64[kMaxLevels]; double* cx64[kMaxLevels]; double* cy64[kMaxLevels];
    float* d[kMaxLevels]; float* cx[kMaxLevels]; float* cy[kMaxLevels];
    float* x[kMaxLevels]; float* t[kMaxLevels]; float* r[kMaxLevels];
    float* r0; float* dl; float* s; float* p; float* q;
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
    unsigned long long epoch;       // sweep launch counter (edge flags)

    // mesh
    const double* dx; const double* dy;
    // quadrature, sorted order
    const double* qmu; const double* qeta; const double* qw;
    const double* omu; const double* oeta; const double* ow;   // original order
    const int* perm;                // s -> original k
    const int* sidx;                // original k -> s
    // per-direction coefficients |mu_s|/dx_i [K][nx], |eta_s|/dy_j [K][ny]
    const double* acoef; const double* bcoef;
    const float* acoef_f; const float* bcoef_f;
    const double* rsw;              // FP64: 1/d in sweep order [K][nb][nx+31][32]
    void* I;                        // [K][N] T, intensities of the last sweep (sorted s)
    void* edge;                     // [K][nb][nx] T, top row of each band
    unsigned long long* flags;      // [K][nb] published edge columns
    // cell data
    const double* sigma_a; const double* sigma_s; const double* q; const double* inflow;
    double* sigt; float* sigt_f;
    double* shift; float* shift_f;
    double* src; float* src_f;      // source of the next sweep (with pseudo-time correction)
    double* rho_m;                  // rho^m
    double* rho_h;                  // rho^{m+1/2}
    double* Fx; double* Fy; double* fb;
    // synthetic
    double* diag; double* cx; double* cy;
    double* hotx; double* hoty; double* b;
    double* x; double* r; double* z; double* p; double* qv;
    double* partials;               // reductions scratch
    double* hist;                   // [max_iter]
    Status* status;
    MgPlan mg;
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
cudaError_t launch_hot_rhs(const Plan& P, const double* rho_h, const double* Fx, const double* Fy,
                           const double* fb, cudaStream_t st);
cudaError_t launch_mg_setup(const Plan& P, cudaStream_t st);
cudaError_t launch_synthetic_solve(const Plan& P, const double* guess, double* out, cudaStream_t st);
int mg_cluster_size();
cudaError_t launch_update(const Plan& P, const double* rho_new, cudaStream_t st);

int device_sm_count();
void set_last_error(int code, const char* msg);   // message returned by gsis_last_error()

// ------------------------------------------------------------ device helpers
#ifdef __CUDACC__
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_int(const int* p)
{
    return *reinterpret_cast<const volatile int*>(p);
}

// Waits (bounded by `limit` clock cycles) until *p >= target.  Returns false
// and raises kErrTimeout if the bound is hit, false if another CTA has
// already raised an error.
__device__ __forceinline__ bool wait_at_least(const unsigned long long* p, unsigned long long target,
                                              long long limit, int* err)
{
    const long long t0 = clock64();
    for (;;) {
        if (ld_acquire_u64(p) >= target) return true;
        if (ld_volatile_int(err)) return false;
        if (clock64() - t0 > limit) {
            atomicOr(err, kErrTimeout);
            return false;
        }
        __nanosleep(32);
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

// Fixed-order sum of n doubles by one warp; identical result in all lanes.
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
