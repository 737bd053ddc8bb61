// Kinetic step of SI / GSIS: the first-order-upwind discrete-ordinate sweep
// (Sec. 4.1, Eqs. (RTE_d), (Iij) with psi = 0, Eq. (RTE_SI) steady) and its
// angular moments (Eqs. (def_rho), (def_F), (RTE_M0)), plus the per-problem
// set-up of the coefficients every iteration reuses.
//
// Sweep layout.  Work unit = (direction s, band of 32 rows).  A warp owns one
// unit: lane l owns row 32*band + l (counted from the upwind wall) and walks
// the row from the upwind wall, one cell per step, lane l lagging lane l-1 by
// one step, so the upwind south value is the value lane l-1 produced one step
// earlier (one warp shuffle) and the upwind west value is the lane's own
// previous result (a register).  Lane 0 takes its south value from the band
// below (its last-row results, handed over value by value through a global
// row whose slots read "unwritten" until stored) or from the inflow on the
// first band.  Each compute warp is paired with a copy warp that stages the
// cell data of the coming steps in shared memory and fetches the south
// values, so the compute warp touches global memory only to store results.
// Every wait is bounded and reports kErrTimeout instead of hanging.
//
// All intensities of the last sweep stay in HBM as I[s][cell] (needed by the
// moment reduction, the pseudo-time delta form of Sec. 4.3 and the final
// second moment).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "gsis_internal.cuh"

namespace gsis {

namespace {

constexpr double kInvFourPi = 0.079577471545947667884441881686257;   // 1 / (4 pi)

// --------------------------------------------------------------- set-up
// |mu_s|/dx_i and |eta_s|/dy_j per sorted direction (both precisions).
__global__ void coef_kernel(int nx, int ny, int K, const double* __restrict__ dx,
                            const double* __restrict__ dy, const double* __restrict__ qmu,
                            const double* __restrict__ qeta, double* acoef, double* bcoef,
                            float* acoef_f, float* bcoef_f)
{
    const int tot_a = K * nx, tot = K * (nx + ny);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
        if (t < tot_a) {
            const int s = t / nx, i = t - s * nx;
            const double v = fabs(qmu[s]) / dx[i];
            acoef[t] = v;
            if (acoef_f) acoef_f[t] = (float)v;
        } else {
            const int u = t - tot_a;
            const int s = u / ny, j = u - s * ny;
            const double v = fabs(qeta[s]) / dy[j];
            bcoef[u] = v;
            if (bcoef_f) bcoef_f[u] = (float)v;
        }
    }
}

// Per cell: sigma_t, pseudo-time shift (Eqs. (cfl_pse), (tau_pse),
// dx_ref = min(dx_i, dy_j)), the finite-volume synthetic operator
// (Eqs. (elem_mtx_M), (Gamma_ij_com2) on the Cartesian mesh:
// Gamma = 2 / (3 (sigma_i h_i + sigma_j h_j)); boundary
// beta = 2/(3 sigma_i h_i) + 1/4 from Eq. (macro_bc_delta_flux)), input checks
// (opacities, sources and inflow finite; opacities non-negative).
__global__ void cell_setup_kernel(int nx, int ny, const double* __restrict__ dx,
                                  const double* __restrict__ dy, const double* __restrict__ sa,
                                  const double* __restrict__ ss, const double* __restrict__ q,
                                  const double* __restrict__ inflow, int n_inflow,
                                  double shift0, double cfl_p, double beta, double* sigt, float* sigt_f,
                                  double* shift, float* shift_f, double* diag, double* cx,
                                  double* cy, double* hw, double* bface, double* gw, float* gw_f,
                                  float* sigt_d, int* err)
{
    const int N = nx * ny;
    if (inflow)
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_inflow; t += gridDim.x * blockDim.x)
            if (!isfinite(inflow[t])) atomicOr(err, kErrBadInput);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const int j = c / nx, i = c - j * nx;
        const double a = sa[c], s = ss[c], st = a + s;
        if (!(a >= 0.0) || !(s >= 0.0) || !(st > 0.0) || !isfinite(st) || !isfinite(q[c]))
            atomicOr(err, kErrBadInput);
        sigt[c] = st;
        if (sigt_f) sigt_f[c] = (float)st;
        const double hx = dx[i], hy = dy[j];
        // neighbour optical distances |sigma_i r^L - sigma_j r^R|
        double th = 0.0;
        double gE = 0.0, gW = 0.0, gN = 0.0, gS = 0.0;
        if (i + 1 < nx) {
            const double o = 0.5 * (st * hx + (sa[c + 1] + ss[c + 1]) * dx[i + 1]);
            th = fmax(th, o);
            gE = 1.0 / (3.0 * o);
        }
        if (i > 0) {
            const double o = 0.5 * (st * hx + (sa[c - 1] + ss[c - 1]) * dx[i - 1]);
            th = fmax(th, o);
            gW = 1.0 / (3.0 * o);
        }
        if (j + 1 < ny) {
            const double o = 0.5 * (st * hy + (sa[c + nx] + ss[c + nx]) * dy[j + 1]);
            th = fmax(th, o);
            gN = 1.0 / (3.0 * o);
        }
        if (j > 0) {
            const double o = 0.5 * (st * hy + (sa[c - nx] + ss[c - nx]) * dy[j - 1]);
            th = fmax(th, o);
            gS = 1.0 / (3.0 * o);
        }
        const double ref = fmin(hx, hy);
        double sh = shift0;   // 1/(c dt) of a time step (0 when steady)
        if (cfl_p > 0.0) sh += 1.0 / (cfl_p * ref);
        if (beta > 0.0) sh += th / (beta * ref);
        shift[c] = sh;
        if (shift_f) shift_f[c] = (float)sh;
        if (sigt_d) sigt_d[c] = (float)(st + sh);
        // D = V sigma_a + sum_int A Gamma + sum_bnd A beta
        double d = hx * hy * a + hy * (gE + gW) + hx * (gN + gS);
        const double bx = 2.0 / (3.0 * st * hx) + 0.25, by = 2.0 / (3.0 * st * hy) + 0.25;
        if (i == 0) d += hy * bx;
        if (i == nx - 1) d += hy * bx;
        if (j == 0) d += hx * by;
        if (j == ny - 1) d += hx * by;
        diag[c] = d;
        cx[c] = hy * gE;
        cy[c] = hx * gN;
        // adaptive least-squares gradient on the Cartesian mesh (Eqs. (shifted_j),
        // (new_vector), (LSF_mdf)): G_x = sum_{E,W} d_j (rho_j - rho_i) / sum d_j^2
        // with d_E = +(hx/2 + (sigma_E/sigma_i) dx_E/2), d_W = -(...); the weights
        // d_j / sum d^2 carry the 1/(3 sigma_t) of the high-order terms (Eq. (GSIS_HoT))
        {
            double dE = 0.0, dW = 0.0, dN = 0.0, dS = 0.0;
            if (i + 1 < nx) dE = 0.5 * hx + ((sa[c + 1] + ss[c + 1]) / st) * 0.5 * dx[i + 1];
            if (i > 0) dW = -(0.5 * hx + ((sa[c - 1] + ss[c - 1]) / st) * 0.5 * dx[i - 1]);
            if (j + 1 < ny) dN = 0.5 * hy + ((sa[c + nx] + ss[c + nx]) / st) * 0.5 * dy[j + 1];
            if (j > 0) dS = -(0.5 * hy + ((sa[c - nx] + ss[c - nx]) / st) * 0.5 * dy[j - 1]);
            const double inv3s = 1.0 / (3.0 * st);
            const double sx = dE * dE + dW * dW, sy = dN * dN + dS * dS;
            const double fx = sx > 0.0 ? inv3s / sx : 0.0, fy = sy > 0.0 ? inv3s / sy : 0.0;
            hw[c] = dE * fx;
            hw[N + c] = dW * fx;
            hw[2 * N + c] = dN * fy;
            hw[3 * N + c] = dS * fy;
            if (gw) {   // the same least-squares gradient for the intensities (no 1/(3 sigma_t))
                const double gx = sx > 0.0 ? 1.0 / sx : 0.0, gy = sy > 0.0 ? 1.0 / sy : 0.0;
                const double g4[4] = {dE * gx, dW * gx, dN * gy, dS * gy};
                for (int t = 0; t < 4; ++t) {
                    gw[(size_t)t * N + c] = g4[t];
                    if (gw_f) gw_f[(size_t)t * N + c] = (float)g4[t];
                }
            }
        }
        // boundary faces: area * beta (Eq. (macro_bc_delta_flux)), faces W, E, S, N
        if (i == 0) bface[j] = hy * bx;
        if (i == nx - 1) bface[ny + j] = hy * bx;
        if (j == 0) bface[2 * ny + i] = hx * by;
        if (j == ny - 1) bface[2 * ny + nx + i] = hx * by;
    }
}

// 1 / (sigma_t + shift + |mu|/dx + |eta|/dy) in sweep order (FP64 sweep).
__global__ void recip_kernel(int nx, int ny, int K, int nb, const int* __restrict__ perm,
                             const double* __restrict__ qmu, const double* __restrict__ qeta,
                             const double* __restrict__ acoef, const double* __restrict__ bcoef,
                             const double* __restrict__ sigt, const double* __restrict__ shift,
                             double* rsw)
{
    const int ns = nx + 31;
    const size_t tot = (size_t)K * nb * ns * 32;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot;
         t += (size_t)gridDim.x * blockDim.x) {
        const int lane = (int)(t & 31);
        size_t u = t >> 5;
        const int step = (int)(u % ns);
        u /= ns;
        const int band = (int)(u % nb);
        const int s = (int)(u / nb);
        const int c = step - lane, jl = band * 32 + lane;
        double v = 0.0;
        if (c >= 0 && c < nx && jl < ny) {
            const int i = qmu[s] >= 0.0 ? c : nx - 1 - c;
            const int j = qeta[s] >= 0.0 ? jl : ny - 1 - jl;
            const int cell = i + nx * j;
            v = 1.0 / (sigt[cell] + shift[cell] + acoef[(size_t)s * nx + i] + bcoef[(size_t)s * ny + j]);
        }
        rsw[t] = v;
    }
}

__global__ void fill_kernel(double* a, size_t n, double v)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        a[t] = v;
}

__global__ void fillf_kernel(float* a, size_t n, float v)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        a[t] = v;
}

// Angular source of the next sweep from rho (Eq. (RTE_SI)):
// src = (sigma_s rho + q)/4pi  (no pseudo-time correction; used by the
// stand-alone kinetic step and at start-up).
__global__ void source_kernel(int N, const double* __restrict__ ss, const double* __restrict__ q,
                              const double* __restrict__ rho, double* src, float* src_f)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const double v = (ss[c] * rho[c] + q[c]) * kInvFourPi;
        src[c] = v;
        if (src_f) src_f[c] = (float)v;
    }
}

// --------------------------------------------------------------- sweep
// Source of the sweep: isotropic (plain), isotropic plus the pseudo-time
// term shift * I^m (delta form), or the adjoint source
// w_s (a - mu_s bx - eta_s by) of the transposed kinetic step.
// kSrcDelta: the increment sweep of the second-order upwind delta form
// (Eqs. (RTE_d_increment), (delta_Iij), (RTE_d_mtx)): source = the residual
// R[s][cell], zero increment on inflow faces, stored result I + corr + dI.
constexpr int kSrcPlain = 0, kSrcPseudoTime = 1, kSrcAdjoint = 2, kSrcDelta = 3;
// Windows per chunk buffer beyond the source (and the FP32 sigma_t): the
// pseudo-time, adjoint and increment forms read two per-cell/per-ordinate
// arrays more, the plain form none.  (A time-step form that read I^n and
// the per-cell source, one window more, with 1/(c dt) as a constant, was
// measured slower: 1024^2 S16 sweep 1.09 -> 1.92 ms against the 0.40 ms of
// the per-ordinate source pass it saved; the sweep is bound by its copy
// pipeline.)
__host__ __device__ constexpr int sweep_xw(int mode) { return mode == kSrcPlain ? 0 : 2; }

template <typename T>
struct SweepArgs {
    int nx, ny, N, K, nb, nsteps;
    const T* acoef; const T* bcoef;
    const double* rsw;
    const T* sigt; const T* shift; const T* src;
    int src_stride;             // elements between ordinates' sources (0: one per-cell source for all)
    const T* iold;              // stored intensities of the delta form: I^m (pseudo-time) or I^n (time step)
    const T* ax; const T* ay;   // adjoint source: bx, by (src holds a)
    const double* qw;           // sorted weights (adjoint source)
    T* I; T* edge;
    const double* inflow;
    const int* perm; const double* qmu; const double* qeta;
    int* err; const int* done;
    unsigned int* tasks;     // unit counter (band-major order)
    unsigned int* exits;     // warps that have left
    unsigned int* arrived;   // CTAs that have started
    int* mode;               // 0 undecided, 1 static placement, 2 counter
    long long wait_cycles;
};

// Several independent problems in one launch: unit u of the launch lies in
// segment g (seg_start[g] <= u < seg_start[g + 1]); a segment is one band of
// one problem, all K_p of its directions.  Within a problem the bands appear
// in increasing order, so a unit's upstream unit has the smaller index.
template <typename T>
struct SweepBatch {
    const SweepArgs<T>* probs;   // [B]
    const int* seg_start;        // [nseg + 1]
    const int* seg_prob;         // [nseg]
    const int* seg_band;         // [nseg]
    int nseg, ntasks;
    int dynamic;                 // 1: counter order even when the grid is resident
    unsigned int* tasks; unsigned int* exits; unsigned int* arrived; int* mode;
    int* err;                    // the launch's own error bits (a wait outside any unit)
    long long wait_cycles;
};

__device__ __forceinline__ double rcp_t(double d) { return 1.0 / d; }
__device__ __forceinline__ float rcp_t(float d) { return __frcp_rn(d); }

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(smem)), "l"(gmem), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Band hand-off slots hold the bit pattern "all ones" (a NaN that no
// arithmetic produces) until the upstream band writes the value.
template <typename T> struct Bits;
template <> struct Bits<double> {
    using U = unsigned long long;
    static constexpr U empty = ~0ull;
    static __device__ __forceinline__ U load(const double* p)
    {
        U v;
        asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p));
        return v;
    }
    static __device__ __forceinline__ void store(double* p, double v)
    {
        asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v));
    }
    static __device__ __forceinline__ double value(U u) { return __longlong_as_double((long long)u); }
    static __device__ __forceinline__ void clear(double* p) { *reinterpret_cast<U*>(p) = empty; }
    // plain store of a result; no compiler memory clobber, so the shared-memory
    // loads of the next steps may be issued ahead of it
    static __device__ __forceinline__ void put(double* p, double v)
    {
        asm volatile("st.global.f64 [%0], %1;" ::"l"(p), "d"(v));
    }
};
template <> struct Bits<float> {
    using U = unsigned int;
    static constexpr U empty = ~0u;
    static __device__ __forceinline__ U load(const float* p)
    {
        U v;
        asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p));
        return v;
    }
    static __device__ __forceinline__ void store(float* p, float v)
    {
        asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v));
    }
    static __device__ __forceinline__ float value(U u) { return __uint_as_float(u); }
    static __device__ __forceinline__ void clear(float* p) { *reinterpret_cast<U*>(p) = empty; }
    static __device__ __forceinline__ void put(float* p, float v)
    {
        asm volatile("st.global.f32 [%0], %1;" ::"l"(p), "f"(v));
    }
};

// Shared-memory plan of one (compute, copy) warp pair.  A chunk is SEG
// consecutive steps (64-byte row segments).  Each of the NBUF chunk buffers
// holds, for the lane's own row, the cell data of the SEG cells the lane
// updates in the chunk (padded rows: conflict-free column access), the
// column coefficients of the SEG + 31 columns the skewed lanes touch, the
// 1/d table rows of the chunk (FP64) and the SEG south values of lane 0.
template <typename T, int XW, bool PRE, bool WIDE = false>
struct SweepSmem {
    static constexpr int SEG = 64 / (int)sizeof(T);
    static constexpr int NBUF = 3;
    static constexpr int RS = SEG + 1;
    static constexpr int AW = SEG + 32;
    static constexpr int NW = (PRE ? 1 : 2) + XW;              // src, [sigt], [shift,] [I^m or I^n]
    static constexpr int W_SRC = 0;                           // window slots
    static constexpr int W_SIGT = 1;                          // FP32 only (no 1/d table)
    static constexpr int W_SHIFT = PRE ? 1 : 2;               // two extra windows only
    static constexpr int W_IOLD = (PRE ? 1 : 2) + (XW >= 2 ? 1 : 0);   // extra windows only
    static constexpr int WIN = 32 * RS;
    static constexpr size_t r16(size_t b) { return (b + 15) / 16 * 16; }
    static constexpr size_t off_r = r16(sizeof(T) * (size_t)NW * WIN);
    static constexpr size_t off_a = off_r + (PRE ? (size_t)SEG * 32 * sizeof(double) : 0);
    static constexpr size_t off_e = off_a + r16(sizeof(T) * (size_t)AW);
    static constexpr size_t off_h = off_e + r16(sizeof(T) * (size_t)SEG);   // unit index of the chunk
    static constexpr size_t buf_bytes = off_h + 16;
    static constexpr size_t bar_bytes = 64;                   // full[NBUF], empty[NBUF]
    static constexpr size_t pair_bytes = bar_bytes + NBUF * buf_bytes;
    // pairs per CTA: 8 (two chains per SM sub-partition), or in the WIDE
    // form as many as the shared memory holds up to kSweepMaxPairs (the
    // batched sweep: 64 problems 0.69 -> 0.55 ms; with staged write-out,
    // the FP64 sweep of a problem with many units, below)
    static constexpr size_t kFit = kSweepSmemCap / pair_bytes;
    static constexpr size_t kWant = WIDE ? (size_t)kSweepMaxPairs : (size_t)8;
    static constexpr int PAIRS = (int)(kFit < kWant ? kFit : kWant);
    static constexpr size_t bytes = PAIRS * pair_bytes;
    static_assert(PAIRS >= 4, "a sweep CTA needs at least one pair per sub-partition");
    static_assert(2 * NBUF * 8 <= bar_bytes, "barrier space");
};

// One persistent CTA per SM runs PAIRS warp pairs; a pair's copy warp
// chooses the units (direction s, band), u = band * K + s, and hands each to
// its compute warp in the header of the unit's first chunk buffer.  When the
// whole grid is resident (every CTA checks in within a few microseconds) the
// units are placed statically: pair p of CTA c takes u = p G + c + i PAIRS G, so
// each SM's first units come from different bands and run at different
// times; every unit is owned by a running pair and waits only on u - K.
// Otherwise (part of the grid held back by other work on the GPU) the pairs
// take units from a counter in increasing order, so a unit only waits on one
// that a running pair took earlier.  One atomic decision picks the mode for
// every CTA; the launch's last warp to leave re-arms the counters.
//
// Copy warp: for each chunk, cp.async of the window data into a free buffer
// (arrival on the buffer's "full" barrier when the copies land), then the
// south values of lane 0: the inflow on band 0, else the upstream band's
// last-row results, polled until written (bounded).  Compute warp: waits on
// "full", runs the SEG steps from shared memory, writes each result straight
// to I, and the last lane also to this band's hand-off row, then arrives on
// "empty".  Every wait is bounded; on time-out kErrTimeout is raised and the
// warp leaves after its copies in flight have landed.
template <typename T, int MODE, bool PRE, bool BATCH, bool WIDE = false>
__global__ void __launch_bounds__(SweepSmem<T, sweep_xw(MODE), PRE, BATCH || WIDE>::PAIRS * 64, 1)
sweep_kernel(const SweepArgs<T> a1, const SweepBatch<T> bt)
{
    constexpr bool PT = MODE == kSrcPseudoTime, ADJ = MODE == kSrcAdjoint, DELTA = MODE == kSrcDelta;
    // FP32 and the WIDE form: results collected in shared memory and written
    // out per chunk in coarser stores (fewer store instructions per step:
    // one 8-byte store per step touches 32 rows); the FP64 latency-bound
    // form writes each result at once (there the write-out would sit on the
    // band hand-off path: 256^2 S12 channel 0.127 -> 0.141 ms when staged)
    constexpr bool STAGE = sizeof(T) == 4 || WIDE;
    using SM = SweepSmem<T, sweep_xw(MODE), PRE, BATCH || WIDE>;
    using B = Bits<T>;
    constexpr int SEG = SM::SEG, NBUF = SM::NBUF, RS = SM::RS, NW = SM::NW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool copier = warp >= SM::PAIRS;
    const int pair = copier ? warp - SM::PAIRS : warp;
    unsigned char* pbase = smem_raw + (size_t)pair * SM::pair_bytes;
    unsigned long long* full = reinterpret_cast<unsigned long long*>(pbase);
    unsigned long long* empty = full + NBUF;
    auto buf = [&](int b) { return pbase + SM::bar_bytes + (size_t)b * SM::buf_bytes; };

    if (threadIdx.x < SM::PAIRS) {
        unsigned long long* f = reinterpret_cast<unsigned long long*>(smem_raw + (size_t)threadIdx.x * SM::pair_bytes);
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(f + b, 64);            // 32 cp.async arrivals + 32 lane arrivals
            mbar_init(f + NBUF + b, 32);     // 32 compute lanes
        }
    }
    __syncthreads();

    const int G = gridDim.x;
    const int ntasks = BATCH ? bt.ntasks : a1.K * a1.nb;
    const long long budget = BATCH ? bt.wait_cycles : a1.wait_cycles;
    unsigned* const c_tasks = BATCH ? bt.tasks : a1.tasks;
    unsigned* const c_exits = BATCH ? bt.exits : a1.exits;
    unsigned* const c_arrived = BATCH ? bt.arrived : a1.arrived;
    int* const c_mode = BATCH ? bt.mode : a1.mode;

    __shared__ int cta_mode;
    if (threadIdx.x == 0) {
        atomicAdd(c_arrived, 1u);
        const long long t0 = clock64();
        int m = 0;
        for (;;) {
            m = *reinterpret_cast<volatile int*>(c_mode);
            if (m != 0) break;
            if (*reinterpret_cast<volatile unsigned*>(c_arrived) >= (unsigned)G) atomicCAS(c_mode, 0, 1);
            else if (clock64() - t0 > 20000) atomicCAS(c_mode, 0, 2);
        }
        cta_mode = m;
    }
    __syncthreads();
    const bool placed = cta_mode == 1 && !(BATCH && bt.dynamic);

    unsigned g = 0;   // chunks this pair has handled (buffer = g % NBUF)
    int next_static = pair * G + (int)blockIdx.x;
    bool first = true;
    auto body = [&]() {
    if (!BATCH) {
        int stop = 0;
        if (lane == 0) stop = ld_volatile_int(a1.done) | ld_volatile_int(a1.err);
        if (__shfl_sync(kFull, stop, 0)) return;
    }
    for (;;) {
        int task, prob = 0, ltask;   // launch unit, its problem and the unit within the problem
        if (copier) {
            // next unit; -1: none left, or an error was raised.  In a batch the
            // units of a problem that has stopped (converged or failed) are skipped.
            int t = -1, pp = 0, lt = 0;
            if (lane == 0) {
                for (;;) {
                    if (placed) {
                        t = next_static;
                        next_static += SM::PAIRS * G;
                    } else {
                        if (first && pair >= SM::PAIRS / 2) {
                            // the second half of the pairs shares sub-partitions with the
                            // first half: let the first half take the first units, so that
                            // concurrently running units start on distinct sub-partitions
                            const unsigned want = min((unsigned)ntasks, (unsigned)(SM::PAIRS / 2) * (unsigned)G);
                            const long long t0 = clock64();
                            while (*reinterpret_cast<volatile unsigned*>(c_tasks) < want && clock64() - t0 < 20000)
                                __nanosleep(64);
                        }
                        first = false;
                        t = (int)atomicAdd(c_tasks, 1u);
                    }
                    if (t >= ntasks) { t = -1; break; }
                    if (!BATCH) {
                        if (ld_volatile_int(a1.err)) t = -1;
                        lt = t;
                        break;
                    }
                    const int sg = batch_find(bt.seg_start, bt.nseg, t);
                    pp = bt.seg_prob[sg];
                    const SweepArgs<T>& q = bt.probs[pp];
                    if (ld_volatile_int(q.done) | ld_volatile_int(q.err)) continue;
                    lt = bt.seg_band[sg] * q.K + (t - bt.seg_start[sg]);
                    break;
                }
            }
            task = __shfl_sync(kFull, t, 0);
            prob = __shfl_sync(kFull, pp, 0);
            ltask = __shfl_sync(kFull, lt, 0);
            first = false;
            if (task < 0) {   // end marker in the next buffer, then leave
                const int b = (int)(g % NBUF);
                if (g >= NBUF && !__all_sync(kFull, mbar_wait(empty + b, ((g / NBUF) - 1) & 1, budget))) {
                    if (lane == 0) atomicOr(BATCH ? bt.err : a1.err, kErrTimeout);
                    return;
                }
                if (lane == 0) *reinterpret_cast<volatile int*>(buf(b) + SM::off_h) = -1;
                cp_async_mbar_arrive(full + b);
                mbar_arrive(full + b);
                return;
            }
        } else {
            // the unit is in the header of its first chunk's buffer
            const int b = (int)(g % NBUF);
            if (!__all_sync(kFull, mbar_wait(full + b, (g / NBUF) & 1, budget))) {
                if (lane == 0) atomicOr(BATCH ? bt.err : a1.err, kErrTimeout);
                return;
            }
            const volatile int* h = reinterpret_cast<const volatile int*>(buf(b) + SM::off_h);
            task = h[0];
            if (task < 0) return;
            prob = h[1];
            ltask = h[2];
        }
        const SweepArgs<T>& a = BATCH ? bt.probs[prob] : a1;
        const int nx = a.nx, ny = a.ny, K = a.K, nb = a.nb, nsteps = a.nsteps;
        const int nchunks = (nsteps + SEG - 1) / SEG;
        const int band = ltask / K;
        const int s = ltask - band * K;
        const bool xpos = a.qmu[s] >= 0.0, ypos = a.qeta[s] >= 0.0;
        const int k = a.perm[s];
        const int jl = band * 32 + lane;
        const bool row_ok = jl < ny;
        const int j = ypos ? jl : ny - 1 - jl;
        T* Is = a.I + (size_t)s * a.N;
        // cell of (band row r, sweep column c) = base0 + r * dr + c * dc
        const bool full_rows = band * 32 + 32 <= ny;
        const int dr = ypos ? nx : -nx, dc = xpos ? 1 : -1;
        const int base0 = (ypos ? band * 32 : ny - 1 - band * 32) * nx + (xpos ? 0 : nx - 1);

        if (copier) {
            // ---------------------------------------------------- copy warp
            const T* wsrc[NW];
            wsrc[SM::W_SRC] = a.src + (size_t)s * a.src_stride;
            if (!PRE) wsrc[SM::W_SIGT] = a.sigt;
            if (PT) {
                wsrc[SM::W_SHIFT] = a.shift;
                wsrc[SM::W_IOLD] = a.iold + (size_t)s * a.N;
            }
            if (ADJ) {
                wsrc[SM::W_SHIFT] = a.ax;
                wsrc[SM::W_IOLD] = a.ay;
            }
            if (DELTA) {   // residual and stored intensity of this ordinate, correction per cell
                wsrc[SM::W_SRC] = a.src + (size_t)s * a.N;
                wsrc[SM::W_SHIFT] = a.shift;
                wsrc[SM::W_IOLD] = a.iold + (size_t)s * a.N;
            }
            const T* arow = a.acoef + (size_t)s * nx;
            const double* rrow = PRE ? a.rsw + ((size_t)s * nb + band) * (size_t)a.nsteps * 32 : nullptr;
            T* edge_in = band > 0 ? a.edge + ((size_t)s * nb + band - 1) * nx : nullptr;
            for (int m = 0; m < nchunks; ++m, ++g) {
                const int b = (int)(g % NBUF);
                if (g >= NBUF) {
                    const bool ok = __all_sync(kFull, mbar_wait(empty + b, ((g / NBUF) - 1) & 1, budget));
                    if (!ok) {
                        if (lane == 0) atomicOr(a.err, kErrTimeout);
                        cp_async_wait_all();
                        return;
                    }
                }
                unsigned char* bp = buf(b);
                T* wb = reinterpret_cast<T*>(bp);
                const int t0 = m * SEG;
                constexpr int RPI = 32 / SEG;   // rows per copy instruction
                const int kk = lane % SEG;
                if (full_rows && t0 >= 31 && t0 + SEG <= nx) {
                    // interior chunk: every row window lies inside the mesh
                    const int r = lane / SEG;
                    int cell = base0 + r * dr + (t0 + kk - r) * dc;
                    const int dcell = RPI * (dr - dc);
                    T* dst = wb + r * RS + kk;
#pragma unroll
                    for (int r0 = 0; r0 < 32; r0 += RPI) {
#pragma unroll
                        for (int w = 0; w < NW; ++w) cp_async<sizeof(T)>(dst + w * SM::WIN, wsrc[w] + cell);
                        cell += dcell;
                        dst += RPI * RS;
                    }
                    T* ab = reinterpret_cast<T*>(bp + SM::off_a);
                    for (int u = lane; u < SEG + 31; u += 32)
                        cp_async<sizeof(T)>(ab + u, arow + (xpos ? t0 - 31 + u : nx - 1 - (t0 - 31 + u)));
                } else {
                    // row r of the band needs columns t0 - r .. t0 - r + SEG - 1
#pragma unroll 4
                    for (int r0 = 0; r0 < 32; r0 += RPI) {
                        const int r = r0 + lane / SEG;
                        const int jr = band * 32 + r;
                        const int c = t0 + kk - r;
                        if (jr < ny && c >= 0 && c < nx) {
                            const size_t cell = (size_t)(ypos ? jr : ny - 1 - jr) * nx + (xpos ? c : nx - 1 - c);
#pragma unroll
                            for (int w = 0; w < NW; ++w) cp_async<sizeof(T)>(wb + w * SM::WIN + r * RS + kk, wsrc[w] + cell);
                        }
                    }
                    T* ab = reinterpret_cast<T*>(bp + SM::off_a);
                    for (int u = lane; u < SEG + 31; u += 32) {
                        const int c = t0 - 31 + u;
                        if (c >= 0 && c < nx) cp_async<sizeof(T)>(ab + u, arow + (xpos ? c : nx - 1 - c));
                    }
                }
                if (PRE) {
                    const int nv = min(SEG, nsteps - t0) * 32;   // doubles, multiple of 32
                    double* rb = reinterpret_cast<double*>(bp + SM::off_r);
                    for (int v = 2 * lane; v < nv; v += 64) cp_async<16>(rb + v, rrow + (size_t)t0 * 32 + v);
                }
                cp_async_mbar_arrive(full + b);
                // south values of lane 0 for columns t0 .. t0 + SEG - 1
                T ev = T(0);
                const bool need = lane < SEG && t0 + lane < nx;
                if (band == 0) {
                    if (need && a.inflow) {
                        const int c = t0 + lane;
                        const int i = xpos ? c : nx - 1 - c;
                        const int f = ypos ? 2 * ny + i : 2 * ny + nx + i;
                        ev = (T)a.inflow[(size_t)f * K + k];
                    }
                } else {
                    bool have = !need;
                    const long long start = clock64();
                    for (;;) {
                        if (!have) {
                            const typename B::U u = B::load(edge_in + t0 + lane);
                            if (u != B::empty) {
                                have = true;
                                ev = B::value(u);
                            }
                        }
                        if (__all_sync(kFull, have)) break;
                        if (__any_sync(kFull, clock64() - start > budget)) {   // warp-uniform exit
                            if (lane == 0) atomicOr(a.err, kErrTimeout);
                            cp_async_wait_all();
                            return;
                        }
                        __nanosleep(20);
                    }
                }
                if (lane < SEG) reinterpret_cast<T*>(bp + SM::off_e)[lane] = ev;
                if (lane == 0) {
                    volatile int* h = reinterpret_cast<volatile int*>(bp + SM::off_h);
                    h[0] = task;
                    h[1] = prob;
                    h[2] = ltask;
                }
                mbar_arrive(full + b);
            }
            // every value of the upstream hand-off row has been taken:
            // mark it unwritten for the next sweep
            if (band > 0)
                for (int c = lane; c < nx; c += 32) B::clear(edge_in + c);
        } else {
            // ------------------------------------------------- compute warp
            const T bj = row_ok ? a.bcoef[(size_t)s * ny + j] : T(0);
            T cw = T(0), cm = T(0), ce = T(0);   // adjoint source w (a - mu bx - eta by)
            if (ADJ) {
                const double ws = a.qw[s];
                cw = (T)ws;
                cm = (T)(-ws * a.qmu[s]);
                ce = (T)(-ws * a.qeta[s]);
            }
            T IW = T(0);
            if (row_ok && a.inflow) IW = (T)a.inflow[(size_t)(xpos ? j : ny + j) * K + k];
            T Iprev = T(0);
            T* eo = a.edge + ((size_t)s * nb + band) * nx;   // this band's last row, by column
            const bool put_edge = lane == 31 && band < nb - 1;
            for (int m = 0; m < nchunks; ++m, ++g) {
                const int b = (int)(g % NBUF);
                const bool ok = __all_sync(kFull, mbar_wait(full + b, (g / NBUF) & 1, budget));
                if (!ok) {
                    if (lane == 0) atomicOr(a.err, kErrTimeout);
                    return;
                }
                unsigned char* bp = buf(b);
                // the lane's row; with STAGE its source slots collect the results
                T* wb = reinterpret_cast<T*>(bp) + lane * RS;
                const T* ab = reinterpret_cast<const T*>(bp + SM::off_a) + 31 - lane;
                const double* rb = reinterpret_cast<const double*>(bp + SM::off_r) + lane;
                const T* ein = reinterpret_cast<const T*>(bp + SM::off_e);
                const int t0 = m * SEG;
                if (full_rows && t0 >= 31 && t0 + SEG <= nx) {
                    // interior chunk: every lane updates a cell at every step
                    T* Ic = Is + base0 + lane * dr + (t0 - lane) * dc;
                    T* ec = eo + (t0 - 31);
                    // the step's source, column coefficient and 1/d depend only on
                    // the chunk's data: they are formed one step ahead, so that
                    // only the two upwind FMAs and the 1/d multiply wait on the
                    // previous step
                    auto operands = [&](int tt, T& sv, T& ai, T& rinv) {
                        sv = wb[SM::W_SRC * SM::WIN + tt];
                        if (ADJ) sv = fma(cm, wb[SM::W_SHIFT * SM::WIN + tt], fma(ce, wb[SM::W_IOLD * SM::WIN + tt], cw * sv));
                        ai = ab[tt];
                        if (PRE) {
                            if (PT) sv = fma(wb[SM::W_SHIFT * SM::WIN + tt], wb[SM::W_IOLD * SM::WIN + tt], sv);
                            rinv = (T)rb[tt * 32];
                        } else {
                            T d = wb[SM::W_SIGT * SM::WIN + tt] + ai + bj;
                            if (PT) {
                                const T sh = wb[SM::W_SHIFT * SM::WIN + tt];
                                sv = fma(sh, wb[SM::W_IOLD * SM::WIN + tt], sv);
                                d += sh;
                            }
                            rinv = rcp_t(d);
                        }
                    };
                    T sv_n, ai_n, rinv_n;
                    operands(0, sv_n, ai_n, rinv_n);
#pragma unroll
                    for (int tt = 0; tt < SEG; ++tt) {
                        const T sv = sv_n, ai = ai_n, rinv = rinv_n;
                        if (tt + 1 < SEG) operands(tt + 1, sv_n, ai_n, rinv_n);
                        // lane l gets lane l-1's previous result; lane 0 the south value
                        const T e = ein[tt];
                        const T Isouth = __shfl_sync(kFull, lane == 31 ? e : Iprev, (lane + 31) & 31);
                        T acc = fma(ai, IW, sv);
                        acc = fma(bj, Isouth, acc);
                        const T Inew = acc * rinv;
                        IW = Inew;
                        Iprev = Inew;
                        const T out = DELTA ? (wb[SM::W_IOLD * SM::WIN + tt] + wb[SM::W_SHIFT * SM::WIN + tt]) + Inew : Inew;
                        if constexpr (STAGE) wb[SM::W_SRC * SM::WIN + tt] = out;   // the slot just read
                        else B::put(Ic + tt * dc, out);
                        if (put_edge) B::store(ec + tt, Inew);
                    }
                } else {
#pragma unroll 4
                    for (int tt = 0; tt < SEG; ++tt) {
                        const int t = t0 + tt;
                        if (t >= nsteps) break;
                        const T e = ein[tt];
                        const T Isouth = __shfl_sync(kFull, lane == 31 ? e : Iprev, (lane + 31) & 31);
                        const int c = t - lane;
                        T Inew = T(0);
                        if (row_ok && c >= 0 && c < nx) {
                            T sv = wb[SM::W_SRC * SM::WIN + tt];
                            if (ADJ) sv = fma(cm, wb[SM::W_SHIFT * SM::WIN + tt], fma(ce, wb[SM::W_IOLD * SM::WIN + tt], cw * sv));
                            const T ai = ab[tt];
                            T rinv;
                            if (PRE) {
                                if (PT) sv = fma(wb[SM::W_SHIFT * SM::WIN + tt], wb[SM::W_IOLD * SM::WIN + tt], sv);
                                    rinv = (T)rb[tt * 32];
                            } else {
                                T d = wb[SM::W_SIGT * SM::WIN + tt] + ai + bj;
                                if (PT) {
                                    const T sh = wb[SM::W_SHIFT * SM::WIN + tt];
                                    sv = fma(sh, wb[SM::W_IOLD * SM::WIN + tt], sv);
                                    d += sh;
                                }
                                rinv = rcp_t(d);
                            }
                            T acc = fma(ai, IW, sv);
                            acc = fma(bj, Isouth, acc);
                            Inew = acc * rinv;
                            IW = Inew;
                            const T out =
                                DELTA ? (wb[SM::W_IOLD * SM::WIN + tt] + wb[SM::W_SHIFT * SM::WIN + tt]) + Inew : Inew;
                            if constexpr (STAGE) wb[SM::W_SRC * SM::WIN + tt] = out;
                            else B::put(Is + base0 + lane * dr + c * dc, out);
                            if (put_edge) B::store(eo + c, Inew);
                        }
                        Iprev = Inew;
                    }
                }
                if constexpr (STAGE) {
                    // write the chunk's results out row by row: RPI rows of SEG
                    // consecutive cells per store instruction instead of one
                    // cell of each of 32 rows
                    __syncwarp();
                    constexpr int RPI = 32 / SEG;
                    const int kk = lane % SEG;
                    const T* stage = reinterpret_cast<const T*>(bp);
#pragma unroll 4
                    for (int r0 = 0; r0 < 32; r0 += RPI) {
                        const int r = r0 + lane / SEG;
                        const int c = t0 + kk - r;
                        if (band * 32 + r < ny && c >= 0 && c < nx)
                            B::put(Is + base0 + r * dr + c * dc, stage[r * RS + kk]);
                    }
                    __syncwarp();
                }
                mbar_arrive(empty + b);
            }
        }
    }
    };
    body();
    if (copier) cp_async_wait_all();
    // the launch's last warp to leave re-arms the counters for the next launch
    __syncwarp();
    if (lane == 0) {
        __threadfence();
        if (atomicAdd(c_exits, 1u) == (unsigned)G * (unsigned)(2 * SM::PAIRS) - 1u) {
            *c_tasks = 0u;
            *c_arrived = 0u;
            *c_mode = 0;
            *c_exits = 0u;
        }
    }
}

// --------------------------------------------------------------- moments
template <typename T>
struct MomArgs {
    int nx, ny, N, K;
    const T* I;
    const int* sidx;
    const double* mu; const double* eta; const double* w;   // original order
    double* rho; double* Fx; double* Fy;                    // may be null (F)
    double* Pxx; double* Pxy; double* Pyy;                  // may be null
    const double* rho_new;                                  // GSIS correction of P (or null)
    const int* done;
    const int* pairs;   // [K/2][2] x-reflection pairs (original k, the first with mu > 0), or null
};

// Per cell, in original direction order k = 0..K-1:
// rho = sum w I, F = sum w Omega I, P = sum w Omega Omega I.
template <typename T, bool WITH_F, bool WITH_P>
__device__ __forceinline__ void moments_body(const MomArgs<T>& a, int bid, int nblk)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* cf = reinterpret_cast<T*>(smem_raw);                     // [K][6]
    int* sk = reinterpret_cast<int*>(cf + 6 * a.K);             // [K]
    if (a.done && ld_volatile_int(a.done)) return;
    if (!WITH_P && a.pairs) {
        // Directions in x-reflection pairs k1 = (mu, eta), k2 = (-mu, eta)
        // with one weight: rho += w (I1 + I2), F_x += w mu (I1 - I2),
        // F_y += w eta (I1 + I2): five FP64 operations per pair instead of
        // six (the FP64 pipe bounds this kernel).
        const int np = a.K / 2;
        T* cp = cf;                                             // [np][3]: w, w mu, w eta of k1
        int* sp = reinterpret_cast<int*>(cf + 3 * np);          // [np][2]: sorted indices of k1, k2
        for (int p = threadIdx.x; p < np; p += blockDim.x) {
            const int k1 = a.pairs[2 * p], k2 = a.pairs[2 * p + 1];
            const double w = a.w[k1];
            cp[3 * p + 0] = (T)w;
            cp[3 * p + 1] = (T)(w * a.mu[k1]);
            cp[3 * p + 2] = (T)(w * a.eta[k1]);
            sp[2 * p] = a.sidx[k1];
            sp[2 * p + 1] = a.sidx[k2];
        }
        __syncthreads();
        for (int c = bid * blockDim.x + threadIdx.x; c < a.N; c += nblk * blockDim.x) {
            T r = T(0), fx = T(0), fy = T(0);
#pragma unroll 4
            for (int p = 0; p < np; ++p) {
                const T v1 = a.I[(size_t)sp[2 * p] * a.N + c];
                const T v2 = a.I[(size_t)sp[2 * p + 1] * a.N + c];
                const T sum = v1 + v2;
                r = fma(cp[3 * p + 0], sum, r);
                if (WITH_F) {
                    fx = fma(cp[3 * p + 1], v1 - v2, fx);
                    fy = fma(cp[3 * p + 2], sum, fy);
                }
            }
            if (a.rho) a.rho[c] = (double)r;
            if (WITH_F) {
                a.Fx[c] = (double)fx;
                a.Fy[c] = (double)fy;
            }
        }
        return;
    }
    for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
        const double w = a.w[k], m = a.mu[k], e = a.eta[k];
        cf[6 * k + 0] = (T)w;
        cf[6 * k + 1] = (T)(w * m);
        cf[6 * k + 2] = (T)(w * e);
        cf[6 * k + 3] = (T)(w * m * m);
        cf[6 * k + 4] = (T)(w * m * e);
        cf[6 * k + 5] = (T)(w * e * e);
        sk[k] = a.sidx[k];
    }
    __syncthreads();
    for (int c = bid * blockDim.x + threadIdx.x; c < a.N; c += nblk * blockDim.x) {
        T r = T(0), fx = T(0), fy = T(0), pxx = T(0), pxy = T(0), pyy = T(0);
#pragma unroll 4
        for (int k = 0; k < a.K; ++k) {
            const T v = a.I[(size_t)sk[k] * a.N + c];
            r = fma(cf[6 * k + 0], v, r);
            if (WITH_F) {
                fx = fma(cf[6 * k + 1], v, fx);
                fy = fma(cf[6 * k + 2], v, fy);
            }
            if (WITH_P) {
                pxx = fma(cf[6 * k + 3], v, pxx);
                pxy = fma(cf[6 * k + 4], v, pxy);
                pyy = fma(cf[6 * k + 5], v, pyy);
            }
        }
        if (a.rho) a.rho[c] = (double)r;
        if (WITH_F) {
            a.Fx[c] = (double)fx;
            a.Fy[c] = (double)fy;
        }
        if (WITH_P) {
            double dxx = (double)pxx, dyy = (double)pyy;
            if (a.rho_new) {   // moments of I + (rho_new - rho_half)/4pi: + drho/3 on the diagonal
                const double d = (a.rho_new[c] - (double)r) / 3.0;
                dxx += d;
                dyy += d;
            }
            a.Pxx[c] = dxx;
            a.Pxy[c] = (double)pxy;
            a.Pyy[c] = dyy;
        }
    }
}

// Kinetic net flux through every boundary face, sum_k w_k (Omega_k . n) I_face,k
// (outgoing: boundary cell intensity, incoming: inflow).  One warp per face;
// lane l sums k = l, l+32, ... in order, then a fixed shuffle tree.
template <typename T>
struct BfArgs {
    int nx, ny, K;
    const T* I;
    const int* sidx;
    const double* mu; const double* eta; const double* w;   // original order
    const double* inflow;
    double* fb;
    const int* done;
};

template <typename T>
__device__ __forceinline__ void bflux_body(const BfArgs<T>& a, int bid, int nblk)
{
    if (a.done && ld_volatile_int(a.done)) return;
    const int nx = a.nx, ny = a.ny, K = a.K;
    const int nbf = 2 * (nx + ny), N = nx * ny;
    const int lane = threadIdx.x & 31;
    const int warps = (nblk * blockDim.x) >> 5;
    for (int f = (bid * blockDim.x + threadIdx.x) >> 5; f < nbf; f += warps) {
        int c, axis;
        double sgn;
        if (f < ny) { c = nx * f; axis = 0; sgn = -1.0; }
        else if (f < 2 * ny) { c = nx - 1 + nx * (f - ny); axis = 0; sgn = 1.0; }
        else if (f < 2 * ny + nx) { c = f - 2 * ny; axis = 1; sgn = -1.0; }
        else { c = (f - 2 * ny - nx) + nx * (ny - 1); axis = 1; sgn = 1.0; }
        T acc = T(0);
        for (int k = lane; k < K; k += 32) {
            const double on = sgn * (axis == 0 ? a.mu[k] : a.eta[k]);
            T Iface;
            if (on >= 0.0) Iface = a.I[(size_t)a.sidx[k] * N + c];
            else Iface = a.inflow ? (T)a.inflow[(size_t)f * K + k] : T(0);
            acc = fma((T)(a.w[k] * on), Iface, acc);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (lane == 0) a.fb[f] = (double)acc;
    }
}

template <typename T, bool WITH_F, bool WITH_P>
__global__ void __launch_bounds__(kRedBlock) moments_kernel(const MomArgs<T> a)
{
    moments_body<T, WITH_F, WITH_P>(a, blockIdx.x, gridDim.x);
}

template <typename T>
__global__ void __launch_bounds__(256) bflux_kernel(const BfArgs<T> a)
{
    bflux_body(a, blockIdx.x, gridDim.x);
}

// Moments and boundary fluxes of one problem in one launch: the first
// mblocks blocks take the cells, the rest the boundary faces.
template <typename T, bool WITH_F, bool WITH_P>
__global__ void __launch_bounds__(kRedBlock) moments_bflux_kernel(const MomArgs<T> m, const BfArgs<T> f, int mblocks)
{
    if ((int)blockIdx.x < mblocks) moments_body<T, WITH_F, WITH_P>(m, blockIdx.x, mblocks);
    else bflux_body(f, blockIdx.x - mblocks, gridDim.x - mblocks);
}

// Batched moments and boundary fluxes: problem p owns blocks
// [bstart[p], bstart[p + 1]); its first mblocks blocks take the cell moments,
// the rest the boundary faces.
template <typename T>
struct MomBatchRec {
    MomArgs<T> m;
    BfArgs<T> f;
    int mblocks;
};

template <typename T, bool WITH_F, bool WITH_P>
__global__ void __launch_bounds__(kRedBlock) moments_batch_kernel(const MomBatchRec<T>* __restrict__ tab,
                                                                  const int* __restrict__ bstart, int B)
{
    const int p = batch_find(bstart, B, blockIdx.x);
    const int b0 = __ldg(bstart + p), nblk = __ldg(bstart + p + 1) - b0, lb = blockIdx.x - b0;
    const int mb = tab[p].mblocks;
    if (lb < mb) {
        const MomArgs<T> a = tab[p].m;
        moments_body<T, WITH_F, WITH_P>(a, lb, mb);
    } else {
        const BfArgs<T> a = tab[p].f;
        bflux_body(a, lb - mb, nblk - mb);
    }
}

int grid_for(long long n, int block, int cap)
{
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

template <typename T, int MODE, bool BATCH = false>
size_t sweep_smem();

// Threads of one sweep CTA of this variant (its pairs x 64).
template <typename T, int MODE, bool BATCH = false>
constexpr int sweep_threads()
{
    return SweepSmem<T, sweep_xw(MODE), sizeof(T) == 8, BATCH>::PAIRS * 64;
}

template <typename T, int MODE>
SweepArgs<T> sweep_args(const Plan& P)
{
    SweepArgs<T> a{};
    a.nx = P.nx; a.ny = P.ny; a.N = P.N; a.K = P.K; a.nb = P.nb; a.nsteps = P.nx + 31;
    if constexpr (sizeof(T) == 8) {
        a.acoef = P.acoef; a.bcoef = P.bcoef; a.sigt = P.sigt; a.shift = P.shift; a.src = P.src;
    } else {
        a.acoef = P.acoef_f; a.bcoef = P.bcoef_f; a.sigt = P.sigt_f; a.shift = P.shift_f; a.src = P.src_f;
    }
    a.rsw = P.rsw;
    a.I = static_cast<T*>(P.I);
    a.iold = P.In ? static_cast<const T*>(P.In) : a.I;
    a.edge = static_cast<T*>(P.edge);
    a.inflow = P.inflow;
    if (MODE == kSrcAdjoint) {   // transposed kinetic step: reflected direction, adjoint source
        if constexpr (sizeof(T) == 8) {
            a.src = P.adj_a; a.ax = P.adj_x; a.ay = P.adj_y;
        } else {
            a.src = P.adj_a_f; a.ax = P.adj_x_f; a.ay = P.adj_y_f;
            if (P.adj_sigt_f) a.sigt = P.adj_sigt_f;
        }
        a.I = static_cast<T*>(P.Iadj);
        a.inflow = P.adj_inflow;
    }
    if (MODE == kSrcDelta) {   // increment sweep: residual source, zero inflow increment, correction
        a.src = static_cast<const T*>(P.R);
        if constexpr (sizeof(T) == 8) a.shift = P.corr;
        else {
            a.shift = P.corr_f;
            a.sigt = P.sigt_d;
        }
        a.inflow = nullptr;
    }
    a.qw = P.qw;
    a.perm = P.perm; a.qmu = P.qmu; a.qeta = P.qeta;
    a.err = &P.status->error;
    a.done = &P.status->done;
    a.tasks = &P.status->sweep_tasks;
    a.exits = &P.status->sweep_exits;
    a.arrived = &P.status->sweep_arrived;
    a.mode = &P.status->sweep_mode;
    a.wait_cycles = P.wait_cycles;
    return a;
}

template <typename T, int MODE, bool PRE>
cudaError_t launch_sweep_t(Plan& P, cudaStream_t st)
{
    const SweepArgs<T> a = sweep_args<T, MODE>(P);
    sweep_kernel<T, MODE, PRE, false><<<P.sweep_grid, sweep_threads<T, MODE>(), sweep_smem<T, MODE>(), st>>>(a, SweepBatch<T>{});
    return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t launch_sweep_batch_t(const BatchTables& bt, cudaStream_t st)
{
    SweepBatch<T> b{};
    b.probs = static_cast<const SweepArgs<T>*>(bt.sweep);
    b.seg_start = bt.seg_start;
    b.seg_prob = bt.seg_prob;
    b.seg_band = bt.seg_band;
    b.nseg = bt.nseg;
    b.ntasks = bt.ntasks;
    b.dynamic = bt.dynamic;
    b.tasks = &bt.status->sweep_tasks;
    b.exits = &bt.status->sweep_exits;
    b.arrived = &bt.status->sweep_arrived;
    b.mode = &bt.status->sweep_mode;
    b.err = &bt.status->error;
    b.wait_cycles = bt.wait_cycles;
    sweep_kernel<T, MODE, sizeof(T) == 8, true><<<bt.sweep_grid, sweep_threads<T, MODE, true>(), sweep_smem<T, MODE, true>(), st>>>(
        SweepArgs<T>{}, b);
    return cudaGetLastError();
}

template <typename T>
size_t moments_smem(int K)
{
    return (size_t)K * (6 * sizeof(T) + sizeof(int)) + 16;
}

template <typename T>
BfArgs<T> bflux_args(const Plan& P, double* fb_out, const int* done)
{
    BfArgs<T> f{};
    f.nx = P.nx; f.ny = P.ny; f.K = P.K;
    f.I = static_cast<const T*>(P.I);
    f.sidx = P.sidx;
    f.mu = P.omu; f.eta = P.oeta; f.w = P.ow;
    f.inflow = P.inflow;
    f.fb = fb_out;
    f.done = done;
    return f;
}

template <typename T>
cudaError_t launch_moments_t(const Plan& P, bool with_F, bool with_P, double* rho_out, double* Fout,
                             double* Pout, bool gsis_correct, double* fb_out, bool force, cudaStream_t st)
{
    MomArgs<T> a{};
    a.nx = P.nx; a.ny = P.ny; a.N = P.N; a.K = P.K;
    a.I = static_cast<const T*>(P.I);
    a.sidx = P.sidx;
    a.pairs = P.has_mpair ? P.mpair : nullptr;
    a.mu = P.omu;
    a.eta = P.oeta;
    a.w = P.ow;
    a.rho = rho_out;
    a.Fx = Fout ? Fout : P.Fx;
    a.Fy = Fout ? Fout + P.N : P.Fy;
    if (with_P) { a.Pxx = Pout; a.Pxy = Pout + P.N; a.Pyy = Pout + 2 * (size_t)P.N; }
    a.rho_new = gsis_correct ? P.rho_m : nullptr;
    a.done = force ? nullptr : &P.status->done;
    const size_t smem = moments_smem<T>(P.K);
    const int grid = grid_for(P.N, kRedBlock, P.num_sms * 8);
    if (P.order != 2) {   // cells and boundary faces in one launch
        static_assert(kRedBlock == 256, "the boundary-flux blocks take 256 threads");
        const BfArgs<T> f = bflux_args<T>(P, fb_out, a.done);
        const int fg = grid_for((long long)P.nbf * 32, 256, P.num_sms * 4);
        if (with_P) moments_bflux_kernel<T, true, true><<<grid + fg, kRedBlock, smem, st>>>(a, f, grid);
        else if (with_F) moments_bflux_kernel<T, true, false><<<grid + fg, kRedBlock, smem, st>>>(a, f, grid);
        else moments_bflux_kernel<T, false, false><<<grid + fg, kRedBlock, smem, st>>>(a, f, grid);
        return cudaGetLastError();
    }
    if (with_P) moments_kernel<T, true, true><<<grid, kRedBlock, smem, st>>>(a);
    else if (with_F) moments_kernel<T, true, false><<<grid, kRedBlock, smem, st>>>(a);
    else moments_kernel<T, false, false><<<grid, kRedBlock, smem, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (P.order == 2) return launch_uw2_bflux(P, fb_out, a.done, st);   // reconstructed outgoing faces
    bflux_kernel<T><<<grid_for((long long)P.nbf * 32, 256, P.num_sms * 4), 256, 0, st>>>(
        bflux_args<T>(P, fb_out, a.done));
    return cudaGetLastError();
}

template <typename T, int MODE, bool BATCH>
size_t sweep_smem()
{
    return SweepSmem<T, sweep_xw(MODE), sizeof(T) == 8, BATCH>::bytes;
}


template <typename T, int MODE, bool BATCH>
cudaError_t sweep_attr()
{
    return cudaFuncSetAttribute(sweep_kernel<T, MODE, sizeof(T) == 8, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sweep_smem<T, MODE, BATCH>());
}

// Raises the dynamic shared-memory limit of fn to at least `bytes` (never
// lowers it: plans of different sizes may launch concurrently).
cudaError_t raise_smem_limit(const void* fn, size_t bytes)
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

template <typename T>
cudaError_t prepare_t(int K)
{
    static std::once_flag once;
    static cudaError_t first = cudaSuccess;
    std::call_once(once, [] {
        cudaError_t e;
        if ((e = sweep_attr<T, kSrcPlain, false>()) != cudaSuccess ||
            (e = sweep_attr<T, kSrcPseudoTime, false>()) != cudaSuccess ||
            (e = sweep_attr<T, kSrcAdjoint, false>()) != cudaSuccess ||
            (e = sweep_attr<T, kSrcDelta, false>()) != cudaSuccess ||
            (e = sweep_attr<T, kSrcPlain, true>()) != cudaSuccess ||
            (e = sweep_attr<T, kSrcPseudoTime, true>()) != cudaSuccess)
            first = e;
        if constexpr (sizeof(T) == 8) {   // the FP64 throughput form
            if (first == cudaSuccess &&
                (e = cudaFuncSetAttribute(sweep_kernel<double, kSrcPlain, true, false, true>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sweep_smem<double, kSrcPlain, true>())) != cudaSuccess)
                first = e;
        }
    });
    if (first != cudaSuccess) return first;
    const size_t ms = moments_smem<T>(K);
    cudaError_t e;
    if ((e = raise_smem_limit((const void*)moments_kernel<T, true, true>, ms)) != cudaSuccess) return e;
    if ((e = raise_smem_limit((const void*)moments_kernel<T, true, false>, ms)) != cudaSuccess) return e;
    if ((e = raise_smem_limit((const void*)moments_kernel<T, false, false>, ms)) != cudaSuccess) return e;
    if ((e = raise_smem_limit((const void*)moments_batch_kernel<T, true, false>, ms)) != cudaSuccess) return e;
    if ((e = raise_smem_limit((const void*)moments_bflux_kernel<T, true, true>, ms)) != cudaSuccess) return e;
    if ((e = raise_smem_limit((const void*)moments_bflux_kernel<T, true, false>, ms)) != cudaSuccess) return e;
    if ((e = raise_smem_limit((const void*)moments_bflux_kernel<T, false, false>, ms)) != cudaSuccess) return e;
    return raise_smem_limit((const void*)moments_batch_kernel<T, false, false>, ms);
}

template <typename T, int MODE, bool BATCH>
int sweep_occupancy()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_kernel<T, MODE, sizeof(T) == 8, BATCH>,
                                                      sweep_threads<T, MODE, BATCH>(), sweep_smem<T, MODE, BATCH>()) != cudaSuccess)
        return 0;
    return n;
}

template <int MODE, bool WIDE>
int sweep_fp64_occupancy()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_kernel<double, MODE, true, false, WIDE>,
                                                      sweep_threads<double, MODE, WIDE>(),
                                                      sweep_smem<double, MODE, WIDE>()) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace

int device_sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_setup(const Plan& P, cudaStream_t st)
{
    const int tot = P.K * (P.nx + P.ny);
    coef_kernel<<<grid_for(tot, 256, 1024), 256, 0, st>>>(
        P.nx, P.ny, P.K, P.dx, P.dy, P.qmu, P.qeta, const_cast<double*>(P.acoef),
        const_cast<double*>(P.bcoef), P.fp32 ? const_cast<float*>(P.acoef_f) : nullptr,
        P.fp32 ? const_cast<float*>(P.bcoef_f) : nullptr);
    return cudaGetLastError();
}

// Per-cell set-up and the FP64 reciprocal table (pseudo-time controls given).
cudaError_t launch_cell_setup(const Plan& P, double cfl_p, double beta, cudaStream_t st)
{
    cell_setup_kernel<<<grid_for(P.N, 256, P.num_sms * 8), 256, 0, st>>>(
        P.nx, P.ny, P.dx, P.dy, P.sigma_a, P.sigma_s, P.q, P.inflow, P.nbf * P.K, P.shift0, cfl_p, beta, P.sigt,
        P.fp32 ? P.sigt_f : nullptr, P.shift, P.fp32 ? P.shift_f : nullptr, P.diag, P.cx, P.cy, P.hw,
        P.bface, P.gw, P.gw_f, P.sigt_d, &P.status->error);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (!P.fp32) {
        const size_t tot = (size_t)P.K * P.nb * (P.nx + 31) * 32;
        recip_kernel<<<grid_for((long long)tot, 256, P.num_sms * 16), 256, 0, st>>>(
            P.nx, P.ny, P.K, P.nb, P.perm, P.qmu, P.qeta, P.acoef, P.bcoef, P.sigt, P.shift,
            const_cast<double*>(P.rsw));
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_init_state(const Plan& P, cudaStream_t st)
{
    const int g = grid_for(P.N, 256, P.num_sms * 8);
    fill_kernel<<<g, 256, 0, st>>>(P.rho_m, P.N, 0.0);
    fill_kernel<<<g, 256, 0, st>>>(P.rho_h, P.N, 0.0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (P.order == 2) {   // no correction of the initial intensities
        fill_kernel<<<g, 256, 0, st>>>(P.corr, P.N, 0.0);
        if (P.fp32) fillf_kernel<<<g, 256, 0, st>>>(P.corr_f, P.N, 0.f);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (P.pt || P.order == 2) {   // I^0 = 0 (the delta form reads it)
        const size_t n = (size_t)P.K * P.N;
        if (P.fp32) fillf_kernel<<<grid_for((long long)n, 256, P.num_sms * 16), 256, 0, st>>>(static_cast<float*>(P.I), n, 0.f);
        else fill_kernel<<<grid_for((long long)n, 256, P.num_sms * 16), 256, 0, st>>>(static_cast<double*>(P.I), n, 0.0);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return launch_source_from(P, P.rho_m, st);
}

cudaError_t launch_source_from(const Plan& P, const double* rho_in, cudaStream_t st)
{
    source_kernel<<<grid_for(P.N, 256, P.num_sms * 8), 256, 0, st>>>(P.N, P.sigma_s, P.q, rho_in, P.src,
                                                                    P.fp32 ? P.src_f : nullptr);
    return cudaGetLastError();
}

// The FP64 sweep's throughput form pays when every pair has several long
// units to run (1024^2 S16: 4608 units, sweep 1.32 -> 1.09 ms); with fewer
// units than two waves of the 8-pair form the band hand-off latency
// dominates and per-result stores are faster (256^2 S12: 672 units).
bool sweep_wide(const Plan& P)
{
    return (long long)P.K * P.nb >= 2LL * P.sweep_grid * 8;
}

cudaError_t launch_sweep(Plan& P, cudaStream_t st)
{
    if (P.pt && P.X && !P.fp32) {
        // FP64 pseudo-time form with its source already combined per ordinate
        // (X = src + shift I^m, formed by the update kernel): the plain sweep
        // over X takes one FP64 operation per update fewer, same bits
        SweepArgs<double> a = sweep_args<double, kSrcPlain>(P);
        a.src = P.X;
        a.src_stride = P.N;
        if (sweep_wide(P)) {   // throughput form: 12 pairs, staged write-out (same bits)
            sweep_kernel<double, kSrcPlain, true, false, true>
                <<<P.sweep_grid, sweep_threads<double, kSrcPlain, true>(), sweep_smem<double, kSrcPlain, true>(), st>>>(
                    a, SweepBatch<double>{});
            return cudaGetLastError();
        }
        sweep_kernel<double, kSrcPlain, true, false>
            <<<P.sweep_grid, sweep_threads<double, kSrcPlain>(), sweep_smem<double, kSrcPlain>(), st>>>(a, SweepBatch<double>{});
        return cudaGetLastError();
    }
    if (P.fp32 && P.pt && P.X_f) {
        // FP32 time step with its source combined per ordinate (X = src +
        // I^n/(c dt)) and its diagonal sigma_t + 1/(c dt): the plain sweep
        // over X reads two cell windows instead of four
        SweepArgs<float> a = sweep_args<float, kSrcPlain>(P);
        a.src = P.X_f;
        a.src_stride = P.N;
        a.sigt = P.sigt_d;
        sweep_kernel<float, kSrcPlain, false, false>
            <<<P.sweep_grid, sweep_threads<float, kSrcPlain>(), sweep_smem<float, kSrcPlain>(), st>>>(a, SweepBatch<float>{});
        return cudaGetLastError();
    }
    if (P.fp32) {
        return P.pt ? launch_sweep_t<float, kSrcPseudoTime, false>(P, st)
                    : launch_sweep_t<float, kSrcPlain, false>(P, st);
    }
    return P.pt ? launch_sweep_t<double, kSrcPseudoTime, true>(P, st) : launch_sweep_t<double, kSrcPlain, true>(P, st);
}

cudaError_t launch_delta_sweep(Plan& P, cudaStream_t st)
{
    return P.fp32 ? launch_sweep_t<float, kSrcDelta, false>(P, st) : launch_sweep_t<double, kSrcDelta, true>(P, st);
}

cudaError_t launch_adjoint_sweep(Plan& P, cudaStream_t st)
{
    return P.fp32 ? launch_sweep_t<float, kSrcAdjoint, false>(P, st) : launch_sweep_t<double, kSrcAdjoint, true>(P, st);
}

template <typename T>
cudaError_t launch_sweep_pt_into_t(Plan& P, const void* src, const void* iold, void* out, cudaStream_t st)
{
    constexpr bool PRE = sizeof(T) == 8;
    SweepArgs<T> a = sweep_args<T, kSrcPseudoTime>(P);
    a.src = static_cast<const T*>(src);
    a.iold = static_cast<const T*>(iold);
    a.I = static_cast<T*>(out);
    a.inflow = nullptr;
    sweep_kernel<T, kSrcPseudoTime, PRE, false>
        <<<P.sweep_grid, sweep_threads<T, kSrcPseudoTime>(), sweep_smem<T, kSrcPseudoTime>(), st>>>(a, SweepBatch<T>{});
    return cudaGetLastError();
}

cudaError_t launch_sweep_pt_into(Plan& P, const void* src, const void* iold, void* out, cudaStream_t st)
{
    return P.fp32 ? launch_sweep_pt_into_t<float>(P, src, iold, out, st)
                  : launch_sweep_pt_into_t<double>(P, src, iold, out, st);
}

// Moments of the last sweep into the given outputs: rho always, F when
// with_F (Fout or the plan's F arrays), P when with_P (plus drho/3 on the
// diagonal when gsis_correct), boundary fluxes into fb_out.  force: run even
// after the device has stopped the iteration (final outputs).
cudaError_t launch_moments_to(const Plan& P, bool with_F, bool with_P, double* rho_out, double* Fout,
                              double* Pout, bool gsis_correct, double* fb_out, bool force, cudaStream_t st)
{
    if (P.fp32)
        return launch_moments_t<float>(P, with_F, with_P, rho_out, Fout, Pout, gsis_correct, fb_out, force, st);
    return launch_moments_t<double>(P, with_F, with_P, rho_out, Fout, Pout, gsis_correct, fb_out, force, st);
}

size_t sweep_batch_rec_bytes(int fp32)
{
    return fp32 ? sizeof(SweepArgs<float>) : sizeof(SweepArgs<double>);
}

void sweep_batch_rec(const Plan& P, void* out)
{
    if (P.fp32) {
        SweepArgs<float> a = P.pt ? sweep_args<float, kSrcPseudoTime>(P) : sweep_args<float, kSrcPlain>(P);
        if (P.pt && P.X_f) {   // the plain sweep over the per-ordinate source, as launch_sweep does
            a = sweep_args<float, kSrcPlain>(P);
            a.src = P.X_f;
            a.src_stride = P.N;
            a.sigt = P.sigt_d;
        }
        std::memcpy(out, &a, sizeof(a));
    } else {
        const SweepArgs<double> a = P.pt ? sweep_args<double, kSrcPseudoTime>(P) : sweep_args<double, kSrcPlain>(P);
        std::memcpy(out, &a, sizeof(a));
    }
}

cudaError_t launch_sweep_batch(const BatchTables& bt, cudaStream_t st)
{
    if (bt.fp32)   // with per-ordinate sources (ord_blocks > 0) the records describe plain sweeps
        return bt.pt && bt.ord_blocks == 0 ? launch_sweep_batch_t<float, kSrcPseudoTime>(bt, st)
                                           : launch_sweep_batch_t<float, kSrcPlain>(bt, st);
    return bt.pt ? launch_sweep_batch_t<double, kSrcPseudoTime>(bt, st) : launch_sweep_batch_t<double, kSrcPlain>(bt, st);
}

size_t mom_batch_rec_bytes(int fp32)
{
    return fp32 ? sizeof(MomBatchRec<float>) : sizeof(MomBatchRec<double>);
}

template <typename T>
int mom_batch_rec_t(const Plan& P, bool with_F, void* out)
{
    MomBatchRec<T> r{};
    r.m.nx = P.nx; r.m.ny = P.ny; r.m.N = P.N; r.m.K = P.K;
    r.m.I = static_cast<const T*>(P.I);
    r.m.sidx = P.sidx;
    r.m.pairs = P.has_mpair ? P.mpair : nullptr;
    r.m.mu = P.omu; r.m.eta = P.oeta; r.m.w = P.ow;
    r.m.rho = P.rho_h;
    r.m.Fx = with_F ? P.Fx : nullptr;
    r.m.Fy = with_F ? P.Fy : nullptr;
    r.m.done = &P.status->done;
    r.f = bflux_args<T>(P, P.fb, &P.status->done);
    r.mblocks = grid_for(P.N, kRedBlock, P.num_sms * 8);
    std::memcpy(out, &r, sizeof(r));
    return r.mblocks + grid_for((long long)P.nbf * 32, kRedBlock, P.num_sms * 4);
}

// Batched record of the moments of one GSIS / SI iteration (rho^{m+1/2},
// F^{m+1/2} when with_F, boundary fluxes); returns the problem's blocks.
int mom_batch_rec(const Plan& P, bool with_F, void* out)
{
    return P.fp32 ? mom_batch_rec_t<float>(P, with_F, out) : mom_batch_rec_t<double>(P, with_F, out);
}

cudaError_t launch_moments_batch(const BatchTables& bt, cudaStream_t st)
{
    const int fp32 = bt.fp32;
    const size_t smem = fp32 ? moments_smem<float>(bt.maxK) : moments_smem<double>(bt.maxK);
    if (fp32) {
        const auto* tab = static_cast<const MomBatchRec<float>*>(bt.mom);
        if (bt.with_F) moments_batch_kernel<float, true, false><<<bt.mom_blocks, kRedBlock, smem, st>>>(tab, bt.mom_bstart, bt.B);
        else moments_batch_kernel<float, false, false><<<bt.mom_blocks, kRedBlock, smem, st>>>(tab, bt.mom_bstart, bt.B);
    } else {
        const auto* tab = static_cast<const MomBatchRec<double>*>(bt.mom);
        if (bt.with_F) moments_batch_kernel<double, true, false><<<bt.mom_blocks, kRedBlock, smem, st>>>(tab, bt.mom_bstart, bt.B);
        else moments_batch_kernel<double, false, false><<<bt.mom_blocks, kRedBlock, smem, st>>>(tab, bt.mom_bstart, bt.B);
    }
    return cudaGetLastError();
}

cudaError_t prepare_kernels(int K, int fp32, int pt)
{
    (void)pt;
    return fp32 ? prepare_t<float>(K) : prepare_t<double>(K);
}

int sweep_max_active_blocks(int fp32, int pt)
{
    // one grid for every variant a plan may launch (forward, pseudo-time,
    // adjoint): every warp pair must be resident, so take the smallest
    (void)pt;
    if (fp32)
        return std::min({sweep_occupancy<float, kSrcPlain, false>(), sweep_occupancy<float, kSrcPseudoTime, false>(),
                         sweep_occupancy<float, kSrcAdjoint, false>(), sweep_occupancy<float, kSrcDelta, false>(),
                         sweep_occupancy<float, kSrcPlain, true>(),
                         sweep_occupancy<float, kSrcPseudoTime, true>()});
    return std::min({sweep_occupancy<double, kSrcPlain, false>(), sweep_occupancy<double, kSrcPseudoTime, false>(),
                     sweep_occupancy<double, kSrcAdjoint, false>(), sweep_occupancy<double, kSrcDelta, false>(),
                     sweep_occupancy<double, kSrcPlain, true>(),
                     sweep_occupancy<double, kSrcPseudoTime, true>(), sweep_fp64_occupancy<kSrcPlain, true>()});
}

}  // namespace gsis
