// Host-side helpers shared by the entry points (single-problem solves in
// api.cu, batched solves in batch.cu): argument checks, the workspace
// layout of one problem and its preparation.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <vector>

#include "gsis.h"
#include "gsis_internal.cuh"

namespace gsis {

constexpr size_t kAlign = 256;
constexpr double kPi = 3.14159265358979323846;

// Records the message returned by gsis_last_error(); returns code.
int fail(int code, const char* fmt, ...);

#define CK(expr)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (expr);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(GSIS_ERR_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));          \
    } while (0)

// Instrumentation: counts the kernels of one class launch and, when
// profiling is on, brackets it with CUDA events on st (gsis_profile_*).
struct ProfScope {
    int cls, nk;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(int c, int n, cudaStream_t s);
    ~ProfScope();
};

#define TIMED(cls, nk, expr)                        \
    do {                                            \
        ProfScope ps_((cls), (nk), st);             \
        CK(expr);                                   \
    } while (0)

struct Sizes {
    int nx, ny, K, fp32, hist, adjoint, td, order;
    int ordsrc;   // the per-ordinate source array of the pseudo-time sweeps (FP32: with its diagonal)
};

// Carves one problem's workspace (base may be null: size query only).
size_t layout(const Sizes& z, char* base, Plan* P);
int check_mesh(const gsis_mesh* m);
int check_quad(const gsis_quadrature* q);
int check_opt(const gsis_options* o);
int check_ws(void* ws, size_t have, size_t need);
// Sizes, grids, sorted quadrature copy, per-cell set-up and the synthetic
// solver's plan of one problem (stream-ordered on st).
int prepare(Plan& P, const gsis_mesh* mesh, const gsis_quadrature* quad, const gsis_options* opt,
            const double* sa, const double* ss, const double* q, const double* inflow, cudaStream_t st);
// Copies the status block back (synchronising st) and maps device error bits.
int read_status(Status& S, const Plan& P, cudaStream_t st);
Sizes sizes_of(const gsis_mesh* m, const gsis_quadrature* q, const gsis_options* o);
// The sizes of gsis_solve: with the FP64 pseudo-time form, also the
// per-ordinate source of the sweep.
Sizes solve_sizes(const gsis_mesh* m, const gsis_quadrature* q, const gsis_options* o);
// The options gsis_transport_sweep runs with (first-order upwind, no
// pseudo-time) and the sizes of its workspace.
gsis_options sweep_options(const gsis_options* o);
Sizes sweep_sizes(const gsis_mesh* m, const gsis_quadrature* q, const gsis_options* o);
// All spacings equal (relative 1e-12).
bool uniform_spacing(const double* h, int n);
// Sorted index (quadrant-major, as in prepare) of the reflected direction
// -Omega of every sorted direction; false if the set is not closed under
// the reflection with equal weights.
bool reflection_table(const gsis_quadrature* quad, std::vector<int>& refl);

}  // namespace gsis
