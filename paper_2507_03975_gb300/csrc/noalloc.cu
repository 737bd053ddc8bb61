// Kinetic step for callers that cannot allocate device memory.
//
// Some callers have no device allocator to hand: a plain C host program that
// links only this library, or a plug-in whose host application owns every
// byte of device memory through its own pool and forbids further
// allocations.  gsis_transport_sweep_static() serves them: it runs exactly
// the work of gsis_transport_sweep(), but its scratch lives in one
// file-scope device array of fixed size instead of a caller workspace.
//
// Properties a caller must know:
//  * the array holds kStaticScratchBytes (GSIS_STATIC_SCRATCH_BYTES, 32 MiB);
//    every GPU on which the library's kernels are loaded keeps it reserved
//    until the process exits;
//  * problems whose kinetic-step workspace exceeds it are rejected with
//    GSIS_ERR_WORKSPACE before any device work; that is the workspace of
//    gsis_transport_sweep() (first-order upwind, no pseudo-time, whatever
//    the options ask), i.e. gsis_workspace_bytes() with spatial_order = 1,
//    cfl_p = beta = 0;
//  * the first call on a device looks the array's device address up with
//    cudaGetSymbolAddress (once per device, that device current); make that
//    first call before any stream capture;
//  * every call shares the one array and it keeps the last call's contents;
//    the status block and the band hand-off rows that must start "unwritten"
//    are reset by every call; calls that overlap on the GPU (other streams,
//    other host threads) race on the array.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "gsis.h"
#include "gsis_internal.cuh"
#include "host.h"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)GSIS_STATIC_SCRATCH_BYTES;
static_assert(kStaticScratchBytes % 256 == 0, "scratch size must keep 256-byte alignment");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device (looked up once).
int scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        gsis::set_last_error(GSIS_ERR_CUDA, cudaGetErrorString(e));
        return GSIS_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        gsis::set_last_error(GSIS_ERR_ARG, "device ordinal beyond the static scratch table");
        return GSIS_ERR_ARG;
    }
    std::lock_guard<std::mutex> g(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            gsis::set_last_error(GSIS_ERR_CUDA, e != cudaSuccess ? cudaGetErrorString(e)
                                                                 : "cudaGetSymbolAddress returned NULL");
            return GSIS_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return GSIS_OK;
}

}  // namespace

extern "C" int gsis_transport_sweep_static(const gsis_mesh* mesh, const gsis_quadrature* quad,
                                           const gsis_options* opt, const double* sigma_a,
                                           const double* sigma_s, const double* q, const double* inflow,
                                           const double* rho_in, double* rho_half, double* F_half,
                                           double* P_half, double* bflux, void* stream)
{
    int rc;
    if ((rc = gsis::check_mesh(mesh)) || (rc = gsis::check_quad(quad)) || (rc = gsis::check_opt(opt))) return rc;
    // the layout gsis_transport_sweep carves (its own option overrides)
    const size_t need = gsis::layout(gsis::sweep_sizes(mesh, quad, opt), nullptr, nullptr);
    if (need > kStaticScratchBytes) {
        char msg[160];
        snprintf(msg, sizeof msg, "problem needs %zu bytes of scratch, the static array holds %zu", need,
                 kStaticScratchBytes);
        gsis::set_last_error(GSIS_ERR_WORKSPACE, msg);
        return GSIS_ERR_WORKSPACE;
    }
    void* scratch = nullptr;
    if ((rc = scratch_address(&scratch)) != GSIS_OK) return rc;
    return gsis_transport_sweep(mesh, quad, opt, sigma_a, sigma_s, q, inflow, rho_in, rho_half, F_half,
                                P_half, bflux, scratch, kStaticScratchBytes, stream);
}
