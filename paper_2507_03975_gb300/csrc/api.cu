// C ABI of libgsis: argument checks, workspace layout, the SI / GSIS
// iteration loop (Sec. 2.2, Sec. 3.1, flowchart of Sec. 4 without the time
// loop) and status reporting.  All device work is stream-ordered on the
// caller's stream; the loop reads the device status block back every
// `check_every` iterations, and kernels launched after the device has
// decided to stop return at once.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "gsis.h"
#include "gsis_internal.cuh"
#include "host.h"

using namespace gsis;

namespace {

thread_local std::string g_last_error;
thread_local gsis_solve_info g_last_info{};

}  // namespace

int gsis::fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

namespace {

// ------------------------------------------------------------ instrumentation
struct Profiler {
    std::mutex mu;
    bool on = false;
    gsis_kernel_stats st[GSIS_KCLASS_COUNT]{};
    struct Pending { int cls; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;
};
Profiler g_prof;

}  // namespace

ProfScope::ProfScope(int c, int n, cudaStream_t s) : cls(c), nk(n), st(s)
{
    std::lock_guard<std::mutex> g(g_prof.mu);
    g_prof.st[cls].kernels += nk;
    g_prof.st[cls].groups += 1;
    if (!g_prof.on) return;
    if (g_prof.pool.empty()) {
        cudaEvent_t x, y;
        if (cudaEventCreate(&x) != cudaSuccess) return;
        if (cudaEventCreate(&y) != cudaSuccess) { cudaEventDestroy(x); return; }
        g_prof.pool.push_back({x, y});
    }
    a = g_prof.pool.back().first;
    b = g_prof.pool.back().second;
    g_prof.pool.pop_back();
    cudaEventRecord(a, st);
}

ProfScope::~ProfScope()
{
    if (!a) return;
    cudaEventRecord(b, st);
    std::lock_guard<std::mutex> g(g_prof.mu);
    g_prof.pending.push_back({cls, a, b});
}

namespace {

// After a stream synchronisation: accumulate the finished event pairs.
void prof_harvest()
{
    std::lock_guard<std::mutex> g(g_prof.mu);
    for (auto& p : g_prof.pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_prof.st[p.cls].timed += 1;
            g_prof.st[p.cls].total_ms += ms;
        }
        g_prof.pool.push_back({p.a, p.b});
    }
    g_prof.pending.clear();
    cudaGetLastError();   // an unfinished pair reports "not ready": not an error of the caller
}


}  // namespace

namespace gsis {


// Carves the workspace (base may be null: size query only).
size_t layout(const Sizes& z, char* base, Plan* P)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off += (bytes + kAlign - 1) / kAlign * kAlign;
        return p;
    };
    const size_t N = (size_t)z.nx * z.ny, K = (size_t)z.K;
    const size_t nb = (size_t)(z.ny + 31) / 32, nbf = 2 * (size_t)(z.nx + z.ny);
    const size_t Ts = z.fp32 ? sizeof(float) : sizeof(double);
    Plan tmp{};
    Plan& p = P ? *P : tmp;
    p.status = reinterpret_cast<Status*>(take(sizeof(Status)));
    double* qbuf = reinterpret_cast<double*>(take(6 * K * sizeof(double)));
    p.qmu = qbuf; p.qeta = qbuf ? qbuf + K : nullptr; p.qw = qbuf ? qbuf + 2 * K : nullptr;
    p.omu = qbuf ? qbuf + 3 * K : nullptr; p.oeta = qbuf ? qbuf + 4 * K : nullptr;
    p.ow = qbuf ? qbuf + 5 * K : nullptr;
    int* ibuf = reinterpret_cast<int*>(take(3 * K * sizeof(int)));
    p.perm = ibuf; p.sidx = ibuf ? ibuf + K : nullptr; p.mpair = ibuf ? ibuf + 2 * K : nullptr;
    p.dx = reinterpret_cast<double*>(take(z.nx * sizeof(double)));
    p.dy = reinterpret_cast<double*>(take(z.ny * sizeof(double)));
    p.acoef = reinterpret_cast<double*>(take(K * z.nx * sizeof(double)));
    p.bcoef = reinterpret_cast<double*>(take(K * z.ny * sizeof(double)));
    p.acoef_f = z.fp32 ? reinterpret_cast<float*>(take(K * z.nx * sizeof(float))) : nullptr;
    p.bcoef_f = z.fp32 ? reinterpret_cast<float*>(take(K * z.ny * sizeof(float))) : nullptr;
    p.rsw = z.fp32 ? nullptr : reinterpret_cast<double*>(take(K * nb * (z.nx + 31) * 32 * sizeof(double)));
    p.I = take(K * N * Ts);
    p.edge = take(K * nb * z.nx * Ts);
    p.sigt = reinterpret_cast<double*>(take(N * sizeof(double)));
    p.shift = reinterpret_cast<double*>(take(N * sizeof(double)));
    p.src = reinterpret_cast<double*>(take(N * sizeof(double)));
    p.sigt_f = z.fp32 ? reinterpret_cast<float*>(take(N * sizeof(float))) : nullptr;
    p.shift_f = z.fp32 ? reinterpret_cast<float*>(take(N * sizeof(float))) : nullptr;
    p.src_f = z.fp32 ? reinterpret_cast<float*>(take(N * sizeof(float))) : nullptr;
    p.rho_m = reinterpret_cast<double*>(take(N * sizeof(double)));
    p.rho_h = reinterpret_cast<double*>(take(N * sizeof(double)));
    p.Fx = reinterpret_cast<double*>(take(N * sizeof(double)));
    p.Fy = reinterpret_cast<double*>(take(N * sizeof(double)));
    p.fb = reinterpret_cast<double*>(take(nbf * sizeof(double)));
    double** syn[] = {&p.diag, &p.cx, &p.cy, &p.hotx, &p.hoty, &p.b, &p.x, &p.r, &p.z, &p.p, &p.qv};
    for (double** d : syn) *d = reinterpret_cast<double*>(take(N * sizeof(double)));
    p.hw = reinterpret_cast<double*>(take(4 * N * sizeof(double)));
    p.bface = reinterpret_cast<double*>(take(nbf * sizeof(double)));
    p.partials = reinterpret_cast<double*>(take(11 * (size_t)kMaxCgBlocks * sizeof(double)));
    p.mg_gslots_d = reinterpret_cast<double*>(take(6 * (size_t)kMaxCgBlocks * sizeof(double)));
    p.mg_gslots_f = reinterpret_cast<float*>(take(6 * (size_t)kMaxCgBlocks * sizeof(float)));
    // multigrid hierarchy: 2x2 aggregation down to a single cell
    {
        MgPlan& g = p.mg;
        int lx = z.nx, ly = z.ny, l = 0;
        for (;;) {
            g.nx[l] = lx;
            g.ny[l] = ly;
            const size_t n = (size_t)lx * ly;
            g.d64[l] = reinterpret_cast<double*>(take(n * sizeof(double)));
            g.cx64[l] = reinterpret_cast<double*>(take(n * sizeof(double)));
            g.cy64[l] = reinterpret_cast<double*>(take(n * sizeof(double)));
            g.d[l] = reinterpret_cast<float*>(take(n * sizeof(float)));
            g.cx[l] = reinterpret_cast<float*>(take(n * sizeof(float)));
            g.cy[l] = reinterpret_cast<float*>(take(n * sizeof(float)));
            g.x[l] = reinterpret_cast<float*>(take(n * sizeof(float)));
            g.t[l] = reinterpret_cast<float*>(take(n * sizeof(float)));
            g.r[l] = reinterpret_cast<float*>(take(n * sizeof(float)));
            ++l;
            if (n == 1 || l == kMaxLevels) break;
            lx = (lx + 1) / 2;
            ly = (ly + 1) / 2;
        }
        g.nl = l;
        g.direct = -1;
        for (int k = 1; k < l; ++k)
            if ((size_t)g.nx[k] * g.ny[k] <= (size_t)kDirectMax) { g.direct = k; break; }
        g.cinv = reinterpret_cast<float*>(take((size_t)kDirectMax * kDirectMax * sizeof(float)));
        g.local_from = l - 1;
        for (int k = 0; k < l; ++k)
            if ((size_t)g.nx[k] * g.ny[k] <= 4 * (size_t)kMgBlock) { g.local_from = k; break; }
        float** v[] = {&g.r0, &g.dl, &g.s, &g.p, &g.q};
        for (float** f : v) *f = reinterpret_cast<float*>(take(N * sizeof(float)));
    }
    p.hist = reinterpret_cast<double*>(take((size_t)std::max(1, z.hist) * sizeof(double)));
    if (z.adjoint) {
        p.Iadj = take(K * N * Ts);
        double** adj[] = {&p.adj_a, &p.adj_x, &p.adj_y, &p.lam, &p.nu};
        for (double** d : adj) *d = reinterpret_cast<double*>(take(N * sizeof(double)));
        if (z.fp32) {
            float** af[] = {&p.adj_a_f, &p.adj_x_f, &p.adj_y_f};
            for (float** f : af) *f = reinterpret_cast<float*>(take(N * sizeof(float)));
        }
        p.adj_inflow = reinterpret_cast<double*>(take(nbf * K * sizeof(double)));
        p.refl = reinterpret_cast<int*>(take(K * sizeof(int)));
    }
    if (z.order == 2) {
        p.R = take(K * N * Ts);
        p.corr = reinterpret_cast<double*>(take(N * sizeof(double)));
        p.gw = reinterpret_cast<double*>(take(4 * N * sizeof(double)));
        if (z.fp32) {
            p.corr_f = reinterpret_cast<float*>(take(N * sizeof(float)));
            p.gw_f = reinterpret_cast<float*>(take(4 * N * sizeof(float)));
            p.sigt_d = reinterpret_cast<float*>(take(N * sizeof(float)));
        }
    }
    if (z.ordsrc) {   // the sweep's source per ordinate (FP32: with its diagonal sigma_t + shift)
        if (z.fp32) {
            p.X_f = reinterpret_cast<float*>(take(K * N * sizeof(float)));
            if (!p.sigt_d) p.sigt_d = reinterpret_cast<float*>(take(N * sizeof(float)));
        } else {
            p.X = reinterpret_cast<double*>(take(K * N * sizeof(double)));
        }
    }
    if (z.td) {
        p.In = take(K * N * Ts);
        double** td[] = {&p.td.rho_n, &p.td.T_n, &p.td.T,   &p.td.cn,  &p.td.cnext, &p.td.qeff,
                         &p.td.diag0, &p.td.hr1, &p.td.hr2, &p.td.ht1, &p.td.ht2, &p.td.ckap,
                         &p.td.cphi,  &p.td.cf};
        for (double** d : td) *d = reinterpret_cast<double*>(take(N * sizeof(double)));
    }
    return off;
}

int check_mesh(const gsis_mesh* m)
{
    if (!m) return fail(GSIS_ERR_ARG, "mesh is NULL");
    if (m->nx < 1 || m->ny < 1 || m->nx > kMaxSide || m->ny > kMaxSide)
        return fail(GSIS_ERR_ARG, "mesh size %d x %d out of range [1, %d]", m->nx, m->ny, kMaxSide);
    if ((long long)m->nx * m->ny > (1LL << 30)) return fail(GSIS_ERR_ARG, "too many cells");
    if (!m->dx || !m->dy) return fail(GSIS_ERR_ARG, "mesh spacing arrays are NULL");
    for (int i = 0; i < m->nx; ++i)
        if (!(m->dx[i] > 0.0) || !std::isfinite(m->dx[i])) return fail(GSIS_ERR_ARG, "dx[%d] not > 0", i);
    for (int j = 0; j < m->ny; ++j)
        if (!(m->dy[j] > 0.0) || !std::isfinite(m->dy[j])) return fail(GSIS_ERR_ARG, "dy[%d] not > 0", j);
    return GSIS_OK;
}

int check_quad(const gsis_quadrature* q)
{
    if (!q) return fail(GSIS_ERR_ARG, "quadrature is NULL");
    if (q->K < 1 || q->K > kMaxK) return fail(GSIS_ERR_ARG, "K = %d out of range [1, %d]", q->K, kMaxK);
    if (!q->mu || !q->eta || !q->w) return fail(GSIS_ERR_ARG, "quadrature arrays are NULL");
    double sw = 0.0;
    for (int k = 0; k < q->K; ++k) {
        const double m = q->mu[k], e = q->eta[k], w = q->w[k];
        if (!std::isfinite(m) || !std::isfinite(e) || !(w > 0.0) || !std::isfinite(w))
            return fail(GSIS_ERR_ARG, "direction %d invalid", k);
        if (m * m + e * e > 1.0 + 1e-12) return fail(GSIS_ERR_ARG, "direction %d: mu^2 + eta^2 > 1", k);
        sw += w;
    }
    if (std::fabs(sw - 4.0 * kPi) > 1e-10 * 4.0 * kPi)
        return fail(GSIS_ERR_ARG, "sum of weights %.17g != 4 pi", sw);
    return GSIS_OK;
}

int check_opt(const gsis_options* o)
{
    if (!o) return fail(GSIS_ERR_ARG, "options are NULL");
    if (o->scheme != GSIS_SCHEME_SI && o->scheme != GSIS_SCHEME_GSIS) return fail(GSIS_ERR_ARG, "bad scheme");
    if (o->precision != GSIS_FP64 && o->precision != GSIS_FP32_SWEEP) return fail(GSIS_ERR_ARG, "bad precision");
    if (!(o->tol > 0.0) && o->fixed_iters <= 0) return fail(GSIS_ERR_ARG, "tol must be > 0");
    if (o->max_iter < 1 || o->max_iter > 100000000) return fail(GSIS_ERR_ARG, "max_iter out of range");
    if (o->fixed_iters < 0 || o->fixed_iters > o->max_iter) return fail(GSIS_ERR_ARG, "fixed_iters out of range");
    if (!(o->synth_rtol >= 0.0) || o->synth_max_iter < 0) return fail(GSIS_ERR_ARG, "bad synthetic controls");
    if (o->check_every < 1) return fail(GSIS_ERR_ARG, "check_every must be >= 1");
    if (!(o->wait_limit_s > 0.0) || o->wait_limit_s > 3600.0) return fail(GSIS_ERR_ARG, "wait_limit_s out of range");
    if (o->spatial_order != 1 && o->spatial_order != 2) return fail(GSIS_ERR_ARG, "spatial_order must be 1 or 2");
    if (o->limiter != 0 && o->limiter != 1) return fail(GSIS_ERR_ARG, "limiter must be 0 or 1");
    if (!std::isfinite(o->cfl_p) || !std::isfinite(o->beta)) return fail(GSIS_ERR_ARG, "bad pseudo-time controls");
    return GSIS_OK;
}

int check_ws(void* ws, size_t have, size_t need)
{
    if (!ws) return fail(GSIS_ERR_WORKSPACE, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(GSIS_ERR_WORKSPACE, "workspace not 256-byte aligned");
    if (have < need) return fail(GSIS_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", have, need);
    return GSIS_OK;
}

// Host-side preparation of the plan: sizes, grids, sorted quadrature copy.
int prepare(Plan& P, const gsis_mesh* mesh, const gsis_quadrature* quad, const gsis_options* opt,
            const double* sa, const double* ss, const double* q, const double* inflow, cudaStream_t st)
{
    P.nx = mesh->nx;
    P.ny = mesh->ny;
    P.N = P.nx * P.ny;
    P.K = quad ? quad->K : 0;
    P.nb = (P.ny + 31) / 32;
    P.nbf = 2 * (P.nx + P.ny);
    P.fp32 = opt->precision == GSIS_FP32_SWEEP;
    P.scheme = opt->scheme;
    P.pt = (opt->cfl_p > 0.0 || opt->beta > 0.0) ? 1 : 0;
    P.tol = opt->tol;
    P.max_iter = opt->max_iter;
    P.fixed_iters = opt->fixed_iters;
    P.synth_rtol = opt->synth_rtol;
    P.synth_max_iter = opt->synth_max_iter;
    P.order = opt->spatial_order;
    P.limiter = opt->limiter;
    P.sigma_a = sa;
    P.sigma_s = ss;
    P.q = q;
    P.inflow = inflow;
    int dev = 0, clk_khz = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev));
    if (clk_khz <= 0) clk_khz = 2000000;
    P.wait_cycles = (long long)(opt->wait_limit_s * clk_khz * 1000.0);
    P.num_sms = device_sm_count();
    if (P.num_sms <= 0) return fail(GSIS_ERR_CUDA, "cannot query the device");
    CK(prepare_kernels(std::max(P.K, 1), P.fp32, P.pt));
    if (P.K > 0) {
        const int per_sm = std::max(1, sweep_max_active_blocks(P.fp32, P.pt));
        const long long units = (long long)P.K * P.nb;   // one unit per warp pair, all pairs resident
        P.sweep_grid = (int)std::max(1LL, std::min<long long>((long long)per_sm * P.num_sms, units));
    }
    P.mg.cluster = mg_cluster_size();
    P.red_grid = std::max(1, std::min({P.num_sms * 8, kMaxCgBlocks, (P.N + kRedBlock - 1) / kRedBlock}));

    CK(cudaMemsetAsync(P.status, 0, sizeof(Status), st));
    CK(cudaMemcpyAsync(const_cast<double*>(P.dx), mesh->dx, P.nx * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(const_cast<double*>(P.dy), mesh->dy, P.ny * sizeof(double), cudaMemcpyHostToDevice, st));
    if (P.K > 0) {
        const int K = P.K;
        std::vector<int> perm;
        perm.reserve(K);
        for (int qd = 0; qd < 4; ++qd)
            for (int k = 0; k < K; ++k) {
                const int kq = (quad->mu[k] < 0.0 ? 1 : 0) + (quad->eta[k] < 0.0 ? 2 : 0);
                if (kq == qd) perm.push_back(k);
            }
        std::vector<double> hq(6 * (size_t)K);
        std::vector<int> hi(3 * (size_t)K, -1);
        for (int s = 0; s < K; ++s) {
            hq[s] = quad->mu[perm[s]];
            hq[K + s] = quad->eta[perm[s]];
            hq[2 * K + s] = quad->w[perm[s]];
            hi[s] = perm[s];
            hi[K + perm[s]] = s;
        }
        for (int k = 0; k < K; ++k) {
            hq[3 * K + k] = quad->mu[k];
            hq[4 * K + k] = quad->eta[k];
            hq[5 * K + k] = quad->w[k];
        }
        // x-reflection pairs (mu, eta) <-> (-mu, eta) with equal weights (every
        // level-symmetric set): the moments then sum each pair once
        P.has_mpair = K % 2 == 0;
        {
            int np = 0;
            std::vector<char> used(K, 0);
            for (int k = 0; k < K && P.has_mpair; ++k) {
                if (used[k]) continue;
                if (!(quad->mu[k] > 0.0)) { P.has_mpair = 0; break; }
                int m = -1;
                for (int t = 0; t < K; ++t)
                    if (!used[t] && t != k && std::fabs(quad->mu[t] + quad->mu[k]) <= 1e-14 &&
                        quad->eta[t] == quad->eta[k] && quad->w[t] == quad->w[k]) { m = t; break; }
                if (m < 0) { P.has_mpair = 0; break; }
                used[k] = used[m] = 1;
                hi[2 * K + 2 * np] = k;
                hi[2 * K + 2 * np + 1] = m;
                ++np;
            }
        }
        CK(cudaMemcpyAsync(const_cast<double*>(P.qmu), hq.data(), hq.size() * sizeof(double),
                           cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(const_cast<int*>(P.perm), hi.data(), hi.size() * sizeof(int),
                           cudaMemcpyHostToDevice, st));
        // band hand-off rows start "unwritten" (all-ones bytes); each sweep
        // restores that state after consuming them
        CK(cudaMemsetAsync(P.edge, 0xff, (size_t)K * P.nb * P.nx * (P.fp32 ? sizeof(float) : sizeof(double)), st));
        CK(cudaStreamSynchronize(st));   // host staging vectors go out of scope
        TIMED(GSIS_KCLASS_SETUP, 1, launch_setup(P, st));
    }
    TIMED(GSIS_KCLASS_SETUP, P.fp32 ? 1 : 2, launch_cell_setup(P, opt->cfl_p, opt->beta, st));
    if (P.scheme == GSIS_SCHEME_GSIS || P.K == 0) {
        TIMED(GSIS_KCLASS_SETUP, mg_setup_launches(P), launch_mg_setup(P, st));
        CK(plan_synthetic(P));
    }
    return GSIS_OK;
}

int read_status(Status& S, const Plan& P, cudaStream_t st)
{
    CK(cudaMemcpyAsync(&S, P.status, sizeof(Status), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    prof_harvest();
    if (S.error & kErrBadInput)
        return fail(GSIS_ERR_ARG, "sigma_a, sigma_s must be >= 0 with sigma_t > 0; q and inflow finite");
    if (S.error & kErrTimeout)
        return fail(GSIS_ERR_DEVICE_TIMEOUT, "a device-side wait exceeded its bound");
    return GSIS_OK;
}

Sizes sizes_of(const gsis_mesh* m, const gsis_quadrature* q, const gsis_options* o)
{
    Sizes z{};
    z.nx = m->nx;
    z.ny = m->ny;
    z.K = q ? q->K : 0;
    z.fp32 = o->precision == GSIS_FP32_SWEEP;
    z.hist = std::max(o->max_iter, o->fixed_iters);
    z.order = o->spatial_order;
    return z;
}

gsis_options sweep_options(const gsis_options* o)
{
    gsis_options r = *o;
    r.cfl_p = 0.0;
    r.beta = 0.0;
    r.spatial_order = 1;
    return r;
}

Sizes sweep_sizes(const gsis_mesh* m, const gsis_quadrature* q, const gsis_options* o)
{
    const gsis_options r = sweep_options(o);
    return sizes_of(m, q, &r);
}

Sizes solve_sizes(const gsis_mesh* m, const gsis_quadrature* q, const gsis_options* o)
{
    Sizes z = sizes_of(m, q, o);
    z.ordsrc = (o->cfl_p > 0.0 || o->beta > 0.0) && o->spatial_order == 1;
    return z;
}

}  // namespace gsis

void gsis::set_last_error(int code, const char* msg)
{
    (void)code;
    g_last_error = msg ? msg : "";
}

namespace gsis {

bool uniform_spacing(const double* h, int n)
{
    for (int i = 1; i < n; ++i)
        if (!(std::fabs(h[i] - h[0]) <= 1e-12 * std::fabs(h[0]))) return false;
    return true;
}

// Sorted index (quadrant-major, as in prepare) of the reflected direction
// -Omega of every sorted direction; false if the set is not closed under
// the reflection with equal weights.
bool reflection_table(const gsis_quadrature* quad, std::vector<int>& refl)
{
    const int K = quad->K;
    std::vector<int> perm;
    perm.reserve(K);
    for (int qd = 0; qd < 4; ++qd)
        for (int k = 0; k < K; ++k) {
            const int kq = (quad->mu[k] < 0.0 ? 1 : 0) + (quad->eta[k] < 0.0 ? 2 : 0);
            if (kq == qd) perm.push_back(k);
        }
    refl.assign(K, -1);
    for (int s = 0; s < K; ++s) {
        const int k = perm[s];
        for (int t = 0; t < K; ++t) {
            const int m = perm[t];
            if (std::fabs(quad->mu[m] + quad->mu[k]) <= 1e-12 && std::fabs(quad->eta[m] + quad->eta[k]) <= 1e-12 &&
                std::fabs(quad->w[m] - quad->w[k]) <= 1e-12 * std::fabs(quad->w[k])) {
                refl[s] = t;
                break;
            }
        }
        if (refl[s] < 0) return false;
    }
    return true;
}

}  // namespace gsis

namespace {

cudaError_t launch_uw2_kinetic(Plan& P, cudaStream_t st)
{
    const cudaError_t e = launch_uw2_residual(P, st);
    return e != cudaSuccess ? e : launch_delta_sweep(P, st);
}

}  // namespace

extern "C" {

void gsis_default_options(gsis_options* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->scheme = GSIS_SCHEME_GSIS;
    o->precision = GSIS_FP64;
    o->tol = 1e-8;
    o->max_iter = 100000;
    o->fixed_iters = 0;
    o->synth_rtol = 1e-12;
    o->synth_max_iter = 20000;
    o->cfl_p = 0.0;
    o->beta = 0.0;
    o->check_every = 16;
    o->stall_window = 0;
    o->wait_limit_s = 2.0;
    o->spatial_order = 1;
    o->limiter = 0;
}

const char* gsis_status_string(int s)
{
    switch (s) {
        case GSIS_OK: return "ok";
        case GSIS_ERR_ARG: return "invalid argument";
        case GSIS_ERR_CUDA: return "CUDA error";
        case GSIS_ERR_MAXITER: return "maximum number of iterations reached";
        case GSIS_ERR_DIVERGED: return "iteration diverged";
        case GSIS_ERR_STALLED: return "iteration stalled";
        case GSIS_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
        case GSIS_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        default: return "unknown status";
    }
}

const char* gsis_last_error(void) { return g_last_error.c_str(); }

int gsis_last_solve_info(gsis_solve_info* out)
{
    if (!out) return GSIS_ERR_ARG;
    *out = g_last_info;
    return GSIS_OK;
}

int gsis_profile_enable(int enable)
{
    std::lock_guard<std::mutex> g(g_prof.mu);
    g_prof.on = enable != 0;
    for (auto& x : g_prof.st) x = gsis_kernel_stats{};
    g_prof.pending.clear();
    return GSIS_OK;
}

int gsis_profile_read(gsis_kernel_stats* out, int n)
{
    if (!out || n < 0) return GSIS_ERR_ARG;
    prof_harvest();
    std::lock_guard<std::mutex> g(g_prof.mu);
    for (int i = 0; i < n && i < GSIS_KCLASS_COUNT; ++i) out[i] = g_prof.st[i];
    return GSIS_OK;
}

int gsis_workspace_bytes(const gsis_mesh* mesh, const gsis_quadrature* quad, const gsis_options* opt,
                         size_t* bytes)
{
    g_last_error.clear();
    int rc;
    if ((rc = check_mesh(mesh)) || (quad && (rc = check_quad(quad))) || (rc = check_opt(opt))) return rc;
    if (!bytes) return fail(GSIS_ERR_ARG, "bytes is NULL");
    *bytes = layout(solve_sizes(mesh, quad, opt), nullptr, nullptr);
    return GSIS_OK;
}

int gsis_solve(const gsis_mesh* mesh, const gsis_quadrature* quad, const gsis_options* opt,
               const double* sigma_a, const double* sigma_s, const double* q, const double* inflow,
               double* rho, double* F, double* P_out, double* history, int* iters_out, double* err_out,
               void* workspace, size_t workspace_bytes, void* stream)
{
    g_last_error.clear();
    int rc;
    if ((rc = check_mesh(mesh)) || (rc = check_quad(quad)) || (rc = check_opt(opt))) return rc;
    if (!sigma_a || !sigma_s || !q || !rho || !F) return fail(GSIS_ERR_ARG, "a required device pointer is NULL");
    const Sizes z = solve_sizes(mesh, quad, opt);
    if ((rc = check_ws(workspace, workspace_bytes, layout(z, nullptr, nullptr)))) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Plan P{};
    layout(z, static_cast<char*>(workspace), &P);
    if ((rc = prepare(P, mesh, quad, opt, sigma_a, sigma_s, q, inflow, st))) return rc;
    TIMED(GSIS_KCLASS_SETUP, P.pt ? 4 : 3, launch_init_state(P, st));
    if (P.X || P.X_f) TIMED(GSIS_KCLASS_SETUP, 1, launch_ordinate_source(P, st));
    Status S{};
    if ((rc = read_status(S, P, st))) return rc;

    const bool gsis = opt->scheme == GSIS_SCHEME_GSIS;
    const int nmax = opt->fixed_iters > 0 ? opt->fixed_iters : opt->max_iter;
    double best = INFINITY;
    int since_best = 0;
    int launched = 0;
    while (launched < nmax) {
        const int batch = std::min(opt->check_every, nmax - launched);
        for (int b = 0; b < batch; ++b) {
            if (P.order == 2) {   // UW2 residual, then the first-order increment sweep
                TIMED(GSIS_KCLASS_SWEEP, 2, launch_uw2_kinetic(P, st));
            } else {
                TIMED(GSIS_KCLASS_SWEEP, 1, launch_sweep(P, st));
            }
            TIMED(GSIS_KCLASS_MOMENTS, P.order == 2 ? 2 : 1,
                  launch_moments_to(P, gsis, false, P.rho_h, nullptr, nullptr, false, P.fb, false, st));
            if (gsis) {
                TIMED(GSIS_KCLASS_HOT_RHS, 1, launch_hot_rhs(P, P.rho_h, P.Fx, P.Fy, P.fb, P.rho_m, st, true));
                TIMED(GSIS_KCLASS_SYNTH, 1, launch_synthetic_solve(P, P.rho_m, P.x, st));
                TIMED(GSIS_KCLASS_UPDATE, 1, launch_update(P, P.x, st));
            } else {
                TIMED(GSIS_KCLASS_UPDATE, 1, launch_update(P, P.rho_h, st));
            }
            // FP64 pseudo-time: the update also formed the next sweep's per-ordinate source
            if (P.X_f) TIMED(GSIS_KCLASS_UPDATE, 1, launch_ordinate_source(P, st));
        }
        launched += batch;
        if ((rc = read_status(S, P, st))) return rc;
        if (S.done) break;
        if (opt->stall_window > 0) {
            if (S.err < best) {
                best = S.err;
                since_best = 0;
            } else if (++since_best >= opt->stall_window) {
                break;
            }
        }
    }
    // outputs: rho^{m+1}; F and P of I^{m+1} from the intensities of the last sweep
    TIMED(GSIS_KCLASS_MOMENTS, P.order == 2 ? 2 : 1, launch_moments_to(P, true, P_out != nullptr, P.rho_h, F, P_out, gsis, P.fb, true, st));
    CK(cudaMemcpyAsync(rho, P.rho_m, (size_t)P.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if ((rc = read_status(S, P, st))) return rc;
    if (history && S.iter > 0)
        CK(cudaMemcpy(history, P.hist, (size_t)S.iter * sizeof(double), cudaMemcpyDeviceToHost));
    g_last_info.iters = S.iter;
    g_last_info.synth_inner_iters = S.synth_iters_total;
    g_last_info.err = S.err;
    g_last_info.synth_relres = S.synth_relres;
    if (iters_out) *iters_out = S.iter;
    if (err_out) *err_out = S.err;
    if (S.reason == kDiverged) return fail(GSIS_ERR_DIVERGED, "Err = %g after %d iterations", S.err, S.iter);
    if (S.reason == kConverged || S.reason == kFixedDone) return GSIS_OK;
    if (S.reason == kMaxIter) return fail(GSIS_ERR_MAXITER, "Err = %g after %d iterations", S.err, S.iter);
    return fail(GSIS_ERR_STALLED, "Err = %g did not decrease for %d checks", S.err, opt->stall_window);
}

int gsis_transport_sweep(const gsis_mesh* mesh, const gsis_quadrature* quad, const gsis_options* opt,
                         const double* sigma_a, const double* sigma_s, const double* q, const double* inflow,
                         const double* rho_in, double* rho_half, double* F_half, double* P_half,
                         double* bflux, void* workspace, size_t workspace_bytes, void* stream)
{
    g_last_error.clear();
    int rc;
    if ((rc = check_mesh(mesh)) || (rc = check_quad(quad)) || (rc = check_opt(opt))) return rc;
    if (!sigma_a || !sigma_s || !q || !rho_in || !rho_half || !F_half)
        return fail(GSIS_ERR_ARG, "a required device pointer is NULL");
    const gsis_options o = sweep_options(opt);
    const Sizes z = sweep_sizes(mesh, quad, opt);
    if ((rc = check_ws(workspace, workspace_bytes, layout(z, nullptr, nullptr)))) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Plan P{};
    layout(z, static_cast<char*>(workspace), &P);
    if ((rc = prepare(P, mesh, quad, &o, sigma_a, sigma_s, q, inflow, st))) return rc;
    TIMED(GSIS_KCLASS_SETUP, 1, launch_source_from(P, rho_in, st));
    TIMED(GSIS_KCLASS_SWEEP, 1, launch_sweep(P, st));
    TIMED(GSIS_KCLASS_MOMENTS, P.order == 2 ? 2 : 1, launch_moments_to(P, true, P_half != nullptr, rho_half, F_half, P_half, false,
                                                    bflux ? bflux : P.fb, true, st));
    return GSIS_OK;
}

int gsis_synthetic_step(const gsis_mesh* mesh, const gsis_options* opt, const double* sigma_a,
                        const double* sigma_s, const double* q, const double* rho_half, const double* F_half,
                        const double* bflux, const double* rho_guess, double* rho_out, double* hot,
                        double* rhs, int* synth_iters_out, void* workspace, size_t workspace_bytes,
                        void* stream)
{
    g_last_error.clear();
    int rc;
    if ((rc = check_mesh(mesh)) || (rc = check_opt(opt))) return rc;
    if (!sigma_a || !sigma_s || !q || !rho_half || !F_half || !bflux || !rho_out)
        return fail(GSIS_ERR_ARG, "a required device pointer is NULL");
    gsis_options o = *opt;
    o.cfl_p = 0.0;
    o.beta = 0.0;
    o.spatial_order = 1;
    const Sizes z = sizes_of(mesh, nullptr, &o);
    if ((rc = check_ws(workspace, workspace_bytes, layout(z, nullptr, nullptr)))) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Plan P{};
    layout(z, static_cast<char*>(workspace), &P);
    if ((rc = prepare(P, mesh, nullptr, &o, sigma_a, sigma_s, q, nullptr, st))) return rc;
    const double* guess = rho_guess ? rho_guess : rho_half;
    TIMED(GSIS_KCLASS_HOT_RHS, 2, launch_hot_rhs(P, rho_half, F_half, F_half + P.N, bflux, guess, st));
    TIMED(GSIS_KCLASS_SYNTH, 1, launch_synthetic_solve(P, guess, rho_out, st));
    if (hot) {
        CK(cudaMemcpyAsync(hot, P.hotx, (size_t)P.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(hot + P.N, P.hoty, (size_t)P.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    if (rhs) CK(cudaMemcpyAsync(rhs, P.b, (size_t)P.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    Status S{};
    if ((rc = read_status(S, P, st))) return rc;
    if (synth_iters_out) *synth_iters_out = S.synth_iters;
    return GSIS_OK;
}

int gsis_adjoint_workspace_bytes(const gsis_mesh* mesh, const gsis_quadrature* quad, const gsis_options* opt,
                                 size_t* bytes)
{
    g_last_error.clear();
    int rc;
    if ((rc = check_mesh(mesh)) || (rc = check_quad(quad)) || (rc = check_opt(opt))) return rc;
    if (!bytes) return fail(GSIS_ERR_ARG, "bytes is NULL");
    Sizes z = sizes_of(mesh, quad, opt);
    z.adjoint = 1;
    *bytes = layout(z, nullptr, nullptr);
    return GSIS_OK;
}

int gsis_adjoint(const gsis_mesh* mesh, const gsis_quadrature* quad, const gsis_options* opt,
                 const double* sigma_a, const double* sigma_s, const double* q, const double* inflow,
                 const double* rho_star, const double* dJ_drho, double* grad_sigma_a, double* grad_sigma_s,
                 int* iters_out, double* err_out, void* workspace, size_t workspace_bytes, void* stream)
{
    g_last_error.clear();
    int rc;
    if ((rc = check_mesh(mesh)) || (rc = check_quad(quad)) || (rc = check_opt(opt))) return rc;
    if (!sigma_a || !sigma_s || !q || !rho_star || !dJ_drho || !grad_sigma_a || !grad_sigma_s)
        return fail(GSIS_ERR_ARG, "a required device pointer is NULL");
    if (opt->scheme != GSIS_SCHEME_GSIS) return fail(GSIS_ERR_ARG, "the adjoint is that of the GSIS solution");
    if (opt->spatial_order != 1) return fail(GSIS_ERR_ARG, "the adjoint covers first-order upwind face values");
    if (opt->cfl_p > 0.0 || opt->beta > 0.0)
        return fail(GSIS_ERR_ARG, "the adjoint is that of the steady GSIS map without pseudo-time");
    if (!uniform_spacing(mesh->dx, mesh->nx) || !uniform_spacing(mesh->dy, mesh->ny))
        return fail(GSIS_ERR_ARG, "the adjoint needs a uniform mesh (transposed sweep = reflected sweep)");
    std::vector<int> refl;
    if (!reflection_table(quad, refl))
        return fail(GSIS_ERR_ARG, "the adjoint needs a quadrature closed under Omega -> -Omega with equal weights");
    Sizes z = sizes_of(mesh, quad, opt);
    z.adjoint = 1;
    if ((rc = check_ws(workspace, workspace_bytes, layout(z, nullptr, nullptr)))) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Plan P{};
    layout(z, static_cast<char*>(workspace), &P);
    if ((rc = prepare(P, mesh, quad, opt, sigma_a, sigma_s, q, inflow, st))) return rc;
    P.g = dJ_drho;
    CK(cudaMemcpyAsync(P.refl, refl.data(), refl.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    // kinetic step at rho*: I_k, rho_1/2, F, F_b
    CK(cudaMemcpyAsync(P.rho_m, rho_star, (size_t)P.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    TIMED(GSIS_KCLASS_SETUP, 1, launch_source_from(P, P.rho_m, st));
    TIMED(GSIS_KCLASS_SWEEP, 1, launch_sweep(P, st));
    TIMED(GSIS_KCLASS_MOMENTS, P.order == 2 ? 2 : 1, launch_moments_to(P, true, false, P.rho_h, nullptr, nullptr, false, P.fb, false, st));
    // lam = g (also the first right-hand side), nu = 0
    CK(cudaMemcpyAsync(P.lam, dJ_drho, (size_t)P.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(P.b, dJ_drho, (size_t)P.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(P.nu, 0, (size_t)P.N * sizeof(double), st));
    CK(cudaStreamSynchronize(st));   // the host table goes out of scope
    Status S{};
    if ((rc = read_status(S, P, st))) return rc;

    // transposed GSIS iteration lam = M^T lam + g
    auto pass = [&](bool update) -> int {
        TIMED(GSIS_KCLASS_HOT_RHS, 1, launch_synth_resid(P, P.b, P.nu, st));
        TIMED(GSIS_KCLASS_SYNTH, 1, launch_synthetic_solve(P, P.nu, P.x, st));
        TIMED(GSIS_KCLASS_HOT_RHS, 2, launch_adjoint_rhs(P, P.x, st));
        TIMED(GSIS_KCLASS_SWEEP, 1, launch_adjoint_sweep(P, st));
        if (update) TIMED(GSIS_KCLASS_UPDATE, 1, launch_adjoint_update(P, st));
        return GSIS_OK;
    };
    const int nmax = opt->fixed_iters > 0 ? opt->fixed_iters : opt->max_iter;
    int launched = 0;
    double best = INFINITY;
    int since_best = 0;
    bool stalled = false;
    while (launched < nmax) {
        const int batch = std::min(opt->check_every, nmax - launched);
        for (int b = 0; b < batch; ++b)
            if ((rc = pass(true))) return rc;
        launched += batch;
        if ((rc = read_status(S, P, st))) return rc;
        if (S.done) break;
        if (opt->stall_window > 0) {
            if (S.err < best) {
                best = S.err;
                since_best = 0;
            } else if (++since_best >= opt->stall_window) {
                stalled = true;
                break;
            }
        }
    }
    // nu and phi at the final lam, then the explicit derivative
    CK(cudaMemsetAsync(&P.status->done, 0, sizeof(int), st));
    if ((rc = pass(false))) return rc;
    TIMED(GSIS_KCLASS_UPDATE, 1, launch_adjoint_gradient(P, grad_sigma_a, grad_sigma_s, st));
    Status S2{};
    if ((rc = read_status(S2, P, st))) return rc;
    g_last_info.iters = S.iter;
    g_last_info.synth_inner_iters = S2.synth_iters_total;
    g_last_info.err = S.err;
    g_last_info.synth_relres = S2.synth_relres;
    if (iters_out) *iters_out = S.iter;
    if (err_out) *err_out = S.err;
    if (S.reason == kDiverged) return fail(GSIS_ERR_DIVERGED, "adjoint Err = %g after %d iterations", S.err, S.iter);
    if (S.reason == kConverged || S.reason == kFixedDone) return GSIS_OK;
    if (stalled) return fail(GSIS_ERR_STALLED, "adjoint Err = %g did not decrease for %d checks", S.err,
                             opt->stall_window);
    return fail(GSIS_ERR_MAXITER, "adjoint Err = %g after %d iterations", S.err, S.iter);
}

}  // extern "C"
