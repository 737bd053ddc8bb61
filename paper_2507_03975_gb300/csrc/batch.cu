// Batched solve of independent steady problems (gsis_solve_batch) and its
// autotuner (gsis_batch_autotune).
//
// Every problem keeps the workspace layout, preparation and iteration of a
// single gsis_solve; what the batch adds is the launch structure.  Each step
// of an iteration is one launch over all problems, driven by per-problem
// argument records that are built once and stay in device memory:
//   sweep      one persistent launch over the units (ordinate, band) of every
//              problem; a unit table lists the bands of all problems in the
//              tuned order (bands of one problem in upwind order);
//   moments    cell moments and boundary fluxes, blocks partitioned by problem;
//   hot / rhs  HoT and the synthetic right-hand side (per-problem reductions);
//   synthetic  the strip solver, one cluster per problem, one launch per
//              cluster size, the launches on concurrent branches;
//   update     Err, convergence decision and next source per problem.
// check_every iterations are captured once as a CUDA graph and replayed; the
// host reads all status blocks with one copy after each replay, and every
// launch skips the problems that have stopped.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "gsis.h"
#include "gsis_internal.cuh"
#include "host.h"

using namespace gsis;

namespace {

constexpr int kMaxBatch = 4096;
constexpr int kStalled = 5;   // host-set stop reason: Err stopped decreasing (per-problem stall window)

size_t al(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

// Device header of a batch workspace (byte offsets), followed by every
// problem's own gsis_solve workspace.
struct Header {
    size_t bstatus, statuses, sweep, seg_start, seg_prob, seg_band, mom, mom_bs, hot, hot_bs, rhs, rhs_bs, upd,
        upd_bs, ord, ord_bs, strip, total;
};

Header header_layout(int B, int nseg, int fp32)
{
    Header h{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += al(bytes);
        return o;
    };
    const size_t bs = (size_t)(B + 1) * sizeof(int);
    h.bstatus = take(sizeof(Status));
    h.statuses = take((size_t)B * sizeof(Status));
    h.sweep = take((size_t)B * sweep_batch_rec_bytes(fp32));
    h.seg_start = take((size_t)(nseg + 1) * sizeof(int));
    h.seg_prob = take((size_t)nseg * sizeof(int));
    h.seg_band = take((size_t)nseg * sizeof(int));
    h.mom = take((size_t)B * mom_batch_rec_bytes(fp32));
    h.mom_bs = take(bs);
    h.hot = take((size_t)B * hot_batch_rec_bytes());
    h.hot_bs = take(bs);
    h.rhs = take((size_t)B * rhs_batch_rec_bytes());
    h.rhs_bs = take(bs);
    h.upd = take((size_t)B * upd_batch_rec_bytes());
    h.upd_bs = take(bs);
    h.ord = take((size_t)B * ord_batch_rec_bytes());
    h.ord_bs = take(bs);
    h.strip = take((size_t)B * strip_batch_rec_bytes());
    h.total = off;
    return h;
}

struct Group {
    int cl;        // CTAs per cluster
    size_t bytes;  // dynamic shared memory (largest member)
    int first, n;  // records [first, first + n) of the strip table
};

struct Batch {
    int B = 0, nseg = 0, fp32 = 0, pt = 0, ordsrc = 0;
    bool gsis = false;
    char* base = nullptr;
    Header h{};
    std::vector<Plan> P;
    Status* bstatus = nullptr;
    Status* statuses = nullptr;
    BatchTables bt{};
    std::vector<Group> groups;
    std::vector<int> fallback;   // problems whose synthetic solve is launched on its own
};

int bands(const gsis_problem& p) { return (p.mesh.ny + 31) / 32; }

int check_problems(const gsis_problem* probs, int n, const gsis_options* opt, bool outputs)
{
    int rc;
    if ((rc = check_opt(opt))) return rc;
    if (opt->spatial_order != 1) return fail(GSIS_ERR_ARG, "the batched solve runs first-order upwind face values");
    if (!probs) return fail(GSIS_ERR_ARG, "probs is NULL");
    if (n < 1 || n > kMaxBatch) return fail(GSIS_ERR_ARG, "batch of %d problems out of range [1, %d]", n, kMaxBatch);
    for (int p = 0; p < n; ++p) {
        const gsis_problem& q = probs[p];
        if ((rc = check_mesh(&q.mesh)) || (rc = check_quad(&q.quad)))
            return fail(rc, "problem %d: %s", p, gsis_last_error());
        if (!q.sigma_a || !q.sigma_s || !q.q || (outputs && !q.rho))
            return fail(GSIS_ERR_ARG, "problem %d: a required device pointer is NULL", p);
    }
    return GSIS_OK;
}

int total_segments(const gsis_problem* probs, int n)
{
    long long s = 0;
    for (int p = 0; p < n; ++p) s += bands(probs[p]);
    return (int)s;
}

// A problem's arrays: gsis_solve's, except that FP64 pseudo-time sweeps keep
// forming src + shift I^m inside the batched sweep (the same bits as the
// single solve's per-ordinate source), so only FP32 plans get X.
Sizes batch_sizes(const gsis_problem& q, const gsis_options* opt)
{
    Sizes z = solve_sizes(&q.mesh, &q.quad, opt);
    if (!z.fp32) z.ordsrc = 0;
    return z;
}

size_t batch_bytes(const gsis_problem* probs, int n, const gsis_options* opt)
{
    size_t tot = header_layout(n, total_segments(probs, n), opt->precision == GSIS_FP32_SWEEP).total;
    for (int p = 0; p < n; ++p) tot += al(layout(batch_sizes(probs[p], opt), nullptr, nullptr));
    return tot;
}

// Carves the workspace and prepares every problem (set-up kernels, rho^0 = 0).
int batch_setup(Batch& b, const gsis_problem* probs, int n, const gsis_options* opt, void* ws, size_t bytes,
                cudaStream_t st)
{
    int rc;
    if ((rc = check_ws(ws, bytes, batch_bytes(probs, n, opt)))) return rc;
    b.B = n;
    b.nseg = total_segments(probs, n);
    b.fp32 = opt->precision == GSIS_FP32_SWEEP;
    b.gsis = opt->scheme == GSIS_SCHEME_GSIS;
    b.base = static_cast<char*>(ws);
    b.h = header_layout(n, b.nseg, b.fp32);
    b.bstatus = reinterpret_cast<Status*>(b.base + b.h.bstatus);
    b.statuses = reinterpret_cast<Status*>(b.base + b.h.statuses);
    b.P.assign(n, Plan{});
    size_t off = b.h.total;
    for (int p = 0; p < n; ++p) {
        const gsis_problem& q = probs[p];
        const Sizes z = batch_sizes(q, opt);
        layout(z, b.base + off, &b.P[p]);
        off += al(layout(z, nullptr, nullptr));
        b.P[p].status = b.statuses + p;   // all status blocks side by side: one read per check
        if ((rc = prepare(b.P[p], &q.mesh, &q.quad, opt, q.sigma_a, q.sigma_s, q.q, q.inflow, st)))
            return fail(rc, "problem %d: %s", p, gsis_last_error());
        // synthetic solves run on concurrent branches: no grid-wide (every-SM) solver here
        b.P[p].synth_grid = 0;
        CK(launch_init_state(b.P[p], st));
        if (b.P[p].X_f) CK(launch_ordinate_source(b.P[p], st));
    }
    b.pt = b.P[0].pt;
    b.ordsrc = b.P[0].X_f != nullptr;   // FP32 pseudo-time sweeps over per-ordinate sources
    CK(cudaMemsetAsync(b.bstatus, 0, sizeof(Status), st));
    return GSIS_OK;
}

// Restarts every problem from rho^0 = 0 (autotuner trials).
int batch_restart(Batch& b, cudaStream_t st)
{
    CK(cudaMemsetAsync(b.statuses, 0, (size_t)b.B * sizeof(Status), st));
    CK(cudaMemsetAsync(b.bstatus, 0, sizeof(Status), st));
    for (int p = 0; p < b.B; ++p) {
        CK(launch_init_state(b.P[p], st));
        if (b.P[p].X_f) CK(launch_ordinate_source(b.P[p], st));
    }
    return GSIS_OK;
}

// Strip-solver cluster of a problem under the tuning (0: its synthetic solve
// is launched on its own).
int choose_cluster(const Plan& P, int cells_per_cta, std::vector<char>& rec, size_t& bytes)
{
    if (cells_per_cta <= 0) {
        if (P.synth_cl > 0 && strip_batch_rec(P, P.synth_cl, rec.data(), &bytes)) return P.synth_cl;
        return 0;
    }
    for (int cl = 2; cl <= 16; cl *= 2) {
        if ((long long)P.N > (long long)cells_per_cta * cl && cl < 16) continue;
        if (cl > P.mg.cluster) break;
        if (strip_batch_rec(P, cl, rec.data(), &bytes)) return cl;
    }
    return 0;
}

// Builds the argument tables of one tuning in host memory and copies them
// into the workspace header.
int batch_tables(Batch& b, const gsis_batch_tuning& t, cudaStream_t st)
{
    const int B = b.B;
    const Header& h = b.h;
    std::vector<char> img(h.total - h.sweep, 0);
    auto at = [&](size_t off) { return img.data() + (off - h.sweep); };

    // sweep: records and unit segments in the tuned order
    const size_t srec = sweep_batch_rec_bytes(b.fp32);
    int maxK = 1, maxnb = 1;
    for (int p = 0; p < B; ++p) {
        sweep_batch_rec(b.P[p], at(h.sweep) + (size_t)p * srec);
        maxK = std::max(maxK, b.P[p].K);
        maxnb = std::max(maxnb, b.P[p].nb);
    }
    std::vector<int> ord(B);
    std::iota(ord.begin(), ord.end(), 0);
    const bool longest = t.sweep_order == GSIS_ORDER_LONGEST || t.sweep_order == GSIS_ORDER_BAND_LONGEST;
    const bool band_major = t.sweep_order == GSIS_ORDER_BAND || t.sweep_order == GSIS_ORDER_BAND_LONGEST;
    if (longest)
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
            return (long long)b.P[x].nb * (b.P[x].nx + 31) > (long long)b.P[y].nb * (b.P[y].nx + 31);
        });
    int* seg_start = reinterpret_cast<int*>(at(h.seg_start));
    int* seg_prob = reinterpret_cast<int*>(at(h.seg_prob));
    int* seg_band = reinterpret_cast<int*>(at(h.seg_band));
    int g = 0;
    long long u = 0;
    auto push = [&](int p, int band) {
        seg_start[g] = (int)u;
        seg_prob[g] = p;
        seg_band[g] = band;
        u += b.P[p].K;
        ++g;
    };
    if (band_major) {
        for (int band = 0; band < maxnb; ++band)
            for (int p : ord)
                if (band < b.P[p].nb) push(p, band);
    } else {
        for (int p : ord)
            for (int band = 0; band < b.P[p].nb; ++band) push(p, band);
    }
    if (g != b.nseg || u > 0x7fffffffLL) return fail(GSIS_ERR_ARG, "batch too large for one sweep launch");
    seg_start[g] = (int)u;

    // per-block tables
    auto blocks = [&](size_t rec_off, size_t rec_bytes, size_t bs_off, auto&& fill) {
        int* bs = reinterpret_cast<int*>(at(bs_off));
        long long tot = 0;
        for (int p = 0; p < B; ++p) {
            bs[p] = (int)tot;
            tot += fill(b.P[p], at(rec_off) + (size_t)p * rec_bytes);
        }
        bs[B] = (int)tot;
        return (int)tot;
    };
    const bool gsis = b.gsis;
    const int mom_blocks = blocks(h.mom, mom_batch_rec_bytes(b.fp32), h.mom_bs,
                                  [&](const Plan& P, void* o) { return mom_batch_rec(P, gsis, o); });
    const int hot_blocks = blocks(h.hot, hot_batch_rec_bytes(), h.hot_bs,
                                  [&](const Plan& P, void* o) { return hot_batch_rec(P, o); });
    const int rhs_blocks = blocks(h.rhs, rhs_batch_rec_bytes(), h.rhs_bs,
                                  [&](const Plan& P, void* o) { return rhs_batch_rec(P, o); });
    const int upd_blocks = blocks(h.upd, upd_batch_rec_bytes(), h.upd_bs,
                                  [&](const Plan& P, void* o) { return upd_batch_rec(P, gsis, o); });
    // FP32 pseudo-time: the next sweeps' per-ordinate sources after every update
    const int ord_blocks = b.ordsrc ? blocks(h.ord, ord_batch_rec_bytes(), h.ord_bs,
                                             [&](const Plan& P, void* o) { return ord_batch_rec(P, o); })
                                    : 0;

    // synthetic: problems grouped by cluster size, one table run per group
    b.groups.clear();
    b.fallback.clear();
    if (gsis) {
        const size_t rb = strip_batch_rec_bytes();
        std::vector<char> rec(rb);
        std::map<int, std::vector<std::pair<int, size_t>>> by_cl;
        for (int p = 0; p < B; ++p) {
            size_t bytes = 0;
            const int cl = choose_cluster(b.P[p], t.synth_cells_per_cta, rec, bytes);
            if (cl > 0) by_cl[cl].push_back({p, bytes});
            else b.fallback.push_back(p);
        }
        int first = 0;
        for (auto& kv : by_cl) {
            size_t bytes = 0;
            for (auto& m : kv.second) bytes = std::max(bytes, m.second);
            if (!prepare_strip_batch(kv.first, bytes)) {
                for (auto& m : kv.second) b.fallback.push_back(m.first);
                continue;
            }
            for (size_t i = 0; i < kv.second.size(); ++i) {
                size_t bb = 0;
                strip_batch_rec(b.P[kv.second[i].first], kv.first, at(h.strip) + (size_t)(first + i) * rb, &bb);
            }
            b.groups.push_back(Group{kv.first, bytes, first, (int)kv.second.size()});
            first += (int)kv.second.size();
        }
    }
    CK(cudaMemcpyAsync(b.base + h.sweep, img.data(), img.size(), cudaMemcpyHostToDevice, st));

    BatchTables& bt = b.bt;
    bt = BatchTables{};
    bt.B = B;
    bt.fp32 = b.fp32;
    bt.pt = b.pt;
    bt.with_F = gsis ? 1 : 0;
    bt.maxK = maxK;
    bt.status = b.bstatus;
    bt.wait_cycles = b.P[0].wait_cycles;
    bt.sweep = b.base + h.sweep;
    bt.seg_start = reinterpret_cast<const int*>(b.base + h.seg_start);
    bt.seg_prob = reinterpret_cast<const int*>(b.base + h.seg_prob);
    bt.seg_band = reinterpret_cast<const int*>(b.base + h.seg_band);
    bt.nseg = b.nseg;
    bt.ntasks = (int)u;
    const int per_sm = std::max(1, sweep_max_active_blocks(b.fp32, b.pt));
    bt.sweep_grid = (int)std::max(1LL, std::min<long long>((long long)per_sm * b.P[0].num_sms, u));
    bt.dynamic = t.sweep_dynamic ? 1 : 0;
    bt.mom = b.base + h.mom;
    bt.mom_bstart = reinterpret_cast<const int*>(b.base + h.mom_bs);
    bt.mom_blocks = mom_blocks;
    bt.hot = b.base + h.hot;
    bt.hot_bstart = reinterpret_cast<const int*>(b.base + h.hot_bs);
    bt.hot_blocks = hot_blocks;
    bt.rhs = b.base + h.rhs;
    bt.rhs_bstart = reinterpret_cast<const int*>(b.base + h.rhs_bs);
    bt.rhs_blocks = rhs_blocks;
    bt.upd = b.base + h.upd;
    bt.upd_bstart = reinterpret_cast<const int*>(b.base + h.upd_bs);
    bt.upd_blocks = upd_blocks;
    bt.ord = b.base + h.ord;
    bt.ord_bstart = reinterpret_cast<const int*>(b.base + h.ord_bs);
    bt.ord_blocks = ord_blocks;
    CK(cudaStreamSynchronize(st));   // the host image goes out of scope
    return GSIS_OK;
}

// Side streams of the synthetic step: one per strip-solver group, plus one
// for the problems solved on their own; the groups run concurrently.
struct Branches {
    std::vector<cudaStream_t> s;
    std::vector<cudaEvent_t> done;
    cudaEvent_t fork = nullptr;
    ~Branches()
    {
        for (cudaStream_t x : s) cudaStreamDestroy(x);
        for (cudaEvent_t x : done) cudaEventDestroy(x);
        if (fork) cudaEventDestroy(fork);
    }
};

int make_branches(const Batch& b, Branches& br)
{
    const int n = b.gsis ? (int)b.groups.size() + (b.fallback.empty() ? 0 : 1) : 0;
    if (n < 2) return GSIS_OK;
    CK(cudaEventCreateWithFlags(&br.fork, cudaEventDisableTiming));
    for (int i = 0; i < n; ++i) {
        cudaStream_t x = nullptr;
        cudaEvent_t e = nullptr;
        CK(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
        br.s.push_back(x);
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        br.done.push_back(e);
    }
    return GSIS_OK;
}

// The synthetic solves of all problems: group i on side stream i (or all on s).
cudaError_t enqueue_synthetic(const Batch& b, cudaStream_t s, const Branches& br)
{
    cudaError_t e;
    const bool fork = !br.s.empty();
    if (fork && (e = cudaEventRecord(br.fork, s)) != cudaSuccess) return e;
    auto side = [&](int k) { return fork ? br.s[k] : s; };
    auto begin = [&](int k) { return fork ? cudaStreamWaitEvent(br.s[k], br.fork, 0) : cudaSuccess; };
    auto end = [&](int k) {
        if (!fork) return cudaSuccess;
        const cudaError_t x = cudaEventRecord(br.done[k], br.s[k]);
        return x != cudaSuccess ? x : cudaStreamWaitEvent(s, br.done[k], 0);
    };
    const size_t rb = strip_batch_rec_bytes();
    int i = 0;
    for (const Group& g : b.groups) {
        if ((e = begin(i)) != cudaSuccess) return e;
        if ((e = launch_strip_batch(b.base + b.h.strip + (size_t)g.first * rb, g.n, g.cl, g.bytes, side(i))) !=
            cudaSuccess)
            return e;
        if ((e = end(i)) != cudaSuccess) return e;
        ++i;
    }
    if (!b.fallback.empty()) {
        if ((e = begin(i)) != cudaSuccess) return e;
        for (int p : b.fallback)
            if ((e = launch_synthetic_solve(b.P[p], b.P[p].rho_m, b.P[p].x, side(i))) != cudaSuccess) return e;
        if ((e = end(i)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// One iteration of every problem: the launches of gsis_solve's loop body, each
// over the whole batch.  ev (optional, 6 events): recorded before the sweep
// and after each class (sweep, moments, HoT / rhs, synthetic, update).
cudaError_t enqueue_iteration(const Batch& b, cudaStream_t s, const Branches& br, cudaEvent_t* ev = nullptr)
{
    cudaError_t e;
    auto mark = [&](int i) { return ev ? cudaEventRecord(ev[i], s) : cudaSuccess; };
    if ((e = mark(0)) != cudaSuccess) return e;
    if ((e = launch_sweep_batch(b.bt, s)) != cudaSuccess || (e = mark(1)) != cudaSuccess) return e;
    if ((e = launch_moments_batch(b.bt, s)) != cudaSuccess || (e = mark(2)) != cudaSuccess) return e;
    if (b.gsis) {
        if ((e = launch_hot_rhs_batch(b.bt, s)) != cudaSuccess || (e = mark(3)) != cudaSuccess) return e;
        if ((e = enqueue_synthetic(b, s, br)) != cudaSuccess) return e;
    } else if ((e = mark(3)) != cudaSuccess) {
        return e;
    }
    if ((e = mark(4)) != cudaSuccess) return e;
    if ((e = launch_update_batch(b.bt, s)) != cudaSuccess) return e;
    if (b.bt.ord_blocks > 0 && (e = launch_ordsrc_batch(b.bt, s)) != cudaSuccess) return e;
    return mark(5);
}

// Captures `iters` iterations as one graph (on a private stream: the caller's
// may be the legacy stream, which cannot capture).
int capture(const Batch& b, int iters, cudaGraphExec_t* exec)
{
    Branches br;
    int rc;
    if ((rc = make_branches(b, br))) return rc;
    cudaStream_t cs = nullptr;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int i = 0; i < iters && e == cudaSuccess; ++i) e = enqueue_iteration(b, cs, br);
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return fail(GSIS_ERR_CUDA, "capturing the batched iteration failed: %s", cudaGetErrorString(e));
    return GSIS_OK;
}

// Copies every status block back (synchronising st); maps device error bits.
int read_statuses(const Batch& b, std::vector<Status>& S, cudaStream_t st)
{
    S.resize(b.B + 1);
    CK(cudaMemcpyAsync(S.data(), b.statuses, (size_t)b.B * sizeof(Status), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&S[b.B], b.bstatus, sizeof(Status), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int p = 0; p <= b.B; ++p) {
        if (S[p].error & kErrBadInput)
            return fail(GSIS_ERR_ARG, "problem %d: sigma_a, sigma_s must be >= 0 with sigma_t > 0; q and inflow finite", p);
        if (S[p].error & kErrTimeout) return fail(GSIS_ERR_DEVICE_TIMEOUT, "a device-side wait exceeded its bound");
    }
    return GSIS_OK;
}

std::string signature(const gsis_problem* probs, int n, const gsis_options* opt)
{
    std::string s = std::to_string(opt->scheme) + "/" + std::to_string(opt->precision) + "/" +
                    std::to_string(opt->cfl_p > 0.0 || opt->beta > 0.0);
    for (int p = 0; p < n; ++p)
        s += ":" + std::to_string(probs[p].mesh.nx) + "x" + std::to_string(probs[p].mesh.ny) + "x" +
             std::to_string(probs[p].quad.K);
    return s;
}

std::mutex g_tune_mu;
std::map<std::string, gsis_batch_tuning> g_tuned;

int status_code(int reason)
{
    switch (reason) {
    case kConverged:
    case kFixedDone: return GSIS_OK;
    case kDiverged: return GSIS_ERR_DIVERGED;
    case kStalled: return GSIS_ERR_STALLED;
    default: return GSIS_ERR_MAXITER;
    }
}

}  // namespace

extern "C" {

void gsis_default_batch_tuning(gsis_batch_tuning* t)
{
    if (!t) return;
    t->sweep_order = GSIS_ORDER_LONGEST;
    t->sweep_dynamic = 1;
    t->synth_cells_per_cta = 0;
}

int gsis_batch_workspace_bytes(const gsis_problem* probs, int n, const gsis_options* opt, size_t* bytes)
{
    int rc;
    if ((rc = check_problems(probs, n, opt, false))) return rc;
    if (!bytes) return fail(GSIS_ERR_ARG, "bytes is NULL");
    *bytes = batch_bytes(probs, n, opt);
    return GSIS_OK;
}

int gsis_solve_batch(gsis_problem* probs, int n, const gsis_options* opt, const gsis_batch_tuning* tuning,
                     void* workspace, size_t workspace_bytes, void* stream)
{
    int rc;
    if ((rc = check_problems(probs, n, opt, true))) return rc;
    if (tuning && (tuning->sweep_order < 0 || tuning->sweep_order > GSIS_ORDER_BAND_LONGEST ||
                   tuning->synth_cells_per_cta < 0))
        return fail(GSIS_ERR_ARG, "bad tuning");
    gsis_batch_tuning t;
    gsis_default_batch_tuning(&t);
    if (tuning) {
        t = *tuning;
    } else {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tuned.find(signature(probs, n, opt));
        if (it != g_tuned.end()) t = it->second;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Batch b;
    if ((rc = batch_setup(b, probs, n, opt, workspace, workspace_bytes, st))) return rc;
    if ((rc = batch_tables(b, t, st))) return rc;
    std::vector<Status> S;
    if ((rc = read_statuses(b, S, st))) return rc;

    const int per_graph = std::max(1, opt->check_every);
    cudaGraphExec_t exec = nullptr;
    if ((rc = capture(b, per_graph, &exec))) return rc;
    const int nmax = opt->fixed_iters > 0 ? opt->fixed_iters : opt->max_iter;
    std::vector<double> best(n, INFINITY);
    std::vector<int> since(n, 0);
    int launched = 0;
    while (launched < nmax) {
        cudaError_t e = cudaGraphLaunch(exec, st);
        if (e != cudaSuccess) {
            cudaGraphExecDestroy(exec);
            return fail(GSIS_ERR_CUDA, "cudaGraphLaunch failed: %s", cudaGetErrorString(e));
        }
        launched += per_graph;
        if ((rc = read_statuses(b, S, st))) {
            cudaGraphExecDestroy(exec);
            return rc;
        }
        bool all = true;
        for (int p = 0; p < n; ++p) {
            if (S[p].done) continue;
            if (opt->stall_window > 0) {
                if (S[p].err < best[p]) {
                    best[p] = S[p].err;
                    since[p] = 0;
                } else if (++since[p] >= opt->stall_window) {
                    // stop this problem like gsis_solve stops a stalled solve
                    const int stop[2] = {1, kStalled};   // done, reason
                    static_assert(offsetof(Status, reason) == offsetof(Status, done) + sizeof(int), "layout");
                    e = cudaMemcpyAsync(&b.statuses[p].done, stop, sizeof stop, cudaMemcpyHostToDevice, st);
                    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                    if (e != cudaSuccess) {
                        cudaGraphExecDestroy(exec);
                        return fail(GSIS_ERR_CUDA, "stopping a stalled problem failed: %s", cudaGetErrorString(e));
                    }
                    S[p].done = 1;
                    S[p].reason = kStalled;
                    continue;
                }
            }
            all = false;
        }
        if (all) break;
    }
    cudaGraphExecDestroy(exec);
    // outputs: rho^{m+1}; F of I^{m+1} from the intensities of the last sweep
    for (int p = 0; p < n; ++p) {
        Plan& P = b.P[p];
        CK(launch_moments_to(P, true, false, P.rho_h, probs[p].F, nullptr, b.gsis, P.fb, true, st));
        CK(cudaMemcpyAsync(probs[p].rho, P.rho_m, (size_t)P.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    if ((rc = read_statuses(b, S, st))) return rc;
    int worst = GSIS_OK;
    for (int p = 0; p < n; ++p) {
        probs[p].iters = S[p].iter;
        probs[p].err = S[p].err;
        probs[p].status = status_code(S[p].reason);
        if (probs[p].status != GSIS_OK && worst == GSIS_OK) worst = probs[p].status;
    }
    if (worst != GSIS_OK) return fail(worst, "%s in at least one problem", gsis_status_string(worst));
    return GSIS_OK;
}

int gsis_batch_autotune(gsis_problem* probs, int n, const gsis_options* opt, int trial_iters,
                        gsis_batch_tuning* best, double* ms_per_iter, double* class_ms, void* workspace,
                        size_t workspace_bytes, void* stream)
{
    int rc;
    if ((rc = check_problems(probs, n, opt, false))) return rc;
    if (!best) return fail(GSIS_ERR_ARG, "best is NULL");
    if (trial_iters < 1 || trial_iters > 1000) return fail(GSIS_ERR_ARG, "trial_iters out of range [1, 1000]");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Batch b;
    if ((rc = batch_setup(b, probs, n, opt, workspace, workspace_bytes, st))) return rc;
    std::vector<gsis_batch_tuning> cand;
    for (int order = 0; order <= GSIS_ORDER_BAND_LONGEST; ++order)
        for (int dyn = 0; dyn <= 1; ++dyn)
            for (int cpc : {0, 4096, 16384}) {
                if (!b.gsis && cpc != 0) continue;
                cand.push_back(gsis_batch_tuning{order, dyn, cpc});
            }
    cudaEvent_t ev[6] = {};
    for (auto& x : ev) CK(cudaEventCreate(&x));
    struct Ev {
        cudaEvent_t* e;
        ~Ev()
        {
            for (int i = 0; i < 6; ++i) cudaEventDestroy(e[i]);
        }
    } ev_guard{ev};
    std::vector<Status> S;
    double best_ms = INFINITY;
    gsis_batch_tuning chosen = cand[0];
    for (const gsis_batch_tuning& t : cand) {
        cudaGraphExec_t exec = nullptr;
        if ((rc = batch_tables(b, t, st)) || (rc = batch_restart(b, st)) || (rc = capture(b, 1, &exec))) return rc;
        cudaError_t e = cudaGraphLaunch(exec, st);   // untimed first iteration
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
        for (int i = 0; i < trial_iters && e == cudaSuccess; ++i) e = cudaGraphLaunch(exec, st);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        cudaGraphExecDestroy(exec);
        if (e != cudaSuccess) return fail(GSIS_ERR_CUDA, "autotune trial failed: %s", cudaGetErrorString(e));
        if ((rc = read_statuses(b, S, st))) return rc;
        const double per = ms / trial_iters;
        if (per < best_ms) {
            best_ms = per;
            chosen = t;
        }
    }
    if (class_ms) {
        // per-class device time of the chosen tuning (launches bracketed by events)
        double acc[GSIS_KCLASS_COUNT] = {};
        if ((rc = batch_tables(b, chosen, st)) || (rc = batch_restart(b, st))) return rc;
        Branches br;
        if ((rc = make_branches(b, br))) return rc;
        cudaError_t e = enqueue_iteration(b, st, br);
        const int cls[5] = {GSIS_KCLASS_SWEEP, GSIS_KCLASS_MOMENTS, GSIS_KCLASS_HOT_RHS, GSIS_KCLASS_SYNTH,
                            GSIS_KCLASS_UPDATE};
        for (int i = 0; i < trial_iters && e == cudaSuccess; ++i) {
            e = enqueue_iteration(b, st, br, ev);
            if (e == cudaSuccess) e = cudaEventSynchronize(ev[5]);
            for (int c = 0; c < 5 && e == cudaSuccess; ++c) {
                float ms = 0.f;
                e = cudaEventElapsedTime(&ms, ev[c], ev[c + 1]);
                acc[cls[c]] += ms;
            }
        }
        if (e != cudaSuccess) return fail(GSIS_ERR_CUDA, "class timing failed: %s", cudaGetErrorString(e));
        for (int c = 0; c < GSIS_KCLASS_COUNT; ++c) class_ms[c] = acc[c] / trial_iters;
        if ((rc = read_statuses(b, S, st))) return rc;
    }
    *best = chosen;
    if (ms_per_iter) *ms_per_iter = best_ms;
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tuned[signature(probs, n, opt)] = chosen;
    return GSIS_OK;
}

}  // extern "C"
