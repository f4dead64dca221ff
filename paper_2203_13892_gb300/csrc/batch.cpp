// batch.cpp -- many independent simulations replayed as one CUDA graph, and the
// autotuner that picks the tile width of a plan by timing trial runs.
//
// A batch plans every circuit (uneven qubit counts and depths are fine), then
// captures all their launches once into a CUDA graph with one branch per
// circuit, so that small circuits run beside large ones and the host issues a
// single graph launch per replay.  Seeds live in device memory, so a replay with
// new seeds needs no re-capture.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "handles.h"

struct tqs_batch {
    std::vector<std::unique_ptr<tqs_plan>> plans;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaStream_t origin = nullptr;
    cudaEvent_t fork = nullptr, ev0 = nullptr, ev1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t *d_seeds = nullptr;
    uint64_t launches = 0;
    double alg_bytes = 0;

    ~tqs_batch()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        plans.clear();  // frees the plans' workspaces
        for (auto s : streams) cudaStreamDestroy(s);
        for (auto e : joins) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (origin) cudaStreamDestroy(origin);
        if (d_seeds) cudaFree(d_seeds);
    }
};

namespace tqs {

namespace {
std::mutex g_tune_mu;
std::map<uint64_t, uint32_t> g_tune_cache;

uint64_t shape_key(const tqs_circuit *c, const tqs_options &o, uint64_t shots)
{
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) {
        h ^= v;
        h *= 1099511628211ull;
    };
    mix(c->c.n);
    mix(c->c.gates.size());
    mix((uint64_t)o.prec);
    mix((uint64_t)o.mode);
    mix((uint64_t)o.part);
    mix((uint64_t)(o.flags & TQS_FLAG_FUSE));
    mix((uint64_t)(std::log2((double)shots) * 4));
    for (const auto &g : c->c.gates) {
        mix(g.kind);
        mix(g.q0);
        mix(g.q1);
    }
    return h;
}
}  // namespace

// Picks tile_qubits (how many qubits a tile pass holds: the split between the
// low, in-tile qubits and the high ones gathered per tile), for FP32 whether
// dense blocks are fused onto the tensor cores, and then the node batch (tree
// nodes per launch) for this circuit shape: each candidate runs the same tree on
// a few whole level-0 subtrees and the fastest per leaf wins.  The cache holds
// tile_qubits | (fuse << 8) | (batch << 16) (batch 0: the library's choice); a
// caller that set TQS_FLAG_FUSE keeps it, one that set batch keeps it.
tqs_status autotune(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, const tqs_options &o,
                    tqs_options &tuned)
{
    tuned = o;
    if (o.tile_qubits)
        return TQS_OK;  // the caller fixed it
    const uint64_t key = shape_key(c, o, shots);
    auto apply = [&](uint32_t v) {
        tuned.tile_qubits = v & 0xffu;
        if ((v >> 8) & 1u)
            tuned.flags |= TQS_FLAG_FUSE;
        if (!o.batch && (v >> 16))
            tuned.batch = v >> 16;
    };
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            apply(it->second);
            return TQS_OK;
        }
    }
    std::vector<uint64_t> arity;
    std::vector<uint32_t> split;
    std::string m = partition(c->c, nz->nz, shots, o, arity, split);
    if (!m.empty())
        return set_error(TQS_EINVAL, m);
    uint64_t below = 1;
    for (size_t i = 1; i < arity.size(); i++)
        below *= arity[i];
    const uint64_t roots = (shots + below - 1) / below;
    const uint64_t trial_roots = std::min<uint64_t>(roots, std::max<uint64_t>(1, 4096 / below));
    const uint64_t trial_shots = std::min<uint64_t>(shots, trial_roots * below);
    const uint32_t n = c->c.n;
    const bool may_fuse = o.prec == TQS_FP32 && !(o.flags & TQS_FLAG_FUSE);
    std::vector<uint32_t> cands;  // tile_qubits | (fuse << 8)
    if (o.prec == TQS_FP64)
        cands = {9, 10, 11, 12};
    else
        cands = {10, 11, 12, 13};
    if (may_fuse)
        for (uint32_t t : {11u, 12u})
            if (t <= n)
                cands.push_back(t | 0x100u);
    const uint32_t fuse_all = (o.flags & TQS_FLAG_FUSE) ? 0x100u : 0u;
    // one trial: the device time of two runs of the trial tree (the second kept)
    auto trial = [&](uint32_t cand, float &ms) -> tqs_status {
        tqs_options tr = o;
        tr.flags &= ~(TQS_FLAG_AUTOTUNE | TQS_FLAG_PROFILE);
        if ((cand >> 8) & 1u)
            tr.flags |= TQS_FLAG_FUSE;
        if (cand >> 16)
            tr.batch = cand >> 16;
        tr.part = TQS_PART_EXPLICIT;
        tr.k = (uint32_t)arity.size() - 1;
        tr.arity = arity.data();
        tr.split = split.data();
        tr.tile_qubits = cand & 0xffu;
        tr.workspace = nullptr;
        tr.workspace_bytes = o.workspace ? 0 : o.workspace_bytes;
        std::unique_ptr<tqs_plan> p;
        tqs_status st = make_plan(c, nz, trial_shots, tr, false, p);
        if (st != TQS_OK)
            return st;
        std::string err;
        for (int rep = 0; rep < 2; rep++) {
            st = p->dp.execute(rep, p->dp.d_counts_internal, true, err);
            if (st != TQS_OK)
                return set_error(st, err);
            cudaError_t e = cudaEventSynchronize(p->dp.ev1);
            if (e == cudaSuccess)
                e = cudaEventElapsedTime(&ms, p->dp.ev0, p->dp.ev1);
            if (e != cudaSuccess)
                return set_error(TQS_ECUDA, cuda_msg("autotune trial", (int)e));
        }
        return TQS_OK;
    };
    uint32_t best = 0;
    double best_t = 1e300;
    bool small_done = false;
    // first the tile width (and fusion) ...
    for (uint32_t cand : cands) {
        const uint32_t t = cand & 0xffu;
        if (t > n) {  // every width >= n gives the same single-tile plan
            if (small_done)
                continue;
            small_done = true;
        }
        float ms = 0;
        tqs_status st = trial(cand, ms);
        if (st != TQS_OK)
            return st;
        if (ms < best_t) {
            best_t = ms;
            best = cand | fuse_all;
        }
    }
    // ... then the node batch with that width (the library's default is the first candidate)
    if (!o.batch) {
        const uint32_t width = best & 0xffffu;
        for (uint32_t b : {32u, 64u, 128u, 512u}) {
            float ms = 0;
            tqs_status st = trial(width | (b << 16), ms);
            if (st != TQS_OK)
                return st;
            if (ms < best_t) {
                best_t = ms;
                best = width | (b << 16);
            }
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    apply(best);
    return TQS_OK;
}

}  // namespace tqs

namespace {
tqs_status fail_cuda(const char *what, cudaError_t e)
{
    return tqs::set_error(TQS_ECUDA, tqs::cuda_msg(what, (int)e));
}
}  // namespace

extern "C" {

tqs_status tqs_batch_create(size_t count, const tqs_circuit *const *circuits, const tqs_noise *const *noises,
                            const uint64_t *shots, const tqs_options *opts, tqs_batch **out)
{
    if (!out || !circuits || !noises || !shots || count == 0)
        return tqs::set_error(TQS_EINVAL, "batch needs count >= 1, circuits, noises, shots and out");
    tqs_options o;
    if (opts)
        o = *opts;
    else
        tqs_options_default(&o);
    if (o.workspace)
        return tqs::set_error(TQS_EINVAL, "a batch allocates its own workspaces; pass workspace = NULL");
    if (o.part == TQS_PART_EXPLICIT)
        return tqs::set_error(TQS_EINVAL, "a batch plans each circuit with DCP/UCP/XCP, not an explicit tree");
    o.flags &= ~TQS_FLAG_PROFILE;
    std::unique_ptr<tqs_batch> b(new (std::nothrow) tqs_batch());
    if (!b)
        return tqs::set_error(TQS_ENOMEM, "host allocation failed");
    cudaError_t e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
    if (e != cudaSuccess)
        return fail_cuda("cudaStreamCreate", e);
    // device memory is shared out in proportion to each circuit's state size
    size_t fr = 0, tot = 0;
    e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess)
        return fail_cuda("cudaMemGetInfo", e);
    double wsum = 0;
    for (size_t i = 0; i < count; i++) {
        if (!circuits[i] || !noises[i])
            return tqs::set_error(TQS_EINVAL, "NULL circuit or noise in the batch");
        wsum += std::ldexp(1.0, (int)circuits[i]->c.n);
    }
    const double budget = 0.7 * (double)fr;
    for (size_t i = 0; i < count; i++) {
        tqs_options oi = o;
        oi.stream = b->origin;
        oi.workspace = nullptr;
        oi.workspace_bytes = (size_t)(budget * std::ldexp(1.0, (int)circuits[i]->c.n) / wsum);
        std::unique_ptr<tqs_plan> p;
        // the batch's plans share the device and run concurrently: each keeps the
        // smaller launches of 2^16 tiles by default
        tqs_status st = tqs::make_plan(circuits[i], noises[i], shots[i], oi, false, p, 65536);
        if (st != TQS_OK)
            return st;
        b->plans.push_back(std::move(p));
    }
    e = cudaMalloc(&b->d_seeds, sizeof(uint64_t) * count);
    if (e != cudaSuccess)
        return fail_cuda("cudaMalloc(seeds)", e);
    b->streams.resize(count, nullptr);
    b->joins.resize(count, nullptr);
    for (size_t i = 0; i < count; i++) {
        if ((e = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking)) != cudaSuccess)
            return fail_cuda("cudaStreamCreate", e);
        if ((e = cudaEventCreateWithFlags(&b->joins[i], cudaEventDisableTiming)) != cudaSuccess)
            return fail_cuda("cudaEventCreate", e);
    }
    if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreate(&b->ev0)) != cudaSuccess || (e = cudaEventCreate(&b->ev1)) != cudaSuccess)
        return fail_cuda("cudaEventCreate", e);
    if (tqs::prepare_kernels() != 0)
        return fail_cuda("kernel attributes", cudaGetLastError());
    if ((e = cudaStreamSynchronize(b->origin)) != cudaSuccess)
        return fail_cuda("plan uploads", e);

    // capture: fork one branch per circuit from the origin stream, join back
    e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess)
        return fail_cuda("cudaStreamBeginCapture", e);
    cudaEventRecord(b->fork, b->origin);
    std::string err;
    tqs_status st = TQS_OK;
    for (size_t i = 0; i < count && st == TQS_OK; i++) {
        tqs::DevicePlan &dp = b->plans[i]->dp;
        cudaStreamWaitEvent(b->streams[i], b->fork, 0);
        dp.stream = b->streams[i];
        dp.seed_dev = b->d_seeds + i;
        st = dp.execute(0, dp.d_counts_internal, false, err);
        b->launches += dp.launches;
        b->alg_bytes += dp.alg_bytes;
        cudaEventRecord(b->joins[i], b->streams[i]);
        cudaStreamWaitEvent(b->origin, b->joins[i], 0);
    }
    cudaGraph_t g = nullptr;
    cudaError_t ec = cudaStreamEndCapture(b->origin, &g);
    if (st != TQS_OK) {
        if (g)
            cudaGraphDestroy(g);
        return tqs::set_error(st, err);
    }
    if (ec != cudaSuccess)
        return fail_cuda("cudaStreamEndCapture", ec);
    b->graph = g;
    if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess)
        return fail_cuda("cudaGraphInstantiate", e);
    *out = b.release();
    return TQS_OK;
}

tqs_status tqs_batch_execute(tqs_batch *b, const uint64_t *seeds, tqs_report *report)
{
    if (!b || !seeds)
        return tqs::set_error(TQS_EINVAL, "batch and seeds are required");
    const size_t count = b->plans.size();
    cudaError_t e = cudaMemcpyAsync(b->d_seeds, seeds, sizeof(uint64_t) * count, cudaMemcpyHostToDevice, b->origin);
    if (e == cudaSuccess)
        e = cudaEventRecord(b->ev0, b->origin);
    if (e == cudaSuccess)
        e = cudaGraphLaunch(b->exec, b->origin);
    if (e == cudaSuccess)
        e = cudaEventRecord(b->ev1, b->origin);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(b->origin);
    if (e != cudaSuccess)
        return fail_cuda("tqs_batch_execute", e);
    for (auto &p : b->plans) {
        std::string err;
        const tqs_status st = p->dp.check_device_error(err);
        if (st != TQS_OK)
            return tqs::set_error(st, err);
    }
    if (report) {
        float ms = 0;
        cudaEventElapsedTime(&ms, b->ev0, b->ev1);
        std::memset(report, 0, sizeof(*report));
        uint64_t shots = 0;
        for (auto &p : b->plans)
            shots += p->shots;
        report->shots_done = shots;
        report->kernel_launches = b->launches;
        report->kernel_ms = ms;
        report->shots_per_s = ms > 0 ? (double)shots / (ms * 1e-3) : 0;
        report->alg_bytes = b->alg_bytes;
        report->fid_norm = report->fid_s = std::nan("");
    }
    return TQS_OK;
}

tqs_status tqs_batch_counts(const tqs_batch *b, size_t i, uint64_t *counts)
{
    if (!b || !counts || i >= b->plans.size())
        return tqs::set_error(TQS_EINVAL, "batch index out of range or NULL counts");
    const tqs_plan &p = *b->plans[i];
    cudaError_t e = cudaMemcpy(counts, p.dp.d_counts_internal, sizeof(uint64_t) * ((size_t)1 << p.c.n),
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return fail_cuda("tqs_batch_counts", e);
    return TQS_OK;
}

const uint64_t *tqs_batch_device_counts(const tqs_batch *b, size_t i)
{
    if (!b || i >= b->plans.size())
        return nullptr;
    return (const uint64_t *)b->plans[i]->dp.d_counts_internal;
}

size_t tqs_batch_size(const tqs_batch *b) { return b ? b->plans.size() : 0; }

void tqs_batch_destroy(tqs_batch *b) { delete b; }

}  // extern "C"
