// executor.cpp -- device plan (workspace layout, uploads) and the tree traversal
// that launches the kernels: depth-first over the tree in chunks of `batch`
// sibling-consecutive node instances per level (Sec. 3.1), so the live state
// pool is one chunk per level.
#include <cuda_runtime.h>
#include <unistd.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <string>

#include "executor.h"
#include "specialize.h"

namespace tqs {

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

std::string cuda_msg(const char *what, int err)
{
    return std::string(what) + ": " + cudaGetErrorString((cudaError_t)err);
}

#define CK(call)                                                        \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) {                                        \
            err = cuda_msg(#call, (int)e_);                             \
            return TQS_ECUDA;                                           \
        }                                                               \
    } while (0)
#define CKL(call)                                                       \
    do {                                                                \
        int e_ = (call);                                                \
        launches++;                                                     \
        if (e_ != 0) {                                                  \
            err = cuda_msg(#call, e_);                                  \
            return TQS_ECUDA;                                           \
        }                                                               \
    } while (0)
// A launch of kernel class `kind` moving `bytes` algorithmic bytes, bracketed by
// CUDA events on the plan's stream when profiling.
#define CKP(kind, bytes, call)                                          \
    do {                                                                \
        cudaEvent_t a_ = nullptr, b_ = nullptr;                         \
        if (profiling()) {                                              \
            a_ = next_event();                                          \
            b_ = next_event();                                          \
            if (a_) cudaEventRecord(a_, stream);                        \
        }                                                               \
        CKL(call);                                                      \
        if (a_ && b_) {                                                 \
            cudaEventRecord(b_, stream);                                \
            prof.push_back(ProfRec{(kind), (bytes), a_, b_});           \
        }                                                               \
    } while (0)

DevicePlan::~DevicePlan() { release(); }

cudaEvent_t DevicePlan::next_event()
{
    if (ev_used == ev_pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess)
            return nullptr;
        ev_pool.push_back(e);
    }
    return ev_pool[ev_used++];
}

void DevicePlan::release()
{
    for (cudaEvent_t e : ev_pool)
        cudaEventDestroy(e);
    ev_pool.clear();
    if (own_ws && ws)
        cudaFree(ws);
    ws = nullptr;
    own_ws = false;
    if (host_pool)
        cudaFreeHost(host_pool);
    host_pool = host_pool_dev = nullptr;
    host_pool_bytes = 0;
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    ev0 = ev1 = nullptr;
}

// Whether level i keeps node states: every level but the leaves, whose last
// pass only measures (unless the leaves need several passes or are kept).
bool DevicePlan::level_needs_state(uint32_t i) const
{
    const PlanHost &H = host;
    const Level &lv = H.levels[i];
    const bool leaf = i + 1 == (uint32_t)H.levels.size();
    return !leaf || lv.pass_end - lv.pass_begin > 1 || store_leaves;
}

size_t DevicePlan::host_state_bytes(uint64_t B) const
{
    const PlanHost &H = host;
    const size_t sbytes = ((size_t)1 << H.n) * (H.prec == TQS_FP64 ? 16 : 8);
    size_t total = 0;
    for (uint32_t i = 0; i < (uint32_t)H.levels.size(); i++)
        if (((host_mask >> i) & 1u) && level_needs_state(i))
            total += align256(sbytes * B);
    return total;
}

// Workspace layout for `B` slots per level (the levels in host_mask keep their
// state slots in the host pool instead).
size_t DevicePlan::layout(uint64_t B, bool assign)
{
    const PlanHost &H = host;
    const uint32_t L = (uint32_t)H.levels.size();
    const size_t esz = H.prec == TQS_FP64 ? 16 : 8;
    const size_t sbytes = ((size_t)1 << H.n) * esz;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    size_t o_instr = take(2 * sizeof(Instr) * std::max<size_t>(H.instrs.size(), 1));
    size_t o_mats = take((H.prec == TQS_FP64 ? 8 : 4) * H.mats64.size());
    size_t o_pst = take(sizeof(uint32_t) * (H.passes.size() + L) + 64);
    size_t o_prog = take(std::max<size_t>(H.prog.size(), 16));
    size_t o_fused = take(sizeof(float) * std::max<size_t>(H.fused.size(), 4));
    size_t o_err = take(sizeof(unsigned int) * 4);
    size_t o_choff = take(sizeof(uint32_t) * std::max<size_t>(H.chunk_off.size(), 1));
    size_t o_fid = take(caller_counts ? 0 : sizeof(double) * (3 + 3 * 256));
    size_t o_perm = take(32);
    size_t o_counts = take(caller_counts ? 0 : sizeof(uint64_t) * ((size_t)1 << H.n));
    std::vector<size_t> o_state(L), o_noise(L), o_meta(L), h_state(L, 0);
    size_t hoff = 0;
    for (uint32_t i = 0; i < L; i++) {
        const Level &lv = H.levels[i];
        const uint32_t np = lv.pass_end - lv.pass_begin;
        if (!level_needs_state(i)) {
            o_state[i] = (size_t)-1;
        } else if ((host_mask >> i) & 1u) {
            o_state[i] = (size_t)-2;
            h_state[i] = hoff;
            hoff = align256(hoff + sbytes * B);
        } else {
            o_state[i] = take(sbytes * B);
        }
        o_noise[i] = take(std::max<size_t>(lv.g1 - lv.g0, 1) * B);
        o_meta[i] = take(sizeof(NodeMeta) * (np + 1) * B);
    }
    size_t o_S = take(sizeof(double) * H.samp.groups * B);
    // every pass of a plan has the same tile width, min(n, tile_max)
    const uint64_t tiles = (uint64_t)1 << (H.n - std::min<uint32_t>(H.n, H.tile_max));
    size_t o_ksum = take(H.kraus ? sizeof(double) * 4 * tiles * B : 0);
    size_t o_kmat = take(H.kraus ? esz * 8 * B : 0);
    if (assign) {
        char *b = (char *)ws;
        d_instr = (Instr *)(b + o_instr);
        d_pinstr = d_instr + std::max<size_t>(H.instrs.size(), 1);
        d_mats = b + o_mats;
        d_pass_start = (uint32_t *)(b + o_pst);
        d_prog = (uint8_t *)(b + o_prog);
        d_fused = (float *)(b + o_fused);
        d_err = (unsigned int *)(b + o_err);
        d_chunk_off = (uint32_t *)(b + o_choff);
        d_fid = caller_counts ? nullptr : (double *)(b + o_fid);
        d_perm = (uint8_t *)(b + o_perm);
        d_counts_internal = caller_counts ? nullptr : (unsigned long long *)(b + o_counts);
        state.assign(L, nullptr);
        noise.assign(L, nullptr);
        meta.assign(L, nullptr);
        for (uint32_t i = 0; i < L; i++) {
            if (o_state[i] == (size_t)-1)
                state[i] = nullptr;
            else if (o_state[i] == (size_t)-2)
                state[i] = (void *)((char *)host_pool_dev + h_state[i]);
            else
                state[i] = (void *)(b + o_state[i]);
            noise[i] = (uint8_t *)(b + o_noise[i]);
            meta[i] = (NodeMeta *)(b + o_meta[i]);
        }
        d_S = (double *)(b + o_S);
        d_ksum = H.kraus ? (double *)(b + o_ksum) : nullptr;
        d_kmat = H.kraus ? (void *)(b + o_kmat) : nullptr;
    }
    return off;
}

tqs_status DevicePlan::create(const tqs_options &o, std::string &err)
{
    opts = o;
    stream = (cudaStream_t)o.stream;
    const PlanHost &H = host;
    // state bytes of one slot across all levels (for the batch choice)
    size_t fixed = layout(0, false);
    size_t per_slot = layout(1, false) - fixed + 256 * 8;
    uint64_t maxact = 1;
    for (auto &lv : H.levels)
        maxact = std::max<uint64_t>(maxact, lv.active);
    const uint64_t tiles = (uint64_t)1 << (H.n - std::min<uint32_t>(H.n, H.tile_max));
    // nodes per launch: about 2^18 tiles per level launch, so that the
    // one-CTA-per-leaf sample pass and the per-level noise launches fill the GPU
    // (2^16 with the pool in pinned host memory, which grows with the batch);
    // the memory budget below caps it
    const uint64_t tiles_per_launch =
        launch_tiles ? launch_tiles : ((o.flags & TQS_FLAG_HOST_POOL) ? 65536 : 262144);
    uint64_t want = o.batch ? o.batch : std::max<uint64_t>(64, tiles_per_launch / tiles);
    want = std::min<uint64_t>(want, 65535);
    want = std::min<uint64_t>(want, maxact);
    const uint32_t L = (uint32_t)H.levels.size();
    host_mask = 0;
    if (o.flags & TQS_FLAG_HOST_POOL) {
        for (uint32_t i = 0; i < L; i++)
            if (level_needs_state(i))
                host_mask |= 1u << i;
        per_slot = layout(1, false) - fixed + 256 * 8;
    }
    size_t budget;
    if (o.workspace) {
        budget = o.workspace_bytes > fixed ? o.workspace_bytes - fixed : 0;
    } else {
        size_t fr = 0, tot = 0;
        CK(cudaMemGetInfo(&fr, &tot));
        budget = (size_t)(0.75 * (double)fr);
        if (o.workspace_bytes && o.workspace_bytes < budget)
            budget = o.workspace_bytes;  // a cap on what the library allocates
        budget = budget > fixed ? budget - fixed : 0;
    }
    if (!o.workspace && !(o.flags & TQS_FLAG_HOST_POOL)) {
        // one node per level does not fit in device memory: move the state slots
        // of the upper levels (the fewest node instances) to the host pool until
        // it does
        for (uint32_t i = 0; i < L && per_slot > budget; i++) {
            if (!level_needs_state(i))
                continue;
            host_mask |= 1u << i;
            per_slot = layout(1, false) - fixed + 256 * 8;
        }
    }
    uint64_t B = std::min<uint64_t>(want, budget / std::max<size_t>(per_slot, 1));
    if (B == 0) {
        err = "workspace too small for one node per level (" + std::to_string(fixed + per_slot) + " bytes needed)";
        return TQS_ENOMEM;
    }
    if (host_mask) {
        // the host pool takes at most a quarter of the host's physical memory
        const long pages = sysconf(_SC_PHYS_PAGES), psz = sysconf(_SC_PAGE_SIZE);
        const size_t cap = (pages > 0 && psz > 0) ? (size_t)pages * (size_t)psz / 4 : ((size_t)16 << 30);
        const size_t per_host = std::max<size_t>(host_state_bytes(1), 1);
        B = std::min<uint64_t>(B, std::max<uint64_t>(1, cap / per_host));
        host_pool_bytes = host_state_bytes(B);
        if (cudaHostAlloc(&host_pool, host_pool_bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            host_pool = nullptr;
            err = "pinned host allocation of " + std::to_string(host_pool_bytes) + " bytes for the state pool failed";
            host_pool_bytes = 0;
            return TQS_ENOMEM;
        }
        CK(cudaHostGetDevicePointer(&host_pool_dev, host_pool, 0));
    }
    batch = B;
    ws_bytes = layout(B, false);
    if (o.workspace) {
        if (((uintptr_t)o.workspace & 255) != 0) {
            err = "workspace must be 256-byte aligned";
            return TQS_EINVAL;
        }
        ws = o.workspace;
        own_ws = false;
    } else {
        CK(cudaMalloc(&ws, ws_bytes));
        own_ws = true;
    }
    layout(B, true);
    // uploads
    CK(cudaMemcpyAsync(d_instr, H.instrs.data(), sizeof(Instr) * H.instrs.size(), cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(d_pinstr, H.prog_instrs.data(), sizeof(Instr) * H.prog_instrs.size(), cudaMemcpyHostToDevice,
                       stream));
    if (H.prec == TQS_FP64)
        CK(cudaMemcpyAsync(d_mats, H.mats64.data(), 8 * H.mats64.size(), cudaMemcpyHostToDevice, stream));
    else
        CK(cudaMemcpyAsync(d_mats, H.mats32.data(), 4 * H.mats32.size(), cudaMemcpyHostToDevice, stream));
    // per level: where each pass starts in the level's instruction table (which
    // runs in pass order; npass + 1 entries), concatenated
    pst_host.clear();
    pst_off.clear();
    for (auto &lv : H.levels) {
        pst_off.push_back((uint32_t)pst_host.size());
        for (uint32_t p = lv.pass_begin; p < lv.pass_end; p++)
            pst_host.push_back(H.passes[p].ibeg - H.passes[lv.pass_begin].ibeg);
        pst_host.push_back(lv.g1 - lv.g0);
    }
    CK(cudaMemcpyAsync(d_pass_start, pst_host.data(), 4 * pst_host.size(), cudaMemcpyHostToDevice, stream));
    if (!H.prog.empty())
        CK(cudaMemcpyAsync(d_prog, H.prog.data(), H.prog.size(), cudaMemcpyHostToDevice, stream));
    if (!H.fused.empty())
        CK(cudaMemcpyAsync(d_fused, H.fused.data(), 4 * H.fused.size(), cudaMemcpyHostToDevice, stream));
    CK(cudaMemsetAsync(d_err, 0, 4 * sizeof(unsigned int), stream));
    CK(cudaMemcpyAsync(d_chunk_off, H.chunk_off.data(), 4 * H.chunk_off.size(), cudaMemcpyHostToDevice, stream));
    uint8_t perm[32] = {0};
    for (uint32_t q = 0; q < H.n; q++)
        perm[q] = H.levels.back().perm[q];
    CK(cudaMemcpyAsync(d_perm, perm, 32, cudaMemcpyHostToDevice, stream));
    CK(cudaEventCreate(&ev0));
    CK(cudaEventCreate(&ev1));
    CK(cudaStreamSynchronize(stream));
    if ((o.flags & TQS_FLAG_SPECIALIZE) && H.prec == TQS_FP32)
        return build_specialized(err);
    return TQS_OK;
}

// TQS_FLAG_SPECIALIZE: one kernel per pass program in the store mode, and the
// leaf's measuring modes for the last pass of the last level, compiled together.
tqs_status DevicePlan::build_specialized(std::string &err)
{
    // host allocations and compiler threads may throw: nothing crosses the C ABI
    try {
        return build_specialized_impl(err);
    } catch (const std::exception &e) {
        err = std::string("specialised pass kernels: ") + e.what();
        return TQS_ENOMEM;
    }
}

tqs_status DevicePlan::build_specialized_impl(std::string &err)
{
    const PlanHost &H = host;
    const std::string why = spec_available();
    if (!why.empty()) {
        err = "specialised pass kernels: " + why;
        return TQS_EUNSUPPORTED;
    }
    spec_fn.assign(H.passes.size() * 3, nullptr);
    std::vector<SpecSource> srcs;
    std::vector<size_t> slot;
    const uint32_t last = H.levels.empty() ? 0 : H.levels.back().pass_end - 1;
    for (uint32_t pi = 0; pi < (uint32_t)H.passes.size(); pi++) {
        for (int mode : {MODE_STORE, MODE_SUMS, MODE_SAMPLE}) {
            if (mode != MODE_STORE && pi != last)
                continue;
            SpecSource s;
            if (!spec_generate(H, H.passes[pi], mode, s).empty())
                continue;  // this pass keeps the generic kernel (fused tensor-core blocks)
            srcs.push_back(std::move(s));
            slot.push_back((size_t)pi * 3 + (size_t)mode);
        }
    }
    std::vector<void *> fns;
    const std::string m = spec_build(srcs, fns);
    if (!m.empty()) {
        err = m;
        return TQS_ECUDA;
    }
    for (size_t i = 0; i < slot.size(); i++)
        spec_fn[slot[i]] = fns[i];
    return TQS_OK;
}

// Index checks and fault injection of the options (TQS_FLAG_DEBUG_BOUNDS,
// TQS_FLAG_FAULT_TIMEOUT, TQS_FLAG_FAULT_BOUNDS) for one pass launch.
void DevicePlan::set_debug(PassLaunch &a) const
{
    a.dbg = 0;
    if (opts.flags & TQS_FLAG_DEBUG_BOUNDS)
        a.dbg |= kDbgBounds;
    if (opts.flags & TQS_FLAG_FAULT_TIMEOUT)
        a.dbg |= kDbgFaultTimeout;
    a.in_slots = batch;
    a.out_slots = batch;
    if ((opts.flags & TQS_FLAG_FAULT_BOUNDS) && batch > 0)
        a.out_slots = batch - 1;  // understated on purpose: the kernels' own check must catch it
}

void DevicePlan::set_kraus(PassLaunch &a, const Pass &ps) const
{
    a.kmat = d_kmat;
    a.ksum = ps.kout_gate >= 0 ? d_ksum : nullptr;
    a.knq = ps.kout_nq;
    a.kp0 = ps.kout_p0;
    a.kp1 = ps.kout_p1;
}

int DevicePlan::launch_choice(const Pass &ps, uint64_t lo, uint64_t nn, uint64_t seed, const uint64_t *sdev)
{
    const PlanHost &H = host;
    KrausLaunch k;
    std::memset(&k, 0, sizeof(k));
    k.ksum = d_ksum;
    k.tiles = (uint64_t)1 << (H.n - ps.t);
    k.kmat = d_kmat;
    k.fp64 = H.prec == TQS_FP64;
    k.node_lo = lo;
    k.nnodes = nn;
    k.seed_dev = sdev;
    k.seed = seed;
    k.gate = (uint32_t)ps.kout_gate;
    k.nq = ps.kout_nq;
    for (int c = 0; c < 4; c++)
        k.rate[c] = H.krate[ps.kout_nq == 2 ? 1 : 0][c];
    return launch_kraus(k, stream);
}

tqs_status DevicePlan::run_level(uint32_t i, uint64_t lo, uint64_t hi, std::vector<uint64_t> &plo,
                                 uint64_t seed, unsigned long long *counts, std::string &err)
{
    const PlanHost &H = host;
    const Level &lv = H.levels[i];
    const uint32_t L = (uint32_t)H.levels.size();
    const uint32_t np = lv.pass_end - lv.pass_begin;
    const uint64_t nn = hi - lo;
    plo[i] = lo;
    node_count[i] += nn;
    NoiseLaunch nl;
    nl.instr = d_instr + H.passes[lv.pass_begin].ibeg;
    nl.sites = lv.g1 - lv.g0;
    nl.pass_start = d_pass_start + pst_off[i];
    nl.npass = np;
    nl.node_lo = lo;
    nl.nnodes = nn;
    nl.parent_meta = i ? meta[i - 1] : nullptr;
    nl.parent_stride = i ? (H.levels[i - 1].pass_end - H.levels[i - 1].pass_begin + 1) : 0;
    nl.parent_end = i ? nl.parent_stride - 1 : 0;
    nl.parent_lo = i ? plo[i - 1] : 0;
    nl.arity = lv.arity;
    nl.noise_out = noise[i];
    nl.meta_out = meta[i];
    nl.seed = seed;
    nl.seed_dev = seed_dev;
    nl.thr1 = H.thr1;
    nl.thr2 = H.thr2;
    CKP(TQS_PROF_NOISE, (double)nn * (nl.sites + 8.0 * (np + 1)), launch_noise(nl, stream));
    const bool leaf = (i + 1 == L) && !store_leaves;
    const double sb = (double)((size_t)1 << H.n) * (H.prec == TQS_FP64 ? 16 : 8);
    for (uint32_t pl = 0; pl < np; pl++) {
        const Pass &ps = H.passes[lv.pass_begin + pl];
        PassLaunch a;
        std::memset(&a, 0, sizeof(a));
        a.fp64 = H.prec == TQS_FP64;
        a.in = pl == 0 ? (i ? state[i - 1] : nullptr) : state[i];
        a.in_from_parent = (pl == 0 && i > 0) ? 1 : 0;
        a.out = state[i];
        a.state_elems = (uint64_t)1 << H.n;
        a.node_lo = lo;
        a.parent_lo = i ? plo[i - 1] : 0;
        a.arity = lv.arity;
        a.nnodes = (uint32_t)nn;
        a.instr = d_pinstr;
        a.ibeg = ps.ibeg;
        a.iend = ps.iend;
        a.prog = d_prog;
        a.chunk_off = d_chunk_off;
        a.chunk_begin = ps.chunk_begin;
        a.chunk_end = ps.chunk_end;
        a.fused = ps.fused_blocks ? d_fused : nullptr;
        a.fused_k = ps.fused_blocks ? H.fused_k : 0;
        a.err = d_err;
        set_debug(a);
        a.n = H.n;
        a.t = ps.t;
        a.L = ps.L;
        std::memcpy(a.tbits, ps.tbits, sizeof(a.tbits));
        std::memcpy(a.hbits, ps.hbits, sizeof(a.hbits));
        a.mats = d_mats;
        a.noise = noise[i];
        a.sites = lv.g1 - lv.g0;
        a.meta = meta[i];
        a.meta_stride = np + 1;
        a.pass_local = pl;
        a.S = d_S;
        a.samp = &H.samp;
        a.counts = counts;
        a.seed = seed;
        a.seed_dev = seed_dev;
        a.thrm = H.thrm;
        // state bytes a pass must move: read its input (nothing when it starts
        // from |0...0>) and, unless it only measures, write its output
        set_kraus(a, ps);
        const double rd = a.in ? sb : 0.0;
        if (leaf && pl + 1 == np) {
            const double sums = 8.0 * (double)H.samp.groups;
            a.mode = MODE_SUMS;
            a.spec_fn = spec_for(lv.pass_begin + pl, a.mode);
            CKP(TQS_PROF_SUMS, (double)nn * (rd + sums), launch_pass(a, stream));
            a.mode = MODE_SAMPLE;
            a.spec_fn = spec_for(lv.pass_begin + pl, a.mode);
            const double blk = rd / (double)((uint64_t)1 << (H.n - ps.t));
            CKP(TQS_PROF_SAMPLE, (double)nn * (sums + blk), launch_pass(a, stream));
            alg_bytes += (double)nn * rd;
        } else {
            a.mode = MODE_STORE;
            a.spec_fn = spec_for(lv.pass_begin + pl, a.mode);
            CKP(TQS_PROF_STORE, (double)nn * (rd + sb), launch_pass(a, stream));
            alg_bytes += (double)nn * (rd + sb);
            if (ps.kout_gate >= 0)
                CKP(TQS_PROF_NOISE, (double)nn * 64.0, launch_choice(ps, lo, nn, seed, seed_dev));
        }
    }
    if (i + 1 < L) {
        const Level &ch = H.levels[i + 1];
        const uint64_t clo = lo * ch.arity;
        const uint64_t chi = std::min<uint64_t>(hi * ch.arity, ch.active);
        for (uint64_t c = clo; c < chi; c += batch) {
            tqs_status st = run_level(i + 1, c, std::min<uint64_t>(c + batch, chi), plo, seed, counts, err);
            if (st != TQS_OK)
                return st;
        }
    }
    return TQS_OK;
}

tqs_status DevicePlan::execute(uint64_t seed, unsigned long long *counts, bool timed, std::string &err)
{
    const PlanHost &H = host;
    const uint32_t L = (uint32_t)H.levels.size();
    launches = 0;
    alg_bytes = 0;
    ev_used = 0;
    prof.clear();
    node_count.assign(L, 0);
    std::vector<uint64_t> plo(L, 0);
    if (timed)
        CK(cudaEventRecord(ev0, stream));
    CKL(launch_fill_u64(counts, (uint64_t)1 << H.n, stream));
    const uint64_t roots = H.levels[0].active;
    for (uint64_t lo = 0; lo < roots; lo += batch) {
        tqs_status st = run_level(0, lo, std::min<uint64_t>(lo + batch, roots), plo, seed, counts, err);
        if (st != TQS_OK)
            return st;
    }
    if (timed)
        CK(cudaEventRecord(ev1, stream));
    return TQS_OK;
}

// State of one node along its ancestor chain (debug / ideal run): every level
// runs as a chunk of one node, all passes store.
tqs_status DevicePlan::run_chain(uint32_t level, uint64_t node, uint64_t seed, std::string &err)
{
    const PlanHost &H = host;
    std::vector<uint64_t> chain(level + 1);
    chain[level] = node;
    for (int i = (int)level; i > 0; i--)
        chain[i - 1] = chain[i] / H.levels[i].arity;
    std::vector<uint64_t> plo(H.levels.size(), 0);
    node_count.assign(H.levels.size(), 0);
    for (uint32_t i = 0; i <= level; i++) {
        // same as run_level but without descending and with stores only
        const Level &lv = H.levels[i];
        const uint32_t np = lv.pass_end - lv.pass_begin;
        plo[i] = chain[i];
        NoiseLaunch nl;
        nl.instr = d_instr + H.passes[lv.pass_begin].ibeg;
        nl.sites = lv.g1 - lv.g0;
        nl.pass_start = d_pass_start + pst_off[i];
        nl.npass = np;
        nl.node_lo = chain[i];
        nl.nnodes = 1;
        nl.parent_meta = i ? meta[i - 1] : nullptr;
        nl.parent_stride = i ? (H.levels[i - 1].pass_end - H.levels[i - 1].pass_begin + 1) : 0;
        nl.parent_end = i ? nl.parent_stride - 1 : 0;
        nl.parent_lo = i ? plo[i - 1] : 0;
        nl.arity = lv.arity;
        nl.noise_out = noise[i];
        nl.meta_out = meta[i];
        nl.seed = seed;
        nl.seed_dev = nullptr;
        nl.thr1 = H.thr1;
        nl.thr2 = H.thr2;
        CKL(launch_noise(nl, stream));
        for (uint32_t pl = 0; pl < np; pl++) {
            const Pass &ps = H.passes[lv.pass_begin + pl];
            PassLaunch a;
            std::memset(&a, 0, sizeof(a));
            a.mode = MODE_STORE;
            a.fp64 = H.prec == TQS_FP64;
            a.in = pl == 0 ? (i ? state[i - 1] : nullptr) : state[i];
            a.in_from_parent = (pl == 0 && i > 0) ? 1 : 0;
            a.out = state[i];
            a.state_elems = (uint64_t)1 << H.n;
            a.node_lo = chain[i];
            a.parent_lo = i ? plo[i - 1] : 0;
            a.arity = lv.arity;
            a.nnodes = 1;
            a.instr = d_pinstr;
            a.ibeg = ps.ibeg;
            a.iend = ps.iend;
            a.prog = d_prog;
            a.chunk_off = d_chunk_off;
            a.chunk_begin = ps.chunk_begin;
            a.chunk_end = ps.chunk_end;
            a.fused = ps.fused_blocks ? d_fused : nullptr;
            a.fused_k = ps.fused_blocks ? H.fused_k : 0;
            a.err = d_err;
            set_debug(a);
            a.n = H.n;
            a.t = ps.t;
            a.L = ps.L;
            std::memcpy(a.tbits, ps.tbits, sizeof(a.tbits));
            std::memcpy(a.hbits, ps.hbits, sizeof(a.hbits));
            a.mats = d_mats;
            a.noise = noise[i];
            a.sites = lv.g1 - lv.g0;
            a.meta = meta[i];
            a.meta_stride = np + 1;
            a.pass_local = pl;
            a.seed = seed;
            set_kraus(a, ps);
            a.spec_fn = spec_for(lv.pass_begin + pl, MODE_STORE);
            CKL(launch_pass(a, stream));
            if (ps.kout_gate >= 0)
                CKL(launch_choice(ps, chain[i], 1, seed, nullptr));
        }
    }
    return TQS_OK;
}

tqs_status DevicePlan::check_device_error(std::string &err)
{
    unsigned int h[3] = {0, 0, 0};
    CK(cudaMemcpyAsync(h, d_err, sizeof(h), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    if (h[0]) {
        CK(cudaMemsetAsync(d_err, 0, 4 * sizeof(unsigned int), stream));
        CK(cudaStreamSynchronize(stream));
        if (h[0] & 2u) {
            err = "internal: a fused-gate record reached a kernel built without the tensor-core path";
            return TQS_ECUDA;
        }
        if (h[0] & 4u) {
            static const char *what[] = {"?", "output slot", "input slot", "tile width", "tile bit",
                                         "outside-tile bit"};
            err = std::string("device index check failed: ") + what[h[1] < 6 ? h[1] : 0] + " " +
                  std::to_string(h[2]) + " out of range; the access was skipped";
            return TQS_EBOUNDS;
        }
        err = "a bounded tensor-core wait gave up (device error word " + std::to_string(h[0]) + ")";
        return TQS_ETIMEOUT;
    }
    return TQS_OK;
}

}  // namespace tqs
