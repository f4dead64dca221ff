// capi.cpp -- the extern "C" boundary declared in include/tqs.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <limits>
#include <memory>
#include <new>
#include <string>

#include "executor.h"
#include "handles.h"
#include "specialize.h"

namespace {
thread_local std::string g_err;

tqs_status fail(tqs_status s, const std::string &m)
{
    g_err = m;
    return s;
}

tqs_status from_msg(const std::string &m, tqs_status kind = TQS_EINVAL)
{
    if (m.empty())
        return TQS_OK;
    if (m.rfind("UNSUPPORTED:", 0) == 0)
        return fail(TQS_EUNSUPPORTED, m.substr(12));
    return fail(kind, m);
}

tqs_options opts_or_default(const tqs_options *o)
{
    tqs_options d;
    if (o)
        return *o;
    tqs_options_default(&d);
    return d;
}

tqs_status make_plan_once(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, const tqs_options &o,
                          bool store_leaves, std::unique_ptr<tqs_plan> &out, uint64_t launch_tiles = 0)
{
    if (!c || !nz)
        return fail(TQS_EINVAL, "circuit and noise handles are required");
    if (shots == 0)
        return fail(TQS_EINVAL, "shots must be >= 1");
    if (o.prec != TQS_FP32 && o.prec != TQS_FP64)
        return fail(TQS_EINVAL, "unknown precision");
    std::unique_ptr<tqs_plan> p(new (std::nothrow) tqs_plan());
    if (!p)
        return fail(TQS_ENOMEM, "host allocation failed");
    p->c = c->c;
    p->nz = nz->nz;
    p->shots = shots;
    tqs_status st = from_msg(tqs::partition(p->c, p->nz, shots, o, p->arity, p->split));
    if (st != TQS_OK)
        return st;
    st = from_msg(tqs::build_plan(p->c, p->nz, shots, o, p->arity, p->split, p->dp.host));
    if (st != TQS_OK)
        return st;
    p->dp.store_leaves = store_leaves;
    p->dp.launch_tiles = launch_tiles;
    std::string err;
    st = p->dp.create(o, err);
    if (st != TQS_OK)
        return fail(st, err);
    out = std::move(p);
    return TQS_OK;
}

void fill_report(const tqs_plan *p, double ms, tqs_report *r)
{
    const tqs::PlanHost &H = p->dp.host;
    std::memset(r, 0, sizeof(*r));
    r->shots_done = p->shots;
    r->levels = (uint32_t)H.levels.size();
    double inst = 0;
    for (uint32_t i = 0; i < r->levels; i++) {
        r->arity[i] = H.levels[i].arity;
        r->split[i] = H.levels[i].g0;
        r->node_instances[i] = i < p->dp.node_count.size() ? p->dp.node_count[i] : 0;
        r->passes[i] = H.levels[i].pass_end - H.levels[i].pass_begin;
        for (uint32_t q = H.levels[i].pass_begin; q < H.levels[i].pass_end; q++)
            r->fused_blocks[i] += H.passes[q].fused_blocks;
        inst += (double)r->node_instances[i];
    }
    r->split[r->levels] = H.levels.back().g1;
    r->kernel_launches = p->dp.launches;
    r->kernel_ms = ms;
    r->shots_per_s = ms > 0 ? (double)p->shots / (ms * 1e-3) : 0.0;
    r->alg_bytes = p->dp.alg_bytes;
    r->fid_norm = std::numeric_limits<double>::quiet_NaN();
    r->fid_s = std::numeric_limits<double>::quiet_NaN();
    r->theo_speedup = inst > 0 ? (double)r->levels * (double)p->shots / inst : 0.0;
    for (const auto &pr : p->dp.prof) {
        float t = 0;
        if (cudaEventElapsedTime(&t, pr.a, pr.b) != cudaSuccess)
            continue;
        r->prof_launches[pr.kind] += 1;
        r->prof_ms[pr.kind] += t;
        r->prof_bytes[pr.kind] += pr.bytes;
    }
}

// Normalised fidelity of the device histogram against a noiseless FP64 run.
tqs_status fidelity(const tqs_circuit *c, uint64_t shots, const unsigned long long *d_counts,
                    cudaStream_t stream, double *F, double *Fs)
{
    tqs_noise quiet;
    quiet.nz = {0.0, 0.0, 0.0};
    tqs_options o;
    tqs_options_default(&o);
    o.mode = TQS_MODE_BASELINE;
    o.prec = TQS_FP64;
    o.stream = stream;
    o.batch = 1;
    std::unique_ptr<tqs_plan> ip;
    tqs_status st = make_plan_once(c, &quiet, 1, o, true, ip);
    if (st != TQS_OK)
        return st;
    std::string err;
    st = ip->dp.run_chain(0, 0, 0, err);
    if (st != TQS_OK)
        return fail(st, err);
    int e = tqs::launch_fidelity(ip->dp.state[0], 1, d_counts, c->c.n, ip->dp.d_perm, shots, ip->dp.d_fid, stream);
    if (e)
        return fail(TQS_ECUDA, tqs::cuda_msg("fidelity kernels", e));
    double h[3];
    cudaError_t ce = cudaMemcpyAsync(h, ip->dp.d_fid, sizeof(h), cudaMemcpyDeviceToHost, stream);
    if (ce == cudaSuccess)
        ce = cudaStreamSynchronize(stream);
    if (ce != cudaSuccess)
        return fail(TQS_ECUDA, tqs::cuda_msg("fidelity readback", (int)ce));
    const double fs = h[0] * h[0], fu = h[1] * h[1];
    *Fs = fs;
    *F = std::fabs(1.0 - fu) < 1e-12 ? std::numeric_limits<double>::quiet_NaN() : (fs - fu) / (1.0 - fu);
    return TQS_OK;
}
}  // namespace

tqs_status tqs::set_error(tqs_status s, const std::string &msg) { return fail(s, msg); }

tqs_status tqs::make_plan(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, const tqs_options &o,
                          bool store_leaves, std::unique_ptr<tqs_plan> &out, uint64_t launch_tiles)
{
    if (!(o.flags & TQS_FLAG_AUTOTUNE) || store_leaves)
        return make_plan_once(c, nz, shots, o, store_leaves, out, launch_tiles);
    tqs_options tuned = o;
    tqs_status st = tqs::autotune(c, nz, shots, o, tuned);
    if (st != TQS_OK)
        return st;
    tuned.flags &= ~TQS_FLAG_AUTOTUNE;
    return make_plan_once(c, nz, shots, tuned, store_leaves, out, launch_tiles);
}

extern "C" {

int tqs_abi_version(void) { return TQS_ABI_VERSION; }

const char *tqs_last_error(void) { return g_err.c_str(); }

void tqs_options_default(tqs_options *o)
{
    if (!o)
        return;
    std::memset(o, 0, sizeof(*o));
    o->mode = TQS_MODE_TREE;
    o->prec = TQS_FP32;
    o->part = TQS_PART_DCP;
    o->z = 1.96;
    o->eps = 0.05;
    o->copy_gates = 10;
}

tqs_status tqs_circuit_create(uint32_t n_qubits, const tqs_gate *gates, size_t n_gates, tqs_circuit **out)
{
    if (!out)
        return fail(TQS_EINVAL, "out is NULL");
    std::unique_ptr<tqs_circuit> c(new (std::nothrow) tqs_circuit());
    if (!c)
        return fail(TQS_ENOMEM, "host allocation failed");
    std::string m = tqs::validate_and_build_circuit(n_qubits, gates, n_gates, c->c);
    if (!m.empty())
        return fail(TQS_EINVAL, m);
    *out = c.release();
    return TQS_OK;
}

void tqs_circuit_destroy(tqs_circuit *c) { delete c; }

tqs_status tqs_noise_model(double p1, double p2, double pm, tqs_noise **out)
{
    if (!out)
        return fail(TQS_EINVAL, "out is NULL");
    for (double p : {p1, p2, pm})
        if (!(p >= 0.0 && p <= 1.0))
            return fail(TQS_EINVAL, "probabilities must lie in [0, 1]");
    tqs_noise *n = new (std::nothrow) tqs_noise();
    if (!n)
        return fail(TQS_ENOMEM, "host allocation failed");
    n->nz.p1 = p1;
    n->nz.p2 = p2;
    n->nz.pm = pm;
    *out = n;
    return TQS_OK;
}

tqs_status tqs_noise_model_ex(const tqs_noise_params *q, tqs_noise **out)
{
    if (!out || !q)
        return fail(TQS_EINVAL, "params and out are required");
    for (double p : {q->p1, q->p2, q->pm, q->ad_gamma, q->pd_lambda})
        if (!(p >= 0.0 && p <= 1.0))
            return fail(TQS_EINVAL, "probabilities and damping rates must lie in [0, 1]");
    for (double t : {q->t1, q->t2, q->time_1q, q->time_2q})
        if (!(t >= 0.0) || !std::isfinite(t))
            return fail(TQS_EINVAL, "times must be finite and >= 0");
    tqs::Noise nz;
    nz.p1 = q->p1;
    nz.p2 = q->p2;
    nz.pm = q->pm;
    nz.ad = q->ad_gamma;
    nz.pd = q->pd_lambda;
    if (q->t1 > 0.0) {
        if (!(q->t2 > 0.0 && q->t2 <= 2.0 * q->t1))
            return fail(TQS_EINVAL, "thermal relaxation needs 0 < T2 <= 2 T1");
        // population decay exp(-t/T1) and coherence decay exp(-t/T2) as amplitude
        // damping followed by phase damping
        auto pair = [&](double t, double &g, double &l) {
            g = 1.0 - std::exp(-t / q->t1);
            l = 1.0 - std::exp(t / q->t1 - 2.0 * t / q->t2);
            if (l < 0.0)
                l = 0.0;
        };
        pair(q->time_1q, nz.tr_g1, nz.tr_l1);
        pair(q->time_2q, nz.tr_g2, nz.tr_l2);
    }
    tqs_noise *n = new (std::nothrow) tqs_noise();
    if (!n)
        return fail(TQS_ENOMEM, "host allocation failed");
    n->nz = nz;
    *out = n;
    return TQS_OK;
}

void tqs_noise_destroy(tqs_noise *nz) { delete nz; }

tqs_status tqs_partition(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, const tqs_options *opts,
                         uint32_t *levels_out, uint64_t *arity_out, uint32_t *split_out)
{
    if (!c || !nz || !levels_out || !arity_out || !split_out)
        return fail(TQS_EINVAL, "NULL argument");
    tqs_options o = opts_or_default(opts);
    std::vector<uint64_t> arity;
    std::vector<uint32_t> split;
    tqs_status st = from_msg(tqs::partition(c->c, nz->nz, shots, o, arity, split));
    if (st != TQS_OK)
        return st;
    *levels_out = (uint32_t)arity.size();
    for (size_t i = 0; i < arity.size(); i++)
        arity_out[i] = arity[i];
    for (size_t i = 0; i < split.size(); i++)
        split_out[i] = split[i];
    return TQS_OK;
}

tqs_status tqs_debug_plan_order(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, const tqs_options *opts,
                                uint32_t *order_out, uint32_t *pass_out, uint32_t *tile_out, uint32_t *npasses_out)
{
    if (!c || !nz || !order_out || !pass_out || !npasses_out)
        return fail(TQS_EINVAL, "NULL argument");
    if (shots == 0)
        return fail(TQS_EINVAL, "shots must be >= 1");
    tqs_options o = opts_or_default(opts);
    std::vector<uint64_t> arity;
    std::vector<uint32_t> split;
    tqs_status st = from_msg(tqs::partition(c->c, nz->nz, shots, o, arity, split));
    if (st != TQS_OK)
        return st;
    tqs::PlanHost H;
    st = from_msg(tqs::build_plan(c->c, nz->nz, shots, o, arity, split, H));
    if (st != TQS_OK)
        return st;
    size_t k = 0;
    for (uint32_t q = 0; q < (uint32_t)H.passes.size(); q++) {
        const tqs::Pass &ps = H.passes[q];
        for (uint32_t i = ps.ibeg; i < ps.iend; i++, k++) {
            order_out[k] = H.prog_instrs[i].gate;
            pass_out[k] = q;
        }
        if (tile_out) {
            uint32_t m = 0;
            for (uint32_t j = 0; j < ps.t; j++)
                m |= 1u << ps.tbits[j];
            tile_out[q] = m;
        }
    }
    *npasses_out = (uint32_t)H.passes.size();
    return TQS_OK;
}

static tqs_status debug_spec_check(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, const tqs_options *opts,
                                   uint32_t *nkernels_out, uint64_t *src_bytes_out)
{
    if (!c || !nz || !nkernels_out)
        return fail(TQS_EINVAL, "NULL argument");
    if (shots == 0)
        return fail(TQS_EINVAL, "shots must be >= 1");
    tqs_options o = opts_or_default(opts);
    if (o.prec != TQS_FP32)
        return fail(TQS_EINVAL, "specialised pass kernels are for FP32 plans");
    const std::string why = tqs::spec_available(false);
    if (!why.empty())
        return fail(TQS_EUNSUPPORTED, why);
    std::vector<uint64_t> arity;
    std::vector<uint32_t> split;
    tqs_status st = from_msg(tqs::partition(c->c, nz->nz, shots, o, arity, split));
    if (st != TQS_OK)
        return st;
    tqs::PlanHost H;
    st = from_msg(tqs::build_plan(c->c, nz->nz, shots, o, arity, split, H));
    if (st != TQS_OK)
        return st;
    std::vector<tqs::SpecSource> srcs;
    uint64_t bytes = 0;
    const uint32_t last = H.levels.empty() ? 0 : H.levels.back().pass_end - 1;
    for (uint32_t pi = 0; pi < (uint32_t)H.passes.size(); pi++)
        for (int mode : {tqs::MODE_STORE, tqs::MODE_SUMS, tqs::MODE_SAMPLE}) {
            if (mode != tqs::MODE_STORE && pi != last)
                continue;
            tqs::SpecSource s;
            if (!tqs::spec_generate(H, H.passes[pi], mode, s).empty())
                continue;
            bytes += s.defs.size() + s.walk.size();
            srcs.push_back(std::move(s));
        }
    const std::string m = tqs::spec_compile_only(srcs);
    if (!m.empty())
        return fail(TQS_ECUDA, m);
    *nkernels_out = (uint32_t)srcs.size();
    if (src_bytes_out)
        *src_bytes_out = bytes;
    return TQS_OK;
}

static tqs_status debug_spec_source(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, const tqs_options *opts,
                                    uint32_t pass, int mode, char *buf, uint64_t cap, uint64_t *len_out)
{
    if (!c || !nz || !len_out)
        return fail(TQS_EINVAL, "NULL argument");
    if (shots == 0)
        return fail(TQS_EINVAL, "shots must be >= 1");
    if (mode < tqs::MODE_STORE || mode > tqs::MODE_SAMPLE)
        return fail(TQS_EINVAL, "mode must be 0 (store), 1 (sums) or 2 (sample)");
    tqs_options o = opts_or_default(opts);
    if (o.prec != TQS_FP32)
        return fail(TQS_EINVAL, "specialised pass kernels are for FP32 plans");
    std::vector<uint64_t> arity;
    std::vector<uint32_t> split;
    tqs_status st = from_msg(tqs::partition(c->c, nz->nz, shots, o, arity, split));
    if (st != TQS_OK)
        return st;
    tqs::PlanHost H;
    st = from_msg(tqs::build_plan(c->c, nz->nz, shots, o, arity, split, H));
    if (st != TQS_OK)
        return st;
    if (pass >= H.passes.size())
        return fail(TQS_EINVAL, "pass index out of range");
    tqs::SpecSource s;
    const std::string why = tqs::spec_generate(H, H.passes[pass], mode, s);
    if (!why.empty())
        return fail(TQS_EUNSUPPORTED, why);
    const std::string text = s.defs + s.walk;
    *len_out = text.size();
    if (buf && cap) {
        const size_t n = std::min<size_t>(text.size(), (size_t)cap - 1);
        std::memcpy(buf, text.data(), n);
        buf[n] = '\0';
    }
    return TQS_OK;
}

tqs_status tqs_debug_spec_check(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, const tqs_options *opts,
                                uint32_t *nkernels_out, uint64_t *src_bytes_out)
{
    try {  // host allocations and compiler threads may throw: nothing crosses the C ABI
        return debug_spec_check(c, nz, shots, opts, nkernels_out, src_bytes_out);
    } catch (const std::exception &e) {
        return fail(TQS_ENOMEM, e.what());
    }
}

tqs_status tqs_debug_spec_source(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, const tqs_options *opts,
                                 uint32_t pass, int mode, char *buf, uint64_t cap, uint64_t *len_out)
{
    try {
        return debug_spec_source(c, nz, shots, opts, pass, mode, buf, cap, len_out);
    } catch (const std::exception &e) {
        return fail(TQS_ENOMEM, e.what());
    }
}

tqs_status tqs_plan_create(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, const tqs_options *opts,
                           tqs_plan **out)
{
    if (!out)
        return fail(TQS_EINVAL, "out is NULL");
    std::unique_ptr<tqs_plan> p;
    tqs_status st = tqs::make_plan(c, nz, shots, opts_or_default(opts), false, p);
    if (st != TQS_OK)
        return st;
    *out = p.release();
    return TQS_OK;
}

size_t tqs_plan_workspace_bytes(const tqs_plan *p) { return p ? p->dp.ws_bytes : 0; }

size_t tqs_plan_host_pool_bytes(const tqs_plan *p) { return p ? p->dp.host_pool_bytes : 0; }

void tqs_plan_destroy(tqs_plan *p) { delete p; }

tqs_status tqs_plan_execute(tqs_plan *p, uint64_t seed, uint64_t *d_counts, tqs_report *report)
{
    if (!p || !d_counts)
        return fail(TQS_EINVAL, "plan and d_counts are required");
    std::string err;
    tqs_status st = p->dp.execute(seed, (unsigned long long *)d_counts, report != nullptr, err);
    if (st != TQS_OK)
        return fail(st, err);
    if (report) {
        st = p->dp.check_device_error(err);
        if (st != TQS_OK)
            return fail(st, err);
        cudaError_t e = cudaEventSynchronize(p->dp.ev1);
        float ms = 0;
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, p->dp.ev0, p->dp.ev1);
        if (e != cudaSuccess)
            return fail(TQS_ECUDA, tqs::cuda_msg("plan execute", (int)e));
        fill_report(p, ms, report);
    }
    return TQS_OK;
}

tqs_status tqs_simulate(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, uint64_t seed,
                        const tqs_options *opts, uint64_t *counts, double *fid, tqs_report *report)
{
    if (!counts)
        return fail(TQS_EINVAL, "counts is NULL");
    tqs_options o = opts_or_default(opts);
    std::unique_ptr<tqs_plan> p;
    tqs_status st = tqs::make_plan(c, nz, shots, o, false, p);
    if (st != TQS_OK)
        return st;
    std::string err;
    cudaStream_t s = p->dp.stream;
    st = p->dp.execute(seed, p->dp.d_counts_internal, true, err);
    if (st != TQS_OK)
        return fail(st, err);
    st = p->dp.check_device_error(err);
    if (st != TQS_OK)
        return fail(st, err);
    // the fidelity (from the device histogram) before any output is written,
    // so that a failure there leaves the caller's buffers untouched
    double F = std::numeric_limits<double>::quiet_NaN(), Fs = F;
    if (!(o.flags & TQS_FLAG_NO_FIDELITY)) {
        st = fidelity(c, shots, p->dp.d_counts_internal, s, &F, &Fs);
        if (st != TQS_OK)
            return st;
    }
    const size_t bytes = sizeof(uint64_t) * ((size_t)1 << c->c.n);
    cudaError_t e = cudaMemcpyAsync(counts, p->dp.d_counts_internal, bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return fail(TQS_ECUDA, tqs::cuda_msg("simulate", (int)e));
    float ms = 0;
    cudaEventElapsedTime(&ms, p->dp.ev0, p->dp.ev1);
    if (fid)
        *fid = F;
    if (report) {
        fill_report(p.get(), ms, report);
        report->fid_norm = F;
        report->fid_s = Fs;
    }
    return TQS_OK;
}

tqs_status tqs_debug_node_state(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, uint64_t seed,
                                const tqs_options *opts, uint32_t level, uint64_t node, double *psi_out)
{
    if (!psi_out)
        return fail(TQS_EINVAL, "psi_out is NULL");
    tqs_options o = opts_or_default(opts);
    o.batch = 1;
    std::unique_ptr<tqs_plan> p;
    tqs_status st = make_plan_once(c, nz, shots, o, true, p);
    if (st != TQS_OK)
        return st;
    const tqs::PlanHost &H = p->dp.host;
    if (level >= H.levels.size())
        return fail(TQS_EINVAL, "level out of range");
    if (node >= H.levels[level].active)
        return fail(TQS_EINVAL, "node is not simulated at this level");
    std::string err;
    st = p->dp.run_chain(level, node, seed, err);
    if (st == TQS_OK)
        st = p->dp.check_device_error(err);
    if (st != TQS_OK)
        return fail(st, err);
    const uint64_t dim = (uint64_t)1 << H.n;
    const bool f64 = H.prec == TQS_FP64;
    std::vector<double> raw(2 * dim);
    std::vector<float> raw32;
    cudaError_t e;
    if (f64) {
        e = cudaMemcpyAsync(raw.data(), p->dp.state[level], 16 * dim, cudaMemcpyDefault, p->dp.stream);
    } else {
        raw32.resize(2 * dim);
        e = cudaMemcpyAsync(raw32.data(), p->dp.state[level], 8 * dim, cudaMemcpyDefault, p->dp.stream);
    }
    const tqs::Level &lv = H.levels[level];
    const uint32_t np = lv.pass_end - lv.pass_begin;
    tqs::NodeMeta m;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&m, p->dp.meta[level] + np, sizeof(m), cudaMemcpyDeviceToHost, p->dp.stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(p->dp.stream);
    if (e != cudaSuccess)
        return fail(TQS_ECUDA, tqs::cuda_msg("debug readback", (int)e));
    if (!f64)
        for (size_t i = 0; i < 2 * dim; i++)
            raw[i] = raw32[i];
    // logical psi(y) = i^phase * phi(phys(y) ^ mask)
    const double ph_re[4] = {1, 0, -1, 0}, ph_im[4] = {0, 1, 0, -1};
    const double wr = ph_re[m.phase & 3], wi = ph_im[m.phase & 3];
    for (uint64_t y = 0; y < dim; y++) {
        uint64_t x = 0;
        for (uint32_t q = 0; q < H.n; q++)
            x |= ((y >> q) & 1ull) << lv.perm[q];
        x ^= m.mask;
        const double a = raw[2 * x], b = raw[2 * x + 1];
        psi_out[2 * y] = wr * a - wi * b;
        psi_out[2 * y + 1] = wr * b + wi * a;
    }
    return TQS_OK;
}

tqs_status tqs_debug_node_noise(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, uint64_t seed,
                                const tqs_options *opts, uint32_t level, uint64_t node, uint8_t *paulis_out)
{
    if (!paulis_out)
        return fail(TQS_EINVAL, "paulis_out is NULL");
    tqs_options o = opts_or_default(opts);
    o.batch = 1;
    std::unique_ptr<tqs_plan> p;
    tqs_status st = make_plan_once(c, nz, shots, o, true, p);
    if (st != TQS_OK)
        return st;
    const tqs::PlanHost &H = p->dp.host;
    if (level >= H.levels.size())
        return fail(TQS_EINVAL, "level out of range");
    if (node >= H.levels[level].active)
        return fail(TQS_EINVAL, "node is not simulated at this level");
    std::string err;
    st = p->dp.run_chain(level, node, seed, err);
    if (st != TQS_OK)
        return fail(st, err);
    const size_t sites = H.levels[level].g1 - H.levels[level].g0;
    cudaError_t e = cudaSuccess;
    if (sites)
        e = cudaMemcpyAsync(paulis_out, p->dp.noise[level], sites, cudaMemcpyDeviceToHost, p->dp.stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(p->dp.stream);
    if (e != cudaSuccess)
        return fail(TQS_ECUDA, tqs::cuda_msg("debug readback", (int)e));
    return TQS_OK;
}

}  // extern "C"
