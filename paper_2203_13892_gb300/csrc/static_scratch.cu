// static_scratch.cu -- tqs_simulate_static: the simulation with every byte of
// device scratch taken from one file-scope __device__ array instead of an
// allocation, for callers that cannot allocate device memory.
//
// The array is TQS_STATIC_SCRATCH_BYTES (32 MiB) and is created with the
// library's module on every GPU that loads it; it stays reserved until the
// process exits.  Host code cannot use the array's name as an address, so the
// first call on each device (with that device current) resolves the address
// with cudaGetSymbolAddress and caches it for the rest of the process; the
// cached address does not survive a cudaDeviceReset of that device.  The call
// uploads tables and synchronises its stream, so it is never issued on a
// stream that is being captured.  All calls on a device share the one array and
// it keeps the last call's contents: calls whose work overlaps on the GPU
// (other streams, other threads) race on it and must be serialised by the
// caller.  The learned partitioner is refused here (TQS_EUNSUPPORTED): its
// network runs through the library's allocating MLP kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "executor.h"
#include "handles.h"

namespace {

constexpr size_t kStaticScratchBytes = TQS_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 128;

__device__ __align__(256) unsigned char g_tqs_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the static scratch on the current device (set up once per device).
tqs_status scratch_address(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return tqs::set_error(TQS_ECUDA, tqs::cuda_msg("cudaGetDevice", (int)e));
    if (dev < 0 || dev >= kMaxDevices)
        return tqs::set_error(TQS_EUNSUPPORTED, "device ordinal out of range for the static scratch");
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_tqs_static_scratch);
        if (e != cudaSuccess || p == nullptr)
            return tqs::set_error(TQS_ECUDA, tqs::cuda_msg("cudaGetSymbolAddress(static scratch)", (int)e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return TQS_OK;
}

}  // namespace

extern "C" tqs_status tqs_simulate_static(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots,
                                          uint64_t seed, const tqs_options *opts, uint64_t *d_counts)
{
    if (!c || !nz || !d_counts)
        return tqs::set_error(TQS_EINVAL, "circuit, noise and d_counts are required");
    if (shots == 0)
        return tqs::set_error(TQS_EINVAL, "shots must be >= 1");
    tqs_options o;
    if (opts)
        o = *opts;
    else
        tqs_options_default(&o);
    if (o.prec != TQS_FP32 && o.prec != TQS_FP64)
        return tqs::set_error(TQS_EINVAL, "unknown precision");
    if (o.part == TQS_PART_LEARNED)
        return tqs::set_error(TQS_EUNSUPPORTED,
                              "the learned partitioner allocates device memory for its network; "
                              "tqs_simulate_static takes DCP, UCP, XCP or an explicit tree");
    if (o.flags & TQS_FLAG_SPECIALIZE)
        return tqs::set_error(TQS_EUNSUPPORTED,
                              "specialised pass kernels are compiled and loaded when a plan is created; "
                              "tqs_simulate_static takes the generic kernels");
    o.workspace = nullptr;  // the scratch is the static array
    o.workspace_bytes = 0;
    o.flags &= ~TQS_FLAG_PROFILE;  // no events are created on this path

    tqs::DevicePlan dp;
    std::vector<uint64_t> arity;
    std::vector<uint32_t> split;
    std::string m = tqs::partition(c->c, nz->nz, shots, o, arity, split);
    if (!m.empty()) {
        if (m.rfind("UNSUPPORTED:", 0) == 0)
            return tqs::set_error(TQS_EUNSUPPORTED, m.substr(12));
        return tqs::set_error(TQS_EINVAL, m);
    }
    m = tqs::build_plan(c->c, nz->nz, shots, o, arity, split, dp.host);
    if (!m.empty())
        return tqs::set_error(TQS_EINVAL, m);
    dp.opts = o;
    dp.stream = (cudaStream_t)o.stream;
    dp.store_leaves = false;
    dp.caller_counts = true;  // the histogram is the caller's d_counts and no fidelity is computed
    const tqs::PlanHost &H = dp.host;

    // the largest batch whose workspace fits the static array
    const size_t one = dp.layout(1, false);
    if (one > kStaticScratchBytes)
        return tqs::set_error(TQS_EINVAL,
                              "request needs " + std::to_string(one) +
                                  " bytes of device scratch for one node per level; the static scratch "
                                  "holds " + std::to_string(kStaticScratchBytes) + " bytes");
    uint64_t maxact = 1;
    for (const auto &lv : H.levels)
        maxact = std::max<uint64_t>(maxact, lv.active);
    const uint64_t tiles = (uint64_t)1 << (H.n - std::min<uint32_t>(H.n, H.tile_max));
    uint64_t want = o.batch ? o.batch : std::max<uint64_t>(64, 65536 / tiles);
    want = std::min<uint64_t>(std::min<uint64_t>(want, 65535), maxact);
    uint64_t lo = 1, hi = want;
    while (lo < hi) {
        const uint64_t mid = (lo + hi + 1) / 2;
        if (dp.layout(mid, false) <= kStaticScratchBytes)
            lo = mid;
        else
            hi = mid - 1;
    }
    dp.batch = lo;

    void *base = nullptr;
    tqs_status st = scratch_address(&base);
    if (st != TQS_OK)
        return st;
    dp.ws = base;
    dp.own_ws = false;
    dp.ws_bytes = dp.layout(dp.batch, false);
    dp.layout(dp.batch, true);

    // gate tables (every region the kernels read is rewritten here or by the
    // kernels before it is read; the histogram is zeroed by execute)
    cudaError_t e = cudaMemcpyAsync(dp.d_instr, H.instrs.data(), sizeof(tqs::Instr) * H.instrs.size(),
                                    cudaMemcpyHostToDevice, dp.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dp.d_pinstr, H.prog_instrs.data(), sizeof(tqs::Instr) * H.prog_instrs.size(),
                            cudaMemcpyHostToDevice, dp.stream);
    if (e == cudaSuccess) {
        if (H.prec == TQS_FP64)
            e = cudaMemcpyAsync(dp.d_mats, H.mats64.data(), 8 * H.mats64.size(), cudaMemcpyHostToDevice, dp.stream);
        else
            e = cudaMemcpyAsync(dp.d_mats, H.mats32.data(), 4 * H.mats32.size(), cudaMemcpyHostToDevice, dp.stream);
    }
    for (const auto &lv : H.levels) {
        dp.pst_off.push_back((uint32_t)dp.pst_host.size());
        for (uint32_t p = lv.pass_begin; p < lv.pass_end; p++)
            dp.pst_host.push_back(H.passes[p].ibeg - H.passes[lv.pass_begin].ibeg);
        dp.pst_host.push_back(lv.g1 - lv.g0);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dp.d_pass_start, dp.pst_host.data(), 4 * dp.pst_host.size(), cudaMemcpyHostToDevice,
                            dp.stream);
    if (e == cudaSuccess && !H.prog.empty())
        e = cudaMemcpyAsync(dp.d_prog, H.prog.data(), H.prog.size(), cudaMemcpyHostToDevice, dp.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dp.d_chunk_off, H.chunk_off.data(), 4 * H.chunk_off.size(), cudaMemcpyHostToDevice,
                            dp.stream);
    if (e == cudaSuccess && !H.fused.empty())
        e = cudaMemcpyAsync(dp.d_fused, H.fused.data(), 4 * H.fused.size(), cudaMemcpyHostToDevice, dp.stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(dp.d_err, 0, 4 * sizeof(unsigned int), dp.stream);
    uint8_t perm[32] = {0};
    for (uint32_t q = 0; q < H.n; q++)
        perm[q] = H.levels.back().perm[q];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dp.d_perm, perm, 32, cudaMemcpyHostToDevice, dp.stream);
    if (e != cudaSuccess)
        return tqs::set_error(TQS_ECUDA, tqs::cuda_msg("static scratch upload", (int)e));

    std::string err;
    st = dp.execute(seed, (unsigned long long *)d_counts, false, err);
    if (st != TQS_OK)
        return tqs::set_error(st, err);
    e = cudaStreamSynchronize(dp.stream);
    if (e != cudaSuccess)
        return tqs::set_error(TQS_ECUDA, tqs::cuda_msg("tqs_simulate_static", (int)e));
    st = dp.check_device_error(err);
    return st == TQS_OK ? TQS_OK : tqs::set_error(st, err);
}
