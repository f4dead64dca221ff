// executor.h -- device-side plan: workspace carve-up, uploads and launches.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "internal.h"

namespace tqs {

std::string cuda_msg(const char *what, int err);

struct DevicePlan {
    PlanHost host;
    tqs_options opts{};
    cudaStream_t stream = nullptr;
    bool store_leaves = false;  // keep leaf states (debug chains)
    bool caller_counts = false; // the layout reserves no internal histogram and no fidelity scratch
    const uint64_t *seed_dev = nullptr;  // device seed read by the kernels (graph replays)
    uint64_t batch = 0;         // node instances per chunk and level
    uint64_t launch_tiles = 0;  // default batch target in tiles per launch (0: the library's choice)
    void *ws = nullptr;
    size_t ws_bytes = 0;
    bool own_ws = false;
    Instr *d_instr = nullptr;   // site order (noise kernel)
    Instr *d_pinstr = nullptr;  // program order (pass kernels)
    void *d_mats = nullptr;
    uint32_t *d_pass_start = nullptr;
    uint8_t *d_prog = nullptr;
    float *d_fused = nullptr;
    unsigned int *d_err = nullptr;
    uint32_t *d_chunk_off = nullptr;
    double *d_fid = nullptr;
    uint8_t *d_perm = nullptr;
    unsigned long long *d_counts_internal = nullptr;
    double *d_S = nullptr;
    double *d_ksum = nullptr;   // damping channels: per-tile sums of the last boundary pass
    void *d_kmat = nullptr;     // damping channels: each node's chosen operators
    // Levels whose state slots live in pinned host memory mapped into the
    // device's address space (bit i = level i): the pass kernels read and write
    // them in place (on a Grace-Blackwell node over NVLink-C2C), so the state pool
    // is no longer bounded by HBM (Sec. 3.3-3.4: idle host memory holds
    // intermediate states).  Set by create() under TQS_FLAG_HOST_POOL, or when
    // the library allocates the workspace and one node per level does not fit.
    uint32_t host_mask = 0;
    void *host_pool = nullptr;      // cudaHostAlloc'd, mapped
    void *host_pool_dev = nullptr;  // its device address
    size_t host_pool_bytes = 0;
    std::vector<void *> state;
    std::vector<uint8_t *> noise;
    std::vector<NodeMeta *> meta;
    std::vector<uint32_t> pst_host, pst_off;
    // TQS_FLAG_SPECIALIZE: per pass, the specialised kernel of each mode (nullptr = generic)
    std::vector<void *> spec_fn;
    void *spec_for(uint32_t pass, int mode) const
    {
        const size_t i = (size_t)pass * 3 + (size_t)mode;
        return i < spec_fn.size() ? spec_fn[i] : nullptr;
    }
    tqs_status build_specialized(std::string &err);
    tqs_status build_specialized_impl(std::string &err);
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // per-launch profiling (TQS_FLAG_PROFILE)
    struct ProfRec { int kind; double bytes; cudaEvent_t a, b; };
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<ProfRec> prof;
    cudaEvent_t next_event();
    // statistics of the last execute
    uint64_t launches = 0;
    double alg_bytes = 0;
    std::vector<uint64_t> node_count;

    ~DevicePlan();
    void release();
    size_t layout(uint64_t B, bool assign);
    bool level_needs_state(uint32_t i) const;
    size_t host_state_bytes(uint64_t B) const;  // host pool for B slots per level
    tqs_status create(const tqs_options &o, std::string &err);
    tqs_status execute(uint64_t seed, unsigned long long *counts, bool timed, std::string &err);
    tqs_status run_level(uint32_t i, uint64_t lo, uint64_t hi, std::vector<uint64_t> &plo,
                         uint64_t seed, unsigned long long *counts, std::string &err);
    tqs_status run_chain(uint32_t level, uint64_t node, uint64_t seed, std::string &err);
    // reads and clears the device error word (synchronises the stream)
    tqs_status check_device_error(std::string &err);
    void set_debug(PassLaunch &a) const;
    // damping channels: the boundary sums of pass `ps` and, after it, the choice launch
    void set_kraus(PassLaunch &a, const Pass &ps) const;
    int launch_choice(const Pass &ps, uint64_t lo, uint64_t nn, uint64_t seed, const uint64_t *seed_dev);
    bool profiling() const { return (opts.flags & TQS_FLAG_PROFILE) != 0; }
};

}  // namespace tqs
