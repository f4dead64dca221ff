// handles.h -- definitions of the opaque handles of include/tqs.h, shared by the
// translation units that implement the C ABI.
#pragma once

#include <string>

#include <memory>
#include <vector>

#include "executor.h"
#include "internal.h"

struct tqs_circuit {
    tqs::Circuit c;
};
struct tqs_noise {
    tqs::Noise nz;
};

struct tqs_plan {
    tqs::Circuit c;
    tqs::Noise nz;
    uint64_t shots = 0;
    std::vector<uint64_t> arity;
    std::vector<uint32_t> split;
    tqs::DevicePlan dp;
};

namespace tqs {
// Records `msg` as the calling thread's tqs_last_error() and returns `s`.
tqs_status set_error(tqs_status s, const std::string &msg);
// Partition, lower and upload one simulation (store_leaves keeps every level's states).
// launch_tiles: the default node batch's target in tiles per launch (0: the
// library's choice for a plan that has the device to itself).
tqs_status make_plan(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, const tqs_options &o,
                     bool store_leaves, std::unique_ptr<tqs_plan> &out, uint64_t launch_tiles = 0);
// Chooses tile_qubits for the circuit's shape by timing trial runs (cached per shape).
tqs_status autotune(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, const tqs_options &o,
                    tqs_options &tuned);
}  // namespace tqs
