// handles.h -- definitions of the opaque handles of include/tqs.h, shared by the
// translation units that implement the C ABI.
#pragma once

#include <string>

#include "internal.h"

struct tqs_circuit {
    tqs::Circuit c;
};
struct tqs_noise {
    tqs::Noise nz;
};

namespace tqs {
// Records `msg` as the calling thread's tqs_last_error() and returns `s`.
tqs_status set_error(tqs_status s, const std::string &msg);
}  // namespace tqs
