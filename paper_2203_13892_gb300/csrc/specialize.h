// specialize.h -- pass kernels specialised per pass program (FP32 states).
//
// The generic pass kernel interprets a pass's records (pass_kernel.cuh): every
// thread decodes every record, and the leaf and store passes of the 20-qubit
// QFT tree spend most of their issue slots there rather than on amplitudes.
// Here the same records are turned into straight-line CUDA statements (each
// record becomes the calls the interpreter would make, with the tile
// positions, matrix entries, phase masks and noise sites as constants), the
// tile layout of the pass becomes a compile-time constant, and the result is
// compiled at plan time by NVRTC for sm_103a and launched through the driver
// API in place of the generic instantiation.  NVRTC and the driver are opened
// at run time (dlopen), so the library loads without them; a request for
// specialised kernels without them fails with TQS_EUNSUPPORTED.
#pragma once

#include <string>
#include <vector>

#include "internal.h"

namespace tqs {

// One specialised kernel: the generated walk (included inside the kernel body),
// the tile-layout constants and the template arguments it is compiled with.
struct SpecSource {
    std::string defs;  // namespace tqs::spec constants (tile layout)
    std::string walk;  // the pass's records as statements
    int mode = MODE_STORE;
    int logr = 0;
    std::string key() const;
};

// The source of the kernel for pass `ps` of plan H in mode `mode`.  Returns an
// empty string on success, else why the pass cannot be specialised (FP64
// states, fused tensor-core blocks, a malformed program).
std::string spec_generate(const PlanHost &H, const Pass &ps, int mode, SpecSource &out);

// Compiles (in parallel) and loads the kernels of `srcs` for the current
// device; fns[i] receives a driver function handle.  Compiled kernels are kept
// for the life of the process, keyed by device and source.  Returns "" or the
// error (compiler log included).
std::string spec_build(const std::vector<SpecSource> &srcs, std::vector<void *> &fns);

// Compiles the kernels of `srcs` without loading them (no device needed).
std::string spec_compile_only(const std::vector<SpecSource> &srcs);

// Whether NVRTC and the driver API could be opened ("" = yes, else why not).
// With `need_driver` false only NVRTC is required.
std::string spec_available(bool need_driver = true);

// Launches a specialised kernel with the pass kernel's parameter block.
int spec_launch(void *fn, const void *params, unsigned gx, unsigned gy, size_t smem, void *stream);

}  // namespace tqs
