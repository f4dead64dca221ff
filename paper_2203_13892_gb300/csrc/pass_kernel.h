// pass_kernel.h -- the parameter block of the state-vector pass kernel and
// the per-(precision, mode) launchers; each pair is instantiated in its own
// translation unit (pass_f32_store.cu ... pass_f64_sample.cu) so that the
// kernel's instantiations compile in parallel.
#pragma once
#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#endif

#include "internal.h"

namespace tqs {

struct PassK {
    const void *in;
    void *out;
    uint64_t state_elems;
    uint64_t node_lo, parent_lo, arity;
    const Instr *instr;
    const uint8_t *prog;
    const uint32_t *chunk_off;
    const void *mats;
    const uint8_t *noise;
    const NodeMeta *meta;
    double *S;
    unsigned long long *counts;
    const uint64_t *seed_dev;
    const float *fused;
    unsigned int *err;
    uint64_t seed, thrm;
    uint64_t in_slots, out_slots;
    double *ksum;
    const void *kmat;
    uint32_t knq, kp0, kp1;
    uint32_t dbg;
    uint32_t fused_k;
    uint32_t ibeg, iend, n, t, L, sites, meta_stride, pass_local;
    uint32_t chunk_begin, chunk_end;
    int in_from_parent;
    uint8_t tbits[kMaxTile];
    uint8_t hbits[32];
    SamplerLayout samp;
};

#ifndef __CUDACC_RTC__
// Launch the pass kernel of element type R (float or double) and mode MODE
// (MODE_STORE, MODE_SUMS or MODE_SAMPLE) for tile width 2^(8 + logr).
template <typename R, int MODE>
int launch_pass_r(const PassK &k, int logr, dim3 grid, size_t smem, cudaStream_t st);
// Raise the dynamic shared-memory limit of every instantiation of (R, MODE).
template <typename R, int MODE> int set_attrs_r();
#endif

}  // namespace tqs
