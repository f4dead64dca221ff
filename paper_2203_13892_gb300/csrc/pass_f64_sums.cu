// pass_f64_sums.cu -- instantiations of the pass kernel for double amplitudes,
// MODE_SUMS (one translation unit per pair, compiled in parallel).
#include "pass_kernel.cuh"

namespace tqs {
template int launch_pass_r<double, MODE_SUMS>(const PassK &, int, dim3, size_t, cudaStream_t);
template int set_attrs_r<double, MODE_SUMS>();
}  // namespace tqs
