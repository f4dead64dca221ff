// mlp.h -- the learned partitioner: network sizes and entry points (mlp.cu,
// learned.cpp).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "internal.h"

namespace tqs {

constexpr int kMlpFeatures = 40;
constexpr int kMlpHidden = 128;
constexpr int kMlpClasses = 20;  // class = 10 * mode + k (k extra levels, mode 0 equal / 1 pass-aligned splits)

size_t mlp_param_count();
tqs_status mlp_predict(const float *w, const float *X, size_t rows, float *logits);
tqs_status mlp_loss_grad(const float *w, const float *X, const int32_t *y, size_t rows, float *loss, float *grad);
tqs_status mlp_train(const float *X, const int32_t *y, size_t rows, uint32_t epochs, uint32_t batch, float lr,
                     uint64_t seed, const float *init, float *w_out, float *final_loss);

// learned.cpp
std::string learned_features(const Circuit &c, const Noise &nz, uint64_t shots, const tqs_options &o, float *feat,
                             uint8_t *allowed);
std::string learned_candidate(const Circuit &c, const Noise &nz, uint64_t shots, const tqs_options &o, uint32_t cls,
                              std::vector<uint64_t> &arity, std::vector<uint32_t> &split);
std::string learned_partition(const Circuit &c, const Noise &nz, uint64_t shots, const tqs_options &o,
                              std::vector<uint64_t> &arity, std::vector<uint32_t> &split);

// planner.cpp helpers shared with the learned partitioner
uint64_t dcp_first_arity(const Circuit &c, const Noise &nz, uint64_t N, double z, double eps, uint32_t K);
std::string dcp_tree(const Circuit &c, const Noise &nz, uint64_t N, double z, double eps, uint32_t cgates,
                     std::vector<uint64_t> &arity, std::vector<uint32_t> &split);
std::vector<uint32_t> pass_starts_one_level(const Circuit &c, uint32_t tile_max);

}  // namespace tqs
