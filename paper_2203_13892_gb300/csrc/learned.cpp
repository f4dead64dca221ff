// learned.cpp -- the learned partitioner: circuit features, the candidate trees
// it chooses between, and the partition step that consults the network with DCP
// as the fallback and the arbiter (Sec. 3.2's DCP stays the reference).
//
// A candidate is class = 10 * mode + k: k extra levels (k + 1 subcircuits) with
// the first-level arity from DCP's sample-size rule for that k, equal arities
// A_r = floor((N / A_0min)^(1/k)) below it and A_0 = ceil(N / A_r^k); mode 0 cuts
// the circuit into equal parts, mode 1 moves every cut to the nearest place where
// the tile-pass planner already starts a new pass (a cut inside a pass costs an
// extra state pass per node).  A candidate is allowed only if its A_0 is at least
// DCP's, i.e. its first-level sample (the Hoeffding width of the estimate) is no
// worse than DCP's.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "handles.h"
#include "mlp.h"

namespace tqs {

namespace {
std::mutex g_model_mu;
std::vector<float> g_model;  // empty: no learned model loaded

bool pow_le(uint64_t a, uint32_t k, uint64_t b, uint64_t N)
{
    unsigned __int128 v = b;
    for (uint32_t i = 0; i < k; i++) {
        v *= a;
        if (v > N)
            return false;
    }
    return true;
}

std::vector<uint32_t> equal_cuts(uint32_t G, uint32_t L)
{
    std::vector<uint32_t> s(L + 1);
    for (uint32_t i = 0; i <= L; i++)
        s[i] = (uint32_t)(((uint64_t)i * G) / L);
    return s;
}
}  // namespace

static std::string candidate_impl(const Circuit &c, const Noise &nz, uint64_t N, const tqs_options &o, uint32_t cls,
                                  const std::vector<uint32_t> *starts_in, std::vector<uint64_t> &arity,
                                  std::vector<uint32_t> &split)
{
    if (cls >= (uint32_t)kMlpClasses)
        return "class out of range";
    const uint32_t k = cls % 10, mode = cls / 10;
    const uint32_t G = (uint32_t)c.gates.size();
    if (k == 0) {
        arity = {N};
        split = {0, G};
        return "";
    }
    if (k + 1 > G || k + 1 > TQS_MAX_LEVELS)
        return "invalid: more subcircuits than gates or levels";
    const uint64_t a0min = dcp_first_arity(c, nz, N, o.z, o.eps, k);
    if (!pow_le(2, k, a0min, N))
        return "invalid: the remaining arity would drop below 2";
    uint64_t ar = 2;
    while (pow_le(ar + 1, k, a0min, N))
        ar++;
    unsigned __int128 pk = 1;
    for (uint32_t i = 0; i < k; i++)
        pk *= ar;
    arity.assign(k + 1, ar);
    arity[0] = (uint64_t)(((unsigned __int128)N + pk - 1) / pk);
    split = equal_cuts(G, k + 1);
    if (mode == 1) {
        std::vector<uint32_t> own;
        if (!starts_in) {
            const uint32_t t = o.tile_qubits ? o.tile_qubits : (o.prec == TQS_FP64 ? 11 : 12);
            own = pass_starts_one_level(c, t);
        }
        const std::vector<uint32_t> &starts = starts_in ? *starts_in : own;
        for (uint32_t i = 1; i <= k; i++) {
            uint32_t best = split[i], bd = 0xffffffffu;
            for (uint32_t s : starts) {
                if (s <= split[i - 1] || s >= G)
                    continue;
                const uint32_t d = s > split[i] ? s - split[i] : split[i] - s;
                if (d < bd) {
                    bd = d;
                    best = s;
                }
            }
            if (best > split[i - 1] && best < G)
                split[i] = best;
        }
        for (uint32_t i = 1; i <= k + 1; i++)
            if (split[i] < split[i - 1])
                return "invalid: aligned cuts collide";
    }
    return "";
}

std::string learned_candidate(const Circuit &c, const Noise &nz, uint64_t N, const tqs_options &o, uint32_t cls,
                              std::vector<uint64_t> &arity, std::vector<uint32_t> &split)
{
    return candidate_impl(c, nz, N, o, cls, nullptr, arity, split);
}

std::string learned_features(const Circuit &c, const Noise &nz, uint64_t N, const tqs_options &o, float *f,
                             uint8_t *allowed)
{
    const uint32_t G = (uint32_t)c.gates.size();
    std::vector<uint64_t> da;
    std::vector<uint32_t> ds;
    std::string m = dcp_tree(c, nz, N, o.z, o.eps, o.copy_gates, da, ds);
    if (!m.empty())
        return m;
    const uint32_t kd = (uint32_t)da.size() - 1;
    const uint64_t a0d = da[0];
    for (int i = 0; i < kMlpFeatures; i++)
        f[i] = 0.f;
    double lam = 0;
    uint32_t dense = 0;
    for (const Gate &g : c.gates) {
        lam += is_two_qubit(g.kind) ? nz.p2 : nz.p1;
        dense += is_diagonal(g.kind) || g.kind == TQS_SWAP ? 0 : 1;
    }
    f[0] = (float)c.n / 24.f;
    f[1] = (float)(std::log2((double)N) / 16.0);
    f[2] = (float)G / 1024.f;
    f[3] = (float)(lam / 8.0);
    f[4] = (float)kd / 16.f;
    f[5] = (float)(std::log2((double)dcp_first_arity(c, nz, N, o.z, o.eps, std::max<uint32_t>(kd, 1))) / 16.0);
    for (uint32_t i = 0; i < G; i++) {
        const uint32_t seg = (uint32_t)(((uint64_t)i * 16) / std::max<uint32_t>(G, 1));
        f[(is_two_qubit(c.gates[i].kind) ? 22 : 6) + seg] += 16.f / (float)std::max<uint32_t>(G, 1);
    }
    f[38] = G ? (float)dense / (float)G : 0.f;
    const uint32_t t = o.tile_qubits ? o.tile_qubits : (o.prec == TQS_FP64 ? 11 : 12);
    const std::vector<uint32_t> starts = pass_starts_one_level(c, t);
    f[39] = (float)starts.size() / 64.f;
    if (allowed) {
        for (uint32_t cls = 0; cls < (uint32_t)kMlpClasses; cls++) {
            std::vector<uint64_t> a;
            std::vector<uint32_t> s;
            allowed[cls] = 0;
            if (!candidate_impl(c, nz, N, o, cls, &starts, a, s).empty())
                continue;
            const uint32_t k = cls % 10;
            if (k > kd)
                continue;  // more levels than DCP: a smaller first-level sample
            if (a[0] < a0d)
                continue;
            allowed[cls] = 1;
        }
    }
    return "";
}

std::string learned_partition(const Circuit &c, const Noise &nz, uint64_t N, const tqs_options &o,
                              std::vector<uint64_t> &arity, std::vector<uint32_t> &split)
{
    std::vector<float> w;
    {
        std::lock_guard<std::mutex> lk(g_model_mu);
        w = g_model;
    }
    if (w.empty())
        return "UNSUPPORTED:no learned partitioner model is loaded (tqs_learned_set_model)";
    float feat[kMlpFeatures];
    uint8_t allowed[kMlpClasses];
    std::string m = learned_features(c, nz, N, o, feat, allowed);
    if (!m.empty())
        return m;
    float logits[kMlpClasses];
    if (mlp_predict(w.data(), feat, 1, logits) != TQS_OK)
        return "learned partitioner: device inference failed";
    int best = -1;
    for (int cls = 0; cls < kMlpClasses; cls++)
        if (allowed[cls] && (best < 0 || logits[cls] > logits[best]))
            best = cls;
    if (best < 0)  // nothing allowed: the paper's DCP decides
        return dcp_tree(c, nz, N, o.z, o.eps, o.copy_gates, arity, split);
    return learned_candidate(c, nz, N, o, (uint32_t)best, arity, split);
}

}  // namespace tqs

extern "C" {

size_t tqs_learned_param_count(void) { return tqs::mlp_param_count(); }

tqs_status tqs_learned_features(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, const tqs_options *opts,
                                float *features, uint8_t *allowed)
{
    if (!c || !nz || !features || shots == 0)
        return tqs::set_error(TQS_EINVAL, "circuit, noise, features and shots >= 1 are required");
    tqs_options o;
    if (opts)
        o = *opts;
    else
        tqs_options_default(&o);
    std::string m = tqs::learned_features(c->c, nz->nz, shots, o, features, allowed);
    return m.empty() ? TQS_OK : tqs::set_error(TQS_EINVAL, m);
}

tqs_status tqs_learned_candidate(const tqs_circuit *c, const tqs_noise *nz, uint64_t shots, const tqs_options *opts,
                                 uint32_t cls, uint32_t *levels_out, uint64_t *arity_out, uint32_t *split_out)
{
    if (!c || !nz || !levels_out || !arity_out || !split_out || shots == 0)
        return tqs::set_error(TQS_EINVAL, "NULL argument or shots == 0");
    tqs_options o;
    if (opts)
        o = *opts;
    else
        tqs_options_default(&o);
    std::vector<uint64_t> a;
    std::vector<uint32_t> s;
    std::string m = tqs::learned_candidate(c->c, nz->nz, shots, o, cls, a, s);
    if (!m.empty())
        return tqs::set_error(TQS_EINVAL, m);
    *levels_out = (uint32_t)a.size();
    std::copy(a.begin(), a.end(), arity_out);
    std::copy(s.begin(), s.end(), split_out);
    return TQS_OK;
}

tqs_status tqs_learned_train(const float *X, const int32_t *labels, size_t rows, uint32_t epochs, uint32_t batch,
                             float lr, uint64_t seed, const float *init, float *weights, float *final_loss)
{
    if (!X || !labels || !weights)
        return tqs::set_error(TQS_EINVAL, "X, labels and weights are required");
    return tqs::mlp_train(X, labels, rows, epochs, batch, lr, seed, init, weights, final_loss);
}

tqs_status tqs_learned_loss_grad(const float *weights, const float *X, const int32_t *labels, size_t rows,
                                 float *loss, float *grad)
{
    if (!weights || !X || !labels || !loss || !grad || rows == 0)
        return tqs::set_error(TQS_EINVAL, "NULL argument or rows == 0");
    for (size_t r = 0; r < rows; r++)
        if (labels[r] < 0 || labels[r] >= tqs::kMlpClasses)
            return tqs::set_error(TQS_EINVAL, "label out of range");
    return tqs::mlp_loss_grad(weights, X, labels, rows, loss, grad);
}

tqs_status tqs_learned_predict(const float *weights, const float *X, size_t rows, float *logits)
{
    if (!weights || !X || !logits || rows == 0)
        return tqs::set_error(TQS_EINVAL, "NULL argument or rows == 0");
    return tqs::mlp_predict(weights, X, rows, logits);
}

tqs_status tqs_learned_set_model(const float *weights)
{
    std::lock_guard<std::mutex> lk(tqs::g_model_mu);
    if (!weights)
        tqs::g_model.clear();
    else
        tqs::g_model.assign(weights, weights + tqs::mlp_param_count());
    return TQS_OK;
}

}  // extern "C"
