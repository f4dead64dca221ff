// mlp.cu -- the learned partitioner's network: a multilayer perceptron
// F -> 128 -> 128 -> C (ReLU hidden layers, softmax cross-entropy), FP32, with
// hand-written forward, backward and Adam kernels.  Sizes are small (a few
// thousand rows), so every reduction is a plain per-thread loop in a fixed order:
// results are deterministic and the gradients can be compared with a CPU oracle.
//
// Parameter layout (one contiguous float array): W1[F][H], b1[H], W2[H][H], b2[H],
// W3[H][C], b3[C]; W[i][o] multiplies input i into output o.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "handles.h"
#include "mlp.h"

namespace tqs {

namespace {

constexpr int kTile = 16;

// Y[r][o] = act(b[o] + sum_i X[r][i] W[i][o])
__global__ void linear_fwd(const float *__restrict__ X, const float *__restrict__ W, const float *__restrict__ b,
                           float *__restrict__ Y, int rows, int in, int out, int relu)
{
    __shared__ float xs[kTile][kTile + 1], ws[kTile][kTile + 1];
    const int r = blockIdx.y * kTile + threadIdx.y, o = blockIdx.x * kTile + threadIdx.x;
    float acc = 0.f;
    for (int k0 = 0; k0 < in; k0 += kTile) {
        const int kx = k0 + threadIdx.x, ky = k0 + threadIdx.y;
        xs[threadIdx.y][threadIdx.x] = (r < rows && kx < in) ? X[(size_t)r * in + kx] : 0.f;
        ws[threadIdx.y][threadIdx.x] = (ky < in && o < out) ? W[(size_t)ky * out + o] : 0.f;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kTile; k++)
            acc = fmaf(xs[threadIdx.y][k], ws[k][threadIdx.x], acc);
        __syncthreads();
    }
    if (r < rows && o < out) {
        float y = acc + b[o];
        Y[(size_t)r * out + o] = relu ? fmaxf(y, 0.f) : y;
    }
}

// per row: loss_r = logsumexp(z) - z[label]; dZ = (softmax(z) - onehot) / rows
__global__ void softmax_xent(const float *__restrict__ Z, const int32_t *__restrict__ labels, int rows, int classes,
                             float *__restrict__ dZ, float *__restrict__ loss_rows)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows)
        return;
    const float *z = Z + (size_t)r * classes;
    float m = z[0];
    for (int c = 1; c < classes; c++)
        m = fmaxf(m, z[c]);
    float s = 0.f;
    for (int c = 0; c < classes; c++)
        s += expf(z[c] - m);
    const int y = labels[r];
    loss_rows[r] = logf(s) + m - z[y];
    if (dZ) {
        const float inv = 1.f / (float)rows;
        for (int c = 0; c < classes; c++) {
            const float p = expf(z[c] - m) / s;
            dZ[(size_t)r * classes + c] = (p - (c == y ? 1.f : 0.f)) * inv;
        }
    }
}

__global__ void sum_rows(const float *__restrict__ v, int n, float *__restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; i++)
            s += v[i];
        out[0] = (float)(s / n);
    }
}

// dW[i][o] = sum_r X[r][i] dY[r][o]
__global__ void linear_bwd_w(const float *__restrict__ X, const float *__restrict__ dY, float *__restrict__ dW,
                             int rows, int in, int out)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= in * out)
        return;
    const int i = idx / out, o = idx % out;
    float acc = 0.f;
    for (int r = 0; r < rows; r++)
        acc = fmaf(X[(size_t)r * in + i], dY[(size_t)r * out + o], acc);
    dW[idx] = acc;
}

__global__ void linear_bwd_b(const float *__restrict__ dY, float *__restrict__ db, int rows, int out)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= out)
        return;
    float acc = 0.f;
    for (int r = 0; r < rows; r++)
        acc += dY[(size_t)r * out + o];
    db[o] = acc;
}

// dX[r][i] = (H[r][i] > 0) * sum_o dY[r][o] W[i][o]   (H = the ReLU output feeding the layer)
__global__ void linear_bwd_x(const float *__restrict__ dY, const float *__restrict__ W, const float *__restrict__ H,
                             float *__restrict__ dX, int rows, int in, int out)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * in)
        return;
    const int r = idx / in, i = idx % in;
    float acc = 0.f;
    for (int o = 0; o < out; o++)
        acc = fmaf(dY[(size_t)r * out + o], W[(size_t)i * out + o], acc);
    dX[idx] = H[idx] > 0.f ? acc : 0.f;
}

__global__ void adam_step(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                          float *__restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void gather_rows(const float *__restrict__ X, const int32_t *__restrict__ y, const int32_t *__restrict__ idx,
                            int rows, int feat, float *__restrict__ Xb, int32_t *__restrict__ yb)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * feat)
        return;
    const int r = t / feat, f = t % feat;
    Xb[t] = X[(size_t)idx[r] * feat + f];
    if (f == 0)
        yb[r] = y[idx[r]];
}

struct Dev {
    std::vector<void *> ptrs;
    ~Dev()
    {
        for (void *p : ptrs)
            cudaFree(p);
    }
    template <typename T> T *alloc(size_t n, cudaError_t &e)
    {
        void *p = nullptr;
        if (e == cudaSuccess)
            e = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
        if (e == cudaSuccess)
            ptrs.push_back(p);
        return (T *)p;
    }
};

struct Layout {
    size_t W1, b1, W2, b2, W3, b3, total;
    Layout()
    {
        W1 = 0;
        b1 = W1 + (size_t)kMlpFeatures * kMlpHidden;
        W2 = b1 + kMlpHidden;
        b2 = W2 + (size_t)kMlpHidden * kMlpHidden;
        W3 = b2 + kMlpHidden;
        b3 = W3 + (size_t)kMlpHidden * kMlpClasses;
        total = b3 + kMlpClasses;
    }
};

// Forward (and, with dZ buffers, backward) on `rows` rows already on the device.
struct Net {
    const Layout L;
    float *H1 = nullptr, *H2 = nullptr, *Z = nullptr, *dZ = nullptr, *dH2 = nullptr, *dH1 = nullptr, *lossr = nullptr;
    int cap = 0;
    cudaError_t reserve(Dev &d, int rows)
    {
        cudaError_t e = cudaSuccess;
        cap = rows;
        H1 = d.alloc<float>((size_t)rows * kMlpHidden, e);
        H2 = d.alloc<float>((size_t)rows * kMlpHidden, e);
        Z = d.alloc<float>((size_t)rows * kMlpClasses, e);
        dZ = d.alloc<float>((size_t)rows * kMlpClasses, e);
        dH2 = d.alloc<float>((size_t)rows * kMlpHidden, e);
        dH1 = d.alloc<float>((size_t)rows * kMlpHidden, e);
        lossr = d.alloc<float>(rows, e);
        return e;
    }
    void forward(const float *w, const float *X, int rows, cudaStream_t st)
    {
        dim3 blk(kTile, kTile);
        linear_fwd<<<dim3((kMlpHidden + kTile - 1) / kTile, (rows + kTile - 1) / kTile), blk, 0, st>>>(
            X, w + L.W1, w + L.b1, H1, rows, kMlpFeatures, kMlpHidden, 1);
        linear_fwd<<<dim3((kMlpHidden + kTile - 1) / kTile, (rows + kTile - 1) / kTile), blk, 0, st>>>(
            H1, w + L.W2, w + L.b2, H2, rows, kMlpHidden, kMlpHidden, 1);
        linear_fwd<<<dim3((kMlpClasses + kTile - 1) / kTile, (rows + kTile - 1) / kTile), blk, 0, st>>>(
            H2, w + L.W3, w + L.b3, Z, rows, kMlpHidden, kMlpClasses, 0);
    }
    void backward(const float *w, const float *X, const int32_t *y, int rows, float *grad, float *loss,
                  cudaStream_t st)
    {
        softmax_xent<<<(rows + 127) / 128, 128, 0, st>>>(Z, y, rows, kMlpClasses, dZ, lossr);
        sum_rows<<<1, 32, 0, st>>>(lossr, rows, loss);
        const int T = 256;
        linear_bwd_w<<<(kMlpHidden * kMlpClasses + T - 1) / T, T, 0, st>>>(H2, dZ, grad + L.W3, rows, kMlpHidden,
                                                                          kMlpClasses);
        linear_bwd_b<<<1, T, 0, st>>>(dZ, grad + L.b3, rows, kMlpClasses);
        linear_bwd_x<<<(rows * kMlpHidden + T - 1) / T, T, 0, st>>>(dZ, w + L.W3, H2, dH2, rows, kMlpHidden,
                                                                    kMlpClasses);
        linear_bwd_w<<<(kMlpHidden * kMlpHidden + T - 1) / T, T, 0, st>>>(H1, dH2, grad + L.W2, rows, kMlpHidden,
                                                                         kMlpHidden);
        linear_bwd_b<<<1, T, 0, st>>>(dH2, grad + L.b2, rows, kMlpHidden);
        linear_bwd_x<<<(rows * kMlpHidden + T - 1) / T, T, 0, st>>>(dH2, w + L.W2, H1, dH1, rows, kMlpHidden,
                                                                    kMlpHidden);
        linear_bwd_w<<<(kMlpFeatures * kMlpHidden + T - 1) / T, T, 0, st>>>(X, dH1, grad + L.W1, rows,
                                                                           kMlpFeatures, kMlpHidden);
        linear_bwd_b<<<1, T, 0, st>>>(dH1, grad + L.b1, rows, kMlpHidden);
    }
};

tqs_status cuda_fail(const char *what, cudaError_t e) { return set_error(TQS_ECUDA, cuda_msg(what, (int)e)); }

}  // namespace

size_t mlp_param_count() { return Layout().total; }

tqs_status mlp_predict(const float *w_host, const float *X_host, size_t rows, float *logits_host)
{
    Dev d;
    cudaError_t e = cudaSuccess;
    const Layout L;
    float *w = d.alloc<float>(L.total, e);
    float *X = d.alloc<float>(rows * kMlpFeatures, e);
    Net net;
    if (e == cudaSuccess)
        e = net.reserve(d, (int)rows);
    if (e == cudaSuccess)
        e = cudaMemcpy(w, w_host, L.total * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(X, X_host, rows * kMlpFeatures * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
        return cuda_fail("mlp predict setup", e);
    net.forward(w, X, (int)rows, 0);
    e = cudaMemcpy(logits_host, net.Z, rows * kMlpClasses * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail("mlp predict", e);
    return TQS_OK;
}

tqs_status mlp_loss_grad(const float *w_host, const float *X_host, const int32_t *y_host, size_t rows, float *loss,
                         float *grad_host)
{
    Dev d;
    cudaError_t e = cudaSuccess;
    const Layout L;
    float *w = d.alloc<float>(L.total, e);
    float *g = d.alloc<float>(L.total, e);
    float *X = d.alloc<float>(rows * kMlpFeatures, e);
    int32_t *y = d.alloc<int32_t>(rows, e);
    float *lo = d.alloc<float>(1, e);
    Net net;
    if (e == cudaSuccess)
        e = net.reserve(d, (int)rows);
    if (e == cudaSuccess)
        e = cudaMemcpy(w, w_host, L.total * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(X, X_host, rows * kMlpFeatures * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(y, y_host, rows * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
        return cuda_fail("mlp grad setup", e);
    net.forward(w, X, (int)rows, 0);
    net.backward(w, X, y, (int)rows, g, lo, 0);
    e = cudaMemcpy(grad_host, g, L.total * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(loss, lo, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail("mlp grad", e);
    return TQS_OK;
}

tqs_status mlp_train(const float *X_host, const int32_t *y_host, size_t rows, uint32_t epochs, uint32_t batch,
                     float lr, uint64_t seed, const float *init, float *w_out, float *final_loss)
{
    if (rows == 0 || batch == 0)
        return set_error(TQS_EINVAL, "training needs rows >= 1 and batch >= 1");
    for (size_t r = 0; r < rows; r++)
        if (y_host[r] < 0 || y_host[r] >= kMlpClasses)
            return set_error(TQS_EINVAL, "label out of range");
    const Layout L;
    std::vector<float> w0(L.total);
    if (init) {
        std::memcpy(w0.data(), init, L.total * 4);
    } else {  // He initialisation from a seeded generator, zero biases
        std::mt19937_64 rng(seed);
        std::normal_distribution<float> nd(0.f, 1.f);
        auto fill = [&](size_t off, size_t fan_in, size_t n) {
            const float s = std::sqrt(2.0f / (float)fan_in);
            for (size_t i = 0; i < n; i++)
                w0[off + i] = nd(rng) * s;
        };
        fill(L.W1, kMlpFeatures, (size_t)kMlpFeatures * kMlpHidden);
        fill(L.W2, kMlpHidden, (size_t)kMlpHidden * kMlpHidden);
        fill(L.W3, kMlpHidden, (size_t)kMlpHidden * kMlpClasses);
        for (size_t i : {L.b1, L.b2})
            for (size_t k = 0; k < (size_t)kMlpHidden; k++)
                w0[i + k] = 0.f;
        for (size_t k = 0; k < (size_t)kMlpClasses; k++)
            w0[L.b3 + k] = 0.f;
    }
    Dev d;
    cudaError_t e = cudaSuccess;
    const int B = (int)std::min<size_t>(batch, rows);
    float *w = d.alloc<float>(L.total, e), *g = d.alloc<float>(L.total, e);
    float *m = d.alloc<float>(L.total, e), *v = d.alloc<float>(L.total, e);
    float *X = d.alloc<float>(rows * kMlpFeatures, e), *Xb = d.alloc<float>((size_t)B * kMlpFeatures, e);
    int32_t *y = d.alloc<int32_t>(rows, e), *yb = d.alloc<int32_t>(B, e), *idx = d.alloc<int32_t>(rows, e);
    float *lo = d.alloc<float>(1, e);
    Net net;
    if (e == cudaSuccess)
        e = net.reserve(d, B);
    if (e == cudaSuccess)
        e = cudaMemcpy(w, w0.data(), L.total * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemset(m, 0, L.total * 4);
    if (e == cudaSuccess)
        e = cudaMemset(v, 0, L.total * 4);
    if (e == cudaSuccess)
        e = cudaMemcpy(X, X_host, rows * kMlpFeatures * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(y, y_host, rows * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
        return cuda_fail("mlp train setup", e);
    std::vector<int32_t> order(rows);
    for (size_t r = 0; r < rows; r++)
        order[r] = (int32_t)r;
    std::mt19937_64 rng(seed ^ 0x5851F42D4C957F2Dull);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    int step = 0;
    for (uint32_t ep = 0; ep < epochs; ep++) {
        std::shuffle(order.begin(), order.end(), rng);
        e = cudaMemcpy(idx, order.data(), rows * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess)
            return cuda_fail("mlp train shuffle", e);
        for (size_t r0 = 0; r0 + (size_t)B <= rows; r0 += B) {
            gather_rows<<<(B * kMlpFeatures + 255) / 256, 256>>>(X, y, idx + r0, B, kMlpFeatures, Xb, yb);
            net.forward(w, Xb, B, 0);
            net.backward(w, Xb, yb, B, g, lo, 0);
            step++;
            const float c1 = 1.f - std::pow(b1, (float)step), c2 = 1.f - std::pow(b2, (float)step);
            adam_step<<<((int)L.total + 255) / 256, 256>>>(w, g, m, v, (int)L.total, lr, b1, b2, eps, c1, c2);
        }
    }
    // final loss over the whole set
    Net full;
    if ((e = full.reserve(d, (int)rows)) != cudaSuccess)
        return cuda_fail("mlp train eval", e);
    full.forward(w, X, (int)rows, 0);
    softmax_xent<<<((int)rows + 127) / 128, 128>>>(full.Z, y, (int)rows, kMlpClasses, nullptr, full.lossr);
    sum_rows<<<1, 32>>>(full.lossr, (int)rows, lo);
    e = cudaMemcpy(w_out, w, L.total * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && final_loss)
        e = cudaMemcpy(final_loss, lo, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail("mlp train", e);
    return TQS_OK;
}

}  // namespace tqs
