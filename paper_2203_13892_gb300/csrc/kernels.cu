// kernels.cu -- sm_103a kernels of the noisy tree Monte-Carlo path other than
// the pass kernel, and the launcher that dispatches a pass to its instantiation.
//
//   noise_kernel   one warp per tree node: Philox4x32-10 draws for every noise
//                  site of the node's subcircuit (Sec. 2.4) and the node's Pauli
//                  frame (X mask, i-power) at every pass boundary
//   launch_pass    picks the pass kernel's instantiation (pass_kernel.cuh) for
//                  the precision, mode and tile width of a pass
//   fidelity       FP64 reductions for F_s and the normalised fidelity (Sec. 4.1)
//
// The Pauli frame: a node's logical state is psi(x) = i^phase * phi(x ^ mask)
// where phi is what is stored.  An X on qubit q only toggles bit q of the mask,
// a Z multiplies phi by -1 where (x ^ mask) has bit q set, and a gate U on
// qubits Q acts on phi with U conjugated by the mask bits of Q
// (U'[r][c] = U[r ^ mu][c ^ mu]); no Pauli ever moves data.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "pass_kernel.h"
#include "specialize.h"

namespace tqs {

// ---------------------------------------------------------------------------
// Noise kernel: one warp per node
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) noise_kernel(const __grid_constant__ NoiseLaunch a)
{
    const uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= a.nnodes)
        return;
    const uint64_t node = a.node_lo + w;
    const uint64_t seed = a.seed_dev ? *a.seed_dev : a.seed;
    NodeMeta par = {0u, 0u};
    if (a.parent_meta) {
        const uint64_t ps = node / a.arity - a.parent_lo;
        par = a.parent_meta[ps * a.parent_stride + a.parent_end];
        par.phase &= 3u;  // the parent's flags are not inherited
    }
    uint8_t *nout = a.noise_out + w * a.sites;
    NodeMeta *mout = a.meta_out + w * (a.npass + 1);
    for (uint32_t p = lane; p <= a.npass; p += 32)
        mout[p] = par;
    __syncwarp();
    uint32_t mask = par.mask, phase = par.phase;
    uint32_t noisy = 0;  // bit p: a Pauli was drawn at some site of pass p (passes >= 31 share bit 31)
    for (uint32_t b = 0; b < a.sites; b += 32) {
        const uint32_t s = b + lane;
        uint32_t xm = 0, yc = 0;
        if (s < a.sites) {
            const Instr I = a.instr[s];
            const uint64_t thr = I.npaulis == 15 ? a.thr2 : a.thr1;
            const uint4 r = draw(seed, node, I.gate, kDomNoise);
            uint32_t pz = 0;
            if ((uint64_t)r.x < thr)
                pz = 1u + (uint32_t)(((uint64_t)r.y * I.npaulis) >> 32);
            if (pz) {
                const uint32_t wa = I.npaulis == 15 ? (pz >> 2) : pz;
                const uint32_t wb = I.npaulis == 15 ? (pz & 3u) : 0u;
                if (wa == 1 || wa == 2) xm ^= 1u << I.np0;
                if (wa == 2) yc++;
                if (wb == 1 || wb == 2) xm ^= 1u << I.np1;
                if (wb == 2) yc++;
            }
            nout[I.site] = (uint8_t)pz;  // the table runs in pass order; the noise row is by site
            if (pz) {
                uint32_t p = 0;  // entry s of the table belongs to pass p: pass_start[p] <= s < pass_start[p+1]
                while (p + 1 < a.npass && a.pass_start[p + 1] <= s)
                    p++;
                noisy |= 1u << (p < 31u ? p : 31u);
            }
        }
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t tx = __shfl_up_sync(0xffffffffu, xm, off);
            const uint32_t ty = __shfl_up_sync(0xffffffffu, yc, off);
            if (lane >= off) {
                xm ^= tx;
                yc += ty;
            }
        }
        if (s < a.sites) {
            // boundary p (1..npass) sits after table entry pass_start[p]-1
            for (uint32_t p = 1; p <= a.npass; p++)
                if (a.pass_start[p] == s + 1)
                    mout[p] = NodeMeta{mask ^ xm, (phase + yc) & 3u};
        }
        mask ^= __shfl_sync(0xffffffffu, xm, 31);
        phase += __shfl_sync(0xffffffffu, yc, 31);
    }
    // Flag, in bit 31 of the frame entry that opens it, every pass of this node
    // with at least one Pauli: the pass kernels skip all noise checks of the others.
    noisy = __reduce_or_sync(0xffffffffu, noisy);
    __syncwarp();
    for (uint32_t p = lane; p < a.npass; p += 32)
        if ((noisy >> (p < 31u ? p : 31u)) & 1u)
            mout[p].phase |= 0x80000000u;
}

int launch_noise(const NoiseLaunch &a, void *stream)
{
    if (a.nnodes == 0)
        return 0;
    const uint64_t threads = a.nnodes * 32;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    noise_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

int prepare_kernels()
{
    int e = set_attrs_r<float, MODE_STORE>() | set_attrs_r<float, MODE_SUMS>() | set_attrs_r<float, MODE_SAMPLE>();
    e |= set_attrs_r<double, MODE_STORE>() | set_attrs_r<double, MODE_SUMS>() | set_attrs_r<double, MODE_SAMPLE>();
    return e;
}


int launch_pass(const PassLaunch &a, void *stream)
{
    if (a.nnodes == 0)
        return 0;
    PassK k;
    k.in = a.in;
    k.out = a.out;
    k.state_elems = a.state_elems;
    k.node_lo = a.node_lo;
    k.parent_lo = a.parent_lo;
    k.arity = a.arity ? a.arity : 1;
    k.instr = a.instr;
    k.prog = a.prog;
    k.chunk_off = a.chunk_off;
    k.chunk_begin = a.chunk_begin;
    k.chunk_end = a.chunk_end;
    k.mats = a.mats;
    k.noise = a.noise;
    k.meta = a.meta;
    k.S = a.S;
    k.counts = a.counts;
    k.seed = a.seed;
    k.seed_dev = a.seed_dev;
    k.fused = a.fused;
    k.fused_k = a.fused ? a.fused_k : 0;
    k.err = a.err;
    k.dbg = a.dbg;
    k.ksum = a.ksum;
    k.kmat = a.kmat;
    k.knq = a.knq;
    k.kp0 = a.kp0;
    k.kp1 = a.kp1;
    k.in_slots = a.in_slots;
    k.out_slots = a.out_slots;
    k.thrm = a.thrm;
    k.ibeg = a.ibeg;
    k.iend = a.iend;
    k.n = a.n;
    k.t = a.t;
    k.L = a.L;
    k.sites = a.sites;
    k.meta_stride = a.meta_stride;
    k.pass_local = a.pass_local;
    k.in_from_parent = a.in_from_parent;
    for (int i = 0; i < kMaxTile; i++)
        k.tbits[i] = a.tbits[i];
    for (int i = 0; i < 32; i++)
        k.hbits[i] = a.hbits[i];
    if (a.samp)
        k.samp = *a.samp;
    else
        k.samp = SamplerLayout{};
    const size_t elem = a.fp64 ? 16 : 8;
    const size_t te = ((size_t)1 << a.t) < (size_t)kThreads ? (size_t)kThreads : ((size_t)1 << a.t);
    const size_t nzst = ((a.sites < (uint32_t)kNoiseStage ? a.sites : (uint32_t)kNoiseStage) + 15u) / 16u * 16u;
    size_t smem = te * elem + 256 * 2 + kThreads * 8 + 4 * 8 + 32 * 4 + nzst + kProgChunkBytes;
    if (k.fused_k) {  // A lo (the tile region doubles as A hi), B hi/lo, mbarrier and TMEM slot
        const size_t K = (size_t)2 << k.fused_k;
        smem = (smem + 127) / 128 * 128 + te * elem + 2 * K * K * 4 + 128;
    }
    const int logr = a.t > 8 ? (int)a.t - 8 : 0;
    const uint64_t tiles = (uint64_t)1 << (a.n - a.t);
    dim3 grid = a.mode == MODE_SAMPLE ? dim3(a.nnodes) : dim3((unsigned)tiles, a.nnodes);
    cudaStream_t st = (cudaStream_t)stream;
    if (a.spec_fn && !a.fp64 && !k.fused_k)
        return spec_launch(a.spec_fn, &k, grid.x, grid.y, smem, stream);
    if (a.fp64) {
        if (a.mode == MODE_STORE) return launch_pass_r<double, MODE_STORE>(k, logr, grid, smem, st);
        if (a.mode == MODE_SUMS) return launch_pass_r<double, MODE_SUMS>(k, logr, grid, smem, st);
        return launch_pass_r<double, MODE_SAMPLE>(k, logr, grid, smem, st);
    }
    if (a.mode == MODE_STORE) return launch_pass_r<float, MODE_STORE>(k, logr, grid, smem, st);
    if (a.mode == MODE_SUMS) return launch_pass_r<float, MODE_SUMS>(k, logr, grid, smem, st);
    return launch_pass_r<float, MODE_SAMPLE>(k, logr, grid, smem, st);
}


// ---------------------------------------------------------------------------
// Damping channels: the trajectory choice after one gate (Sec. 4.3)
// ---------------------------------------------------------------------------
// One warp per node.  The lanes add the per-tile sums in a fixed order (lane
// l takes tiles l, l+32, ...; then a fixed butterfly), so the result does not
// depend on scheduling.  Lane 0 then goes through the channels of the gate's
// qubits in order: with P the normalised joint distribution of the (one or
// two) qubits' logical values, a channel of rate r on qubit i jumps iff
// u < r * P(bit i = 1), u drawn from counter (node_lo, node_hi, 16 g + 8 i + c,
// 4); the jump operator is sqrt(r)|0><1| (damping) or sqrt(r)|1><1|
// (dephasing), otherwise diag(1, sqrt(1-r)), each divided by the square root
// of the probability of the choice, and P follows the choice.  The operators
// of each qubit are multiplied up (the first also carries 1/sqrt(total), which
// renormalises the state as it stands) and stored for the next pass.
__global__ void __launch_bounds__(256) kraus_kernel(const __grid_constant__ KrausLaunch a)
{
    const uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= a.nnodes)
        return;
    const double *S = a.ksum + w * a.tiles * 4;
    double s4[4] = {0.0, 0.0, 0.0, 0.0};
    for (uint64_t t = lane; t < a.tiles; t += 32)
        for (int j = 0; j < 4; j++)
            s4[j] += S[t * 4 + j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        for (int j = 0; j < 4; j++)
            s4[j] += __shfl_xor_sync(0xffffffffu, s4[j], off);
    if (lane != 0)
        return;
    const uint64_t node = a.node_lo + w;
    const uint64_t seed = a.seed_dev ? *a.seed_dev : a.seed;
    const double total = s4[0] + s4[1] + s4[2] + s4[3];
    double P[4];
    for (int j = 0; j < 4; j++)
        P[j] = total > 0.0 ? s4[j] / total : 0.0;
    // M[q] = [[m00, m01], [m10, m11]] as doubles (the operators are real)
    double M[2][4] = {{1.0, 0.0, 0.0, 1.0}, {1.0, 0.0, 0.0, 1.0}};
    double scale = total > 0.0 ? 1.0 / sqrt(total) : 1.0;
    for (uint32_t i = 0; i < a.nq; i++) {
        const uint32_t bit = 1u << i;
        for (uint32_t c = 0; c < 4; c++) {
            const double r = a.rate[c];
            if (!(r > 0.0))
                continue;
            const bool damping = (c & 1u) == 0u;  // thermal damping, amplitude damping
            double P1 = 0.0;
            for (uint32_t x = 0; x < 4; x++)
                if (x & bit)
                    P1 += P[x];
            const double pj = r * P1;
            const uint4 rr = draw(seed, node, 16u * a.gate + 8u * i + c, kDomKraus);
            const double u = ((double)(rr.x >> 5) * 67108864.0 + (double)(rr.y >> 6)) * (1.0 / 9007199254740992.0);
            double K[4];
            double Pn[4] = {0.0, 0.0, 0.0, 0.0};
            if (u < pj) {
                const double sc = sqrt(r / pj);
                if (damping) {
                    K[0] = 0.0; K[1] = sc; K[2] = 0.0; K[3] = 0.0;
                    for (uint32_t x = 0; x < 4; x++)
                        if (x & bit)
                            Pn[x ^ bit] = P[x] * r / pj;
                } else {
                    K[0] = 0.0; K[1] = 0.0; K[2] = 0.0; K[3] = sc;
                    for (uint32_t x = 0; x < 4; x++)
                        if (x & bit)
                            Pn[x] = P[x] * r / pj;
                }
            } else {
                const double s0 = 1.0 / sqrt(1.0 - pj);
                K[0] = s0; K[1] = 0.0; K[2] = 0.0; K[3] = sqrt(1.0 - r) * s0;
                for (uint32_t x = 0; x < 4; x++)
                    Pn[x] = P[x] * ((x & bit) ? (1.0 - r) : 1.0) / (1.0 - pj);
            }
            for (int x = 0; x < 4; x++)
                P[x] = Pn[x];
            double *m = M[i];
            const double n00 = K[0] * m[0] + K[1] * m[2], n01 = K[0] * m[1] + K[1] * m[3];
            const double n10 = K[2] * m[0] + K[3] * m[2], n11 = K[2] * m[1] + K[3] * m[3];
            m[0] = n00; m[1] = n01; m[2] = n10; m[3] = n11;
        }
    }
    for (int j = 0; j < 4; j++)
        M[0][j] *= scale;
    if (a.fp64) {
        double2 *out = reinterpret_cast<double2 *>(a.kmat) + w * 8;
        for (int q = 0; q < 2; q++)
            for (int j = 0; j < 4; j++)
                out[q * 4 + j] = make_double2(M[q][j], 0.0);
    } else {
        float2 *out = reinterpret_cast<float2 *>(a.kmat) + w * 8;
        for (int q = 0; q < 2; q++)
            for (int j = 0; j < 4; j++)
                out[q * 4 + j] = make_float2((float)M[q][j], 0.0f);
    }
}

int launch_kraus(const KrausLaunch &a, void *stream)
{
    if (a.nnodes == 0)
        return 0;
    const uint64_t threads = a.nnodes * 32;
    kraus_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Utility kernels
// ---------------------------------------------------------------------------
__global__ void fill_u64_kernel(unsigned long long *p, uint64_t n)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        p[i] = 0ull;
}

int launch_fill_u64(unsigned long long *p, uint64_t n, void *stream)
{
    if (!n)
        return 0;
    const unsigned blocks = (unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    fill_u64_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(p, n);
    return (int)cudaGetLastError();
}

// F_s = (sum_y sqrt(P_id(y) Q(y)))^2 and F_s(P_id, uniform), FP64.  Each block
// writes partial sums; a one-block kernel adds them in a fixed order.
constexpr int kFidBlocks = 256;

template <typename R>
__global__ void __launch_bounds__(256) fidelity_partial(const typename CT<R>::T *ideal,
                                                        const unsigned long long *counts, uint32_t n,
                                                        const uint8_t *perm, double inv_shots,
                                                        double *part)
{
    __shared__ double sh[3][256];
    __shared__ uint8_t P[32];
    if (threadIdx.x < n)
        P[threadIdx.x] = perm[threadIdx.x];
    __syncthreads();
    const uint64_t dim = 1ull << n;
    const double inv_dim = 1.0 / (double)dim;
    double a = 0.0, b = 0.0, t = 0.0;
    for (uint64_t y = (uint64_t)blockIdx.x * 256 + threadIdx.x; y < dim; y += (uint64_t)gridDim.x * 256) {
        uint64_t ph = 0;
        for (uint32_t q = 0; q < n; q++)
            ph |= ((y >> q) & 1ull) << P[q];
        const typename CT<R>::T v = ideal[ph];
        const double p = (double)v.x * (double)v.x + (double)v.y * (double)v.y;
        const double qv = (double)counts[y] * inv_shots;
        a += sqrt(p * qv);
        b += sqrt(p * inv_dim);
        t += p;
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    sh[2][threadIdx.x] = t;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off)
            for (int k = 0; k < 3; k++)
                sh[k][threadIdx.x] += sh[k][threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x < 3)
        part[blockIdx.x * 3 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void fidelity_final(const double *part, int blocks, double *out3)
{
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int i = 0; i < blocks; i++)
            s += part[i * 3 + threadIdx.x];
        out3[threadIdx.x] = s;
    }
}

int launch_fidelity(const void *ideal, int fp64, const unsigned long long *counts, uint32_t n,
                    const uint8_t *perm_dev, uint64_t shots, double *out3, void *stream)
{
    // out3 must have room for 3 + 3*kFidBlocks doubles (partials follow the result)
    double *part = out3 + 3;
    cudaStream_t st = (cudaStream_t)stream;
    const double inv = 1.0 / (double)shots;
    if (fp64)
        fidelity_partial<double><<<kFidBlocks, 256, 0, st>>>((const double2 *)ideal, counts, n, perm_dev, inv, part);
    else
        fidelity_partial<float><<<kFidBlocks, 256, 0, st>>>((const float2 *)ideal, counts, n, perm_dev, inv, part);
    fidelity_final<<<1, 32, 0, st>>>(part, kFidBlocks, out3);
    return (int)cudaGetLastError();
}

}  // namespace tqs
