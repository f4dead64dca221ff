// kernels.cu -- sm_103a kernels of the noisy tree Monte-Carlo path.
//
//   noise_kernel   one warp per tree node: Philox4x32-10 draws for every noise
//                  site of the node's subcircuit (Sec. 2.4) and the node's Pauli
//                  frame (X mask, i-power) at every pass boundary
//   pass_kernel    one CTA per (tile, node): loads a 2^t-amplitude tile of the
//                  parent's (or the node's own) state into shared memory, applies
//                  a run of gates whose non-diagonal qubits all lie in the tile
//                  plus the sampled Paulis (X/Y flip the frame mask, Z/Y flip
//                  signs), then either stores the tile (STORE), writes FP64 block
//                  sums of |a|^2 for measurement (SUMS), or, one CTA per leaf,
//                  picks the outcome from the block sums, recomputes the chosen
//                  tile and samples within it (SAMPLE)
//   fidelity       FP64 reductions for F_s and the normalised fidelity (Sec. 4.1)
//
// The Pauli frame: a node's logical state is psi(x) = i^phase * phi(x ^ mask)
// where phi is what is stored.  An X on qubit q only toggles bit q of the mask,
// a Z multiplies phi by -1 where (x ^ mask) has bit q set, and a gate U on
// qubits Q acts on phi with U conjugated by the mask bits of Q
// (U'[r][c] = U[r ^ mu][c ^ mu]); no Pauli ever moves data.
#include <cuda_runtime.h>

#include "internal.h"

namespace tqs {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the 4x32
// multiply-xor S-box with the Weyl key schedule.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 draw(uint64_t seed, uint64_t id, uint32_t index, uint32_t dom)
{
    return philox4x32_10(make_uint4((uint32_t)id, (uint32_t)(id >> 32), index, dom),
                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// ---------------------------------------------------------------------------
// Complex helpers
// ---------------------------------------------------------------------------
template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };

__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b)
{
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cmadd(C a, C b, C acc)  // acc + a*b
{
    return mk(acc.x + a.x * b.x - a.y * b.y, acc.y + a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cneg(C a) { return mk(-a.x, -a.y); }
template <typename R> __device__ __forceinline__ R norm2(typename CT<R>::T a)
{
    return a.x * a.x + a.y * a.y;
}

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
    NodeMeta par = {0u, 0u};
    if (a.parent_meta) {
        const uint64_t ps = node / a.arity - a.parent_lo;
        par = a.parent_meta[ps * a.parent_stride + a.parent_end];
    }
    uint8_t *nout = a.noise_out + w * a.sites;
    NodeMeta *mout = a.meta_out + w * (a.npass + 1);
    for (uint32_t p = lane; p <= a.npass; p += 32)
        mout[p] = par;
    __syncwarp();
    uint32_t mask = par.mask, phase = par.phase;
    for (uint32_t b = 0; b < a.sites; b += 32) {
        const uint32_t s = b + lane;
        uint32_t xm = 0, yc = 0;
        if (s < a.sites) {
            const Instr I = a.instr[s];
            const uint64_t thr = I.npaulis == 15 ? a.thr2 : a.thr1;
            const uint4 r = draw(a.seed, node, I.gate, kDomNoise);
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
            nout[s] = (uint8_t)pz;
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
            // boundary p (1..npass) sits after site pass_start[p]-1
            for (uint32_t p = 1; p <= a.npass; p++)
                if (a.pass_start[p] == s + 1)
                    mout[p] = NodeMeta{mask ^ xm, (phase + yc) & 3u};
        }
        mask ^= __shfl_sync(0xffffffffu, xm, 31);
        phase += __shfl_sync(0xffffffffu, yc, 31);
    }
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

// ---------------------------------------------------------------------------
// Pass kernel
// ---------------------------------------------------------------------------
struct PassK {
    const void *in;
    void *out;
    uint64_t state_elems;
    uint64_t node_lo, parent_lo, arity;
    const Instr *instr;
    const void *mats;
    const uint8_t *noise;
    const NodeMeta *meta;
    double *S;
    unsigned long long *counts;
    uint64_t seed, thrm;
    uint32_t ibeg, iend, n, t, L, sites, meta_stride, pass_local;
    int in_from_parent;
    uint8_t tbits[kMaxTile];
    uint8_t hbits[32];
    SamplerLayout samp;
};

// Block-wide inclusive scan of one double per thread (kThreads threads).
__device__ __forceinline__ double block_incl_scan(double v, double *wsum)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off)
            v += t;
    }
    if (lane == 31)
        wsum[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double x = lane < kThreads / 32 ? wsum[lane] : 0.0;
#pragma unroll
        for (int off = 1; off < kThreads / 32; off <<= 1) {
            const double t = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off)
                x += t;
        }
        if (lane < kThreads / 32)
            wsum[lane] = x;
    }
    __syncthreads();
    const double r = v + (wid ? wsum[wid - 1] : 0.0);
    __syncthreads();
    return r;
}

// Smallest index in [0, count) of the sequence `val(i)` (nonnegative) whose
// running sum exceeds `target`, computed as per-thread contiguous chunks, a
// block scan of the chunk sums, and a sequential walk inside the winning chunk.
// Returns the index and (via *resid) target minus the sum before it; if the
// rounding leaves no such index it returns the last index with a nonzero value
// and resid = +inf.  All threads get the result.
template <typename F>
__device__ uint64_t block_pick(uint64_t count, double target, F val, double *resid, double *sh,
                               unsigned long long *shu)
{
    const uint64_t chunk = (count + kThreads - 1) / kThreads;
    const uint64_t b = (uint64_t)threadIdx.x * chunk;
    const uint64_t e = b + chunk < count ? b + chunk : count;
    double local = 0.0;
    uint64_t lastnz = ~0ull;
    for (uint64_t i = b; i < e; i++) {
        const double v = val(i);
        local += v;
        if (v > 0.0)
            lastnz = i;
    }
    if (threadIdx.x == 0) {
        shu[0] = ~0ull;  // winner thread
        shu[1] = 0ull;   // last nonzero + 1 (max)
    }
    const double incl = block_incl_scan(local, sh);
    // exclusive = inclusive of the previous thread, exactly
    sh[threadIdx.x] = incl;
    __syncthreads();
    const double excl = threadIdx.x ? sh[threadIdx.x - 1] : 0.0;
    if (b < e && excl <= target && incl > target)
        atomicMin(&shu[0], (unsigned long long)threadIdx.x);
    if (lastnz != ~0ull)
        atomicMax(&shu[1], lastnz + 1);
    __syncthreads();
    if (threadIdx.x == shu[0]) {
        double acc = excl;
        uint64_t pick = ~0ull;
        double rs = 0.0;
        for (uint64_t i = b; i < e; i++) {
            const double v = val(i);
            const double before = acc;
            acc += v;
            if (acc > target) {
                pick = i;
                rs = target - before;
                break;
            }
        }
        if (pick == ~0ull) {
            pick = lastnz;
            rs = __longlong_as_double(0x7ff0000000000000ll);
        }
        shu[2] = pick;
        sh[0] = rs;
    }
    __syncthreads();
    uint64_t pick;
    double rs;
    if (shu[0] == ~0ull) {
        pick = shu[1] ? shu[1] - 1 : 0;
        rs = __longlong_as_double(0x7ff0000000000000ll);
    } else {
        pick = shu[2];
        rs = sh[0];
    }
    __syncthreads();
    *resid = rs;
    return pick;
}

template <typename R, int MODE>
__global__ void __launch_bounds__(kThreads) pass_kernel(const __grid_constant__ PassK a)
{
    using C = typename CT<R>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t TE = 1u << a.t;
    const uint32_t nhi = a.t - a.L;
    C *s = reinterpret_cast<C *>(smem);
    uint32_t *dep = reinterpret_cast<uint32_t *>(s + TE);
    uint16_t *lut = reinterpret_cast<uint16_t *>(dep + ((1u << nhi) < 4u ? 4u : (1u << nhi)));  // 256 entries
    double *red = reinterpret_cast<double *>(lut + 256);                   // kThreads doubles
    unsigned long long *shu = reinterpret_cast<unsigned long long *>(red + kThreads);  // 4
    const int tid = threadIdx.x;
    const uint32_t lomask = (1u << a.L) - 1u;

    const uint32_t slot = (MODE == MODE_SAMPLE) ? blockIdx.x : blockIdx.y;
    const uint64_t node = a.node_lo + slot;
    const NodeMeta m0 = a.meta[(uint64_t)slot * a.meta_stride + a.pass_local];
    const NodeMeta m1 = a.meta[(uint64_t)slot * a.meta_stride + a.pass_local + 1];

    for (uint32_t i = tid; i < (1u << nhi); i += kThreads) {
        uint32_t d = 0;
        for (uint32_t b = 0; b < nhi; b++)
            if ((i >> b) & 1u)
                d |= 1u << a.tbits[a.L + b];
        dep[i] = d;
    }
    const SamplerLayout &SL = a.samp;
    if (MODE != MODE_STORE) {
        // unkey tables: rank bits 0..6 -> tile positions (lut[0..127]), 7..13 -> lut[128..255]
        for (uint32_t i = tid; i < 256; i += kThreads) {
            const uint32_t rb = i < 128 ? 0 : 7, v = i & 127;
            uint32_t e = 0;
            for (uint32_t b = 0; b < 7 && rb + b < a.t; b++)
                if ((v >> b) & 1u)
                    e |= 1u << SL.rank_pos[rb + b];
            lut[i] = (uint16_t)e;
        }
    }

    // ---- which tile ------------------------------------------------------
    uint32_t base = 0;
    uint64_t gstar = 0;
    double resid = 0.0;
    if (MODE != MODE_SAMPLE) {
        const uint32_t h = blockIdx.x;
        for (uint32_t b = 0; b < a.n - a.t; b++)
            if ((h >> b) & 1u)
                base |= 1u << a.hbits[b];
    } else {
        // stage 1: outcome block from the block sums of this leaf
        const double *Sl = a.S + (uint64_t)slot * SL.groups;
        const uint4 r = draw(a.seed, node, 0u, kDomMeas);
        const double u = ((double)(r.x >> 5) * 67108864.0 + (double)(r.y >> 6)) * (1.0 / 9007199254740992.0);
        // total (same chunked order as the pick)
        const uint64_t chunk = (SL.groups + kThreads - 1) / kThreads;
        double local = 0.0;
        for (uint64_t i = (uint64_t)tid * chunk; i < SL.groups && i < (uint64_t)(tid + 1) * chunk; i++)
            local += Sl[i];
        const double tot = block_incl_scan(local, red);
        if (tid == kThreads - 1)
            red[kThreads / 32] = tot;  // slot after the warp sums
        __syncthreads();
        const double total = red[kThreads / 32];
        __syncthreads();
        gstar = block_pick(SL.groups, u * total, [&](uint64_t i) { return Sl[i]; }, &resid, red, shu);
        const uint32_t fm = m1.mask;
        for (uint32_t q = SL.gamma; q < a.n; q++) {
            const uint32_t bit = (uint32_t)(gstar >> (q - SL.gamma)) & 1u;
            if (SL.rank_of_logical[q] < 0) {
                const uint32_t pb = SL.phys_of_logical[q];
                base |= (bit ^ ((fm >> pb) & 1u)) << pb;
            }
        }
    }
    __syncthreads();

    // ---- load ------------------------------------------------------------
    const uint64_t in_slot = a.in_from_parent ? (node / a.arity - a.parent_lo) : slot;
    const bool synth = a.in == nullptr;
    const bool zero_tile = synth && base != 0;
    {
        const C *src = synth ? nullptr : reinterpret_cast<const C *>(a.in) + in_slot * a.state_elems;
        for (uint32_t e = tid; e < TE; e += kThreads) {
            const uint32_t ph = base | dep[e >> a.L] | (e & lomask);
            C v;
            if (synth)
                v = mk((R)(ph == 0 ? 1 : 0), (R)0);
            else
                v = src[ph];
            s[e] = v;
        }
    }

    // ---- gates and noise -----------------------------------------------
    uint32_t mask = m0.mask;
    const R *mats = reinterpret_cast<const R *>(a.mats);
    const uint8_t *nz = a.noise + (uint64_t)slot * a.sites;
    bool last_dense = true;  // the load wrote with element ownership; dense ops re-pair
    if (!zero_tile) {
        for (uint32_t ii = a.ibeg; ii < a.iend; ii++) {
            const Instr I = a.instr[ii];
            const R *M = mats + (size_t)I.gate * 32;
            if (I.op == OP_DENSE1) {
                __syncthreads();
                const uint32_t mu = (mask >> I.p0) & 1u;
                const C u00 = mk(M[2 * (0 ^ (mu * 3))], M[2 * (0 ^ (mu * 3)) + 1]);
                const C u01 = mk(M[2 * (1 ^ (mu * 3))], M[2 * (1 ^ (mu * 3)) + 1]);
                const C u10 = mk(M[2 * (2 ^ (mu * 3))], M[2 * (2 ^ (mu * 3)) + 1]);
                const C u11 = mk(M[2 * (3 ^ (mu * 3))], M[2 * (3 ^ (mu * 3)) + 1]);
                const uint32_t j = I.j0, lm = (1u << j) - 1u;
                for (uint32_t pi = tid; pi < TE / 2; pi += kThreads) {
                    const uint32_t e0 = ((pi & ~lm) << 1) | (pi & lm), e1 = e0 | (1u << j);
                    const C x0 = s[e0], x1 = s[e1];
                    s[e0] = cmadd(u01, x1, cmul(u00, x0));
                    s[e1] = cmadd(u11, x1, cmul(u10, x0));
                }
                last_dense = true;
            } else if (I.op == OP_DENSE2) {
                __syncthreads();
                const uint32_t mu = ((mask >> I.p0) & 1u) | (((mask >> I.p1) & 1u) << 1);
                C u[16];
#pragma unroll
                for (int r = 0; r < 4; r++)
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        const int k = ((r ^ mu) * 4 + (c ^ mu));
                        u[r * 4 + c] = mk(M[2 * k], M[2 * k + 1]);
                    }
                const uint32_t ja = I.j0 < I.j1 ? I.j0 : I.j1, jb = I.j0 < I.j1 ? I.j1 : I.j0;
                const uint32_t la = (1u << ja) - 1u, lb = (1u << jb) - 1u;
                for (uint32_t qi = tid; qi < TE / 4; qi += kThreads) {
                    uint32_t e = ((qi & ~la) << 1) | (qi & la);
                    e = ((e & ~lb) << 1) | (e & lb);
                    uint32_t idx[4];
                    C x[4];
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        idx[k] = e | ((k & 1) ? (1u << I.j0) : 0u) | ((k & 2) ? (1u << I.j1) : 0u);
                        x[k] = s[idx[k]];
                    }
#pragma unroll
                    for (int r = 0; r < 4; r++) {
                        C acc = cmul(u[r * 4], x[0]);
#pragma unroll
                        for (int c = 1; c < 4; c++)
                            acc = cmadd(u[r * 4 + c], x[c], acc);
                        s[idx[r]] = acc;
                    }
                }
                last_dense = true;
            } else if (I.op == OP_DIAG1 || I.op == OP_DIAG2) {
                if (last_dense)
                    __syncthreads();
                const C d0 = mk(M[0], M[1]), d1 = mk(M[2], M[3]);
                C d2 = d0, d3 = d1;
                if (I.op == OP_DIAG2) {
                    d2 = mk(M[4], M[5]);
                    d3 = mk(M[6], M[7]);
                }
                const uint32_t p1 = I.op == OP_DIAG2 ? I.p1 : I.p0;
                for (uint32_t e = tid; e < TE; e += kThreads) {
                    const uint32_t x = (base | dep[e >> a.L] | (e & lomask)) ^ mask;
                    const uint32_t k = ((x >> I.p0) & 1u) | (I.op == OP_DIAG2 ? (((x >> p1) & 1u) << 1) : 0u);
                    const C d = k == 0 ? d0 : (k == 1 ? d1 : (k == 2 ? d2 : d3));
                    s[e] = cmul(s[e], d);
                }
                last_dense = false;
            }
            // the noise site after this gate
            const uint32_t pz = nz[I.site];
            if (pz) {
                const uint32_t wa = I.npaulis == 15 ? (pz >> 2) : pz;
                const uint32_t wb = I.npaulis == 15 ? (pz & 3u) : 0u;
                const uint32_t zmask = ((wa >= 2) ? (1u << I.np0) : 0u) | ((wb >= 2) ? (1u << I.np1) : 0u);
                if (zmask) {
                    if (last_dense)
                        __syncthreads();
                    for (uint32_t e = tid; e < TE; e += kThreads) {
                        const uint32_t x = (base | dep[e >> a.L] | (e & lomask)) ^ mask;
                        if (__popc(x & zmask) & 1)
                            s[e] = cneg(s[e]);
                    }
                    last_dense = false;
                }
                if (wa == 1 || wa == 2) mask ^= 1u << I.np0;
                if (wb == 1 || wb == 2) mask ^= 1u << I.np1;
            }
        }
    } else {
        mask = m1.mask;
    }
    __syncthreads();

    // ---- epilogue ------------------------------------------------------
    if (MODE == MODE_STORE) {
        C *dst = reinterpret_cast<C *>(a.out) + (uint64_t)slot * a.state_elems;
        for (uint32_t e = tid; e < TE; e += kThreads)
            dst[base | dep[e >> a.L] | (e & lomask)] = s[e];
        return;
    }

    // tile-coordinate frame mask (final frame)
    uint32_t mT = 0;
    for (uint32_t j = 0; j < a.t; j++)
        mT |= ((mask >> a.tbits[j]) & 1u) << j;
    const uint32_t G = 1u << SL.gamma;
    auto elem_of_key = [&](uint32_t key) -> uint32_t {
        return ((uint32_t)lut[key & 127] | (uint32_t)lut[128 + ((key >> 7) & 127)]) ^ mT;
    };

    if (MODE == MODE_SUMS) {
        // H-bit part of the global group index of this tile
        uint64_t hpart = 0;
        for (uint32_t b = 0; b < a.n - a.t; b++) {
            const uint32_t pb = a.hbits[b];
            hpart |= (uint64_t)(((base ^ mask) >> pb) & 1u) << (SL.logical_of_hbit[b] - SL.gamma);
        }
        const uint32_t GPT = TE >> SL.gamma;                 // groups in this tile
        uint32_t TPG = GPT >= kThreads ? 1u : kThreads / GPT; // threads per group
        if (TPG > G) TPG = G;
        const uint32_t KPT = G / TPG;                         // keys per thread
        const uint32_t nwork = GPT * TPG;
        for (uint32_t wbase = 0; wbase < nwork; wbase += kThreads) {
            const uint32_t wi = wbase + tid;
            double part = 0.0;
            uint32_t grp = 0;
            if (wi < nwork) {
                grp = wi / TPG;
                const uint32_t k0 = grp * G + (wi % TPG) * KPT;
                R acc = 0;
                for (uint32_t k = 0; k < KPT; k++) {
                    acc += norm2<R>(s[elem_of_key(k0 + k)]);
                    if (((k + 1) & 15u) == 0) {
                        part += (double)acc;
                        acc = 0;
                    }
                }
                part += (double)acc;
            }
            // reduce over the TPG consecutive threads of each group
            if (TPG <= 32) {
                for (uint32_t off = 1; off < TPG; off <<= 1)
                    part += __shfl_xor_sync(0xffffffffu, part, off);
                if (wi < nwork && (wi % TPG) == 0) {
                    uint64_t g = hpart;
                    const uint32_t keyhi = grp;  // rank bits >= gamma of this group
                    for (uint32_t r = SL.gamma; r < a.t; r++)
                        g |= (uint64_t)((keyhi >> (r - SL.gamma)) & 1u) << (SL.rank_q[r] - SL.gamma);
                    a.S[(uint64_t)slot * SL.groups + g] = part;
                }
            } else {
                red[tid] = part;
                __syncthreads();
                if (wi < nwork && (wi % TPG) == 0) {
                    double sum = 0.0;
                    for (uint32_t k = 0; k < TPG; k++)
                        sum += red[tid + k];
                    uint64_t g = hpart;
                    for (uint32_t r = SL.gamma; r < a.t; r++)
                        g |= (uint64_t)((grp >> (r - SL.gamma)) & 1u) << (SL.rank_q[r] - SL.gamma);
                    a.S[(uint64_t)slot * SL.groups + g] = sum;
                }
                __syncthreads();
            }
        }
        return;
    }

    // MODE_SAMPLE stage 2: inside the chosen block of 2^gamma outcomes
    uint32_t keyhi = 0;
    for (uint32_t q = SL.gamma; q < a.n; q++) {
        const int r = SL.rank_of_logical[q];
        if (r >= 0)
            keyhi |= (uint32_t)((gstar >> (q - SL.gamma)) & 1u) << (r - SL.gamma);
    }
    const uint32_t kbase = keyhi << SL.gamma;
    double r2;
    const uint64_t wstar = block_pick(G, resid, [&](uint64_t w) {
        return (double)norm2<R>(s[elem_of_key(kbase + (uint32_t)w)]);
    }, &r2, red, shu);
    if (tid < 32) {
        const uint64_t y = (gstar << SL.gamma) | wstar;
        bool flip = false;
        if ((uint32_t)tid < a.n) {
            const uint4 rr = draw(a.seed, node, (uint32_t)tid, kDomRead);
            flip = (uint64_t)rr.x < a.thrm;
        }
        const uint32_t fl = __ballot_sync(0xffffffffu, flip);
        if (tid == 0)
            atomicAdd(&a.counts[y ^ (uint64_t)fl], 1ull);
    }
}

template <typename R, int MODE>
static int launch_pass_t(const PassK &k, dim3 grid, size_t smem, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(pass_kernel<R, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    pass_kernel<R, MODE><<<grid, kThreads, smem, st>>>(k);
    return (int)cudaGetLastError();
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
    k.mats = a.mats;
    k.noise = a.noise;
    k.meta = a.meta;
    k.S = a.S;
    k.counts = a.counts;
    k.seed = a.seed;
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
    const size_t ndep = ((size_t)1 << (a.t - a.L)) < 4 ? 4 : ((size_t)1 << (a.t - a.L));
    const size_t smem = ((size_t)1 << a.t) * elem + ndep * 4 + 256 * 2 + kThreads * 8 + 4 * 8;
    const uint64_t tiles = (uint64_t)1 << (a.n - a.t);
    dim3 grid = a.mode == MODE_SAMPLE ? dim3(a.nnodes) : dim3((unsigned)tiles, a.nnodes);
    cudaStream_t st = (cudaStream_t)stream;
    if (a.fp64) {
        if (a.mode == MODE_STORE) return launch_pass_t<double, MODE_STORE>(k, grid, smem, st);
        if (a.mode == MODE_SUMS) return launch_pass_t<double, MODE_SUMS>(k, grid, smem, st);
        return launch_pass_t<double, MODE_SAMPLE>(k, grid, smem, st);
    }
    if (a.mode == MODE_STORE) return launch_pass_t<float, MODE_STORE>(k, grid, smem, st);
    if (a.mode == MODE_SUMS) return launch_pass_t<float, MODE_SUMS>(k, grid, smem, st);
    return launch_pass_t<float, MODE_SAMPLE>(k, grid, smem, st);
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
