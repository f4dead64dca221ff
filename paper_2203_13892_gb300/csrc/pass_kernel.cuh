// pass_kernel.cuh -- the state-vector pass kernel (definitions).
//
//   pass_kernel    one CTA per (tile, node): loads a 2^t-amplitude tile of the
//                  parent's (or the node's own) state into shared memory, applies
//                  a run of gates whose non-diagonal qubits all lie in the tile
//                  plus the sampled Paulis (X/Y flip the frame mask, Z/Y flip
//                  signs), then either stores the tile (STORE), writes FP64 block
//                  sums of |a|^2 for measurement (SUMS), or, one CTA per leaf,
//                  picks the outcome from the block sums, recomputes the chosen
//                  tile and samples within it (SAMPLE)
//
// The Pauli frame: a node's logical state is psi(x) = i^phase * phi(x ^ mask)
// where phi is what is stored.  An X on qubit q only toggles bit q of the mask,
// a Z multiplies phi by -1 where (x ^ mask) has bit q set, and a gate U on
// qubits Q acts on phi with U conjugated by the mask bits of Q
// (U'[r][c] = U[r ^ mu][c ^ mu]); no Pauli ever moves data.
#pragma once
#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>

#include <atomic>
#endif

#include "device_common.cuh"
#include "pass_kernel.h"

namespace tqs {

// ---------------------------------------------------------------------------
// Blackwell tensor-core helpers (tcgen05 / TMEM / mbarrier), used by fused gates
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major operand without swizzle; lbo / sbo are
// the byte distances between core matrices adjacent in K / in the row dimension.
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of tcgen05.mma .kind::tf32: D F32, A and B TF32, both K-major.
__host__ __device__ constexpr uint32_t tc_idesc_tf32(uint32_t M, uint32_t N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void tc_alloc(uint32_t slot_saddr, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_saddr), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar_saddr)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_saddr)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar_saddr, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar_saddr), "r"(count) : "memory");
}

// Bounded wait for phase `parity` of an mbarrier: true when it completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar_saddr, uint32_t parity, uint32_t max_iter)
{
    for (uint32_t it = 0; it < max_iter; it++) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(mbar_saddr), "r"(parity)
            : "memory");
        if (ok)
            return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 lanes x 32 bits x 16 columns from TMEM (this warp's lane quarter).
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&r)[16])
{
    uint32_t u[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
          "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++)
        r[i] = __uint_as_float(u[i]);
}

__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// ---------------------------------------------------------------------------
// Pass kernel
// ---------------------------------------------------------------------------

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
        if (__double_as_longlong(v) != 0)  // values are >= 0: nonzero iff any bit set
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

// Per-thread accumulator of a run of diagonal factors (Pauli Z signs included).
// A diagonal block is D(x) = prod_g G_g * prod_q a_q^{x_q} * prod_{q<r} c_qr^{x_q x_r}
// over logical bits x.  The thread knows its own bits on thread positions and
// the CTA's bits outside the tile, so those factors collapse into `base`; a
// factor on a slot bit s (register index bit) goes to E[s]; slot-slot pairs go to
// Gs.  Applying the block costs one complex product per amplitude.
template <typename C, int NS> struct DiagAcc {
    using V = C;  // a factor's value: the complex number itself
    C base;
    C E[NS > 0 ? NS : 1];
    C Gs[NS > 1 ? NS * (NS - 1) / 2 : 1];
    bool has_gs;
    bool base_used;    // some factor went to `base` (uniform, whatever its condition gave)
    uint32_t e_used;   // slot factors that some gate touched (uniform)
    uint32_t gs_used;  // slot pairs that some gate touched (uniform)
    __device__ __forceinline__ void reset()
    {
        base = mk((decltype(base.x))1, (decltype(base.x))0);
#pragma unroll
        for (int s = 0; s < NS; s++)
            E[s] = base;
#pragma unroll
        for (int i = 0; i < (NS > 1 ? NS * (NS - 1) / 2 : 1); i++)
            Gs[i] = base;
        has_gs = false;
        base_used = false;
        e_used = 0;
        gs_used = 0;
    }
    static __device__ __forceinline__ C minus_one() { return mk((decltype(C{}.x))-1, (decltype(C{}.x))0); }
    __device__ __forceinline__ void mul_base(C f)
    {
        base = cmul(base, f);
        base_used = true;
    }
    // a factor on fixed bits: applies to this thread iff `c`, but marks `base` as
    // used on every thread so that the flush stays uniform
    __device__ __forceinline__ void mul_base_if(bool c, C f)
    {
        base_used = true;
        if (c)
            base = cmul(base, f);
    }
    __device__ __forceinline__ void mul_E(int s, C f)
    {
        e_used |= 1u << s;
        // s is uniform across the CTA: a branch, not predicated copies
        switch (s) {
        case 0: if (NS > 0) E[0] = cmul(E[0], f); break;
        case 1: if (NS > 1) E[NS > 1 ? 1 : 0] = cmul(E[NS > 1 ? 1 : 0], f); break;
        case 2: if (NS > 2) E[NS > 2 ? 2 : 0] = cmul(E[NS > 2 ? 2 : 0], f); break;
        case 3: if (NS > 3) E[NS > 3 ? 3 : 0] = cmul(E[NS > 3 ? 3 : 0], f); break;
        default: if (NS > 4) E[NS > 4 ? 4 : 0] = cmul(E[NS > 4 ? 4 : 0], f); break;
        }
    }
    __device__ __forceinline__ void mul_Gs(int s0, int s1, C f)
    {
        const int hi = s0 > s1 ? s0 : s1, lo = s0 > s1 ? s1 : s0;
        const int idx = hi * (hi - 1) / 2 + lo;
#pragma unroll
        for (int k = 0; k < (NS > 1 ? NS * (NS - 1) / 2 : 1); k++)
            if (k == idx)
                Gs[k] = cmul(Gs[k], f);
        has_gs = true;
        gs_used |= 1u << idx;
        e_used |= (1u << s0) | (1u << s1);
    }
};

// FP32 states: every diagonal factor of the gates this library classes as
// diagonal (Z, S, T, RZ, P, CZ, CP and their noise Z parts) has modulus one, so
// the block is accumulated as a phase: an unsigned 32-bit fraction of a full
// turn per accumulator (addition modulo 2^32 is addition of angles modulo 2 pi,
// exact), and turned into complex factors only when the block is applied.
// Compared with complex accumulators this halves the registers the block
// holds (11 instead of 22 for 16 register slots) and replaces each factor's
// complex product by one integer add.
template <int NS> struct DiagAcc<float2, NS> {
    using V = uint32_t;  // a factor's phase in units of 2^-32 turns
    uint32_t base;
    uint32_t E[NS > 0 ? NS : 1];
    uint32_t Gs[NS > 1 ? NS * (NS - 1) / 2 : 1];
    bool has_gs;
    bool base_used;    // some factor went to `base` (uniform)
    uint32_t e_used;   // slot factors that some gate touched (uniform)
    uint32_t gs_used;  // slot pairs that some gate touched (uniform)
    __device__ __forceinline__ void reset()
    {
        base = 0u;
#pragma unroll
        for (int s = 0; s < NS; s++)
            E[s] = 0u;
#pragma unroll
        for (int i = 0; i < (NS > 1 ? NS * (NS - 1) / 2 : 1); i++)
            Gs[i] = 0u;
        has_gs = false;
        base_used = false;
        e_used = 0;
        gs_used = 0;
    }
    static __device__ __forceinline__ uint32_t minus_one() { return 0x80000000u; }  // half a turn
    __device__ __forceinline__ void mul_base(uint32_t f)
    {
        base += f;
        base_used = true;
    }
    __device__ __forceinline__ void mul_base_if(bool c, uint32_t f)
    {
        base_used = true;
        if (c)
            base += f;
    }
    __device__ __forceinline__ void mul_E(int s, uint32_t f)
    {
        e_used |= 1u << s;
        switch (s) {
        case 0: if (NS > 0) E[0] += f; break;
        case 1: if (NS > 1) E[NS > 1 ? 1 : 0] += f; break;
        case 2: if (NS > 2) E[NS > 2 ? 2 : 0] += f; break;
        case 3: if (NS > 3) E[NS > 3 ? 3 : 0] += f; break;
        default: if (NS > 4) E[NS > 4 ? 4 : 0] += f; break;
        }
    }
    __device__ __forceinline__ void mul_Gs(int s0, int s1, uint32_t f)
    {
        const int hi = s0 > s1 ? s0 : s1, lo = s0 > s1 ? s1 : s0;
        const int idx = hi * (hi - 1) / 2 + lo;
#pragma unroll
        for (int k = 0; k < (NS > 1 ? NS * (NS - 1) / 2 : 1); k++)
            if (k == idx)
                Gs[k] += f;
        has_gs = true;
        gs_used |= 1u << idx;
    }
    // The frame mask bit of slot s flips (an X or Y drawn on that qubit) while
    // phases are pending.  They were accumulated against the logical slot bit
    // x_s of the old frame, which is 1 - y_s in the new one; substituting gives
    // base += E_s, E_s -> -E_s, and for every pair (s, t): E_t += G_st,
    // G_st -> -G_st.  So X noise needs no flush of the pending phases.
    __device__ __forceinline__ void flip(int s)
    {
#pragma unroll
        for (int q = 0; q < NS; q++) {
            if (q != s)
                continue;
            if ((e_used >> q) & 1u) {
                base += E[q];
                base_used = true;
                E[q] = 0u - E[q];
            }
#pragma unroll
            for (int t = 0; t < NS; t++) {
                if (t == q)
                    continue;
                const int hi = q > t ? q : t, lo = q > t ? t : q, idx = hi * (hi - 1) / 2 + lo;
                if ((gs_used >> idx) & 1u) {
                    E[t] += Gs[idx];
                    e_used |= 1u << t;
                    Gs[idx] = 0u - Gs[idx];
                }
            }
        }
    }
};

// exp(2 pi i a / 2^32) for a phase a in units of 2^-32 turns.  The phase is
// taken into [-pi, pi) as a signed integer and converted to float (rounded to
// 24 bits: at most 1e-7 rad off), then passed to the hardware sine and cosine
// (absolute error about 4e-7 on [-pi, pi]).  The conversion runs on the
// transcendental unit, which the passes leave mostly idle, not on the integer
// pipe they saturate.
__device__ __forceinline__ float2 expi_turn(uint32_t a)
{
    float sn, cs;
    __sincosf((float)(int32_t)a * 1.4629181e-09f, &sn, &cs);  // 2 pi / 2^32
    return make_float2(cs, sn);
}

// Phase of a unit complex number in units of 2^-32 turns (rare paths only).
__device__ __forceinline__ uint32_t turn_of(float re, float im)
{
    const double t = (double)atan2f(im, re) * (4294967296.0 / 6.283185307179586);
    return (uint32_t)(int64_t)llrint(t);
}

// tile position j: thread bit (j < 8 or tile smaller than the CTA), slot bit s = j-8, or outside (0xff)
__device__ __forceinline__ bool thread_or_outside(uint32_t j) { return j == 0xffu || j < 8u; }

template <typename C, int NS>
__device__ __forceinline__ void acc_alpha(DiagAcc<C, NS> &A, uint32_t j, uint32_t p, uint32_t xt,
                                          typename DiagAcc<C, NS>::V f)
{
    if (thread_or_outside(j))
        A.mul_base_if(((xt >> p) & 1u) != 0u, f);
    else
        A.mul_E((int)j - 8, f);
}

template <typename C, int NS>
__device__ __forceinline__ void acc_gamma(DiagAcc<C, NS> &A, uint32_t j0, uint32_t p0, uint32_t j1, uint32_t p1,
                                          uint32_t xt, typename DiagAcc<C, NS>::V f)
{
    const bool a = thread_or_outside(j0), b = thread_or_outside(j1);
    if (a && b) {
        A.mul_base_if(((xt >> p0) & (xt >> p1) & 1u) != 0u, f);
    } else if (a) {
        if ((xt >> p0) & 1u)
            A.mul_E((int)j1 - 8, f);
    } else if (b) {
        if ((xt >> p1) & 1u)
            A.mul_E((int)j0 - 8, f);
    } else {
        A.mul_Gs((int)j0 - 8, (int)j1 - 8, f);
    }
}

template <typename C> __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }

// Multiply the NR register amplitudes by the accumulated diagonal.  msig: the
// frame mask restricted to the slot bits (bit s = mask bit of slot position s).
template <typename C, int LOGR>
__device__ __forceinline__ void acc_flush(DiagAcc<C, LOGR> &A, C (&v)[1 << LOGR], uint32_t msig)
{
    constexpr int NR = 1 << LOGR;
    // rewrite the slot factors from logical bits x_s = b_s ^ m_s to register bits b_s
    C Eb[LOGR > 0 ? LOGR : 1];
    C base = A.base;
#pragma unroll
    for (int s = 0; s < LOGR; s++) {
        if ((msig >> s) & 1u) {
            base = cmul(base, A.E[s]);
            Eb[s] = cconj(A.E[s]);
        } else {
            Eb[s] = A.E[s];
        }
    }
    bool bmul = A.base_used || (msig & A.e_used) != 0u;  // uniform: does base differ from 1?
    C Gb[LOGR > 1 ? LOGR * (LOGR - 1) / 2 : 1];
    if (A.has_gs) {
#pragma unroll
        for (int hi = 1; hi < LOGR; hi++)
#pragma unroll
            for (int lo = 0; lo < hi; lo++) {
                const int idx = hi * (hi - 1) / 2 + lo;
                if (!((A.gs_used >> idx) & 1u)) {
                    Gb[idx] = A.Gs[idx];
                    continue;
                }
                const C g = A.Gs[idx];
                const uint32_t mh = (msig >> hi) & 1u, ml = (msig >> lo) & 1u;
                if (!mh && !ml) {
                    Gb[idx] = g;
                } else if (mh && !ml) {
                    Eb[lo] = cmul(Eb[lo], g);
                    Gb[idx] = cconj(g);
                } else if (!mh && ml) {
                    Eb[hi] = cmul(Eb[hi], g);
                    Gb[idx] = cconj(g);
                } else {
                    base = cmul(base, g);
                    bmul = true;
                    Eb[lo] = cmul(Eb[lo], cconj(g));
                    Eb[hi] = cmul(Eb[hi], cconj(g));
                    Gb[idx] = g;
                }
            }
    }
    // v[k] *= base * prod_{s in k} Eb[s] * prod_{s<s' in k} Gb: one pass per factor
    if (bmul) {
#pragma unroll
        for (int k = 0; k < NR; k++)
            v[k] = cmul(v[k], base);
    }
#pragma unroll
    for (int sb = 0; sb < LOGR; sb++) {
        if (!((A.e_used >> sb) & 1u) && !((msig >> sb) & 1u))
            continue;  // untouched slot factor: exactly 1
#pragma unroll
        for (int k = 0; k < NR; k++)
            if ((k >> sb) & 1)
                v[k] = cmul(v[k], Eb[sb]);
    }
    if (A.has_gs) {
#pragma unroll
        for (int hi = 1; hi < LOGR; hi++)
#pragma unroll
            for (int lo = 0; lo < hi; lo++) {
                if (!((A.gs_used >> (hi * (hi - 1) / 2 + lo)) & 1u))
                    continue;
#pragma unroll
                for (int k = 0; k < NR; k++)
                    if (((k >> hi) & 1) && ((k >> lo) & 1))
                        v[k] = cmul(v[k], Gb[hi * (hi - 1) / 2 + lo]);
            }
    }
    A.reset();
}

// v[k] *= exp(i B) on the registers without bit S, exp(i (B + Es)) on those with it.
template <int LOGR, int S>
__device__ __forceinline__ void apply_one_slot(float2 (&v)[1 << LOGR], uint32_t B, uint32_t Es, bool bmul)
{
    if constexpr (S < LOGR) {
        const float2 f1 = expi_turn(B + Es);
        float2 f0 = make_float2(1.0f, 0.0f);
        if (bmul)
            f0 = expi_turn(B);
#pragma unroll
        for (int k = 0; k < (1 << LOGR); k++) {
            if ((k >> S) & 1)
                v[k] = cmul(v[k], f1);
            else if (bmul)
                v[k] = cmul(v[k], f0);
        }
    }
}

// FP32: multiply the NR register amplitudes by exp(i * phase(k)) where the
// phase of register k is the accumulated quadratic form
//   Q(x) = base + sum_s E_s x_s + sum_{s<t} G_st x_s x_t  at logical slot bits
// x = k ^ msig.  With a frame mask the form is first rewritten in the register
// bits b (x_s = 1 - b_s where m_s = 1): base' = Q(m), G'_st = -G_st when exactly
// one of m_s, m_t is set, E'_s = (-1)^{m_s} (E_s + sum_{t != s, m_t} G_st).
template <int LOGR>
__device__ __forceinline__ void acc_flush(DiagAcc<float2, LOGR> &A, float2 (&v)[1 << LOGR], uint32_t msig)
{
    constexpr int NR = 1 << LOGR;
    if (A.e_used == 0u && A.gs_used == 0u) {
        // the common case of runs on thread and outside-tile bits only: one
        // phase per thread, whatever the frame mask
        if (A.base_used) {
            const float2 eb = expi_turn(A.base);
#pragma unroll
            for (int k = 0; k < NR; k++)
                v[k] = cmul(v[k], eb);
        }
        A.reset();
        return;
    }
    constexpr int NP = LOGR > 1 ? LOGR * (LOGR - 1) / 2 : 1;
    uint32_t B = A.base;
    uint32_t E[LOGR > 0 ? LOGR : 1], G[NP];
#pragma unroll
    for (int s = 0; s < LOGR; s++)
        E[s] = A.E[s];
#pragma unroll
    for (int i = 0; i < NP; i++)
        G[i] = A.Gs[i];
    // Slot factors in use (uniform): those some gate touched and, under a frame
    // mask, those a masked pair partner turns into linear ones.
    uint32_t eu = A.e_used;
#pragma unroll
    for (int hi = 1; hi < LOGR; hi++)
#pragma unroll
        for (int lo = 0; lo < hi; lo++)
            if ((A.gs_used >> (hi * (hi - 1) / 2 + lo)) & 1u) {
                if ((msig >> hi) & 1u)
                    eu |= 1u << lo;
                if ((msig >> lo) & 1u)
                    eu |= 1u << hi;
            }
    const bool bmul = A.base_used || (msig & eu) != 0u;  // base may differ from 0 (uniform)
    if (msig != 0u) {
        uint32_t En[LOGR > 0 ? LOGR : 1];
#pragma unroll
        for (int s = 0; s < LOGR; s++) {
            const bool ms = (msig >> s) & 1u;
            if (ms)
                B += E[s];
            uint32_t e = E[s];
#pragma unroll
            for (int t = 0; t < LOGR; t++) {
                if (t == s)
                    continue;
                const int hi = s > t ? s : t, lo = s > t ? t : s;
                if ((msig >> t) & 1u) {
                    e += G[hi * (hi - 1) / 2 + lo];
                    if (ms && t < s)
                        B += G[hi * (hi - 1) / 2 + lo];
                }
            }
            En[s] = ms ? 0u - e : e;
        }
#pragma unroll
        for (int s = 0; s < LOGR; s++)
            E[s] = En[s];
#pragma unroll
        for (int hi = 1; hi < LOGR; hi++)
#pragma unroll
            for (int lo = 0; lo < hi; lo++)
                if (((msig >> hi) ^ (msig >> lo)) & 1u)
                    G[hi * (hi - 1) / 2 + lo] = 0u - G[hi * (hi - 1) / 2 + lo];
    }
    // Apply.  Without slot terms every register takes the thread's base phase:
    // one sine/cosine and a multiply per register.  With slot terms each
    // register's whole phase is summed in integers and turned into its factor
    // on its own: 2^LOGR independent chains, so the hardware sine/cosine and the
    // multiplies of different registers overlap instead of waiting on one
    // another factor by factor.
    if (eu == 0u && A.gs_used == 0u) {
        if (bmul) {
            const float2 eb = expi_turn(B);
#pragma unroll
            for (int k = 0; k < NR; k++)
                v[k] = cmul(v[k], eb);
        }
    } else if (A.gs_used == 0u && (eu & (eu - 1u)) == 0u) {
        // one slot term: the registers without the bit take the base phase, those
        // with it the base plus the slot's phase (two sines/cosines)
        switch (__ffs(eu) - 1) {
        case 0: apply_one_slot<LOGR, 0>(v, B, E[0], bmul); break;
        case 1: apply_one_slot<LOGR, 1>(v, B, E[LOGR > 1 ? 1 : 0], bmul); break;
        case 2: apply_one_slot<LOGR, 2>(v, B, E[LOGR > 2 ? 2 : 0], bmul); break;
        case 3: apply_one_slot<LOGR, 3>(v, B, E[LOGR > 3 ? 3 : 0], bmul); break;
        default: apply_one_slot<LOGR, 4>(v, B, E[LOGR > 4 ? 4 : 0], bmul); break;
        }
    } else {
#pragma unroll
        for (int k = 0; k < NR; k++) {
            uint32_t a = B;
#pragma unroll
            for (int sb = 0; sb < LOGR; sb++)
                if ((k >> sb) & 1)
                    a += E[sb];
#pragma unroll
            for (int hi = 1; hi < LOGR; hi++)
#pragma unroll
                for (int lo = 0; lo < hi; lo++)
                    if (((k >> hi) & 1) && ((k >> lo) & 1))
                        a += G[hi * (hi - 1) / 2 + lo];
            v[k] = cmul(v[k], expi_turn(a));
        }
    }
    A.reset();
}

// Two-by-two butterfly on register bit r (pairs of slots k, k | 2^r).
template <typename C, int LOGR>
__device__ __forceinline__ void reg_butterfly(C (&v)[1 << LOGR], int r, C u00, C u01, C u10, C u11)
{
#pragma unroll
    for (int rr = 0; rr < LOGR; rr++) {
        if (rr == r) {
#pragma unroll
            for (int k = 0; k < (1 << LOGR); k++) {
                if (!((k >> rr) & 1)) {
                    const int k1 = k | (1 << rr);
                    const C x0 = v[k], x1 = v[k1];
                    v[k] = cmadd(u01, x1, cmul(u00, x0));
                    v[k1] = cmadd(u11, x1, cmul(u10, x0));
                }
            }
        }
    }
}

template <typename C, typename R, int LOGR>
__device__ __forceinline__ void reg_butterfly_real(C (&v)[1 << LOGR], int r, R u00, R u01, R u10, R u11)
{
#pragma unroll
    for (int rr = 0; rr < LOGR; rr++) {
        if (rr == r) {
#pragma unroll
            for (int k = 0; k < (1 << LOGR); k++) {
                if (!((k >> rr) & 1)) {
                    const int k1 = k | (1 << rr);
                    const C x0 = v[k], x1 = v[k1];
                    v[k] = mk(u00 * x0.x + u01 * x1.x, u00 * x0.y + u01 * x1.y);
                    v[k1] = mk(u10 * x0.x + u11 * x1.x, u10 * x0.y + u11 * x1.y);
                }
            }
        }
    }
}

template <typename C> __device__ __forceinline__ C shfl_xor_c(C a, int m)
{
    return mk(__shfl_xor_sync(0xffffffffu, a.x, m), __shfl_xor_sync(0xffffffffu, a.y, m));
}

#ifndef TQS_FP32_MIN_CTAS
#define TQS_FP32_MIN_CTAS 4  // resident CTAs per SM asked of ptxas for FP32 tiles of 2^12 amplitudes
#endif
// FUSE: the pass holds REC_FUSED records (FP32 tiles of 2^11 or 2^12 only); a
// separate instantiation so that the tensor-core code does not weigh on the
// register allocation of the passes without fused gates.
// The fused instantiations hold about 107 KB of shared memory per CTA (tile,
// TF32 hi/lo operands), so at most two fit an SM: they are given the registers
// of two CTAs instead of spilling to fit four.
template <typename R, int MODE, int LOGR, bool FUSE>
__global__ void __launch_bounds__(kThreads, FUSE ? 2
                                            : sizeof(R) == 4 ? (LOGR >= 5 ? 2 : LOGR == 4 ? TQS_FP32_MIN_CTAS : (LOGR == 3 ? 3 : 4))
                                                             : (LOGR >= 3 ? 1 : 2))
    pass_kernel(const __grid_constant__ PassK a)
{
    using C = typename CT<R>::T;
    constexpr int NR = 1 << LOGR;
    extern __shared__ __align__(16) unsigned char smem[];
#ifdef TQS_SPEC
    // a kernel specialised for one pass: its tile layout is a compile-time constant
    constexpr uint32_t kT = spec::kT, kN = spec::kN;
#define TQS_TBIT(j) spec::tbit(j)
#define TQS_HBIT(b) spec::hbit(b)
#define TQS_SOFF(k) spec::soff(k)
#else
    const uint32_t kT = a.t, kN = a.n;
#define TQS_TBIT(j) ((uint32_t)a.tbits[j])
#define TQS_HBIT(b) ((uint32_t)a.hbits[b])
#define TQS_SOFF(k) soff[k]
#endif
    const uint32_t TE = 1u << kT;
    C *s = reinterpret_cast<C *>(smem);
    uint16_t *lut = reinterpret_cast<uint16_t *>(s + (TE < (uint32_t)kThreads ? (uint32_t)kThreads : TE));
    double *red = reinterpret_cast<double *>(lut + 256);
    unsigned long long *shu = reinterpret_cast<unsigned long long *>(red + kThreads);
    const uint32_t tid = threadIdx.x;
    const bool active = tid < TE;

    const uint32_t slot = (MODE == MODE_SAMPLE) ? blockIdx.x : blockIdx.y;
    const uint64_t node = a.node_lo + slot;
    if (a.dbg & kDbgBounds) {
        // index check before the first memory access: every state index this CTA
        // forms is (outside-tile bits | tile bits) of its slot's state, so checking
        // the slots and the bit positions covers all of them
        uint32_t code = 0;
        uint64_t val = 0;
        if ((uint64_t)slot >= a.out_slots) {
            code = 1;
            val = slot;
        } else if (a.in && a.in_from_parent && node / a.arity - a.parent_lo >= a.in_slots) {
            code = 2;
            val = node / a.arity - a.parent_lo;
        } else if (a.t > a.n || a.state_elems != (1ull << a.n)) {
            code = 3;
            val = a.t;
        } else {
            for (uint32_t j = 0; j < a.t && !code; j++)
                if (a.tbits[j] >= a.n) {
                    code = 4;
                    val = a.tbits[j];
                }
            for (uint32_t b = 0; b < a.n - a.t && !code; b++)
                if (a.hbits[b] >= a.n) {
                    code = 5;
                    val = a.hbits[b];
                }
        }
        if (code) {
            if (threadIdx.x == 0 && a.err) {
                atomicOr(a.err, 4u);
                if (atomicCAS(a.err + 1, 0u, code) == 0u)
                    a.err[2] = (unsigned int)val;
            }
            return;  // uniform: nothing of this CTA touches memory
        }
    }
    const uint64_t seed = a.seed_dev ? *a.seed_dev : a.seed;
    const NodeMeta m0 = a.meta[(uint64_t)slot * a.meta_stride + a.pass_local];
    const NodeMeta m1 = a.meta[(uint64_t)slot * a.meta_stride + a.pass_local + 1];

    // physical offsets: thread bits (tile positions 0..7) and slot bits (8..t-1)
    uint32_t tphys = 0;
    const uint32_t tb = kT < 8u ? kT : 8u;
#pragma unroll
    for (uint32_t j = 0; j < tb; j++)
        tphys |= ((tid >> j) & 1u) << TQS_TBIT(j);
    // physical offsets of the register slots (uniform), kept in shared memory
    uint32_t *soff = reinterpret_cast<uint32_t *>(shu + 4);
    if (tid < (uint32_t)NR) {
        uint32_t o = 0;
        for (int b = 0; b < LOGR; b++)
            if ((tid >> b) & 1u)
                o |= 1u << TQS_TBIT(8 + b);
        soff[tid] = o;
    }

    const SamplerLayout &SL = a.samp;
    if (MODE == MODE_SUMS) {
        // rank (position in ascending logical order) of each tile position
        if (tid < a.t)
            lut[SL.rank_pos[tid]] = (uint16_t)tid;
    }
    if (MODE == MODE_SAMPLE) {
        // unkey tables: rank bits 0..6 -> tile positions (lut[0..127]), 7..13 -> lut[128..255]
        for (uint32_t i = tid; i < 256; i += kThreads) {
            const uint32_t rb = i < 128 ? 0 : 7, vv = i & 127;
            uint32_t e = 0;
            for (uint32_t b = 0; b < 7 && rb + b < a.t; b++)
                if ((vv >> b) & 1u)
                    e |= 1u << SL.rank_pos[rb + b];
            lut[i] = (uint16_t)e;
        }
    }

    // ---- tensor-core resources of fused gates (FP32 passes that have them) --
    const uint32_t nzst_k = ((a.sites < (uint32_t)kNoiseStage ? a.sites : (uint32_t)kNoiseStage) + 15u) / 16u * 16u;
    unsigned char *fz = nullptr;
    uint32_t tc_cols = 0, tc_phase = 0;
    bool tc_failed = false;  // CTA-uniform: a bounded tensor-core wait gave up; no more fused blocks
    if (FUSE && a.fused_k) {
        const size_t te_b = (size_t)(TE < (uint32_t)kThreads ? (uint32_t)kThreads : TE) * sizeof(C);
        size_t off = te_b + 256 * 2 + kThreads * 8 + 4 * 8 + 32 * 4 + nzst_k + kProgChunkBytes;
        off = (off + 127) / 128 * 128;
        fz = smem + off;
        const uint32_t K = 2u << a.fused_k;
        unsigned char *tail = fz + te_b + 2 * (size_t)K * K * 4;  // mbarrier (8 B), TMEM slot (4 B)
        tc_cols = K < 32u ? 32u : K;
        if (tid < 32)
            tc_alloc(smem_u32(tail + 8), tc_cols);
        if (tid == 0) {
            mbar_init(smem_u32(tail), 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        tc_fence_before();
    }

    // ---- which tile ------------------------------------------------------
    uint32_t base = 0;
    uint64_t gstar = 0;
    double resid = 0.0;
    if (MODE != MODE_SAMPLE) {
        const uint32_t h = blockIdx.x;
#pragma unroll
        for (uint32_t b = 0; b < kN - kT; b++)
            if ((h >> b) & 1u)
                base |= 1u << TQS_HBIT(b);
    } else {
        // stage 1: the block of 2^gamma outcomes, from this leaf's block sums
        const double *Sl = a.S + (uint64_t)slot * SL.groups;
        const uint4 r = draw(seed, node, 0u, kDomMeas);
        const double u = ((double)(r.x >> 5) * 67108864.0 + (double)(r.y >> 6)) * (1.0 / 9007199254740992.0);
        const uint64_t chunk = (SL.groups + kThreads - 1) / kThreads;
        double local = 0.0;
        for (uint64_t i = (uint64_t)tid * chunk; i < SL.groups && i < (uint64_t)(tid + 1) * chunk; i++)
            local += Sl[i];
        const double tot = block_incl_scan(local, red);
        if (tid == kThreads - 1)
            red[kThreads / 32] = tot;
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
    C v[NR];
    {
        const C *src = synth ? nullptr : reinterpret_cast<const C *>(a.in) + in_slot * a.state_elems;
        const uint32_t tb0 = base | tphys;
#pragma unroll
        for (int k = 0; k < NR; k++) {
            const uint32_t ph = tb0 | TQS_SOFF(k);
            if (!active)
                v[k] = mk((R)0, (R)0);
            else if (synth)
                v[k] = mk((R)(ph == 0 ? 1 : 0), (R)0);
            else
                v[k] = src[ph];
        }
    }

    // ---- gates and noise -----------------------------------------------
    uint32_t mask = m0.mask;
    uint32_t xt = (base | tphys) ^ mask;  // logical bits at thread and outside-tile positions
    const R *mats = reinterpret_cast<const R *>(a.mats);
    const uint8_t *nzg = a.noise + (uint64_t)slot * a.sites;
    uint8_t *nzs = reinterpret_cast<uint8_t *>(soff + 32);
    const bool nz_staged = a.sites <= (uint32_t)kNoiseStage;
    uint8_t *pbuf = nzs + ((a.sites < (uint32_t)kNoiseStage ? a.sites : (uint32_t)kNoiseStage) + 15u) / 16u * 16u;
    // passes in which this node drew no Pauli (most of them) skip every noise check
    const bool pnoisy = (m0.phase & kMetaNoisy) != 0u;
    if (nz_staged && pnoisy)
        for (uint32_t x = tid; x < a.sites; x += kThreads)
            nzs[x] = nzg[x];
    auto noise_at = [&](uint32_t site) -> uint32_t { return nz_staged ? nzs[site] : nzg[site]; };

    using Acc = DiagAcc<C, LOGR>;
    using V = typename Acc::V;  // a diagonal factor: complex (FP64) or a phase in 2^-32 turns (FP32)
    Acc acc;
    acc.reset();
    // a factor value of the compiled program / a per-gate matrix entry
    auto fv_mat = [&](R re, R im) -> V {
        if constexpr (sizeof(R) == 4)
            return turn_of(re, im);
        else
            return mk(re, im);
    };
    auto fv_is_one = [&](V f) -> bool {
        if constexpr (sizeof(R) == 4)
            return f == 0u;
        else
            return f.x == (R)1 && f.y == (R)0;
    };
    bool pending = false;
    auto slot_mask = [&]() {
        uint32_t m = 0;
#pragma unroll
        for (int b = 0; b < LOGR; b++)
            m |= ((mask >> TQS_TBIT(8 + b)) & 1u) << b;
        return m;
    };
    auto flush = [&]() {
        if (pending) {
            acc_flush(acc, v, slot_mask());
            pending = false;
        }
    };
    // the Pauli drawn at a noise site: Z parts join the diagonal run, X parts
    // toggle the frame (after applying what is pending)
    auto apply_noise = [&](uint32_t pz, uint32_t npaulis, uint32_t j0, uint32_t p0, uint32_t j1, uint32_t p1) {
        const uint32_t wa = npaulis == 15 ? (pz >> 2) : pz;
        const uint32_t wb = npaulis == 15 ? (pz & 3u) : 0u;
        const V minus = Acc::minus_one();
        if (wa >= 2) {
            acc_alpha(acc, j0, p0, xt, minus);
            pending = true;
        }
        if (wb >= 2) {
            acc_alpha(acc, j1, p1, xt, minus);
            pending = true;
        }
        const bool xa = wa == 1 || wa == 2, xb = wb == 1 || wb == 2;
        const uint32_t xm = (xa ? (1u << p0) : 0u) | (xb ? (1u << p1) : 0u);
        if (xm) {
            if constexpr (sizeof(R) == 4) {
                if (xa && !thread_or_outside(j0))
                    acc.flip((int)j0 - 8);
                if (xb && !thread_or_outside(j1))
                    acc.flip((int)j1 - 8);
            } else {
                flush();
            }
            mask ^= xm;
            xt ^= xm;
        }
    };
    auto dense1 = [&](uint32_t j, uint32_t p, C u00, C u01, C u10, C u11) {
        // the caller has applied the pending diagonal phases
        if ((mask >> p) & 1u) {  // frame conjugation U'[r][c] = U[r^1][c^1]
            const C t0 = u00, t1 = u01;
            u00 = u11;
            u01 = u10;
            u10 = t1;
            u11 = t0;
        }
        if (j >= 8) {
            reg_butterfly<C, LOGR>(v, (int)j - 8, u00, u01, u10, u11);
        } else if (j < 5) {
            const uint32_t b = (tid >> j) & 1u;
            const C cs = b ? u11 : u00, co = b ? u10 : u01;
#pragma unroll
            for (int k = 0; k < NR; k++) {
                const C o = shfl_xor_c(v[k], 1 << j);
                v[k] = cmadd(co, o, cmul(cs, v[k]));
            }
        } else {
            const uint32_t b = (tid >> j) & 1u;
            const C cs = b ? u11 : u00, co = b ? u10 : u01;
            __syncthreads();
            if (active) {
#pragma unroll
                for (int k = 0; k < NR; k++)
                    s[tid + k * kThreads] = v[k];
            }
            __syncthreads();
            if (active) {
#pragma unroll
                for (int k = 0; k < NR; k++) {
                    const C o = s[(tid ^ (1u << j)) + k * kThreads];
                    v[k] = cmadd(co, o, cmul(cs, v[k]));
                }
            }
        }
    };
    // real 2x2 matrix (H, RY, X, ...): half the multiplies
    auto dense1_real = [&](uint32_t j, uint32_t p, R u00, R u01, R u10, R u11) {
        // the caller has applied the pending diagonal phases
        if ((mask >> p) & 1u) {
            const R t0 = u00, t1 = u01;
            u00 = u11;
            u01 = u10;
            u10 = t1;
            u11 = t0;
        }
        if (j >= 8) {
            reg_butterfly_real<C, R, LOGR>(v, (int)j - 8, u00, u01, u10, u11);
        } else if (j < 5) {
            const uint32_t b = (tid >> j) & 1u;
            const R cs = b ? u11 : u00, co = b ? u10 : u01;
#pragma unroll
            for (int k = 0; k < NR; k++) {
                const C o = shfl_xor_c(v[k], 1 << j);
                v[k] = mk(cs * v[k].x + co * o.x, cs * v[k].y + co * o.y);
            }
        } else {
            const uint32_t b = (tid >> j) & 1u;
            const R cs = b ? u11 : u00, co = b ? u10 : u01;
            __syncthreads();
            if (active) {
#pragma unroll
                for (int k = 0; k < NR; k++)
                    s[tid + k * kThreads] = v[k];
            }
            __syncthreads();
            if (active) {
#pragma unroll
                for (int k = 0; k < NR; k++) {
                    const C o = s[(tid ^ (1u << j)) + k * kThreads];
                    v[k] = mk(cs * v[k].x + co * o.x, cs * v[k].y + co * o.y);
                }
            }
        }
    };
    // U: 16 complex values, row-major, read through `get`
    auto dense2 = [&](uint32_t j0, uint32_t j1, uint32_t p0, uint32_t p1, auto get) {
        // the caller has applied the pending diagonal phases
        const uint32_t mu = ((mask >> p0) & 1u) | (((mask >> p1) & 1u) << 1);
        __syncthreads();
        if (active) {
#pragma unroll
            for (int k = 0; k < NR; k++)
                s[tid + k * kThreads] = v[k];
        }
        __syncthreads();
        if (active) {
            const uint32_t m0b = 1u << j0, m1b = 1u << j1;
#pragma unroll
            for (int k = 0; k < NR; k++) {
                const uint32_t e = tid + (uint32_t)k * kThreads;
                const uint32_t r = ((e >> j0) & 1u) | (((e >> j1) & 1u) << 1);
                const uint32_t eb = e & ~(m0b | m1b);
                C acc2 = mk((R)0, (R)0);
#pragma unroll
                for (uint32_t c = 0; c < 4; c++) {
                    const C x = s[eb | ((c & 1u) ? m0b : 0u) | ((c & 2u) ? m1b : 0u)];
                    acc2 = cmadd(get((r ^ mu) * 4 + (c ^ mu)), x, acc2);
                }
                v[k] = acc2;
            }
        }
    };
    // one diagonal gate from the per-gate tables (runs holding an X or Y noise event)
    auto diag_gate = [&](const Instr &I) {
        const R *M = mats + (size_t)I.gate * 32;
        const uint32_t fl = I.pad;
        if (fl & 1u)
            acc.mul_base(fv_mat(M[0], M[1]));
        if (fl & 2u)
            acc_alpha(acc, I.j0, I.p0, xt, fv_mat(M[2], M[3]));
        if (I.op == OP_DIAG2) {
            if (fl & 4u)
                acc_alpha(acc, I.j1, I.p1, xt, fv_mat(M[4], M[5]));
            if (fl & 8u)
                acc_gamma(acc, I.j0, I.p0, I.j1, I.p1, xt, fv_mat(M[6], M[7]));
        }
        pending = true;
    };
    // One fused gate on the tensor cores: the tile seen as a 2^kf x 128 complex
    // matrix X (rows: the fused qubits' local index, columns: the other tile
    // bits), Y = U X computed as the real product [Yr; Yi]^T = [Xr; Xi]^T [[Ur,-Ui],[Ui,Ur]]^T
    // (M = 128 columns, N = K = 2^(kf+1)) in three TF32 products
    // (hi*hi + hi*lo + lo*hi, FP32 accumulation in TMEM).
    auto fused_apply = [&](const unsigned char *pay, uint32_t kf) {
        if constexpr (sizeof(R) == 4 && FUSE) {
            const uint32_t Kc = 1u << kf, Kr = 2u * Kc;
            uint32_t jpos[5], phys[5];
            uint32_t jmask = 0, mu = 0;
            for (uint32_t i = 0; i < kf; i++) {
                jpos[i] = pay[i];
                phys[i] = pay[8 + i];
                jmask |= 1u << jpos[i];
                mu |= ((mask >> phys[i]) & 1u) << i;
            }
            const uint32_t foff = *reinterpret_cast<const uint32_t *>(pay + 16);
            const size_t te_b = (size_t)TE * sizeof(C);
            float *A_hi = reinterpret_cast<float *>(s);
            float *A_lo = reinterpret_cast<float *>(fz);
            float *B_hi = reinterpret_cast<float *>(fz + te_b);
            float *B_lo = B_hi + (size_t)Kr * Kr;
            const uint32_t mbar = smem_u32(B_lo + (size_t)Kr * Kr);
            const uint32_t tmem = *reinterpret_cast<const uint32_t *>(reinterpret_cast<const unsigned char *>(B_lo + (size_t)Kr * Kr) + 8);
            // split of a tile position set: fused bits -> local index, the rest -> column
            auto gather = [&](uint32_t e) {
                uint32_t r = 0;
                for (uint32_t i = 0; i < kf; i++)
                    r |= ((e >> jpos[i]) & 1u) << i;
                return r;
            };
            auto compress = [&](uint32_t e) {
                uint32_t r = 0, o = 0;
                for (uint32_t j = 0; j < a.t; j++)
                    if (!((jmask >> j) & 1u))
                        r |= ((e >> j) & 1u) << (o++);
                return r;
            };
            auto offA = [&](uint32_t c, uint32_t kk) {
                return (c >> 3) * (Kr / 4) * 32 + (kk >> 2) * 32 + (c & 7u) * 4 + (kk & 3u);
            };
            __syncthreads();  // the tile region is free (all earlier exchanges finished)
            {
                const float4 *src = reinterpret_cast<const float4 *>(a.fused + foff);
                float4 *dst = reinterpret_cast<float4 *>(B_hi);
                for (uint32_t x = tid; x < Kr * Kr / 2; x += kThreads)  // hi and lo, 4 floats each
                    dst[x] = src[x];
            }
            const uint32_t at = gather(tid), ct = compress(tid);
#pragma unroll
            for (int k = 0; k < NR; k++) {
                const uint32_t ek = (uint32_t)k * kThreads;
                const uint32_t aa = (at | gather(ek)) ^ mu, cc = ct | compress(ek);
                const float re = v[k].x, im = v[k].y;
                const float hr = tf32_rna(re), hm = tf32_rna(im);
                A_hi[offA(cc, aa)] = hr;
                A_lo[offA(cc, aa)] = tf32_rna(re - hr);
                A_hi[offA(cc, Kc + aa)] = hm;
                A_lo[offA(cc, Kc + aa)] = tf32_rna(im - hm);
            }
            fence_async_smem();
            __syncthreads();
            tc_fence_after();
            const bool fault = (a.dbg & kDbgFaultTimeout) != 0u;  // test: nothing is issued, the wait runs out
            if (tid == 0 && !fault) {
                const uint32_t idesc = tc_idesc_tf32(128, Kr);
                const uint32_t sbo = Kr / 4 * 128;
                const uint32_t sa[3] = {smem_u32(A_hi), smem_u32(A_hi), smem_u32(A_lo)};
                const uint32_t sb[3] = {smem_u32(B_hi), smem_u32(B_lo), smem_u32(B_hi)};
                for (uint32_t term = 0; term < 3; term++)
                    for (uint32_t ks = 0; ks < Kr / 8; ks++)
                        tc_mma_tf32(tmem, tc_smem_desc(sa[term] + ks * 256, 128, sbo),
                                    tc_smem_desc(sb[term] + ks * 256, 128, sbo), idesc, (term | ks) != 0);
                tc_commit(mbar);
            }
            const uint32_t cap = fault ? (1u << 10) : (1u << 22);
            // one outcome for the whole CTA, so that every thread takes the same branch
            const bool ok = __syncthreads_and(mbar_wait_bounded(mbar, tc_phase, cap) ? 1 : 0) != 0;
            tc_fence_after();
            if (!ok) {
                if (tid == 0 && a.err)
                    atomicOr(a.err, 1u);
                // products possibly still in flight get a second bounded wait before the
                // TMEM they write is released at the end of the kernel
                if (!fault)
                    (void)__syncthreads_and(mbar_wait_bounded(mbar, tc_phase, cap) ? 1 : 0);
                tc_failed = true;  // later fused blocks are skipped; the host reports TQS_ETIMEOUT
                return;            // from fused_apply: v[] keeps the block's input, the tile region is stale
            }
            tc_phase ^= 1u;
            // D[c][o] from TMEM: warp w reads rows 32*(w%4)..+31 (its lane quarter) and
            // one half of the Kr columns
            const uint32_t w = tid >> 5, lane = tid & 31u;
            const uint32_t c = 32u * (w & 3u) + lane;
            float *sf = reinterpret_cast<float *>(s);
            uint32_t dc = 0;  // tile positions of column c
            {
                uint32_t o = 0;
                for (uint32_t j = 0; j < a.t; j++)
                    if (!((jmask >> j) & 1u))
                        dc |= ((c >> (o++)) & 1u) << j;
            }
            const uint32_t half = Kr / 2, col0 = (w >> 2) * half;
            for (uint32_t cb = 0; cb < half; cb += 16) {
                float r[16];
                tc_ld16(tmem + ((32u * (w & 3u)) << 16) + col0 + cb, r);
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    const uint32_t o = col0 + cb + (uint32_t)i;
                    const uint32_t ast = (o & (Kc - 1u)) ^ mu;
                    uint32_t e = dc;
                    for (uint32_t b = 0; b < kf; b++)
                        e |= ((ast >> b) & 1u) << jpos[b];
                    sf[2 * e + (o >= Kc ? 1 : 0)] = r[i];
                }
            }
            tc_fence_before();
            __syncthreads();
#pragma unroll
            for (int k = 0; k < NR; k++)
                v[k] = s[tid + k * kThreads];
            __syncthreads();
        }
    };
    constexpr uint32_t CS = (uint32_t)sizeof(C);
#ifdef TQS_SPEC
    // the pass's records as straight-line code (generated from the same program)
    if (!zero_tile) {
        __syncthreads();  // the staged noise bytes
#include "tqs_spec_walk.inc"
    } else {
        mask = m1.mask;
    }
#else
    if (!zero_tile) {
        for (uint32_t c = a.chunk_begin; c < a.chunk_end; c++) {
            const uint32_t o0 = a.chunk_off[c], o1 = a.chunk_off[c + 1];
            __syncthreads();
            for (uint32_t x = tid; x < (o1 - o0) / 16u; x += kThreads)
                reinterpret_cast<uint4 *>(pbuf)[x] = reinterpret_cast<const uint4 *>(a.prog + o0)[x];
            __syncthreads();
            uint32_t p = 0;
            while (p < o1 - o0) {
                const uint4 hw = *reinterpret_cast<const uint4 *>(pbuf + p);
                const uint32_t htype = hw.x & 0xffu, ha = (hw.x >> 8) & 0xffu, hb = (hw.x >> 16) & 0xffu,
                               hc = hw.x >> 24, hd = hw.y & 0xffu, he = (hw.y >> 8) & 0xffu, hsite = hw.y >> 16;
                const uint32_t hibeg = hw.z, hiend = hw.w;
                const unsigned char *pay = pbuf + p + 16;
                auto pc = [&](uint32_t i) -> C { return *reinterpret_cast<const C *>(pay + i * CS); };
                // The one place pending diagonal phases are applied (FP32; FP64 also
                // flushes at X noise): before every record that is not a diagonal run,
                // the end-of-pass record included.  A single call site keeps the
                // kernel's code small.
                if (sizeof(R) == 4 && MODE != MODE_STORE && htype == REC_END) {
                    acc.reset();  // a final diagonal run changes phases only, not the measured |a|^2
                    pending = false;
                }
                if (htype != REC_RUN)
                    flush();
                if (htype == REC_END)
                    break;
                if (htype == REC_DENSE1) {
                    if (hc)
                        dense1_real(ha, hb, pc(0).x, pc(1).x, pc(2).x, pc(3).x);
                    else
                        dense1(ha, hb, pc(0), pc(1), pc(2), pc(3));
                    const uint32_t pz = pnoisy ? noise_at(hsite) : 0u;
                    if (pz)
                        apply_noise(pz, 3, ha, hb, ha, hb);
                    p += 16u + ((4u * CS + 15u) & ~15u);
                } else if (htype == REC_DENSE2) {
                    dense2(ha, hb, hc, hd, pc);
                    const uint32_t pz = pnoisy ? noise_at(hsite) : 0u;
                    if (pz)
                        apply_noise(pz, 15, ha, hc, hb, hd);
                    p += 16u + 16u * CS;
                } else if (htype == REC_KRAUS) {
                    // this node's damping operators after the previous gate (real 2x2)
                    const C *km = reinterpret_cast<const C *>(a.kmat) + (uint64_t)slot * 8;
                    dense1_real(ha, hc, km[0].x, km[1].x, km[2].x, km[3].x);
                    if (he == 2)
                        dense1_real(hb, hd, km[4].x, km[5].x, km[6].x, km[7].x);
                    p += 16u;
                } else if (htype == REC_FUSED) {
                  if constexpr (!FUSE) {  // the host launches the FUSE instantiation for these
                    if (tid == 0 && a.err)
                        atomicOr(a.err, 2u);
                  } else {
                    uint32_t anyf = 0;  // the block's gates need not have consecutive sites
                    for (uint32_t x = hibeg + (tid & 31u); pnoisy && x < hiend; x += 32u)
                        anyf |= noise_at(a.instr[x].site);
                    const bool any = __any_sync(0xffffffffu, anyf != 0u);
                    bool done = tc_failed;  // after a failed wait nothing more is computed
                    if constexpr (sizeof(R) == 4) {
                        if (!done && !any && a.fused_k == ha) {
                            fused_apply(pay, ha);
                            done = true;
                        }
                    }
                    if (!done) {  // a noise site inside the block: the gates one by one
                        for (uint32_t ii = hibeg; ii < hiend; ii++) {
                            const Instr I = a.instr[ii];
                            const R *M = mats + (size_t)I.gate * 32;
                            if (I.op == OP_DENSE1) {
                                flush();
                                dense1(I.j0, I.p0, mk(M[0], M[1]), mk(M[2], M[3]), mk(M[4], M[5]), mk(M[6], M[7]));
                            } else if (I.op == OP_DENSE2) {
                                flush();
                                dense2(I.j0, I.j1, I.p0, I.p1, [&](uint32_t kk) { return mk(M[2 * kk], M[2 * kk + 1]); });
                            } else if (I.op == OP_DIAG1 || I.op == OP_DIAG2) {
                                diag_gate(I);
                            }
                            const uint32_t pz = noise_at(I.site);
                            if (pz)
                                apply_noise(pz, I.npaulis, I.j0, I.np0, I.j1, I.np1);
                        }
                    }
                  }
                    p += 48u;
                } else if constexpr (sizeof(R) == 4) {
                    // FP32 run: phases grouped by accumulator (RunHdr32), no per-factor
                    // dispatch; a node with a Pauli inside the run goes gate by gate
                    const RunHdr32 &rh = *reinterpret_cast<const RunHdr32 *>(pay);
                    const uint32_t nent = rh.pad[1];
                    constexpr uint32_t ES = 16u + 4u * (uint32_t)sizeof(V);  // GateEnt + 4 phases
                    const unsigned char *gents = pay + 80 + (nent * 8u + 15u) / 16u * 16u;
                    const uint32_t ngates = hiend - hibeg;
                    uint32_t anyn = 0;
                    for (uint32_t x = tid & 31u; pnoisy && x < ngates; x += 32u)
                        anyn |= noise_at(*reinterpret_cast<const uint32_t *>(gents + x * ES + 12));
                    if (!__any_sync(0xffffffffu, anyn != 0u)) {
                        if (rh.g0)
                            acc.mul_base(rh.g0);
                        const uint2 *en = reinterpret_cast<const uint2 *>(pay + 80);
                        const uint32_t nb = rh.nbase;
                        if (rh.pad[0]) {  // base entries only (no slot terms): the usual run in the leaves
                            if (nb)
                                acc.base_used = true;
                            uint32_t add = 0;  // (the run's global phase was added above)
                            for (uint32_t i = 0; i < nb; i++) {
                                const uint2 e = en[i];
                                if ((xt & e.x) == e.x)
                                    add += e.y;
                            }
                            acc.base += add;
                            pending = true;
                            p += 96u + (nent * 8u + 15u) / 16u * 16u + ngates * ES;
                            continue;
                        }
                        if (nb) {
                            acc.base_used = true;
                            uint32_t add = 0;
                            for (uint32_t i = 0; i < nb; i++) {
                                const uint2 e = en[i];
                                if ((xt & e.x) == e.x)
                                    add += e.y;
                            }
                            acc.base += add;
                            en += nb;
                        }
#pragma unroll
                        for (int q = 0; q < LOGR; q++) {
                            const uint32_t nq = rh.ne[q];
                            if (nq == 0u && !((rh.eused >> q) & 1u))
                                continue;
                            uint32_t add = rh.econst[q];
                            for (uint32_t i = 0; i < nq; i++) {
                                const uint2 e = en[i];
                                if ((xt & e.x) == e.x)
                                    add += e.y;
                            }
                            en += nq;
                            acc.E[q] += add;
                            acc.e_used |= 1u << q;
                        }
                        if (rh.gused) {
#pragma unroll
                            for (int i = 0; i < (LOGR > 1 ? LOGR * (LOGR - 1) / 2 : 1); i++)
                                if ((rh.gused >> i) & 1u)
                                    acc.Gs[i] += rh.gp[i];
                            acc.gs_used |= rh.gused;
                            acc.has_gs = true;
                        }
                        pending = true;
                    } else {  // gate by gate from the entries after the factors
                        const unsigned char *gq = gents;
                        for (uint32_t ii = 0; ii < ngates; ii++, gq += ES) {
                            const uint4 e = *reinterpret_cast<const uint4 *>(gq);
                            const uint32_t op = e.x & 0xffu, fl = (e.x >> 8) & 0xffu, j0 = (e.x >> 16) & 0xffu,
                                           p0 = e.x >> 24, j1 = e.y & 0xffu, p1 = (e.y >> 8) & 0xffu,
                                           np0 = (e.y >> 16) & 0xffu, np1 = e.y >> 24, npl = e.z & 0xffu;
                            const V *M = reinterpret_cast<const V *>(gq + 16);
                            if (op == OP_DIAG1 || op == OP_DIAG2) {
                                if (fl & 1u)
                                    acc.mul_base(M[0]);
                                if (fl & 2u)
                                    acc_alpha(acc, j0, p0, xt, M[1]);
                                if (op == OP_DIAG2) {
                                    if (fl & 4u)
                                        acc_alpha(acc, j1, p1, xt, M[2]);
                                    if (fl & 8u)
                                        acc_gamma(acc, j0, p0, j1, p1, xt, M[3]);
                                }
                                pending = true;
                            }
                            const uint32_t pz = noise_at(e.w);
                            if (pz)
                                apply_noise(pz, npl, j0, np0, j1, np1);
                        }
                    }
                    p += 96u + (nent * 8u + 15u) / 16u * 16u + ngates * ES;
                } else {
                    const uint32_t nfac = ha + hb + hc + hd + he;
                    constexpr uint32_t ES = 16u + 4u * (uint32_t)sizeof(V);  // GateEnt + 4 factors
                    const unsigned char *gents = pay + 16 + nfac * (CS == 8 ? 16u : 32u);
                    const uint32_t ngates = hiend - hibeg;
                    uint32_t anyn = 0;  // a Pauli at any site of the run? (the lanes split the gates)
                    for (uint32_t x = tid & 31u; pnoisy && x < ngates; x += 32u)
                        anyn |= noise_at(*reinterpret_cast<const uint32_t *>(gents + x * ES + 12));
                    if (!__any_sync(0xffffffffu, anyn != 0u)) {
                        const V g0 = *reinterpret_cast<const V *>(pay);
                        if (!fv_is_one(g0))
                            acc.mul_base(g0);
                        if (ha + hc)
                            acc.base_used = true;
                        const unsigned char *fp = pay + 16;
                        constexpr uint32_t FS = CS == 8 ? 16u : 32u;
                        auto fval = [&](const unsigned char *q) -> V {
                            return *reinterpret_cast<const V *>(q + (CS == 8 ? 8 : 16));
                        };
                        // FacHdr as one 64-bit word: kind | j0<<8 | p0<<16 | j1<<24 | p1<<32
                        for (uint32_t f = 0; f < ha; f++, fp += FS) {  // a^{x_p}, p fixed
                            const uint32_t w0 = *reinterpret_cast<const uint32_t *>(fp);
                            acc.mul_base_if(((xt >> ((w0 >> 16) & 0xffu)) & 1u) != 0u, fval(fp));
                        }
                        for (uint32_t f = 0; f < hb; f++, fp += FS) {  // a^{x_s}, slot s
                            const uint32_t w0 = *reinterpret_cast<const uint32_t *>(fp);
                            acc.mul_E((int)((w0 >> 8) & 0xffu) - 8, fval(fp));
                        }
                        for (uint32_t f = 0; f < hc; f++, fp += FS) {  // c^{x_p0 x_p1}, both fixed
                            const uint2 w = *reinterpret_cast<const uint2 *>(fp);
                            acc.mul_base_if(((xt >> ((w.x >> 16) & 0xffu)) & (xt >> (w.y & 0xffu)) & 1u) != 0u,
                                            fval(fp));
                        }
                        for (uint32_t f = 0; f < hd; f++, fp += FS) {  // c^{x_p0 x_s1}
                            const uint32_t w0 = *reinterpret_cast<const uint32_t *>(fp);
                            if ((xt >> ((w0 >> 16) & 0xffu)) & 1u)
                                acc.mul_E((int)(w0 >> 24) - 8, fval(fp));
                        }
                        for (uint32_t f = 0; f < he; f++, fp += FS) {  // c^{x_s0 x_s1}
                            const uint32_t w0 = *reinterpret_cast<const uint32_t *>(fp);
                            acc.mul_Gs((int)((w0 >> 8) & 0xffu) - 8, (int)(w0 >> 24) - 8, fval(fp));
                        }
                        pending = true;
                    } else {  // gate by gate from the entries after the factors (in shared memory)
                        const unsigned char *gq = gents;
                        for (uint32_t ii = 0; ii < ngates; ii++, gq += ES) {
                            const uint4 e = *reinterpret_cast<const uint4 *>(gq);
                            const uint32_t op = e.x & 0xffu, fl = (e.x >> 8) & 0xffu, j0 = (e.x >> 16) & 0xffu,
                                           p0 = e.x >> 24, j1 = e.y & 0xffu, p1 = (e.y >> 8) & 0xffu,
                                           np0 = (e.y >> 16) & 0xffu, np1 = e.y >> 24, npl = e.z & 0xffu;
                            const V *M = reinterpret_cast<const V *>(gq + 16);
                            if (op == OP_DIAG1 || op == OP_DIAG2) {
                                if (fl & 1u)
                                    acc.mul_base(M[0]);
                                if (fl & 2u)
                                    acc_alpha(acc, j0, p0, xt, M[1]);
                                if (op == OP_DIAG2) {
                                    if (fl & 4u)
                                        acc_alpha(acc, j1, p1, xt, M[2]);
                                    if (fl & 8u)
                                        acc_gamma(acc, j0, p0, j1, p1, xt, M[3]);
                                }
                                pending = true;
                            }
                            const uint32_t pz = noise_at(e.w);
                            if (pz)
                                apply_noise(pz, npl, j0, np0, j1, np1);
                        }
                    }
                    p += 32u + nfac * (CS == 8 ? 16u : 32u) + ngates * ES;
                }
            }
        }
    } else {
        mask = m1.mask;
    }
#endif
    if (FUSE && a.fused_k) {  // every path reaches here: free the tensor memory
        tc_fence_before();
        __syncthreads();
        if (tid < 32) {
            const uint32_t K = 2u << a.fused_k;
            const uint32_t tmem = *reinterpret_cast<const uint32_t *>(fz + (size_t)TE * sizeof(C) + 2 * (size_t)K * K * 4 + 8);
            tc_dealloc(tmem, tc_cols);
        }
    }

    // ---- epilogue ------------------------------------------------------
    if (MODE == MODE_STORE && a.ksum) {
        // damping channels: this tile's |a|^2 summed by the logical values of
        // the next choice's qubits (bit kp0 -> index bit 0, kp1 -> bit 1)
        double s4[4] = {0.0, 0.0, 0.0, 0.0};
        if (active) {
            const uint32_t tb0 = base | tphys;
#pragma unroll
            for (int k = 0; k < NR; k++) {
                const uint32_t lg = (tb0 | TQS_SOFF(k)) ^ mask;
                const uint32_t ix = ((lg >> a.kp0) & 1u) | (a.knq == 2 ? ((lg >> a.kp1) & 1u) << 1 : 0u);
                const double w = (double)norm2<R>(v[k]);
                s4[0] += ix == 0 ? w : 0.0;
                s4[1] += ix == 1 ? w : 0.0;
                s4[2] += ix == 2 ? w : 0.0;
                s4[3] += ix == 3 ? w : 0.0;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            for (int j = 0; j < 4; j++)
                s4[j] += __shfl_xor_sync(0xffffffffu, s4[j], off);
        __syncthreads();
        if ((tid & 31u) == 0)
            for (int j = 0; j < 4; j++)
                red[(tid >> 5) * 4 + j] = s4[j];
        __syncthreads();
        if (tid < 4) {
            double t = 0.0;
            for (int wi = 0; wi < kThreads / 32; wi++)
                t += red[wi * 4 + tid];
            a.ksum[((uint64_t)slot * gridDim.x + blockIdx.x) * 4 + tid] = t;
        }
    }
    if (MODE == MODE_STORE) {
        C *dst = reinterpret_cast<C *>(a.out) + (uint64_t)slot * a.state_elems;
        if (active) {
            const uint32_t tb0 = base | tphys;
#pragma unroll
            for (int k = 0; k < NR; k++)
                dst[tb0 | TQS_SOFF(k)] = v[k];
        }
        return;
    }
    // tile-coordinate frame mask (final frame)
    uint32_t mT = 0;
#pragma unroll
    for (uint32_t j = 0; j < kT; j++)
        mT |= ((mask >> TQS_TBIT(j)) & 1u) << j;
    if (MODE == MODE_SAMPLE) {
        __syncthreads();
        if (active) {
#pragma unroll
            for (int k = 0; k < NR; k++)
                s[tid + k * kThreads] = v[k];
        }
        __syncthreads();
    }
    const uint32_t G = 1u << SL.gamma;
    auto elem_of_key = [&](uint32_t key) -> uint32_t {
        return ((uint32_t)lut[key & 127] | (uint32_t)lut[128 + ((key >> 7) & 127)]) ^ mT;
    };

#ifdef TQS_SPEC
    if constexpr (MODE == MODE_SUMS && sizeof(R) == 4) {
        // Block sums of |a|^2 (FP32 states), reduced where the amplitudes live.  A
        // block is the 2^gamma outcomes that share every logical bit above gamma;
        // its in-tile bits are the tile positions of logical ranks 0..gamma-1,
        // each a register slot, a lane bit or a warp bit of this layout.  So the
        // block sum is a sum over those slots (adds between registers), those
        // lanes (shuffles) and those warps (shared memory); the thread whose
        // in-block thread bits are 0 then writes one FP64 sum per combination of
        // the other slots.  The frame mask does not change which amplitudes share
        // a block, only the block's index (logical = physical ^ frame).
        uint32_t in_slot = 0, in_thr = 0;
        for (uint32_t r = 0; r < SL.gamma; r++) {
            const uint32_t j = SL.rank_pos[r];
            if (j >= 8u)
                in_slot |= 1u << (j - 8u);
            else
                in_thr |= 1u << j;
        }
        float w[NR];
#pragma unroll
        for (int k = 0; k < NR; k++)
            w[k] = active ? norm2<R>(v[k]) : 0.0f;
#pragma unroll
        for (int sb = 0; sb < LOGR; sb++) {
            if (!((in_slot >> sb) & 1u))
                continue;
#pragma unroll
            for (int k = 0; k < NR; k++)
                if (!((k >> sb) & 1))
                    w[k] += w[k | (1 << sb)];
        }
        // live partials: registers whose in-block slot bits are all 0
        const uint32_t in_lane = in_thr & 31u, in_warp = in_thr & ~31u;
        for (uint32_t l = 0; l < 5u; l++) {
            if (!((in_lane >> l) & 1u))
                continue;
#pragma unroll
            for (int k = 0; k < NR; k++)
                if (((uint32_t)k & in_slot) == 0u)
                    w[k] += __shfl_xor_sync(0xffffffffu, w[k], 1 << l);
        }
        if (in_warp) {
            float *sp = reinterpret_cast<float *>(s);  // the tile region: kThreads x NR floats
            __syncthreads();
#pragma unroll
            for (int k = 0; k < NR; k++)
                if (((uint32_t)k & in_slot) == 0u)
                    sp[(uint32_t)k * kThreads + tid] = w[k];
            __syncthreads();
            if ((tid & in_warp) == 0u) {
#pragma unroll
                for (int k = 0; k < NR; k++) {
                    if (((uint32_t)k & in_slot) != 0u)
                        continue;
                    float acc = 0.0f;
                    // every subset of the in-block warp bits, in a fixed order
                    for (uint32_t sub = in_warp;; sub = (sub - 1u) & in_warp) {
                        acc += sp[(uint32_t)k * kThreads + (tid | sub)];
                        if (sub == 0u)
                            break;
                    }
                    w[k] = acc;
                }
            }
        }
        if (active && (tid & in_thr) == 0u) {
            uint64_t hpart = 0;
            for (uint32_t b = 0; b < kN - kT; b++) {
                const uint32_t pb = TQS_HBIT(b);
                hpart |= (uint64_t)(((base ^ mask) >> pb) & 1u) << (SL.logical_of_hbit[b] - SL.gamma);
            }
            // the logical tile bits above gamma: this thread's part, the frame's
            // part on the slots, and per slot the block-index bit it sets
            uint64_t g0 = hpart;
            uint32_t dsh[LOGR > 0 ? LOGR : 1];
#pragma unroll
            for (int sb = 0; sb < LOGR; sb++)
                dsh[sb] = 63u;  // an in-block slot: never used
            const uint32_t et = tid ^ mT;
            for (uint32_t r = SL.gamma; r < kT; r++) {
                const uint32_t j = SL.rank_pos[r], sh = SL.rank_q[r] - SL.gamma;
                if (j < 8u) {
                    g0 |= (uint64_t)((et >> j) & 1u) << sh;
                } else {
                    g0 |= (uint64_t)((mT >> j) & 1u) << sh;
#pragma unroll
                    for (int sb = 0; sb < LOGR; sb++)
                        if ((uint32_t)sb == j - 8u)
                            dsh[sb] = sh;
                }
            }
            double *Srow = a.S + (uint64_t)slot * SL.groups;
#pragma unroll
            for (int k = 0; k < NR; k++) {
                if (((uint32_t)k & in_slot) != 0u)
                    continue;
                uint64_t g = g0;
#pragma unroll
                for (int sb = 0; sb < LOGR; sb++)
                    if ((k >> sb) & 1)
                        g ^= (uint64_t)1 << dsh[sb];
                Srow[g] = (double)w[k];
            }
        }
        return;
    }
#endif
    if (MODE == MODE_SUMS) {
        // Block sums of |a|^2 over the 2^gamma outcomes that share every logical
        // bit above gamma.  Each |a|^2 is staged in shared memory at its logical
        // tile index (tile element ^ frame, bits in rank = ascending logical
        // order), so block b of this tile is the run [b 2^gamma, (b+1) 2^gamma).
        // Each thread adds its run of consecutive values, the threads of one
        // block combine with shuffles, and one thread per block writes the sum
        // as FP64.  The index map is linear over XOR: thread part ^ slot part.
        uint32_t Lt = 0;
        {
            const uint32_t et = tid ^ (mT & 0xffu), tb = kT < 8u ? kT : 8u;
            for (uint32_t j = 0; j < tb; j++)
                Lt |= ((et >> j) & 1u) << lut[j];
        }
        uint32_t img[LOGR > 0 ? LOGR : 1];
#pragma unroll
        for (int sb = 0; sb < LOGR; sb++) {
            img[sb] = 1u << lut[8 + sb];
            if ((mT >> (8 + sb)) & 1u)
                Lt ^= img[sb];
        }
        R *P = reinterpret_cast<R *>(s);
        // bank swizzle: folds the index bits above the 32 banks into the bank
        // bits, so the scattered writes (a permutation of the tile bits) and the
        // runs read per thread both spread over the banks
        auto sw = [](uint32_t L) { return L ^ (((L >> 5) ^ (L >> 10)) & 31u); };
        __syncthreads();
        if (active) {
#pragma unroll
            for (int k = 0; k < NR; k++) {
                uint32_t L = Lt;
#pragma unroll
                for (int sb = 0; sb < LOGR; sb++)
                    if ((k >> sb) & 1)
                        L ^= img[sb];
                P[sw(L)] = norm2<R>(v[k]);
            }
        }
        uint64_t hpart = 0;
#pragma unroll
        for (uint32_t b = 0; b < kN - kT; b++) {
            const uint32_t pb = TQS_HBIT(b);
            hpart |= (uint64_t)(((base ^ mask) >> pb) & 1u) << (SL.logical_of_hbit[b] - SL.gamma);
        }
        const uint32_t gam = SL.gamma, B = 1u << gam;
        // block index of this tile's block bl: its bits deposited at the logical bits above gamma
        auto block_index = [&](uint32_t bl) -> uint64_t {
            uint64_t g = hpart;
            for (uint32_t i = 0; bl; i++, bl >>= 1)
                if (bl & 1u)
                    g |= (uint64_t)1 << (SL.rank_q[gam + i] - gam);
            return g;
        };
        double *Srow = a.S + (uint64_t)slot * SL.groups;
        const uint32_t nper = TE < (uint32_t)kThreads ? 1u : (uint32_t)NR;  // values per thread
        const uint32_t e0 = tid * nper;
        __syncthreads();
        if (B <= nper) {  // whole blocks inside each thread's run
            if (e0 < TE)
                for (uint32_t b0 = 0; b0 < nper; b0 += B) {
                    R acc = (R)0;
                    for (uint32_t i = 0; i < B; i++)
                        acc += P[sw(e0 + b0 + i)];
                    Srow[block_index((e0 + b0) >> gam)] = (double)acc;
                }
        } else {
            R acc = (R)0;
            if (e0 < TE) {
#pragma unroll
                for (int i = 0; i < NR; i++)
                    if ((uint32_t)i < nper)
                        acc += P[sw(e0 + (uint32_t)i)];
            }
            const uint32_t tpb = B / nper;  // threads per block
            if (tpb <= 32u) {
                for (uint32_t off = 1; off < tpb; off <<= 1)
                    acc += __shfl_xor_sync(0xffffffffu, acc, off);
                if (e0 < TE && (tid & (tpb - 1u)) == 0)
                    Srow[block_index(e0 >> gam)] = (double)acc;
            } else {
                R *part = reinterpret_cast<R *>(red);
                part[tid] = acc;
                __syncthreads();
                if (e0 < TE && (tid & (tpb - 1u)) == 0) {
                    R t2 = (R)0;
                    for (uint32_t i = 0; i < tpb; i++)
                        t2 += part[tid + i];
                    Srow[block_index(e0 >> gam)] = (double)t2;
                }
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
        if (tid < a.n) {
            const uint4 rr = draw(seed, node, tid, kDomRead);
            flip = (uint64_t)rr.x < a.thrm;
        }
        const uint32_t fl = __ballot_sync(0xffffffffu, flip);
        if (tid == 0)
            atomicAdd(&a.counts[y ^ (uint64_t)fl], 1ull);
    }
}

#undef TQS_TBIT
#undef TQS_HBIT
#undef TQS_SOFF

#ifndef __CUDACC_RTC__
template <typename R, int MODE, int LOGR, bool FUSE> static int set_pass_attr()
{
    return (int)cudaFuncSetAttribute(pass_kernel<R, MODE, LOGR, FUSE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     200 * 1024);
}

template <typename R, int MODE, int LOGR, bool FUSE>
static int launch_pass_t(const PassK &k, dim3 grid, size_t smem, cudaStream_t st)
{
    // the dynamic shared-memory limit is an attribute of the function on each
    // device: raise it once per device that launches this instantiation
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(done.load(std::memory_order_acquire) & bit)) {
        set_pass_attr<R, MODE, LOGR, FUSE>();
        done.fetch_or(bit, std::memory_order_acq_rel);
    }
    pass_kernel<R, MODE, LOGR, FUSE><<<grid, kThreads, smem, st>>>(k);
    return (int)cudaGetLastError();
}

template <typename R, int MODE> int set_attrs_r()
{
    int e = set_pass_attr<R, MODE, 0, false>();
    e |= set_pass_attr<R, MODE, 1, false>();
    e |= set_pass_attr<R, MODE, 2, false>();
    e |= set_pass_attr<R, MODE, 3, false>();
    e |= set_pass_attr<R, MODE, 4, false>();
    e |= set_pass_attr<R, MODE, 5, false>();
    if (sizeof(R) == 4) {
        e |= set_pass_attr<R, MODE, 3, true>();
        e |= set_pass_attr<R, MODE, 4, true>();
    }
    return e;
}


template <typename R, int MODE>
int launch_pass_r(const PassK &k, int logr, dim3 grid, size_t smem, cudaStream_t st)
{
    if (sizeof(R) == 4 && k.fused_k) {  // the planner fuses only in tiles of 2^11 and 2^12
        if (logr == 3) return launch_pass_t<R, MODE, 3, true>(k, grid, smem, st);
        if (logr == 4) return launch_pass_t<R, MODE, 4, true>(k, grid, smem, st);
        return (int)cudaErrorInvalidValue;
    }
    switch (logr) {
    case 0: return launch_pass_t<R, MODE, 0, false>(k, grid, smem, st);
    case 1: return launch_pass_t<R, MODE, 1, false>(k, grid, smem, st);
    case 2: return launch_pass_t<R, MODE, 2, false>(k, grid, smem, st);
    case 3: return launch_pass_t<R, MODE, 3, false>(k, grid, smem, st);
    case 4: return launch_pass_t<R, MODE, 4, false>(k, grid, smem, st);
    default: return launch_pass_t<R, MODE, 5, false>(k, grid, smem, st);
    }
}
#endif  // __CUDACC_RTC__

}  // namespace tqs
