// planner.cpp -- host planning for the tree Monte-Carlo path:
//   circuit validation and gate matrices (Sec. 2.2), circuit partitioners
//   (DCP / UCP / XCP / explicit, Sec. 3.2 and 3.6), the noise-site table and
//   the lowering of every subcircuit into shared-memory tile passes.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <string>

#include "internal.h"
#include "mlp.h"

namespace tqs {

bool is_two_qubit(uint32_t k)
{
    return k == TQS_CX || k == TQS_CZ || k == TQS_CP || k == TQS_SWAP || k == TQS_U2;
}

bool is_diagonal(uint32_t k)
{
    switch (k) {
    case TQS_Z: case TQS_S: case TQS_SDG: case TQS_T: case TQS_TDG: case TQS_RZ: case TQS_P:
    case TQS_CZ: case TQS_CP:
        return true;
    default:
        return false;
    }
}

uint64_t threshold32(double p)
{
    return (uint64_t)std::floor(p * 4294967296.0);
}

// Textbook matrices; interleaved (re, im), row-major; two-qubit gates act on the
// local index k = bit(q0) + 2 bit(q1) with q0 the control of CX.
void gate_matrix(uint32_t kind, double th, const double *mat, double *m)
{
    std::memset(m, 0, 32 * sizeof(double));
    auto set = [&](int i, double re, double im) { m[2 * i] = re; m[2 * i + 1] = im; };
    const double r = 1.0 / std::sqrt(2.0);
    const double c = std::cos(th / 2), s = std::sin(th / 2);
    switch (kind) {
    case TQS_H: set(0, r, 0); set(1, r, 0); set(2, r, 0); set(3, -r, 0); break;
    case TQS_X: set(1, 1, 0); set(2, 1, 0); break;
    case TQS_Y: set(1, 0, -1); set(2, 0, 1); break;
    case TQS_Z: set(0, 1, 0); set(3, -1, 0); break;
    case TQS_S: set(0, 1, 0); set(3, 0, 1); break;
    case TQS_SDG: set(0, 1, 0); set(3, 0, -1); break;
    case TQS_T: set(0, 1, 0); set(3, r, r); break;
    case TQS_TDG: set(0, 1, 0); set(3, r, -r); break;
    case TQS_RX: set(0, c, 0); set(1, 0, -s); set(2, 0, -s); set(3, c, 0); break;
    case TQS_RY: set(0, c, 0); set(1, -s, 0); set(2, s, 0); set(3, c, 0); break;
    case TQS_RZ: set(0, std::cos(th / 2), -std::sin(th / 2)); set(3, std::cos(th / 2), std::sin(th / 2)); break;
    case TQS_P: set(0, 1, 0); set(3, std::cos(th), std::sin(th)); break;
    case TQS_U1: std::memcpy(m, mat, 8 * sizeof(double)); break;
    case TQS_CX: set(0, 1, 0); set(1 * 4 + 3, 1, 0); set(2 * 4 + 2, 1, 0); set(3 * 4 + 1, 1, 0); break;
    case TQS_CZ: set(0, 1, 0); set(5, 1, 0); set(10, 1, 0); set(15, -1, 0); break;
    case TQS_CP: set(0, 1, 0); set(5, 1, 0); set(10, 1, 0); set(15, std::cos(th), std::sin(th)); break;
    case TQS_SWAP: set(0, 1, 0); set(1 * 4 + 2, 1, 0); set(2 * 4 + 1, 1, 0); set(15, 1, 0); break;
    case TQS_U2: std::memcpy(m, mat, 32 * sizeof(double)); break;
    default: break;
    }
}

std::string validate_and_build_circuit(uint32_t n, const tqs_gate *gates, size_t ng, Circuit &out)
{
    if (n < 1 || n > TQS_MAX_QUBITS)
        return "n_qubits must be in [1, " + std::to_string(TQS_MAX_QUBITS) + "]";
    if (ng > 0 && gates == nullptr)
        return "gates is NULL";
    if (ng > 60000)
        return "at most 60000 gates are supported";
    out.n = n;
    out.gates.resize(ng);
    for (size_t i = 0; i < ng; i++) {
        const tqs_gate &g = gates[i];
        std::string at = "gate " + std::to_string(i) + ": ";
        if (g.kind > TQS_U2)
            return at + "unknown kind " + std::to_string(g.kind);
        if (g.q0 >= n)
            return at + "q0 out of range";
        bool two = is_two_qubit(g.kind);
        if (two && (g.q1 >= n || g.q1 == g.q0))
            return at + "q1 out of range or equal to q0";
        if (!std::isfinite(g.theta))
            return at + "non-finite angle";
        int d = (g.kind == TQS_U1) ? 4 : (g.kind == TQS_U2 ? 16 : 0);
        if (d && g.mat == nullptr)
            return at + "U1/U2 need a matrix";
        for (int j = 0; j < 2 * d; j++)
            if (!std::isfinite(g.mat[j]))
                return at + "non-finite matrix entry";
        Gate &o = out.gates[i];
        o.kind = g.kind;
        o.q0 = g.q0;
        o.q1 = two ? g.q1 : g.q0;
        o.theta = g.theta;
        gate_matrix(g.kind, g.theta, g.mat, o.m);
    }
    return "";
}

// --------------------------------------------------------------------------
// Partitioners
// --------------------------------------------------------------------------
static std::vector<uint32_t> equal_split(uint32_t G, uint32_t L)
{
    std::vector<uint32_t> s(L + 1);
    for (uint32_t i = 0; i <= L; i++)
        s[i] = (uint32_t)(((uint64_t)i * G) / L);
    return s;
}

// a^k * b <= N without overflow
static bool pow_times_le(uint64_t a, uint32_t k, uint64_t b, uint64_t N)
{
    unsigned __int128 v = b;
    for (uint32_t i = 0; i < k; i++) {
        v *= a;
        if (v > N)
            return false;
    }
    return v <= N;
}

// Dynamic Circuit Partition (Sec. 3.2): the first-subcircuit error rate
// (Eq. error_rate) sets the minimum first-level arity by the sample-size formula
// (Eq. sample_size_formula); the remaining k levels take the equal arity
// floor((N / A_0)^(1/k)) (Eq. subcirc_shots) with k as large as keeps it >= 2
// and no larger than the state-copy limit (at least c gates per subcircuit,
// Sec. 3.6); A_0 is then raised to ceil(N / A_r^k) so that the tree has N
// leaves, and the circuit is cut into k+1 subcircuits of equal length.
// Error rate e_i of gate i for DCP's first-subcircuit estimate (Sec. 3.2,
// Eq. error_rate): its depolarizing probability and, with damping channels, the
// probability that any of them jumps, bounded by its rate on each of the gate's
// qubits (a jump's probability is rate * P1 <= rate).
double gate_error_rate(const Noise &nz, uint32_t kind)
{
    const bool two = is_two_qubit(kind);
    double keep = 1.0 - (two ? nz.p2 : nz.p1);
    const double rates[4] = {two ? nz.tr_g2 : nz.tr_g1, two ? nz.tr_l2 : nz.tr_l1, nz.ad, nz.pd};
    for (int q = 0; q < (two ? 2 : 1); q++)
        for (double r : rates)
            keep *= 1.0 - r;
    return 1.0 - keep;
}

static std::string dcp(const Circuit &c, const Noise &nz, uint64_t N, double z, double eps,
                       uint32_t cgates, std::vector<uint64_t> &arity, std::vector<uint32_t> &split)
{
    const uint32_t G = (uint32_t)c.gates.size();
    std::vector<double> e(G);
    for (uint32_t i = 0; i < G; i++)
        e[i] = gate_error_rate(nz, c.gates[i].kind);
    uint32_t cap = (cgates ? G / cgates : G);
    cap = cap >= 1 ? cap - 1 : 0;
    uint32_t K = cap;
    uint64_t a0min = 1;
    for (;;) {
        uint32_t first = G ? (G + K) / (K + 1) : 0;  // ceil(G / (K+1))
        double prod = 1.0;
        for (uint32_t i = 0; i < first; i++)
            prod *= (1.0 - e[i]);
        double ph = 1.0 - prod;
        double n0 = z * z * ph * (1.0 - ph) / (eps * eps);
        double a = std::ceil(n0 / (1.0 + n0 / (double)N));
        a0min = a < 1.0 ? 1 : (uint64_t)a;
        uint32_t ks = 0;
        while (ks < 63 && pow_times_le(2, ks + 1, a0min, N))
            ks++;
        uint32_t Kn = std::min(std::min(ks, cap), K);
        if (Kn == K)
            break;
        K = Kn;
    }
    if (K == 0) {
        arity = {N};
        split = {0, G};
        return "";
    }
    // the ABI holds at most TQS_MAX_LEVELS levels; a deeper fixed point is cut there
    if (K > TQS_MAX_LEVELS - 1)
        K = TQS_MAX_LEVELS - 1;
    uint64_t ar = 2;
    while (pow_times_le(ar + 1, K, a0min, N))
        ar++;
    unsigned __int128 pk = 1;
    for (uint32_t i = 0; i < K; i++)
        pk *= ar;
    uint64_t a0 = (uint64_t)(((unsigned __int128)N + pk - 1) / pk);
    arity.assign(K + 1, ar);
    arity[0] = a0;
    split = equal_split(G, K + 1);
    return "";
}

uint64_t dcp_first_arity(const Circuit &c, const Noise &nz, uint64_t N, double z, double eps, uint32_t K)
{
    const uint32_t G = (uint32_t)c.gates.size();
    uint32_t first = G ? (G + K) / (K + 1) : 0;
    double prod = 1.0;
    for (uint32_t i = 0; i < first; i++)
        prod *= (1.0 - gate_error_rate(nz, c.gates[i].kind));
    double ph = 1.0 - prod;
    double n0 = z * z * ph * (1.0 - ph) / (eps * eps);
    double a = std::ceil(n0 / (1.0 + n0 / (double)N));
    return a < 1.0 ? 1 : (uint64_t)a;
}

std::string dcp_tree(const Circuit &c, const Noise &nz, uint64_t N, double z, double eps, uint32_t cgates,
                     std::vector<uint64_t> &arity, std::vector<uint32_t> &split)
{
    return dcp(c, nz, N, z, eps, cgates, arity, split);
}

std::string partition(const Circuit &c, const Noise &nz, uint64_t N, const tqs_options &o,
                      std::vector<uint64_t> &arity, std::vector<uint32_t> &split)
{
    const uint32_t G = (uint32_t)c.gates.size();
    if (N == 0)
        return "shots must be >= 1";
    if (o.mode == TQS_MODE_BASELINE) {
        arity = {N};
        split = {0, G};
        return "";
    }
    if (o.mode != TQS_MODE_TREE)
        return "unknown mode";
    switch (o.part) {
    case TQS_PART_DCP:
        if (!(o.z > 0) || !(o.eps > 0) || !std::isfinite(o.z) || !std::isfinite(o.eps))
            return "DCP needs z > 0 and eps > 0";
        return dcp(c, nz, N, o.z, o.eps, o.copy_gates, arity, split);
    case TQS_PART_UCP:
    case TQS_PART_XCP: {
        uint32_t L = o.k + 1;
        if (L > TQS_MAX_LEVELS)
            return "too many levels";
        uint64_t ratio = o.part == TQS_PART_XCP ? 2 : 1;
        for (uint64_t a = 1;; a++) {
            unsigned __int128 prod = 1;
            std::vector<uint64_t> ar(L);
            for (uint32_t i = 0; i < L; i++) {
                unsigned __int128 v = a;
                for (uint32_t j = 0; j + 1 + i < L; j++)
                    v *= ratio;
                ar[i] = (uint64_t)v;
                prod *= v;
                if (prod > ((unsigned __int128)1 << 100))
                    break;
            }
            if (prod >= N) {
                arity = ar;
                split = equal_split(G, L);
                return "";
            }
        }
    }
    case TQS_PART_EXPLICIT: {
        uint32_t L = o.k + 1;
        if (L > TQS_MAX_LEVELS || !o.arity || !o.split)
            return "explicit tree needs k < 17, arity and split";
        arity.assign(o.arity, o.arity + L);
        split.assign(o.split, o.split + L + 1);
        unsigned __int128 prod = 1;
        for (uint64_t a : arity) {
            if (a == 0)
                return "arity must be >= 1";
            prod *= a;
            if (prod > ((unsigned __int128)1 << 100))
                prod = ((unsigned __int128)1 << 100);
        }
        if (prod < N)
            return "prod(arity) must be >= shots";
        if (split[0] != 0 || split[L] != G)
            return "split must start at 0 and end at n_gates";
        for (uint32_t i = 0; i < L; i++)
            if (split[i + 1] < split[i])
                return "split must be non-decreasing";
        return "";
    }
    case TQS_PART_LEARNED:
        return learned_partition(c, nz, N, o, arity, split);
    default:
        return "unknown partitioner";
    }
}

// --------------------------------------------------------------------------
// Lowering: lazy SWAPs, noise sites, tile passes, sampler layout
// --------------------------------------------------------------------------
static void choose_tile(uint32_t n, uint32_t tmax, uint32_t need_mask, const uint8_t *prefer,
                        uint32_t nprefer, Pass &p)
{
    uint32_t t = std::min(n, tmax);
    uint32_t lmin = std::min<uint32_t>(n, 4);
    uint32_t T = need_mask;
    for (uint32_t b = 0; b < lmin; b++)
        T |= 1u << b;
    for (uint32_t i = 0; i < nprefer && (uint32_t)__builtin_popcount(T) < t; i++)
        T |= 1u << prefer[i];
    for (uint32_t b = 0; b < n && (uint32_t)__builtin_popcount(T) < t; b++)
        T |= 1u << b;
    p.t = (uint32_t)__builtin_popcount(T);
    uint32_t j = 0, h = 0;
    for (uint32_t b = 0; b < n; b++) {
        if (T & (1u << b))
            p.tbits[j++] = (uint8_t)b;
        else
            p.hbits[h++] = (uint8_t)b;
    }
    uint32_t L = 0;
    while (L < p.t && p.tbits[L] == L)
        L++;
    p.L = L;
}

// TF32 rounding (nearest, ties to even on the 10-bit mantissa) of an FP32 value.
static float tf32_round(float x)
{
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) != 0x7f800000u)
        u = (u + 0x0fffu + ((u >> 13) & 1u)) & 0xffffe000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

// Dense 2^k x 2^k unitary of a block of gates on the physical bits q[0..k-1]
// (local index bit i <-> q[i]), FP64, row-major.
static std::vector<std::complex<double>> fused_unitary(const PlanHost &P, const std::vector<uint32_t> &ids,
                                                       const uint8_t *q, uint32_t k)
{
    const uint32_t d = 1u << k;
    std::vector<std::complex<double>> U(d * d, 0.0), T(d * d);
    for (uint32_t i = 0; i < d; i++)
        U[i * d + i] = 1.0;
    auto loc = [&](uint8_t p) {
        for (uint32_t i = 0; i < k; i++)
            if (q[i] == p)
                return i;
        return 0u;
    };
    for (uint32_t id : ids) {
        const Instr &in = P.prog_instrs[id];
        if (in.op == OP_NOP)
            continue;
        const double *m = &P.mats64[(size_t)in.gate * 32];
        auto cx = [&](int e) { return std::complex<double>(m[2 * e], m[2 * e + 1]); };
        const bool two = in.op == OP_DENSE2 || in.op == OP_DIAG2;
        const uint32_t l0 = loc(in.p0), l1 = two ? loc(in.p1) : l0;
        std::complex<double> M[16];
        const int gd = two ? 4 : 2;
        if (in.op == OP_DIAG1 || in.op == OP_DIAG2) {
            for (int e = 0; e < 16; e++)
                M[e] = 0.0;
            for (int x = 0; x < gd; x++) {  // D[x] = G a0^{x0} a1^{x1} c^{x0 x1}
                const int x0 = x & 1, x1 = (x >> 1) & 1;
                std::complex<double> v = cx(0);
                if (x0) v *= cx(1);
                if (two && x1) v *= cx(2);
                if (two && x0 && x1) v *= cx(3);
                M[x * gd + x] = v;
            }
        } else {
            for (int e = 0; e < gd * gd; e++)
                M[e] = cx(e);
        }
        const uint32_t gmask = two ? ((1u << l0) | (1u << l1)) : (1u << l0);
        for (uint32_t r = 0; r < d; r++)
            for (uint32_t c = 0; c < d; c++) {
                std::complex<double> acc = 0.0;
                const int kr = (int)(((r >> l0) & 1u) | (two ? (((r >> l1) & 1u) << 1) : 0u));
                for (uint32_t x = 0; x < d; x++) {
                    if ((x & ~gmask) != (r & ~gmask))
                        continue;
                    const int kx = (int)(((x >> l0) & 1u) | (two ? (((x >> l1) & 1u) << 1) : 0u));
                    acc += M[kr * gd + kx] * U[x * d + c];
                }
                T[r * d + c] = acc;
            }
        U.swap(T);
    }
    return U;
}

// Tensor-core operand of a fused gate: the real 2^(k+1)-square matrix
// [[Re U, -Im U], [Im U, Re U]] as TF32 hi and lo parts, each in the K-major
// core-matrix layout (8 rows x 16 bytes per core matrix; core matrices adjacent
// in K are 128 bytes apart, 8-row groups K/4 * 128 bytes apart).
static void append_fused_operand(std::vector<float> &out, const std::vector<std::complex<double>> &U, uint32_t k)
{
    const uint32_t d = 1u << k, K = 2 * d;
    const size_t base = out.size();
    out.resize(base + 2 * (size_t)K * K, 0.f);
    for (uint32_t o = 0; o < K; o++)
        for (uint32_t kk = 0; kk < K; kk++) {
            const std::complex<double> u = U[(o % d) * d + (kk % d)];
            double val;
            if (o < d)
                val = kk < d ? u.real() : -u.imag();
            else
                val = kk < d ? u.imag() : u.real();
            const float f = (float)val, hi = tf32_round(f), lo = tf32_round(f - hi);
            const size_t off = (size_t)(o / 8) * (K / 4) * 32 + (size_t)(kk / 4) * 32 + (o % 8) * 4 + (kk % 4);
            out[base + off] = hi;
            out[base + (size_t)K * K + off] = lo;
        }
}

// Lower every pass into the record program the kernels walk (see RecHdr):
// dense gates with their matrix inline, and each run of consecutive diagonal
// gates (lazy SWAPs included) merged into one record of per-qubit and
// per-pair factors classified by the tile position of their bits.
// Physical qubits an instruction and its noise site act on.
static uint32_t instr_qubits(const Instr &in)
{
    uint32_t m = 1u << in.np0;
    if (in.npaulis == 15)
        m |= 1u << in.np1;
    if (in.op == OP_DENSE1 || in.op == OP_DIAG1)
        m |= 1u << in.p0;
    else if (in.op == OP_DENSE2 || in.op == OP_DIAG2)
        m |= (1u << in.p0) | (1u << in.p1);
    return m;
}

// Reorders each pass so that diagonal gates (and lazy SWAP noise sites) wait
// until the first later dense gate that shares a qubit with them, or the end of
// the pass.  An instruction and its noise site only move past instructions on
// disjoint qubits, and instructions sharing a qubit keep their relative order,
// so every node's result is unchanged (up to rounding): the Pauli drawn at a
// site still acts between the same gates on its qubits.  Effect: the diagonal
// run flushed before a dense gate holds only the factors that touch it, and the
// rest merge into one run at the end of the pass.
static void sink_diagonals(PlanHost &P)
{
    P.prog_instrs = P.instrs;
    for (const Pass &ps : P.passes) {
        std::vector<Instr> out, pend;
        out.reserve(ps.iend - ps.ibeg);
        for (uint32_t k = ps.ibeg; k < ps.iend; k++) {
            const Instr &in = P.instrs[k];
            if (in.op != OP_DENSE1 && in.op != OP_DENSE2) {
                pend.push_back(in);
                continue;
            }
            const uint32_t qd = instr_qubits(in);
            std::vector<char> go(pend.size(), 0);
            for (size_t i = 0; i < pend.size(); i++)
                go[i] = (instr_qubits(pend[i]) & qd) != 0;
            // an earlier pending instruction sharing a qubit with one that goes must go too
            for (size_t i = pend.size(); i-- > 0;) {
                if (!go[i])
                    continue;
                const uint32_t qi = instr_qubits(pend[i]);
                for (size_t j = 0; j < i; j++)
                    if (!go[j] && (instr_qubits(pend[j]) & qi))
                        go[j] = 1;
            }
            std::vector<Instr> keep;
            for (size_t i = 0; i < pend.size(); i++)
                (go[i] ? out : keep).push_back(pend[i]);
            pend.swap(keep);
            out.push_back(in);
        }
        out.insert(out.end(), pend.begin(), pend.end());
        std::copy(out.begin(), out.end(), P.prog_instrs.begin() + ps.ibeg);
    }
}

#ifndef TQS_FUSE_MIN_DENSE
#define TQS_FUSE_MIN_DENSE 2  // dense gates a block needs before it is fused onto the tensor cores
#endif
// A unit complex number as a phase in units of 2^-32 turns (rounded), the form
// in which FP32 programs carry diagonal factors.
static uint32_t turn32(std::complex<double> z)
{
    const double t = std::arg(z) / (2.0 * M_PI);  // (-1/2, 1/2]
    return (uint32_t)(int64_t)std::llround(t * 4294967296.0);
}

static void compile_programs(PlanHost &P)
{
    const bool f64 = P.prec == TQS_FP64;
    // FP64: diagonal factors are complex doubles; FP32: phases (turn32), 4 bytes
    const size_t csz = f64 ? 16 : 8, fsz = f64 ? 32 : 16, esz = 16 + 4 * (f64 ? csz : 4);
    const size_t kMaxFactors = 200;  // also keeps an FP32 run's entry count within RunHdr32's byte
    std::vector<uint8_t> &out = P.prog;
    out.clear();
    P.chunk_off.clear();
    P.fused.clear();
    P.fused_k = 0;
    auto put = [&](const void *p, size_t n) {
        const uint8_t *b = (const uint8_t *)p;
        out.insert(out.end(), b, b + n);
    };
    auto putc = [&](std::complex<double> z) {
        if (f64) {
            double v[2] = {z.real(), z.imag()};
            put(v, 16);
        } else {
            float v[2] = {(float)z.real(), (float)z.imag()};
            put(v, 8);
        }
    };
    auto pad16 = [&]() {
        while (out.size() % 16)
            out.push_back(0);
    };
    // a diagonal factor in the program's form
    auto putd = [&](std::complex<double> z) {
        if (f64) {
            putc(z);
        } else {
            const uint32_t a = turn32(z);
            put(&a, 4);
        }
    };
    auto cplx = [&](uint32_t gate, int k) {
        return std::complex<double>(P.mats64[(size_t)gate * 32 + 2 * k], P.mats64[(size_t)gate * 32 + 2 * k + 1]);
    };
    size_t chunk_start = 0;
    auto reserve = [&](size_t bytes) {  // open a new chunk if `bytes` do not fit the current one
        if (out.size() > chunk_start && out.size() - chunk_start + bytes > (size_t)kProgChunkBytes) {
            P.chunk_off.push_back((uint32_t)out.size());
            chunk_start = out.size();
        }
    };
    for (Pass &ps : P.passes) {
        uint8_t pos[32];
        std::memset(pos, 0xff, sizeof(pos));
        for (uint32_t j = 0; j < ps.t; j++)
            pos[ps.tbits[j]] = (uint8_t)j;
        auto is_slot = [&](uint8_t p) { return pos[p] != 0xff && pos[p] >= 8; };
        ps.chunk_begin = (uint32_t)P.chunk_off.size();
        ps.fused_blocks = 0;
        P.chunk_off.push_back((uint32_t)out.size());
        chunk_start = out.size();
        if (ps.kin_nq) {  // the damping operators chosen after the previous gate
            RecHdr h;
            std::memset(&h, 0, sizeof(h));
            h.type = REC_KRAUS;
            h.a = pos[ps.kin_p0];
            h.b = ps.kin_nq == 2 ? pos[ps.kin_p1] : 0xff;
            h.c = ps.kin_p0;
            h.d = ps.kin_p1;
            h.e = ps.kin_nq;
            h.ibeg = h.iend = ps.ibeg;
            put(&h, 16);
        }
        // tensor-core fusion: FP32 states and tiles with 128 columns beside k = t - 7 fused qubits
        const uint32_t kf = (P.fuse && !f64 && (ps.t == 11 || ps.t == 12)) ? ps.t - 7 : 0;
        uint32_t k = ps.ibeg;
        while (k < ps.iend) {
            const Instr &in = P.prog_instrs[k];
            if (kf && (in.op == OP_DENSE1 || in.op == OP_DENSE2)) {
                uint32_t qmask = 0, dense_cnt = 0, kk = k;
                for (; kk < ps.iend; kk++) {
                    const Instr &g = P.prog_instrs[kk];
                    if (g.op == OP_NOP)
                        continue;
                    const bool two = g.op == OP_DENSE2 || g.op == OP_DIAG2;
                    const uint32_t gm = (1u << g.p0) | (two ? (1u << g.p1) : 0u);
                    if (pos[g.p0] == 0xff || (two && pos[g.p1] == 0xff))
                        break;
                    if ((uint32_t)__builtin_popcount(qmask | gm) > kf)
                        break;
                    qmask |= gm;
                    dense_cnt += (g.op == OP_DENSE1 || g.op == OP_DENSE2) ? 1 : 0;
                }
                if (dense_cnt >= (uint32_t)TQS_FUSE_MIN_DENSE) {
                    // pad the fused set to exactly kf tile qubits (identity on the extra ones)
                    for (uint32_t j = 0; j < ps.t && (uint32_t)__builtin_popcount(qmask) < kf; j++)
                        qmask |= 1u << ps.tbits[j];
                    uint8_t q[8] = {0}, jp[8] = {0};
                    uint32_t nq = 0;
                    for (uint32_t b = 0; b < 32; b++)
                        if (qmask & (1u << b)) {
                            q[nq] = (uint8_t)b;
                            jp[nq] = pos[b];
                            nq++;
                        }
                    std::vector<uint32_t> ids;
                    for (uint32_t x = k; x < kk; x++)
                        ids.push_back(x);
                    const uint32_t off = (uint32_t)P.fused.size();
                    append_fused_operand(P.fused, fused_unitary(P, ids, q, kf), kf);
                    P.fused_k = kf;
                    ps.fused_blocks++;
                    reserve(48);
                    RecHdr h;
                    std::memset(&h, 0, sizeof(h));
                    h.type = REC_FUSED;
                    h.a = (uint8_t)kf;
                    h.site = in.site;
                    h.ibeg = k;
                    h.iend = kk;
                    put(&h, 16);
                    uint8_t pj[16] = {0};
                    for (uint32_t i = 0; i < 8; i++) {
                        pj[i] = jp[i];
                        pj[8 + i] = q[i];
                    }
                    put(pj, 16);
                    uint32_t w4[4] = {off, 0, 0, 0};
                    put(w4, 16);
                    k = kk;
                    continue;
                }
            }
            if (in.op == OP_DENSE1 || in.op == OP_DENSE2) {
                const bool two = in.op == OP_DENSE2;
                reserve(16 + (two ? 16 : 4) * csz);
                RecHdr h;
                std::memset(&h, 0, sizeof(h));
                h.type = two ? REC_DENSE2 : REC_DENSE1;
                h.a = in.j0;
                h.b = two ? in.j1 : in.p0;
                h.c = in.p0;
                h.d = in.p1;
                h.site = in.site;
                h.ibeg = k;
                h.iend = k + 1;
                if (!two) {
                    bool real = true;
                    for (int e = 0; e < 4; e++)
                        real = real && cplx(in.gate, e).imag() == 0.0;
                    h.c = real ? 1 : 0;
                }
                put(&h, 16);
                for (int e = 0; e < (two ? 16 : 4); e++)
                    putc(cplx(in.gate, e));
                pad16();
                k++;
                continue;
            }
            // a run of diagonal gates / lazy SWAPs, cut so that its factors stay bounded
            std::complex<double> G = 1.0;
            std::complex<double> alpha[32];
            for (auto &a : alpha)
                a = 1.0;
            std::vector<std::pair<std::pair<uint8_t, uint8_t>, std::complex<double>>> pairs;
            auto pair_mul = [&](uint8_t a, uint8_t b, std::complex<double> f) {
                if (a > b)
                    std::swap(a, b);
                for (auto &e : pairs)
                    if (e.first.first == a && e.first.second == b) {
                        e.second *= f;
                        return;
                    }
                pairs.push_back({{a, b}, f});
            };
            const uint32_t r0 = k;
            // the record (header, G, factors, one gate entry per gate) must fit one chunk
            uint32_t touched = 0;
            auto fits_one_more = [&]() {
                const size_t nfac = (size_t)__builtin_popcount(touched) + pairs.size() + 3;
                return 32 + nfac * fsz + (size_t)(k - r0 + 1) * esz + 16 <= (size_t)kProgChunkBytes;
            };
            while (k < ps.iend && P.prog_instrs[k].op != OP_DENSE1 && P.prog_instrs[k].op != OP_DENSE2 &&
                   pairs.size() + 32 < kMaxFactors && (k == r0 || fits_one_more())) {
                const Instr &d = P.prog_instrs[k];
                if (d.op == OP_DIAG1 || d.op == OP_DIAG2)
                    touched |= 1u << d.p0;
                if (d.op == OP_DIAG2)
                    touched |= 1u << d.p1;
                if (d.op == OP_DIAG1 || d.op == OP_DIAG2) {
                    G *= cplx(d.gate, 0);
                    alpha[d.p0] *= cplx(d.gate, 1);
                    if (d.op == OP_DIAG2) {
                        alpha[d.p1] *= cplx(d.gate, 2);
                        if (d.pad & 8u)
                            pair_mul(d.p0, d.p1, cplx(d.gate, 3));
                    }
                }
                k++;
            }
            std::vector<std::pair<FacHdr, std::complex<double>>> facs;
            for (uint32_t q = 0; q < 32; q++) {
                if (alpha[q] == std::complex<double>(1.0, 0.0))
                    continue;
                FacHdr f;
                std::memset(&f, 0, sizeof(f));
                f.kind = is_slot((uint8_t)q) ? FAC_A_SLOT : FAC_A_FIXED;
                f.p0 = (uint8_t)q;
                f.j0 = pos[q];
                facs.push_back({f, alpha[q]});
            }
            for (auto &e : pairs) {
                if (e.second == std::complex<double>(1.0, 0.0))
                    continue;
                uint8_t a = e.first.first, b = e.first.second;
                FacHdr f;
                std::memset(&f, 0, sizeof(f));
                const bool sa = is_slot(a), sb = is_slot(b);
                if (!sa && !sb)
                    f.kind = FAC_C_FIXED;
                else if (sa && sb)
                    f.kind = FAC_C_SLOTS;
                else {
                    f.kind = FAC_C_MIXED;
                    if (sa)
                        std::swap(a, b);  // p0 fixed, p1 on a slot
                }
                f.p0 = a;
                f.j0 = pos[a];
                f.p1 = b;
                f.j1 = pos[b];
                facs.push_back({f, e.second});
            }
            std::stable_sort(facs.begin(), facs.end(),
                             [](const std::pair<FacHdr, std::complex<double>> &x,
                                const std::pair<FacHdr, std::complex<double>> &y) { return x.first.kind < y.first.kind; });
            if (!f64) {
                // FP32 runs: the factors grouped by the phase accumulator they feed,
                // each with the mask of fixed physical bits whose logical values
                // must all be 1 for it to apply (one or two bits), and the uniform
                // ones (slot-only) summed here.  See RunHdr32.
                std::vector<std::pair<uint32_t, uint32_t>> lists[1 + kMaxSlots];
                uint32_t econst[kMaxSlots] = {0}, gp[kMaxSlots * (kMaxSlots - 1) / 2] = {0};
                uint32_t eused = 0, gused = 0;
                for (auto &f : facs) {
                    const FacHdr &fh = f.first;
                    const uint32_t ang = turn32(f.second);
                    switch (fh.kind) {
                    case FAC_A_FIXED: lists[0].push_back({1u << fh.p0, ang}); break;
                    case FAC_C_FIXED: lists[0].push_back({(1u << fh.p0) | (1u << fh.p1), ang}); break;
                    case FAC_A_SLOT: econst[fh.j0 - 8] += ang; eused |= 1u << (fh.j0 - 8); break;
                    case FAC_C_MIXED: lists[1 + fh.j1 - 8].push_back({1u << fh.p0, ang}); break;
                    default: {  // FAC_C_SLOTS
                        const uint32_t a = fh.j0 - 8u, b = fh.j1 - 8u, hi = a > b ? a : b, lo = a > b ? b : a;
                        gp[hi * (hi - 1) / 2 + lo] += ang;
                        gused |= 1u << (hi * (hi - 1) / 2 + lo);
                    }
                    }
                }
                size_t nent = 0;
                for (auto &l : lists)
                    nent += l.size();
                const size_t body = 16 + 16 + 64 + (nent * 8 + 15) / 16 * 16 + (size_t)(k - r0) * esz;
                reserve(body);
                RecHdr h;
                std::memset(&h, 0, sizeof(h));
                h.type = REC_RUN;
                h.site = P.prog_instrs[r0].site;
                h.ibeg = r0;
                h.iend = k;
                put(&h, 16);
                RunHdr32 rh;
                std::memset(&rh, 0, sizeof(rh));
                rh.nbase = (uint8_t)lists[0].size();
                for (uint32_t q = 0; q < kMaxSlots; q++)
                    rh.ne[q] = (uint8_t)lists[1 + q].size();
                rh.gused = (uint16_t)gused;
                rh.eused = (uint8_t)eused;
                bool slot_terms = gused || eused;
                for (uint32_t q = 0; q < kMaxSlots; q++)
                    slot_terms = slot_terms || !lists[1 + q].empty();
                rh.pad[0] = slot_terms ? 0 : 1;
                rh.pad[1] = (uint8_t)nent;
                rh.g0 = turn32(G);
                for (uint32_t q = 0; q < kMaxSlots; q++)
                    rh.econst[q] = econst[q];
                for (uint32_t q = 0; q < kMaxSlots * (kMaxSlots - 1) / 2; q++)
                    rh.gp[q] = gp[q];
                put(&rh, sizeof(rh));
                for (auto &l : lists)
                    for (auto &e : l) {
                        put(&e.first, 4);
                        put(&e.second, 4);
                    }
                pad16();
            } else {
            uint8_t cnt[8] = {0};
            for (auto &f : facs)
                cnt[f.first.kind]++;
            reserve(32 + facs.size() * fsz + (size_t)(k - r0) * esz + 16);
            RecHdr h;
            std::memset(&h, 0, sizeof(h));
            h.type = REC_RUN;
            h.a = cnt[FAC_A_FIXED];
            h.b = cnt[FAC_A_SLOT];
            h.c = cnt[FAC_C_FIXED];
            h.d = cnt[FAC_C_MIXED];
            h.e = cnt[FAC_C_SLOTS];
            h.site = P.prog_instrs[r0].site;
            h.ibeg = r0;
            h.iend = k;
            put(&h, 16);
            putd(G);
            pad16();
            for (auto &f : facs) {
                put(&f.first, 8);
                if (f64)
                    out.insert(out.end(), 8, 0);  // the value sits 16-byte aligned
                putd(f.second);
                pad16();
            }
            }
            // the run gate by gate, for nodes with a Pauli inside it (see GateEnt)
            for (uint32_t x = r0; x < k; x++) {
                const Instr &d = P.prog_instrs[x];
                GateEnt g;
                std::memset(&g, 0, sizeof(g));
                g.op = d.op;
                g.fl = (uint8_t)d.pad;
                g.j0 = d.j0;
                g.p0 = d.p0;
                g.j1 = d.j1;
                g.p1 = d.p1;
                g.np0 = d.np0;
                g.np1 = d.np1;
                g.npaulis = d.npaulis;
                g.site = d.site;
                put(&g, 16);
                for (int e = 0; e < 4; e++)
                    putd(d.op == OP_DIAG1 || d.op == OP_DIAG2 ? cplx(d.gate, e) : std::complex<double>(1.0, 0.0));
            }
        }
        reserve(16);
        RecHdr endh;
        std::memset(&endh, 0, sizeof(endh));
        endh.type = REC_END;
        endh.ibeg = endh.iend = ps.iend;
        put(&endh, 16);
        ps.chunk_end = (uint32_t)P.chunk_off.size();
    }
    P.chunk_off.push_back((uint32_t)out.size());
}

std::vector<uint32_t> pass_starts_one_level(const Circuit &c, uint32_t tile_max)
{
    PlanHost P;
    tqs_options o;
    tqs_options_default(&o);
    o.tile_qubits = tile_max;
    Noise nz = {0, 0, 0};
    std::vector<uint64_t> arity = {1};
    std::vector<uint32_t> split = {0, (uint32_t)c.gates.size()};
    std::vector<uint32_t> starts;
    if (!build_plan(c, nz, 1, o, arity, split, P).empty())
        return starts;
    for (const Pass &ps : P.passes)
        starts.push_back(ps.site_begin);
    return starts;
}

std::string build_plan(const Circuit &c, const Noise &nz, uint64_t shots, const tqs_options &o,
                       const std::vector<uint64_t> &arity, const std::vector<uint32_t> &split,
                       PlanHost &P)
{
    const uint32_t n = c.n, G = (uint32_t)c.gates.size();
    const uint32_t L = (uint32_t)arity.size();
    P = PlanHost();
    P.n = n;
    P.prec = o.prec;
    P.mode = o.mode;
    P.shots = shots;
    uint32_t tdef = o.prec == TQS_FP64 ? 11 : 12;
    uint32_t tmax = o.tile_qubits ? o.tile_qubits : tdef;
    if (tmax < 6 || tmax > (uint32_t)kMaxTile)
        return "tile_qubits must be in [6, 13]";
    P.tile_max = tmax;
    P.thr1 = threshold32(nz.p1);
    P.thr2 = threshold32(nz.p2);
    P.thrm = threshold32(nz.pm);

    // lowered matrices: dense gates keep the full matrix, diagonal gates their diagonal
    P.mats64.assign((size_t)std::max<uint32_t>(G, 1) * 32, 0.0);
    std::vector<uint8_t> op(G);
    std::vector<uint16_t> diag_flags(G, 0);
    for (uint32_t g = 0; g < G; g++) {
        const Gate &gt = c.gates[g];
        bool two = is_two_qubit(gt.kind);
        double *dst = &P.mats64[(size_t)g * 32];
        if (gt.kind == TQS_SWAP) {
            op[g] = OP_NOP;
            continue;
        }
        int d = two ? 4 : 2;
        bool diag = is_diagonal(gt.kind);
        if (gt.kind == TQS_U1 || gt.kind == TQS_U2) {
            diag = true;
            for (int r = 0; r < d; r++)
                for (int k = 0; k < d; k++)
                    if (r != k && (gt.m[2 * (r * d + k)] != 0.0 || gt.m[2 * (r * d + k) + 1] != 0.0))
                        diag = false;
        }
        if (diag) {
            // D[x] (x = local index) as G * a0^{x0} * a1^{x1} * c^{x0 x1}: the
            // kernels fold runs of diagonal gates into these factors
            op[g] = two ? OP_DIAG2 : OP_DIAG1;
            std::complex<double> dd[4];
            for (int r = 0; r < d; r++)
                dd[r] = {gt.m[2 * (r * d + r)], gt.m[2 * (r * d + r) + 1]};
            std::complex<double> f[4] = {dd[0], dd[1] / dd[0], 1.0, 1.0};
            if (two) {
                f[2] = dd[2] / dd[0];
                f[3] = dd[3] * dd[0] / (dd[1] * dd[2]);
            }
            uint16_t flags = 0;
            for (int k = 0; k < 4; k++) {
                dst[2 * k] = f[k].real();
                dst[2 * k + 1] = f[k].imag();
                if (f[k] != std::complex<double>(1.0, 0.0))
                    flags |= (uint16_t)(1u << k);
            }
            diag_flags[g] = flags;
        } else {
            op[g] = two ? OP_DENSE2 : OP_DENSE1;
            std::memcpy(dst, gt.m, sizeof(double) * 2 * d * d);
        }
    }
    P.mats32.resize(P.mats64.size());
    for (size_t i = 0; i < P.mats64.size(); i++)
        P.mats32[i] = (float)P.mats64[i];

    // physical qubit of every gate with SWAPs made lazy (a relabelling only)
    std::vector<uint8_t> perm(n);
    for (uint32_t q = 0; q < n; q++)
        perm[q] = (uint8_t)q;
    struct Lowered { uint8_t p0, p1, np0, np1; };
    std::vector<Lowered> low(G);
    std::vector<std::vector<uint8_t>> perm_after(G + 1);
    perm_after[0] = perm;
    for (uint32_t g = 0; g < G; g++) {
        const Gate &gt = c.gates[g];
        if (gt.kind == TQS_SWAP)
            std::swap(perm[gt.q0], perm[gt.q1]);
        low[g].p0 = perm[gt.q0];
        low[g].p1 = perm[gt.q1];
        low[g].np0 = perm[gt.q0];
        low[g].np1 = perm[gt.q1];
        perm_after[g + 1] = perm;
    }

    // levels
    uint64_t below = 1;
    P.levels.resize(L);
    for (int i = (int)L - 1; i >= 0; i--) {
        Level &lv = P.levels[i];
        lv.g0 = split[i];
        lv.g1 = split[i + 1];
        lv.arity = arity[i];
        lv.below = below;
        unsigned __int128 act = ((unsigned __int128)shots + below - 1) / below;
        lv.active = (uint64_t)act;
        unsigned __int128 nb = (unsigned __int128)below * arity[i];
        below = nb > ((unsigned __int128)1 << 63) ? ((uint64_t)1 << 63) : (uint64_t)nb;
        lv.perm = perm_after[lv.g1];
    }

    // tile passes per level, by list scheduling: a pass takes, in gate order,
    // every gate whose qubits no earlier untaken gate touches and whose dense
    // qubits still fit the tile (diagonal gates and lazy SWAP noise sites fit
    // any tile).  Gates that share a (physical) qubit keep their order, so each
    // gate and the Pauli drawn after it act between the same neighbours as in
    // the circuit; gates on disjoint qubits commute.  A pass can thus run ahead
    // on the qubits it holds instead of stopping at the first gate that does
    // not fit.
    auto gate_qubits = [&](uint32_t g) {
        const bool two = is_two_qubit(c.gates[g].kind);
        uint32_t q = (1u << low[g].np0) | (two ? (1u << low[g].np1) : 0u);
        if (op[g] != OP_NOP)
            q |= (1u << low[g].p0) | (two ? (1u << low[g].p1) : 0u);
        return q;
    };
    // With damping channels (Sec. 4.3) every gate's channel choice needs a
    // reduction over the whole state after it, so every gate ends a pass and
    // gates keep circuit order: pass k of a level holds gate g0+k, opened by the
    // operators chosen after the previous gate of the level; one more pass,
    // holding only those of the level's last gate, closes the level.
    P.kraus = nz.kraus();
    P.krate[0][0] = nz.tr_g1; P.krate[0][1] = nz.tr_l1; P.krate[0][2] = nz.ad; P.krate[0][3] = nz.pd;
    P.krate[1][0] = nz.tr_g2; P.krate[1][1] = nz.tr_l2; P.krate[1][2] = nz.ad; P.krate[1][3] = nz.pd;
    for (uint32_t i = 0; i < L; i++) {
        Level &lv = P.levels[i];
        lv.pass_begin = (uint32_t)P.passes.size();
        std::vector<uint32_t> rem;
        for (uint32_t g = lv.g0; g < lv.g1; g++)
            rem.push_back(g);
        uint8_t kin_nq = 0, kin_p0 = 0, kin_p1 = 0;
        do {
            uint32_t need = 0, blocked = 0;
            const uint32_t lowbits = (1u << std::min<uint32_t>(n, 4)) - 1;
            std::vector<uint32_t> take, left;
            if (P.kraus) {
                need = kin_nq ? ((1u << kin_p0) | (kin_nq == 2 ? (1u << kin_p1) : 0u)) : 0u;
                if (!rem.empty()) {
                    const uint32_t g = rem[0];
                    if (op[g] == OP_DENSE1)
                        need |= 1u << low[g].p0;
                    else if (op[g] == OP_DENSE2)
                        need |= (1u << low[g].p0) | (1u << low[g].p1);
                    take.push_back(g);
                    left.assign(rem.begin() + 1, rem.end());
                }
                rem.clear();
            }
            for (uint32_t g : rem) {
                const uint32_t q = gate_qubits(g);
                uint32_t add = 0;
                if (op[g] == OP_DENSE1)
                    add = 1u << low[g].p0;
                else if (op[g] == OP_DENSE2)
                    add = (1u << low[g].p0) | (1u << low[g].p1);
                if ((q & blocked) || (uint32_t)__builtin_popcount(need | add | lowbits) > std::min(n, tmax)) {
                    blocked |= q;
                    left.push_back(g);
                    continue;
                }
                need |= add;
                take.push_back(g);
            }
            if (take.empty() && !rem.empty())
                return "internal: pass scheduling made no progress";  // an empty level gets one empty pass
            Pass ps;
            std::memset(&ps, 0, sizeof(ps));
            ps.kout_gate = -1;
            ps.level = i;
            ps.site_begin = take.empty() ? 0u : take[0] - lv.g0;
            if (P.kraus) {
                ps.kin_nq = kin_nq;
                ps.kin_p0 = kin_p0;
                ps.kin_p1 = kin_p1;
                kin_nq = 0;
                if (!take.empty()) {
                    const uint32_t g = take[0];
                    const bool two = is_two_qubit(c.gates[g].kind);
                    ps.kout_gate = (int32_t)g;
                    ps.kout_nq = two ? 2 : 1;
                    ps.kout_p0 = low[g].np0;
                    ps.kout_p1 = two ? low[g].np1 : low[g].np0;
                    kin_nq = ps.kout_nq;
                    kin_p0 = ps.kout_p0;
                    kin_p1 = ps.kout_p1;
                }
            }
            choose_tile(n, tmax, need, nullptr, 0, ps);
            ps.ibeg = (uint32_t)P.instrs.size();
            uint8_t pos[32];
            std::memset(pos, 0xff, sizeof(pos));
            for (uint32_t j = 0; j < ps.t; j++)
                pos[ps.tbits[j]] = (uint8_t)j;
            for (uint32_t k : take) {
                Instr in;
                std::memset(&in, 0, sizeof(in));
                in.op = op[k];
                in.p0 = low[k].p0;
                in.p1 = low[k].p1;
                in.j0 = pos[low[k].p0];
                in.j1 = pos[low[k].p1];
                in.np0 = low[k].np0;
                in.np1 = low[k].np1;
                in.npaulis = is_two_qubit(c.gates[k].kind) ? 15 : 3;
                in.site = (uint16_t)(k - lv.g0);
                in.pad = diag_flags[k];
                in.gate = k;
                P.instrs.push_back(in);
            }
            ps.iend = (uint32_t)P.instrs.size();
            P.passes.push_back(ps);
            rem.swap(left);
        } while (!rem.empty() || (P.kraus && kin_nq));  // damping: a closing pass applies the last choice
        lv.pass_end = (uint32_t)P.passes.size();
    }

    // final pass: prefer the physical homes of the lowest logical outcome bits
    Pass &fin = P.passes.back();
    const std::vector<uint8_t> &pf = P.levels.back().perm;
    {
        uint32_t need = 0;
        for (uint32_t k = fin.ibeg; k < fin.iend; k++) {
            const Instr &in = P.instrs[k];
            if (in.op == OP_DENSE1)
                need |= 1u << in.p0;
            else if (in.op == OP_DENSE2)
                need |= (1u << in.p0) | (1u << in.p1);
        }
        if (fin.kin_nq)
            need |= (1u << fin.kin_p0) | (1u << fin.kin_p1);
        choose_tile(n, tmax, need, pf.data(), std::min<uint32_t>(n, kMaxGamma), fin);
        uint8_t pos[32];
        std::memset(pos, 0xff, sizeof(pos));
        for (uint32_t j = 0; j < fin.t; j++)
            pos[fin.tbits[j]] = (uint8_t)j;
        for (uint32_t k = fin.ibeg; k < fin.iend; k++) {
            P.instrs[k].j0 = pos[P.instrs[k].p0];
            P.instrs[k].j1 = pos[P.instrs[k].p1];
        }
    }

    // sampler layout of the final pass
    SamplerLayout &S = P.samp;
    std::memset(&S, 0, sizeof(S));
    uint8_t inv[32];
    for (uint32_t q = 0; q < n; q++) {
        S.phys_of_logical[q] = pf[q];
        inv[pf[q]] = (uint8_t)q;
    }
    uint32_t qH = n;
    for (uint32_t h = 0; h < n - fin.t; h++) {
        S.logical_of_hbit[h] = inv[fin.hbits[h]];
        qH = std::min<uint32_t>(qH, inv[fin.hbits[h]]);
    }
    S.gamma = std::min<uint32_t>(qH, kMaxGamma);
    S.groups = (uint64_t)1 << (n - S.gamma);
    // ranks: tile positions ordered by their logical bit
    std::vector<std::pair<uint8_t, uint8_t>> lr;
    for (uint32_t j = 0; j < fin.t; j++)
        lr.push_back({inv[fin.tbits[j]], (uint8_t)j});
    std::sort(lr.begin(), lr.end());
    for (uint32_t q = 0; q < 32; q++)
        S.rank_of_logical[q] = -1;
    for (uint32_t r = 0; r < fin.t; r++) {
        S.rank_q[r] = lr[r].first;
        S.rank_pos[r] = lr[r].second;
        S.rank_of_logical[lr[r].first] = (int8_t)r;
    }
    for (uint32_t r = 0; r < S.gamma; r++)
        if (S.rank_q[r] != r)
            return "internal: sampler layout invariant broken";
    P.fuse = (o.flags & TQS_FLAG_FUSE) != 0 && !P.kraus;
    sink_diagonals(P);
    compile_programs(P);
    return "";
}

}  // namespace tqs
