// specialize.cpp -- the pass-program compiler: a pass's records (the bytes the
// generic pass kernel interprets) -> CUDA statements and tile-layout constants
// for a kernel specialised to that pass (see specialize.h).  The NVRTC and
// driver-API side that builds, caches and launches the kernels is in
// spec_runtime.cpp.
#include "specialize.h"

#include <cstdio>
#include <cstring>
#include <sstream>

namespace tqs {

// ---------------------------------------------------------------------------
// Code generation
// ---------------------------------------------------------------------------
namespace {

// An FP32 constant as an exact hexadecimal literal.
std::string flit(float f)
{
    char b[64];
    std::snprintf(b, sizeof b, "%af", (double)f);
    return b;
}

std::string u32lit(uint32_t v)
{
    char b[32];
    std::snprintf(b, sizeof b, "0x%xu", v);
    return b;
}

template <typename T> T rd(const uint8_t *p)
{
    T v;
    std::memcpy(&v, p, sizeof(T));
    return v;
}

// The conditional phase terms of one accumulator: add PH where all bits of M
// are 1 in the thread's logical index (the interpreter's entry loop, unrolled).
void emit_entries(std::ostringstream &o, const uint8_t *en, uint32_t count)
{
    for (uint32_t i = 0; i < count; i++) {
        const uint32_t m = rd<uint32_t>(en + 8 * i), ph = rd<uint32_t>(en + 8 * i + 4);
        o << "        if ((xt & " << u32lit(m) << ") == " << u32lit(m) << ") add += " << u32lit(ph) << ";\n";
    }
}

void emit_noise(std::ostringstream &o, uint32_t site, uint32_t npaulis, uint32_t j0, uint32_t p0, uint32_t j1,
                uint32_t p1, bool guarded)
{
    if (guarded)
        o << "    if (pnoisy) ";
    else
        o << "    ";
    o << "{ const uint32_t pz = noise_at(" << site << "u); if (pz) apply_noise(pz, " << npaulis << "u, " << j0
      << "u, " << p0 << "u, " << j1 << "u, " << p1 << "u); }\n";
}

// One FP32 diagonal run (RunHdr32 layout), as the interpreter walks it: the
// grouped phase entries when no Pauli of this node falls inside the run, else
// gate by gate from the run's gate entries.
// `avail` = the bytes of the chunk from the record's header on: the record's
// length (from its header) is checked against it before any entry is read.
bool emit_run(std::ostringstream &o, const RecHdr &h, const uint8_t *pay, uint32_t avail, int logr, uint32_t &len,
              std::string &why)
{
    if (avail < 96u || h.iend < h.ibeg) {
        why = "truncated run record";
        return false;
    }
    RunHdr32 rh;
    std::memcpy(&rh, pay, sizeof rh);
    const uint32_t nent = rh.pad[1];
    const uint32_t ngates = h.iend - h.ibeg;
    const uint32_t ent_bytes = (nent * 8u + 15u) / 16u * 16u;
    constexpr uint32_t ES = 32;  // GateEnt + four u32 phases
    const uint8_t *en = pay + 80;
    const uint8_t *gents = pay + 80 + ent_bytes;
    len = 96u + ent_bytes + ngates * ES;
    if ((uint64_t)96u + ent_bytes + (uint64_t)ngates * ES > avail) {
        why = "run record runs past its chunk";
        return false;
    }
    uint32_t nsum = rh.nbase;
    for (int q = 0; q < logr; q++)
        nsum += rh.ne[q];
    if (nsum > nent) {
        why = "run record: more entries than its header declares";
        return false;
    }
    o << "    {  // diagonal run: sites " << h.ibeg << ".." << h.iend << "\n";
    o << "    bool anyn = false;\n";
    if (ngates) {
        o << "    if (pnoisy) anyn = (";
        for (uint32_t x = 0; x < ngates; x++)
            o << (x ? " | " : "") << "noise_at(" << rd<uint32_t>(gents + x * ES + 12) << "u)";
        o << ") != 0u;\n";
    }
    o << "    if (!anyn) {\n";
    if (rh.g0)
        o << "        acc.mul_base(" << u32lit(rh.g0) << ");\n";
    const uint32_t nb = rh.nbase;
    if (rh.pad[0]) {
        if (nb)
            o << "        acc.base_used = true;\n";
        o << "        { uint32_t add = 0u;\n";
        emit_entries(o, en, nb);
        o << "        acc.base += add; }\n";
        o << "        pending = true;\n";
    } else {
        const uint8_t *e = en;
        if (nb) {
            o << "        acc.base_used = true;\n        { uint32_t add = 0u;\n";
            emit_entries(o, e, nb);
            o << "        acc.base += add; }\n";
            e += 8 * nb;
        }
        for (int q = 0; q < logr; q++) {
            const uint32_t nq = rh.ne[q];
            if (nq == 0u && !((rh.eused >> q) & 1u))
                continue;
            o << "        { uint32_t add = " << u32lit(rh.econst[q]) << ";\n";
            emit_entries(o, e, nq);
            e += 8 * nq;
            o << "        acc.E[" << q << "] += add; acc.e_used |= " << (1u << q) << "u; }\n";
        }
        if (rh.gused) {
            const int npairs = logr > 1 ? logr * (logr - 1) / 2 : 1;
            for (int i = 0; i < npairs; i++)
                if ((rh.gused >> i) & 1u)
                    o << "        acc.Gs[" << i << "] += " << u32lit(rh.gp[i]) << ";\n";
            o << "        acc.gs_used |= " << u32lit(rh.gused) << "; acc.has_gs = true;\n";
        }
        o << "        pending = true;\n";
    }
    o << "    } else {\n";
    for (uint32_t x = 0; x < ngates; x++) {
        const uint8_t *gq = gents + x * ES;
        const uint32_t ex = rd<uint32_t>(gq), ey = rd<uint32_t>(gq + 4), ez = rd<uint32_t>(gq + 8),
                       ew = rd<uint32_t>(gq + 12);
        const uint32_t op = ex & 0xffu, fl = (ex >> 8) & 0xffu, j0 = (ex >> 16) & 0xffu, p0 = ex >> 24,
                       j1 = ey & 0xffu, p1 = (ey >> 8) & 0xffu, np0 = (ey >> 16) & 0xffu, np1 = ey >> 24,
                       npl = ez & 0xffu;
        uint32_t M[4];
        for (int k = 0; k < 4; k++)
            M[k] = rd<uint32_t>(gq + 16 + 4 * k);
        if (op == OP_DIAG1 || op == OP_DIAG2) {
            if (fl & 1u)
                o << "        acc.mul_base(" << u32lit(M[0]) << ");\n";
            if (fl & 2u)
                o << "        acc_alpha(acc, " << j0 << "u, " << p0 << "u, xt, " << u32lit(M[1]) << ");\n";
            if (op == OP_DIAG2) {
                if (fl & 4u)
                    o << "        acc_alpha(acc, " << j1 << "u, " << p1 << "u, xt, " << u32lit(M[2]) << ");\n";
                if (fl & 8u)
                    o << "        acc_gamma(acc, " << j0 << "u, " << p0 << "u, " << j1 << "u, " << p1 << "u, xt, "
                      << u32lit(M[3]) << ");\n";
            }
            o << "        pending = true;\n";
        }
        o << "    ";
        emit_noise(o, ew, npl, j0, np0, j1, np1, false);
    }
    o << "    }\n    }\n";
    return true;
}

}  // namespace

std::string SpecSource::key() const
{
    return std::to_string(mode) + "/" + std::to_string(logr) + "\n" + defs + walk;
}

std::string spec_generate(const PlanHost &H, const Pass &ps, int mode, SpecSource &out)
{
    if (H.prec != TQS_FP32)
        return "only FP32 states have specialised kernels";
    if (ps.fused_blocks)
        return "the pass holds fused tensor-core blocks";
    if (ps.t > (uint32_t)kMaxTile || ps.t > H.n)
        return "tile wider than the state";
    out = SpecSource{};
    out.mode = mode;
    out.logr = ps.t > 8 ? (int)ps.t - 8 : 0;
    {
        std::ostringstream d;
        d << "namespace tqs { namespace spec {\n";
        d << "constexpr uint32_t kT = " << ps.t << "u, kN = " << H.n << "u;\n";
        d << "__host__ __device__ constexpr uint32_t tbit(uint32_t j) { return ";
        for (uint32_t j = 0; j < ps.t; j++)
            d << "j == " << j << "u ? " << (uint32_t)ps.tbits[j] << "u : ";
        d << "0u; }\n";
        d << "__host__ __device__ constexpr uint32_t hbit(uint32_t b) { return ";
        for (uint32_t b = 0; b < H.n - ps.t; b++)
            d << "b == " << b << "u ? " << (uint32_t)ps.hbits[b] << "u : ";
        d << "0u; }\n";
        // physical offset of register slot k: its bits deposited at the slot positions' physical bits
        d << "__host__ __device__ constexpr uint32_t soff(uint32_t k) { return 0u";
        for (int b = 0; b < out.logr; b++)
            d << " | (((k >> " << b << ") & 1u) << " << (uint32_t)ps.tbits[8 + b] << ")";
        d << "; }\n} }\n";
        out.defs = d.str();
    }
    std::ostringstream o;
    const uint8_t *prog = H.prog.data();
    bool ended = false;
    for (uint32_t c = ps.chunk_begin; c < ps.chunk_end; c++) {
        const uint32_t o0 = H.chunk_off[c], o1 = H.chunk_off[c + 1];
        if (ended) {
            if (o1 > o0)
                return "records after the end of the pass";
            continue;
        }
        bool staged = false;  // this chunk's bytes in shared memory (4x4 matrices are read from there)
        uint32_t p = 0;
        while (p < o1 - o0) {
            if (o1 - o0 - p < 16)
                return "truncated record";
            const uint8_t *rec = prog + o0 + p;
            RecHdr h;
            std::memcpy(&h, rec, sizeof h);
            const uint8_t *pay = rec + 16;
            if (h.type == REC_END) {
                // a final diagonal run changes phases only, not the measured |a|^2
                o << "    if (MODE != MODE_STORE) { acc.reset(); pending = false; }\n    flush();\n";
                ended = true;
                break;
            }
            if (h.type != REC_RUN)
                o << "    flush();\n";
            // each record's length is checked against the chunk before its payload is read
            const uint32_t avail = o1 - o0 - p;
            uint32_t len = 0;
            if (h.type == REC_DENSE1 && avail < 48u)
                return "truncated one-qubit gate record";
            if (h.type == REC_DENSE2 && avail < 16u + 16u * 8u)
                return "truncated two-qubit gate record";
            if (h.type == REC_DENSE1) {
                float u[8];
                std::memcpy(u, pay, sizeof u);
                if (h.c)
                    o << "    dense1_real(" << (uint32_t)h.a << "u, " << (uint32_t)h.b << "u, " << flit(u[0]) << ", "
                      << flit(u[2]) << ", " << flit(u[4]) << ", " << flit(u[6]) << ");\n";
                else
                    o << "    dense1(" << (uint32_t)h.a << "u, " << (uint32_t)h.b << "u, mk(" << flit(u[0]) << ", "
                      << flit(u[1]) << "), mk(" << flit(u[2]) << ", " << flit(u[3]) << "), mk(" << flit(u[4])
                      << ", " << flit(u[5]) << "), mk(" << flit(u[6]) << ", " << flit(u[7]) << "));\n";
                emit_noise(o, h.site, 3, h.a, h.b, h.a, h.b, true);
                len = 48;
            } else if (h.type == REC_DENSE2) {
                if (!staged) {
                    o << "    __syncthreads();\n    for (uint32_t x = tid; x < " << (o1 - o0) / 16u
                      << "u; x += kThreads)\n        reinterpret_cast<uint4 *>(pbuf)[x] = "
                         "reinterpret_cast<const uint4 *>(a.prog + "
                      << o0 << "u)[x];\n    __syncthreads();\n";
                    staged = true;
                }
                o << "    dense2(" << (uint32_t)h.a << "u, " << (uint32_t)h.b << "u, " << (uint32_t)h.c << "u, "
                  << (uint32_t)h.d << "u, [&](uint32_t kk) -> C { return *reinterpret_cast<const C *>(pbuf + "
                  << (p + 16) << "u + kk * 8u); });\n";
                emit_noise(o, h.site, 15, h.a, h.c, h.b, h.d, true);
                len = 16 + 16 * 8;
            } else if (h.type == REC_KRAUS) {
                o << "    { const C *km = reinterpret_cast<const C *>(a.kmat) + (uint64_t)slot * 8;\n";
                o << "      dense1_real(" << (uint32_t)h.a << "u, " << (uint32_t)h.c
                  << "u, km[0].x, km[1].x, km[2].x, km[3].x);\n";
                if (h.e == 2)
                    o << "      dense1_real(" << (uint32_t)h.b << "u, " << (uint32_t)h.d
                      << "u, km[4].x, km[5].x, km[6].x, km[7].x);\n";
                o << "    }\n";
                len = 16;
            } else if (h.type == REC_RUN) {
                std::string why;
                if (!emit_run(o, h, pay, avail, out.logr, len, why))
                    return why;
            } else {
                return "record type " + std::to_string((int)h.type) + " has no specialised form";
            }
            p += len;
        }
    }
    if (!ended)
        return "the pass program has no end record";
    out.walk = o.str();
    return "";
}

}  // namespace tqs
