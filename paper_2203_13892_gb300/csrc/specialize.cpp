// specialize.cpp -- the pass-program compiler (records -> CUDA statements) and
// the NVRTC / driver-API runtime that builds, caches and launches the
// specialised pass kernels (see specialize.h).
#include "specialize.h"

#include <cuda.h>
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <sstream>
#include <thread>

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
bool emit_run(std::ostringstream &o, const RecHdr &h, const uint8_t *pay, int logr, uint32_t &len, std::string &why)
{
    RunHdr32 rh;
    std::memcpy(&rh, pay, sizeof rh);
    const uint32_t nent = rh.pad[1];
    const uint32_t ngates = h.iend - h.ibeg;
    const uint32_t ent_bytes = (nent * 8u + 15u) / 16u * 16u;
    constexpr uint32_t ES = 32;  // GateEnt + four u32 phases
    const uint8_t *en = pay + 80;
    const uint8_t *gents = pay + 80 + ent_bytes;
    len = 96u + ent_bytes + ngates * ES;
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
    if (ps.t > (uint32_t)kMaxTile || ps.t + 0u > H.n)
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
            uint32_t len = 0;
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
                if (o1 - o0 - p < 96 || !emit_run(o, h, pay, out.logr, len, why))
                    return why.empty() ? std::string("truncated run record") : why;
            } else {
                return "record type " + std::to_string((int)h.type) + " has no specialised form";
            }
            if (len > o1 - o0 - p)
                return "record runs past its chunk";
            p += len;
        }
    }
    if (!ended)
        return "the pass program has no end record";
    out.walk = o.str();
    return "";
}

// ---------------------------------------------------------------------------
// NVRTC and the driver API, opened at run time
// ---------------------------------------------------------------------------
namespace {

#include "tqs_jit_sources.inc"  // kJitNames / kJitTexts: the kernel's headers, embedded at build time

struct Api {
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    decltype(&nvrtcAddNameExpression) add_name = nullptr;
    decltype(&nvrtcGetLoweredName) lowered = nullptr;
    decltype(&cuModuleLoadData) load = nullptr;
    decltype(&cuModuleGetFunction) get_function = nullptr;
    decltype(&cuFuncSetAttribute) set_attr = nullptr;
    decltype(&cuLaunchKernel) launch = nullptr;
    decltype(&cuGetErrorString) err_string = nullptr;
    std::string why;      // "" = usable (NVRTC and the driver)
    std::string why_rtc;  // "" = NVRTC usable
};

void *open_first(const char *const *names)
{
    for (const char *const *n = names; *n; n++)
        if (void *h = dlopen(*n, RTLD_NOW | RTLD_LOCAL))
            return h;
    return nullptr;
}

const Api &api()
{
    static Api a;
    static std::once_flag once;
    std::call_once(once, [] {
        static const char *const rtc[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                                          nullptr};
        static const char *const drv[] = {"libcuda.so.1", "libcuda.so", nullptr};
        void *hr = open_first(rtc), *hd = open_first(drv);
        if (!hr) {
            a.why = a.why_rtc = "NVRTC (libnvrtc.so.13) could not be opened";
            return;
        }
        bool ok = true;
        auto sym = [&](void *h, const char *name, auto &f) {
            f = reinterpret_cast<std::remove_reference_t<decltype(f)>>(dlsym(h, name));
            ok = ok && f != nullptr;
        };
        sym(hr, "nvrtcCreateProgram", a.create);
        sym(hr, "nvrtcCompileProgram", a.compile);
        sym(hr, "nvrtcGetProgramLogSize", a.log_size);
        sym(hr, "nvrtcGetProgramLog", a.log);
        sym(hr, "nvrtcGetCUBINSize", a.cubin_size);
        sym(hr, "nvrtcGetCUBIN", a.cubin);
        sym(hr, "nvrtcDestroyProgram", a.destroy);
        sym(hr, "nvrtcAddNameExpression", a.add_name);
        sym(hr, "nvrtcGetLoweredName", a.lowered);
        if (!ok) {
            a.why = a.why_rtc = "a symbol of NVRTC is missing";
            return;
        }
        if (!hd) {
            a.why = "the CUDA driver (libcuda.so.1) could not be opened";
            return;
        }
        sym(hd, "cuModuleLoadData", a.load);
        sym(hd, "cuModuleGetFunction", a.get_function);
        sym(hd, "cuFuncSetAttribute", a.set_attr);
        sym(hd, "cuLaunchKernel", a.launch);
        sym(hd, "cuGetErrorString", a.err_string);
        if (!ok)
            a.why = "a symbol of the CUDA driver is missing";
    });
    return a;
}

std::string cu_msg(const char *what, CUresult r)
{
    const char *s = nullptr;
    if (api().err_string)
        api().err_string(r, &s);
    return std::string(what) + ": " + (s ? s : "CUDA driver error " + std::to_string((int)r));
}

struct Compiled {
    std::string cubin, lowered, err;
};

// NVRTC: the kernel's headers plus the generated pieces, the instantiation
// pass_kernel<float, MODE, LOGR, false> by name expression, a cubin for sm_103a.
Compiled compile_one(const SpecSource &s)
{
    const Api &A = api();
    Compiled out;
    const std::string main_src = "#define TQS_SPEC 1\n#include \"internal.h\"\n#include \"tqs_spec_defs.inc\"\n"
                                 "#include \"pass_kernel.cuh\"\n";
    std::vector<const char *> names, texts;
    for (size_t i = 0; i < sizeof(kJitNames) / sizeof(kJitNames[0]); i++) {
        names.push_back(kJitNames[i]);
        texts.push_back(kJitTexts[i]);
    }
    names.push_back("tqs_spec_defs.inc");
    texts.push_back(s.defs.c_str());
    names.push_back("tqs_spec_walk.inc");
    texts.push_back(s.walk.c_str());
    nvrtcProgram prog = nullptr;
    if (A.create(&prog, main_src.c_str(), "tqs_pass_spec.cu", (int)names.size(), texts.data(), names.data()) !=
        NVRTC_SUCCESS) {
        out.err = "nvrtcCreateProgram failed";
        return out;
    }
    const std::string expr = "tqs::pass_kernel<float, " + std::to_string(s.mode) + ", " + std::to_string(s.logr) +
                             ", false>";
    A.add_name(prog, expr.c_str());
    const char *opts[] = {"-arch=sm_103a", "-std=c++17", "-default-device", "-diag-suppress=177,550"};
    const nvrtcResult r = A.compile(prog, (int)(sizeof(opts) / sizeof(opts[0])), opts);
    if (r != NVRTC_SUCCESS) {
        size_t n = 0;
        A.log_size(prog, &n);
        std::string log(n, '\0');
        A.log(prog, &log[0]);
        out.err = "NVRTC failed on a specialised pass kernel: " + log.substr(0, 4000);
        A.destroy(&prog);
        return out;
    }
    const char *low = nullptr;
    A.lowered(prog, expr.c_str(), &low);
    out.lowered = low ? low : "";
    size_t n = 0;
    A.cubin_size(prog, &n);
    out.cubin.resize(n);
    A.cubin(prog, &out.cubin[0]);
    A.destroy(&prog);
    if (out.lowered.empty() || n == 0)
        out.err = "NVRTC produced no kernel";
    return out;
}

std::mutex g_mu;
std::map<std::string, void *> g_cache;  // device + source -> CUfunction

}  // namespace

std::string spec_available(bool need_driver) { return need_driver ? api().why : api().why_rtc; }

std::string spec_compile_only(const std::vector<SpecSource> &srcs)
{
    if (!api().why_rtc.empty())
        return api().why_rtc;
    std::vector<std::string> errs(srcs.size());
    const size_t nthr = std::max<size_t>(1, std::min<size_t>(srcs.size(), std::max(1u, std::thread::hardware_concurrency())));
    std::atomic<size_t> next{0};
    std::vector<std::thread> pool;
    for (size_t t = 0; t < nthr; t++)
        pool.emplace_back([&] {
            for (size_t k; (k = next.fetch_add(1)) < srcs.size();)
                errs[k] = compile_one(srcs[k]).err;
        });
    for (auto &th : pool)
        th.join();
    for (auto &e : errs)
        if (!e.empty())
            return e;
    return "";
}

std::string spec_build(const std::vector<SpecSource> &srcs, std::vector<void *> &fns)
{
    const Api &A = api();
    if (!A.why.empty())
        return A.why;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaFree(nullptr) != cudaSuccess) {  // a current context
        cudaGetLastError();
        return "no CUDA device for the specialised kernels";
    }
    fns.assign(srcs.size(), nullptr);
    std::vector<std::string> keys(srcs.size());
    std::vector<size_t> todo;
    {
        std::lock_guard<std::mutex> g(g_mu);
        std::map<std::string, size_t> first;  // identical sources in one request compile once
        for (size_t i = 0; i < srcs.size(); i++) {
            keys[i] = std::to_string(dev) + "\n" + srcs[i].key();
            auto it = g_cache.find(keys[i]);
            if (it != g_cache.end())
                fns[i] = it->second;
            else if (first.emplace(keys[i], i).second)
                todo.push_back(i);
        }
    }
    std::vector<Compiled> res(todo.size());
    {
        const size_t nthr = std::max<size_t>(1, std::min<size_t>(todo.size(), std::max(1u, std::thread::hardware_concurrency())));
        std::atomic<size_t> next{0};
        std::vector<std::thread> pool;
        for (size_t t = 0; t < nthr; t++)
            pool.emplace_back([&] {
                for (size_t k; (k = next.fetch_add(1)) < todo.size();)
                    res[k] = compile_one(srcs[todo[k]]);
            });
        for (auto &th : pool)
            th.join();
    }
    std::lock_guard<std::mutex> g(g_mu);
    for (size_t k = 0; k < todo.size(); k++) {
        if (!res[k].err.empty())
            return res[k].err;
        CUmodule mod = nullptr;
        CUresult r = A.load(&mod, res[k].cubin.data());
        if (r != CUDA_SUCCESS)
            return cu_msg("cuModuleLoadData (specialised pass kernel)", r);
        CUfunction fn = nullptr;
        r = A.get_function(&fn, mod, res[k].lowered.c_str());
        if (r != CUDA_SUCCESS)
            return cu_msg("cuModuleGetFunction (specialised pass kernel)", r);
        r = A.set_attr(fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, 200 * 1024);
        if (r != CUDA_SUCCESS)
            return cu_msg("cuFuncSetAttribute (specialised pass kernel)", r);
        g_cache[keys[todo[k]]] = (void *)fn;
    }
    for (size_t i = 0; i < srcs.size(); i++)
        if (!fns[i])
            fns[i] = g_cache.at(keys[i]);
    return "";
}

int spec_launch(void *fn, const void *params, unsigned gx, unsigned gy, size_t smem, void *stream)
{
    void *args[] = {const_cast<void *>(params)};
    const CUresult r = api().launch((CUfunction)fn, gx, gy, 1, (unsigned)kThreads, 1, 1, (unsigned)smem,
                                    (CUstream)stream, args, nullptr);
    // the runtime's error codes for the two launch failures callers distinguish
    if (r == CUDA_SUCCESS)
        return 0;
    if (r == CUDA_ERROR_INVALID_VALUE)
        return (int)cudaErrorInvalidValue;
    return (int)cudaErrorLaunchFailure;
}

}  // namespace tqs
