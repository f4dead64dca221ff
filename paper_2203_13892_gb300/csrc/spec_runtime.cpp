// spec_runtime.cpp -- builds, caches and launches the specialised pass kernels
// (see specialize.h): NVRTC compiles the generated sources for sm_103a, the
// driver API loads and launches them.  Both libraries are opened at run time, so
// libtqs loads on hosts without them.
#include <cuda.h>
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <type_traits>

#include "specialize.h"

namespace tqs {

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
        // the driver's versioned name only: an unversioned libcuda.so on a host
        // without a driver is the toolkit's link stub
        static const char *const drv[] = {"libcuda.so.1", nullptr};
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
    // the plan's uploads made the device's primary context current on this thread
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
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
    // the driver's launch errors have the runtime's numbers (invalid value, out of
    // resources, ...), so callers report them with cudaGetErrorString
    return (int)r;
}

}  // namespace tqs
