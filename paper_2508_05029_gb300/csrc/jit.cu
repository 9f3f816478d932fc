// Run-time compilation of plan-specialised kernels.
//
// Paper basis: Section 3.1 (operators are GPU kernels over batches of
// columns).  The aggregate kernels of the ahead-of-time build read the plan's
// shape (column types, join kind, group fields, aggregate kinds) from their
// parameters on every row.  Here a kernel is compiled once per shape with
// NVRTC, the shape fixed as a compile-time struct (JS) in front of the kernel
// source, and loaded as a CUDA library; the kernel text is the library's own
// device headers, embedded at build time.  NVRTC is loaded with dlopen on
// first use, so a process without it still runs the ahead-of-time kernels.
//
// Kernels are cached for the life of the process, keyed by the generated
// source: a library loaded with cudaLibraryLoadData is not tied to a context,
// so one entry serves every engine and device.  Compilation happens under the
// cache lock: concurrent executions of a new shape wait for the first.
#include <dlfcn.h>
#include <nvrtc.h>

#include <chrono>

#include "tp_internal.h"

namespace {

// Embedded sources: {include name, text} pairs, generated by the build from
// the device headers the run-time compiled kernels include.
#include "jit_sources.inc"

struct Nvrtc {
    bool loaded = false;
    std::string why;   // why NVRTC is unavailable
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    decltype(&nvrtcGetErrorString) err = nullptr;
};

struct Entry {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kernel = nullptr;
    std::string error;   // non-empty: this shape failed to compile or load
};

std::mutex g_mu;
Nvrtc g_nvrtc;
bool g_nvrtc_tried = false;
std::map<std::string, Entry> g_cache;

// Loads NVRTC (caller holds g_mu).
void load_nvrtc() {
    if (g_nvrtc_tried) return;
    g_nvrtc_tried = true;
    const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                           "/usr/local/cuda/lib64/libnvrtc.so"};
    void* h = nullptr;
    for (const char* n : names)
        if ((h = dlopen(n, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    if (!h) {
        g_nvrtc.why = "NVRTC library not found";
        return;
    }
    Nvrtc& n = g_nvrtc;
    bool ok = true;
    auto sym = [&](auto& fn, const char* name) {
        fn = reinterpret_cast<std::remove_reference_t<decltype(fn)>>(dlsym(h, name));
        ok = ok && fn != nullptr;
    };
    sym(n.create, "nvrtcCreateProgram");
    sym(n.compile, "nvrtcCompileProgram");
    sym(n.log_size, "nvrtcGetProgramLogSize");
    sym(n.log, "nvrtcGetProgramLog");
    sym(n.cubin_size, "nvrtcGetCUBINSize");
    sym(n.cubin, "nvrtcGetCUBIN");
    sym(n.destroy, "nvrtcDestroyProgram");
    sym(n.err, "nvrtcGetErrorString");
    if (!ok) {
        n.why = "NVRTC library lacks an expected entry point";
        return;
    }
    n.loaded = true;
}

// Compiles `prelude` (shape structs, then the include of the kernel's header)
// for this device's architecture and loads it (caller holds g_mu).
Entry build_entry(const std::string& prelude, const char* entry, int device) {
    Entry en;
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
    std::vector<const char*> hdr_text, hdr_name;
    for (const JitSource& s : kJitSources) {
        hdr_name.push_back(s.name);
        hdr_text.push_back(s.text);
    }
    const std::string& src = prelude;   // shape structs and the kernel's include
    nvrtcProgram prog = nullptr;
    nvrtcResult r = g_nvrtc.create(&prog, src.c_str(), "tp_jit.cu", (int)hdr_text.size(), hdr_text.data(),
                                   hdr_name.data());
    if (r != NVRTC_SUCCESS) {
        en.error = std::string("nvrtcCreateProgram: ") + g_nvrtc.err(r);
        return en;
    }
    char arch[64], d_cons[64], d_rpl[64], d_ctas[64];
    // the architecture-specific target (sm_XXXa): the kernels use sm_90+ PTX
    snprintf(arch, sizeof(arch), "--gpu-architecture=sm_%d%da", major, minor);
    // the kernel's own geometry (the host sized its layout with the same)
    snprintf(d_cons, sizeof(d_cons), "-DTP_ST_CONSUMERS=%d", tpk::JIT_DENSE_GEOM.consumers);
    snprintf(d_rpl, sizeof(d_rpl), "-DTP_ST_RPL=%d", tpk::JIT_DENSE_GEOM.rpl);
    snprintf(d_ctas, sizeof(d_ctas), "-DTP_ST_CTAS=%d", tpk::JIT_DENSE_GEOM.ctas);
    const char* opts[] = {arch, "-std=c++17", "--device-int128", d_cons, d_rpl, d_ctas};
    r = g_nvrtc.compile(prog, (int)(sizeof(opts) / sizeof(opts[0])), opts);
    if (r != NVRTC_SUCCESS) {
        size_t n = 0;
        g_nvrtc.log_size(prog, &n);
        std::string log(n, '\0');
        if (n) g_nvrtc.log(prog, &log[0]);
        en.error = std::string("nvrtcCompileProgram: ") + g_nvrtc.err(r) + ": " + log.substr(0, 600);
        g_nvrtc.destroy(&prog);
        return en;
    }
    size_t bytes = 0;
    g_nvrtc.cubin_size(prog, &bytes);
    std::vector<char> cubin(bytes);
    g_nvrtc.cubin(prog, cubin.data());
    g_nvrtc.destroy(&prog);
    cudaError_t ce = cudaLibraryLoadData(&en.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (ce == cudaSuccess) ce = cudaLibraryGetKernel(&en.kernel, en.lib, entry);
    cudaFuncAttributes fa;   // the handle must be usable where the runtime takes a kernel
    if (ce == cudaSuccess) ce = cudaFuncGetAttributes(&fa, (const void*)en.kernel);
    if (ce != cudaSuccess) {
        en.error = std::string("loading the compiled kernel: ") + cudaGetErrorString(ce);
        en.kernel = nullptr;
    }
    return en;
}

}  // namespace

namespace tp {

const void* jit_kernel(tp_engine* e, const std::string& prelude, const char* entry, std::string* why) {
    std::lock_guard<std::mutex> lk(g_mu);
    const std::string key = std::string(entry) + "\n" + prelude;
    auto it = g_cache.find(key);
    if (it == g_cache.end()) {
        load_nvrtc();
        if (!g_nvrtc.loaded) {
            if (why) *why = g_nvrtc.why;
            return nullptr;
        }
        const auto t0 = std::chrono::steady_clock::now();
        Entry en = build_entry(prelude, entry, e->device);
        const auto us =
            std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
        e->jit_us += (uint64_t)us;
        if (en.error.empty()) e->jit_compiles++;
        else e->jit_failures++;
        it = g_cache.emplace(key, std::move(en)).first;
    }
    if (!it->second.error.empty()) {
        if (why) *why = it->second.error;
        return nullptr;
    }
    return (const void*)it->second.kernel;
}

}  // namespace tp
