// srmc_rtc.cu -- step kernels for user models, compiled at run time.
//
// A user model supplies g and f as source (srmc_user_g, srmc_user_f over the
// type srmc_real).  The library compiles its own step-kernel source with that
// source in front (NVRTC, -DSRMC_USER_MODEL), once per solver and variant
// (precision, basis, control), loads the cubin with the runtime's library
// API and launches the entry kernel srmc_user_step like the built-in ones.
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdio>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "srmc_internal.h"

// The step-kernel sources, embedded at build time (generated unit).
extern const char srmc_rtc_device_cuh[];
extern const char srmc_rtc_step_cu[];

#ifndef SRMC_CUDA_INCLUDE
#define SRMC_CUDA_INCLUDE "/usr/local/cuda/include"
#endif
#ifndef SRMC_NVRTC_LIB
#define SRMC_NVRTC_LIB "libnvrtc.so"
#endif

namespace srmc {
namespace {
// NVRTC is opened on first use (dlopen), so that the library itself does
// not depend on it and only user models need it.
struct Nvrtc {
    nvrtcResult (*create)(nvrtcProgram *, const char *, const char *, int, const char *const *,
                          const char *const *) = nullptr;
    nvrtcResult (*compile)(nvrtcProgram, int, const char *const *) = nullptr;
    nvrtcResult (*log_size)(nvrtcProgram, size_t *) = nullptr;
    nvrtcResult (*log)(nvrtcProgram, char *) = nullptr;
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t *) = nullptr;
    nvrtcResult (*cubin)(nvrtcProgram, char *) = nullptr;
    nvrtcResult (*destroy)(nvrtcProgram *) = nullptr;
    const char *(*error_string)(nvrtcResult) = nullptr;
    bool ok = false;
};

const Nvrtc &nvrtc()
{
    static Nvrtc n;
    static std::once_flag once;
    std::call_once(once, [] {
        void *h = nullptr;
        for (const char *name : {"libnvrtc.so.13", SRMC_NVRTC_LIB, "libnvrtc.so"})
            if ((h = dlopen(name, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
        if (!h) return;
        auto get = [&](auto &fn, const char *sym) {
            fn = reinterpret_cast<std::remove_reference_t<decltype(fn)>>(dlsym(h, sym));
        };
        get(n.create, "nvrtcCreateProgram");
        get(n.compile, "nvrtcCompileProgram");
        get(n.log_size, "nvrtcGetProgramLogSize");
        get(n.log, "nvrtcGetProgramLog");
        get(n.cubin_size, "nvrtcGetCUBINSize");
        get(n.cubin, "nvrtcGetCUBIN");
        get(n.destroy, "nvrtcDestroyProgram");
        get(n.error_string, "nvrtcGetErrorString");
        n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy &&
               n.error_string;
    });
    return n;
}
}  // namespace

void rtc_release(RtcKernel &k)
{
    if (k.lib) cudaLibraryUnload(k.lib);
    k.lib = nullptr;
    k.kernel = nullptr;
}

bool rtc_compile(const std::string &user_source, int d, bool fp64, bool lp1, bool cv, bool user_dynamics,
                 RtcKernel &out, std::string &log)
{
    rtc_release(out);
    const Nvrtc &rt = nvrtc();
    if (!rt.ok) {
        log = "NVRTC (libnvrtc) not found";
        return false;
    }
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
        log = "no CUDA device";
        return false;
    }
    const char *real = fp64 ? "double" : "float";
    const std::string src = std::string("typedef ") + real + " srmc_real;\n"
                            "#define SRMC_USER static __device__ __forceinline__\n"
                            "#line 1 \"user_model\"\n" + user_source + "\n"
                            "#include \"srmc_step.cu\"\n";
    const char *headers[] = {srmc_rtc_device_cuh, srmc_rtc_step_cu};
    const char *names[] = {"srmc_device.cuh", "srmc_step.cu"};
    nvrtcProgram prog = nullptr;
    if (rt.create(&prog, src.c_str(), "srmc_user_model.cu", 2, headers, names) != NVRTC_SUCCESS) {
        log = "nvrtcCreateProgram failed";
        return false;
    }
    const char *inc = getenv("SRMC_CUDA_INCLUDE");
    const std::string o_arch = "--gpu-architecture=sm_" + std::to_string(major * 10 + minor);
    const std::string o_inc = std::string("-I") + (inc ? inc : SRMC_CUDA_INCLUDE);
    const std::string o_d = "-DSRMC_STEP_D=" + std::to_string(d);
    const std::string o_r = std::string("-DSRMC_RTC_REAL=") + real;
    const std::string o_lp1 = std::string("-DSRMC_RTC_LP1=") + (lp1 ? "1" : "0");
    const std::string o_cv = std::string("-DSRMC_RTC_CV=") + (cv ? "1" : "0");
    const char *opts[] = {o_arch.c_str(), "-std=c++17", "-default-device", o_inc.c_str(), o_d.c_str(),
                          "-DSRMC_USER_MODEL", o_r.c_str(), o_lp1.c_str(), o_cv.c_str(),
                          user_dynamics ? "-DSRMC_USER_DYNAMICS" : "-DSRMC_USER_DYNAMICS_OFF"};
    const nvrtcResult r = rt.compile(prog, (int)(sizeof(opts) / sizeof(opts[0])), opts);
    size_t n = 0;
    rt.log_size(prog, &n);
    std::vector<char> text(n + 1, 0);
    if (n) rt.log(prog, text.data());
    log.assign(text.data());
    if (r != NVRTC_SUCCESS) {
        rt.destroy(&prog);
        if (log.empty()) log = rt.error_string(r);
        return false;
    }
    size_t bytes = 0;
    rt.cubin_size(prog, &bytes);
    std::vector<char> cubin(bytes);
    rt.cubin(prog, cubin.data());
    rt.destroy(&prog);
    cudaError_t e = cudaLibraryLoadData(&out.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&out.kernel, out.lib, "srmc_user_step");
    if (e != cudaSuccess) {
        log = std::string("loading the compiled kernel: ") + cudaGetErrorString(e);
        rtc_release(out);
        return false;
    }
    return true;
}

cudaError_t rtc_launch(const RtcKernel &k, const Params &P, int i, int grid, int threads, cudaStream_t st)
{
    Params p = P;
    int step = i;
    void *args[] = {&p, &step};
    return cudaLaunchKernel((const void *)k.kernel, dim3((unsigned)grid), dim3((unsigned)threads), args, 0, st);
}

}  // namespace srmc
