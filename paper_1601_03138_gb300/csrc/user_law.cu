// user_law.cu -- user interaction laws compiled from source at run time.
//
// The paper's user writes the interaction law as functors handed to the
// force calculation (Sect. 2.2).  fdps_user_law_compile takes such a law as
// CUDA source text (a `struct Force` and a `struct Law`, as for the header
// template fdps_user_force.cuh), compiles it with NVRTC for sm_103a together
// with the template's device part, and loads the result; fdps_user_law_run
// launches it over the lists of a tree.  The two public headers are built
// into the library as text, so the compiler sees exactly the declarations
// the library was built with.
#include <nvrtc.h>

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fdps_internal.cuh"
#include "fdps_embedded_headers.inc"  // kHeaderGpu, kHeaderUserForce (generated)

struct fdps_user_law {
    fdps_ctx* ctx = nullptr;
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    int64_t force_size = 0;
    int per_sm = 0;
};

namespace fdps {
namespace {

// fixed-width integer names for the compiler, which has no system headers
const char kStdint[] =
    "#pragma once\n"
    "typedef signed char int8_t;\ntypedef short int16_t;\ntypedef int int32_t;\n"
    "typedef long long int64_t;\ntypedef unsigned char uint8_t;\n"
    "typedef unsigned short uint16_t;\ntypedef unsigned int uint32_t;\n"
    "typedef unsigned long long uint64_t;\n";

std::string program_text(const char* user) {
    std::string s;
    s += "#include \"fdps_user_force.cuh\"\n";
    s += "using fdps_user::Epi;\nusing fdps_user::Epj;\nusing fdps_user::Spj;\n";
    s += "#line 1 \"user_law\"\n";
    s += user;
    s += "\n#line 1 \"fdps_user_entry\"\n";
    s += "extern \"C\" __global__ void __launch_bounds__(fdps_user::detail::kWarps * 32)\n"
         "fdps_user_entry(fdps_tree_view v, Force* out) {\n"
         "    fdps_user::detail::calc_force_body<Force>(v, Law{}, Law{}, out);\n}\n";
    s += "extern \"C\" __device__ const long long fdps_user_force_size = (long long)sizeof(Force);\n";
    return s;
}

void copy_log(const std::string& log, char* out, int64_t cap) {
    if (!out || cap <= 0) return;
    const size_t k = log.size() < (size_t)(cap - 1) ? log.size() : (size_t)(cap - 1);
    memcpy(out, log.data(), k);
    out[k] = '\0';
}

}  // namespace
}  // namespace fdps

using namespace fdps;

extern "C" {

int fdps_user_law_compile(fdps_ctx* ctx, const char* source, fdps_user_law** out, char* log,
                          int64_t log_cap) {
    if (!ctx || !source || !out) return FDPS_EINVAL;
    *out = nullptr;
    copy_log("", log, log_cap);
    if (!*source) return set_error(ctx, FDPS_EINVAL, "empty user law source");
    cudaSetDevice(ctx->device);
    const std::string text = program_text(source);
    const char* hdrs[3] = {kHeaderUserForce, kHeaderGpu, kStdint};
    const char* names[3] = {"fdps_user_force.cuh", "fdps_gpu.h", "stdint.h"};
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, text.c_str(), "user_law.cu", 3, hdrs, names) != NVRTC_SUCCESS)
        return set_error(ctx, FDPS_ECUDA, "NVRTC could not create the program");
    const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device"};
    const nvrtcResult cr = nvrtcCompileProgram(prog, 3, opts);
    size_t ls = 0;
    nvrtcGetProgramLogSize(prog, &ls);
    std::string lg(ls, '\0');
    if (ls) nvrtcGetProgramLog(prog, &lg[0]);
    while (!lg.empty() && lg.back() == '\0') lg.pop_back();
    copy_log(lg, log, log_cap);
    if (cr != NVRTC_SUCCESS) {
        nvrtcDestroyProgram(&prog);
        return set_error(ctx, FDPS_EINVAL, "user law does not compile: %s", nvrtcGetErrorString(cr));
    }
    size_t cs = 0;
    std::vector<char> cubin;
    if (nvrtcGetCUBINSize(prog, &cs) == NVRTC_SUCCESS && cs) {
        cubin.resize(cs);
        if (nvrtcGetCUBIN(prog, cubin.data()) != NVRTC_SUCCESS) cubin.clear();
    }
    nvrtcDestroyProgram(&prog);
    if (cubin.empty()) return set_error(ctx, FDPS_ECUDA, "NVRTC returned no cubin");
    fdps_user_law* law = new (std::nothrow) fdps_user_law();
    if (!law) return FDPS_ENOMEM;
    law->ctx = ctx;
    if (cudaLibraryLoadData(&law->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess ||
        cudaLibraryGetKernel(&law->kern, law->lib, "fdps_user_entry") != cudaSuccess) {
        cudaGetLastError();
        if (law->lib) cudaLibraryUnload(law->lib);
        delete law;
        return set_error(ctx, FDPS_ECUDA, "loading the compiled user law failed");
    }
    void* dsize = nullptr;
    size_t bytes = 0;
    long long fs = 0;
    if (cudaLibraryGetGlobal(&dsize, &bytes, law->lib, "fdps_user_force_size") != cudaSuccess ||
        bytes != sizeof(fs) || cudaMemcpy(&fs, dsize, sizeof(fs), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&law->per_sm, (const void*)law->kern, 128, 0) !=
            cudaSuccess) {
        cudaGetLastError();
        cudaLibraryUnload(law->lib);
        delete law;
        return set_error(ctx, FDPS_ECUDA, "querying the compiled user law failed");
    }
    law->force_size = fs;
    if (law->per_sm < 1) law->per_sm = 1;
    *out = law;
    return FDPS_OK;
}

int64_t fdps_user_law_force_size(const fdps_user_law* law) { return law ? law->force_size : -1; }

int fdps_user_law_run(fdps_user_law* law, const fdps_tree* tree, const fdps_psys* ps, void* out) {
    if (!law || !tree || !ps || !out) return FDPS_EINVAL;
    fdps_ctx* ctx = law->ctx;
    cudaSetDevice(ctx->device);
    fdps_tree_view v;
    const int rc = fdps_tree_get_view(tree, ps, &v);
    if (rc) return rc;
    if (v.n_groups <= 0) return FDPS_OK;
    const int64_t need = (v.n_groups + 3) / 4;
    const int64_t cap = (int64_t)ctx->sm_count * law->per_sm;
    const unsigned int blocks = (unsigned int)(need < cap ? need : cap);
    void* args[2] = {&v, &out};
    if (cudaLaunchKernel((const void*)law->kern, dim3(blocks), dim3(128), args, 0, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, FDPS_ECUDA, "user law launch failed");
    }
    ++ctx->launches;
    return FDPS_OK;
}

int fdps_user_law_destroy(fdps_user_law* law) {
    if (!law) return FDPS_EINVAL;
    cudaSetDevice(law->ctx->device);
    cudaLibraryUnload(law->lib);
    delete law;
    return FDPS_OK;
}

}  // extern "C"
