// Model-specialised step kernels, compiled at run time.
//
// The step body (steps_step.cuh) reads the model through a policy class. The
// generic kernels use RtModel, which looks reactants, flags and
// stoichiometry up in a per-tile table. Here, for one model, a policy is
// generated as C++ source: the species count, the diffusive set, each
// reaction's reactant rows, propensity form and changes become constants.
// The same step body, specialised with it, is then compiled for the device
// by NVRTC. The rate constants stay kernel parameters, so
// steps_set_reac_rate needs no recompilation. The arithmetic is the generic
// kernel's, operation for operation, so both give the same bits.
//
// NVRTC is opened with dlopen: without it the library still loads and the
// generic kernels run. The code is loaded with the runtime's library API
// (cudaLibraryLoadData), and kernels are cached per generated source.
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "steps_internal.h"

namespace steps {

extern const char *const kSrcDeviceH;  // steps_device.h, embedded at build time
extern const char *const kSrcStepCuh;  // steps_step.cuh, embedded at build time

namespace {

// The few NVRTC entry points used (C ABI of libnvrtc).
typedef int nvrtc_result;
typedef struct nvrtc_program_st *nvrtc_program;
struct Nvrtc {
    void *handle = nullptr;
    nvrtc_result (*create)(nvrtc_program *, const char *, const char *, int, const char *const *,
                           const char *const *) = nullptr;
    nvrtc_result (*compile)(nvrtc_program, int, const char *const *) = nullptr;
    nvrtc_result (*log_size)(nvrtc_program, size_t *) = nullptr;
    nvrtc_result (*log)(nvrtc_program, char *) = nullptr;
    nvrtc_result (*cubin_size)(nvrtc_program, size_t *) = nullptr;
    nvrtc_result (*cubin)(nvrtc_program, char *) = nullptr;
    nvrtc_result (*destroy)(nvrtc_program *) = nullptr;
    std::string why;
};

Nvrtc &nvrtc() {
    static Nvrtc n = [] {
        Nvrtc x;
        const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "libnvrtc.so.12"};
        for (const char *nm : names)
            if ((x.handle = dlopen(nm, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
        if (!x.handle) {
            x.why = "libnvrtc not found";
            return x;
        }
        x.create = reinterpret_cast<decltype(x.create)>(dlsym(x.handle, "nvrtcCreateProgram"));
        x.compile = reinterpret_cast<decltype(x.compile)>(dlsym(x.handle, "nvrtcCompileProgram"));
        x.log_size = reinterpret_cast<decltype(x.log_size)>(dlsym(x.handle, "nvrtcGetProgramLogSize"));
        x.log = reinterpret_cast<decltype(x.log)>(dlsym(x.handle, "nvrtcGetProgramLog"));
        x.cubin_size = reinterpret_cast<decltype(x.cubin_size)>(dlsym(x.handle, "nvrtcGetCUBINSize"));
        x.cubin = reinterpret_cast<decltype(x.cubin)>(dlsym(x.handle, "nvrtcGetCUBIN"));
        x.destroy = reinterpret_cast<decltype(x.destroy)>(dlsym(x.handle, "nvrtcDestroyProgram"));
        if (!x.create || !x.compile || !x.log_size || !x.log || !x.cubin_size || !x.cubin || !x.destroy) {
            x.why = "libnvrtc lacks an entry point";
            x.handle = nullptr;
        }
        return x;
    }();
    return n;
}

}  // namespace

// Models with many species keep the trial counts in a global buffer: their
// tile's shared memory then fits more resident blocks per SM.
bool spec_global_trial(const HostModel &hm) { return hm.dev.S >= 16; }

namespace {

std::string hex_u32(uint32_t v) {
    std::ostringstream o;
    o << "0x" << std::hex << v << "u";
    return o.str();
}

// The generated policy: the same functions as RtModel with the model's
// structure as constants. Propensity forms (all in float, as RtModel):
//   order 0: k / inv_nav            order 1: k x
//   order 2: ((k inv_nav) x) y      dimer:   ((k inv_nav) x) (x - 1)
// (RtModel's extra factors of 1 are exact and left out.)
std::string policy_source(const HostModel &hm, int block) {
    const ModelDev &m = hm.dev;
    std::ostringstream o;
    o << "namespace steps {\nnamespace {\nstruct SpecModel {\n";
    o << "    static constexpr bool kGlobalTrial = " << (spec_global_trial(hm) ? "true" : "false") << ";\n";
    o << "    static constexpr bool kExpLeave = " << (hm.leave_exp ? "true" : "false") << ";\n";
    o << "    __device__ static int S(const ModelDev &) { return " << m.S << "; }\n";
    o << "    __device__ static int R(const ModelDev &) { return " << m.R << "; }\n";
    o << "    __device__ static uint32_t diffusive(const ModelDev &) { return " << hex_u32(m.diffusive) << "; }\n";
    o << "    __device__ static uint32_t need(const RxnTab &tb, int r) { return tb.need[r]; }\n";
    o << "    template <int BLOCK>\n    __device__ static void build(const ModelDev &m, RxnTab &tb) {\n";
    o << "        build_rxn_tab<BLOCK>(m, tb);\n    }\n";
    o << "    __device__ static float prop(const RxnTab &, const ModelDev &m, int r, const int32_t *cnt, float inv_nav) {\n";
    o << "        switch (r) {\n";
    for (int r = 0; r < m.R; ++r) {
        const ReacDesc &d = m.reac[r];
        const std::string k = "m.reac[" + std::to_string(r) + "].k";
        const std::string x = "__int2float_rn(cnt[" + std::to_string(d.ia * block) + "])";
        o << "        case " << r << ": return ";
        switch (d.type) {
        case kOrder0: o << "__fdiv_rn(" << k << ", inv_nav)"; break;
        case kOrder1: o << "__fmul_rn(" << k << ", " << x << ")"; break;
        case kOrder2:
            o << "__fmul_rn(__fmul_rn(__fmul_rn(" << k << ", inv_nav), " << x << "), __int2float_rn(cnt["
              << d.ib * block << "]))";
            break;
        default:
            o << "__fmul_rn(__fmul_rn(__fmul_rn(" << k << ", inv_nav), " << x << "), __int2float_rn(cnt["
              << d.ib * block << "] - 1))";
            break;
        }
        o << ";\n";
    }
    o << "        default: return 0.0f;\n        }\n    }\n";
    // the stoichiometry from the tile's table: a switch over reactions inside the
    // SSA loop would inline every reaction's occupancy update there
    o << "    template <class F>\n    __device__ static void for_changes(const RxnTab &tb, int r, F f) {\n";
    o << "        RtModel<false>::for_changes(tb, r, f);\n    }\n";
    o << "};\n}  // namespace\n}  // namespace steps\n";

    return o.str();
}

int reaction_bucket(int R) { return R <= 8 ? 8 : R <= 16 ? 16 : R <= 24 ? 24 : 32; }

std::string program_source(const HostModel &hm, int block) {
    std::ostringstream o;
    // models with many species keep trial counts in global memory; at 256
    // threads their tiles then fit five resident blocks per SM with a 32-entry
    // block map and 48 registers per thread
    const bool five = spec_global_trial(hm) && block == 256;
    if (five) o << "#define STEPS_MAP_CAP 32\n";
    o << "#include \"steps_step.cuh\"\n" << policy_source(hm, block);
    o << "extern \"C\" __global__ void __launch_bounds__(" << block << ", " << (five ? 5 : 2048 / block / 2) << ")\n"
      << "steps_spec_step(const __grid_constant__ steps::ModelDev m, const __grid_constant__ steps::StepArgs a) {\n"
      << "    steps::step_tile<" << block << ", " << reaction_bucket(hm.dev.R) << ", steps::SpecModel>(m, a, "
      << "(int64_t)blockIdx.x);\n}\n";
    o << "extern \"C\" __global__ void __launch_bounds__(" << block << ", " << (five ? 5 : 2048 / block / 2) << ")\n"
      << "steps_spec_flow(const __grid_constant__ steps::ModelDev m, const __grid_constant__ steps::StepArgs a, "
      << "const __grid_constant__ steps::FlowArgs f) {\n"
      << "    steps::flow_tiles<" << block << ", " << reaction_bucket(hm.dev.R) << ", steps::SpecModel>(m, a, f);\n}\n";
    o << "extern \"C\" __global__ void __launch_bounds__(" << block << ", " << 2048 / block / 2 << ")\n"
      << "steps_spec_batch(const steps::BlockWork *__restrict__ work, const steps::RepEntry *__restrict__ reps, "
      << "int32_t prefetch) {\n"
      << "    steps::batch_tile<" << block << ", " << reaction_bucket(hm.dev.R) << ", steps::SpecModel>(work, reps, "
      << "prefetch);\n}\n";
    o << "extern \"C\" __global__ void __launch_bounds__(" << block << ", " << 2048 / block / 2 << ")\n"
      << "steps_spec_batch_flow(const steps::BlockWork *__restrict__ work, const steps::RepEntry *__restrict__ reps, "
      << "const __grid_constant__ steps::FlowArgs f, uint32_t work0, int32_t prefetch) {\n"
      << "    steps::batch_flow_tile<" << block << ", " << reaction_bucket(hm.dev.R) << ", steps::SpecModel>(work, reps, "
      << "f, work0, prefetch);\n}\n";
    return o.str();
}

struct Compiled {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;        // plain step kernel
    cudaKernel_t kern_batch = nullptr;  // batched step kernel
    cudaKernel_t kern_flow = nullptr;   // flow kernel of a simulation's full windows
    cudaKernel_t kern_batch_flow = nullptr;  // flow kernel of a group of batch members
    size_t smem_set = 0;                // dynamic shared memory the plain kernel was opted in to
    size_t smem_set_flow = 0;           // the flow kernel
    size_t smem_set_batch_flow = 0;     // the batched flow kernel
    size_t smem_set_batch = 0;          // and the batched one
    bool global_trial = false;          // trial counts in StepArgs::trial, not shared memory
};

std::mutex g_mu;
std::map<std::string, std::shared_ptr<Compiled>> g_cache;

}  // namespace

std::string spec_program_source(const HostModel &hm, int block) { return program_source(hm, block); }

namespace {

// Compiles (once per generated source) and loads the plain and batched kernels.
Compiled *compiled(const HostModel &hm, int block, std::string *why) {
    Nvrtc &nv = nvrtc();
    if (!nv.handle) {
        if (why) *why = nv.why;
        return nullptr;
    }
    const std::string src = program_source(hm, block);
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_cache.find(src);
    if (it != g_cache.end()) {
        if (!it->second && why) *why = "an earlier build of this kernel failed";
        return it->second.get();
    }
    nvrtc_program prog = nullptr;
    const char *hdr_src[2] = {kSrcDeviceH, kSrcStepCuh};
    const char *hdr_name[2] = {"steps_device.h", "steps_step.cuh"};
    if (nv.create(&prog, src.c_str(), "steps_spec.cu", 2, hdr_src, hdr_name) != 0) {
        if (why) *why = "nvrtcCreateProgram failed";
        g_cache[src] = nullptr;
        return nullptr;
    }
    // the generic kernels' flags: no contraction, C++17, this GPU only
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-fmad=false", "-lineinfo", "--device-int128"};
    const int rc = nv.compile(prog, 5, opts);
    std::vector<char> cubin;
    if (rc == 0) {
        size_t n = 0;
        if (nv.cubin_size(prog, &n) == 0 && n > 0) {
            cubin.resize(n);
            if (nv.cubin(prog, cubin.data()) != 0) cubin.clear();
        }
    } else if (why) {
        size_t n = 0;
        nv.log_size(prog, &n);
        std::string lg(n, '\0');
        if (n) nv.log(prog, &lg[0]);
        *why = "NVRTC compile failed: " + lg.substr(0, 2000);
    }
    nv.destroy(&prog);
    if (cubin.empty()) {
        g_cache[src] = nullptr;
        return nullptr;
    }
    auto c = std::make_shared<Compiled>();
    c->global_trial = spec_global_trial(hm);
    if (cudaLibraryLoadData(&c->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess ||
        cudaLibraryGetKernel(&c->kern, c->lib, "steps_spec_step") != cudaSuccess ||
        cudaLibraryGetKernel(&c->kern_batch, c->lib, "steps_spec_batch") != cudaSuccess ||
        cudaLibraryGetKernel(&c->kern_flow, c->lib, "steps_spec_flow") != cudaSuccess ||
        cudaLibraryGetKernel(&c->kern_batch_flow, c->lib, "steps_spec_batch_flow") != cudaSuccess) {
        cudaGetLastError();
        if (why) *why = "loading the compiled kernel failed";
        g_cache[src] = nullptr;
        return nullptr;
    }
    g_cache[src] = c;
    return c.get();
}

// Opts a kernel in to `smem` bytes of dynamic shared memory (once per size).
bool opt_in(const void *fn, size_t smem, size_t *done) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (*done >= smem) return true;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        set_error("specialised step kernel shared memory: " + std::string(cudaGetErrorString(cudaGetLastError())));
        return false;
    }
    *done = smem;
    return true;
}

}  // namespace

void *spec_kernel(const HostModel &hm, int block, std::string *why) {
    Compiled *c = compiled(hm, block, why);
    return c ? (void *)c : nullptr;
}

int launch_spec(void *spec, const ModelDev &m, const StepArgs &a, int block, void *stream) {
    if (a.T <= 0) return STEPS_OK;
    Compiled *c = static_cast<Compiled *>(spec);
    const void *fn = (const void *)c->kern;
    const size_t smem = ((size_t)m.S + 1 + (c->global_trial ? 0 : (size_t)m.S)) * (size_t)block * sizeof(int32_t);
    if (!opt_in(fn, smem, &c->smem_set)) return STEPS_ERR_CUDA;
    StepArgs b = a;
    if (b.prefetch) b.prefetch = prefetch_distance(fn, block, smem);
    ModelDev mm = m;
    void *args[2] = {(void *)&mm, (void *)&b};
    const unsigned grid = (unsigned)((a.T + block - 1) / block);
    // programmatic dependent launch, as the generic step kernel
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = (cudaStream_t)stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelExC(&cfg, fn, args);
    if (e != cudaSuccess) {
        set_error(std::string("specialised step kernel launch: ") + cudaGetErrorString(e));
        return STEPS_ERR_CUDA;
    }
    return STEPS_OK;
}

int launch_spec_flow(void *spec, const ModelDev &m, const StepArgs &a, const FlowArgs &f, int block, void *stream) {
    if (a.T <= 0 || f.nwin == 0) return STEPS_OK;
    Compiled *c = static_cast<Compiled *>(spec);
    const void *fn = (const void *)c->kern_flow;
    const size_t smem = ((size_t)m.S + 1 + (c->global_trial ? 0 : (size_t)m.S)) * (size_t)block * sizeof(int32_t);
    if (!opt_in(fn, smem, &c->smem_set_flow)) return STEPS_ERR_CUDA;
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1) {
        set_error("flow kernel occupancy: " + std::string(cudaGetErrorString(cudaGetLastError())));
        return STEPS_ERR_CUDA;
    }
    StepArgs b = a;
    b.window_base = nullptr;
    // the item taken about half a resident wave later: its tables into L2
    if (b.prefetch) b.prefetch = std::max(1, per_sm * sms / 2);
    ModelDev mm = m;
    FlowArgs ff = f;
    void *args[3] = {(void *)&mm, (void *)&b, (void *)&ff};
    const unsigned grid = f.nwin * f.ntiles;  // one item per block
    cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3((unsigned)block), args, smem, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_error(std::string("flow step kernel launch: ") + cudaGetErrorString(e));
        return STEPS_ERR_CUDA;
    }
    return STEPS_OK;
}

int launch_spec_batch_flow(void *spec, const BlockWork *work, RepEntry *reps, const FlowArgs &f, uint32_t work0, int S,
                           int block, void *stream) {
    if (f.nwin == 0 || f.ntiles == 0) return STEPS_OK;
    Compiled *c = static_cast<Compiled *>(spec);
    const void *fn = (const void *)c->kern_batch_flow;
    const size_t smem = ((size_t)S + 1 + (c->global_trial ? 0 : (size_t)S)) * (size_t)block * sizeof(int32_t);
    if (!opt_in(fn, smem, &c->smem_set_batch_flow)) return STEPS_ERR_CUDA;
    int32_t prefetch = prefetch_distance(fn, block, smem);
    FlowArgs ff = f;
    void *args[5] = {(void *)&work, (void *)&reps, (void *)&ff, (void *)&work0, (void *)&prefetch};
    const unsigned grid = f.nwin * f.ntiles;  // one item per block
    cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3((unsigned)block), args, smem, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_error(std::string("batched flow step kernel launch: ") + cudaGetErrorString(e));
        return STEPS_ERR_CUDA;
    }
    return STEPS_OK;
}

int launch_spec_batch(void *spec, const BlockWork *work, int64_t nblocks, RepEntry *reps, int S, int block,
                      void *stream) {
    if (nblocks <= 0) return STEPS_OK;
    Compiled *c = static_cast<Compiled *>(spec);
    const void *fn = (const void *)c->kern_batch;
    const size_t smem = ((size_t)S + 1 + (c->global_trial ? 0 : (size_t)S)) * (size_t)block * sizeof(int32_t);
    if (!opt_in(fn, smem, &c->smem_set_batch)) return STEPS_ERR_CUDA;
    int32_t prefetch = prefetch_distance(fn, block, smem);
    void *args[3] = {(void *)&work, (void *)&reps, (void *)&prefetch};
    cudaError_t e = cudaLaunchKernel(fn, dim3((unsigned)nblocks), dim3((unsigned)block), args, smem, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_error(std::string("specialised batched step kernel launch: ") + cudaGetErrorString(e));
        return STEPS_ERR_CUDA;
    }
    return STEPS_OK;
}

}  // namespace steps
