// Plain step kernel (one simulation per launch), its launchers, and the
// device test hooks.
#include <algorithm>

#include "steps_step.cuh"

namespace steps {

namespace {

template <int BLOCK, int RM, bool Z>
__global__ void __launch_bounds__(BLOCK, 2048 / BLOCK / 2)
    step_kernel(const __grid_constant__ ModelDev m, const __grid_constant__ StepArgs a) {
    step_tile<BLOCK, RM, RtModel<Z>>(m, a, (int64_t)blockIdx.x);
}

// The flow form of the generic kernel (256-thread blocks only): one block per
// item (window, tile) of a run's full windows.
template <int RM, bool Z>
__global__ void __launch_bounds__(256, 4)
    flow_kernel(const __grid_constant__ ModelDev m, const __grid_constant__ StepArgs a,
                const __grid_constant__ FlowArgs f) {
    flow_tiles<256, RM, RtModel<Z>>(m, a, f);
}

__global__ void philox_test_kernel(uint32_t k0, uint32_t k1, const uint4 *ctr, int64_t n, uint4 *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = ctr[i];
    out[i] = philox4x32_10(k0, k1, c.x, c.y, c.z, c.w);
}

__global__ void logf_test_kernel(const float *x, int64_t n, float *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = steps_logf(x[i]);
}

// The step kernel's bounded wait on its own: one thread arms an mbarrier for
// a 16-byte bulk copy. With `deliver` it issues the copy and the wait
// completes; without, nothing completes the phase and the wait gives up
// after `limit` cycles. No copy is left in flight when the block exits.
// status: 0 completed, 4 timed out (the step kernel's error bit).
__global__ void wait_test_kernel(const uint4 *src, int deliver, long long limit, uint32_t *status) {
    __shared__ __align__(16) uint4 buf;
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, 16u);
    if (deliver) bulk_g2s(&buf, src, 16u, &bar);
    *status = mbar_wait_bounded(&bar, 0, limit) ? 0u : 4u;
}

// The flow kernel's bounded dependency wait on its own: one warp waits for
// the tiles listed for tile 0 to reach window word 5. status: 0 completed,
// 8 timed out (the flow kernel's error bit).
__global__ void flow_wait_test_kernel(const int32_t *tnb_off, const int32_t *tnb, uint32_t *tile_done,
                                      long long limit, uint32_t *status) {
    FlowArgs f;
    f.tnb_off = tnb_off;
    f.tnb = tnb;
    f.tile_done = tile_done;
    f.fetch = nullptr;
    f.nwin = 1;
    f.ntiles = 1;
    const bool ok = flow_deps_wait(f, 0u, 5u, limit);
    if (threadIdx.x == 0) *status = ok ? 0u : 8u;
}

__global__ void add_u64_kernel(uint64_t *p, uint64_t v) { *p += v; }

template <int BLOCK, int RM, bool Z>
int launch_step_t(const ModelDev &m, const StepArgs &a, void *stream) {
    const int64_t grid = (a.T + BLOCK - 1) / BLOCK;
    const size_t smem = (2 * (size_t)m.S + 1) * BLOCK * sizeof(int32_t);
    static size_t static_smem = [] {
        cudaFuncAttributes fa{};
        return cudaFuncGetAttributes(&fa, step_kernel<BLOCK, RM, Z>) == cudaSuccess ? fa.sharedSizeBytes
                                                                                         : (size_t)0;
    }();
    if (smem + static_smem > 48 * 1024) {  // opt in to more than the default 48 KB per block
        cudaError_t e = cudaFuncSetAttribute(step_kernel<BLOCK, RM, Z>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            set_error(std::string("step kernel shared memory: ") + cudaGetErrorString(e));
            return STEPS_ERR_CUDA;
        }
    }
    StepArgs b = a;
    if (b.prefetch) {
        // about half a resident wave ahead
        b.prefetch = prefetch_distance(reinterpret_cast<const void *>(step_kernel<BLOCK, RM, Z>), BLOCK, smem);
    }
    // programmatic dependent launch: overlaps this window's set-up with the
    // previous window's tail (the kernel waits for it before reading counts)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(BLOCK);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = (cudaStream_t)stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, step_kernel<BLOCK, RM, Z>, m, b);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("step kernel launch: ") + cudaGetErrorString(e));
        return STEPS_ERR_CUDA;
    }
    return STEPS_OK;
}

// reaction loops are unrolled to the smallest bucket of 8, 16, 24 or 32 that holds the model
// (and to models with or without order-0 reactions)
template <int BLOCK, bool Z>
int launch_step_z(const ModelDev &m, const StepArgs &a, void *stream) {
    if (m.R <= 8) return launch_step_t<BLOCK, 8, Z>(m, a, stream);
    if (m.R <= 16) return launch_step_t<BLOCK, 16, Z>(m, a, stream);
    if (m.R <= 24) return launch_step_t<BLOCK, 24, Z>(m, a, stream);
    return launch_step_t<BLOCK, 32, Z>(m, a, stream);
}

template <int BLOCK>
int launch_step_b(const ModelDev &m, const StepArgs &a, void *stream) {
    return m.order0 ? launch_step_z<BLOCK, true>(m, a, stream) : launch_step_z<BLOCK, false>(m, a, stream);
}

template <int RM, bool Z>
int launch_flow_t(const ModelDev &m, const StepArgs &a, const FlowArgs &f, void *stream) {
    const size_t smem = (2 * (size_t)m.S + 1) * 256 * sizeof(int32_t);
    static size_t static_smem = [] {
        cudaFuncAttributes fa{};
        return cudaFuncGetAttributes(&fa, flow_kernel<RM, Z>) == cudaSuccess ? fa.sharedSizeBytes : (size_t)0;
    }();
    if (smem + static_smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(flow_kernel<RM, Z>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            set_error(std::string("flow kernel shared memory: ") + cudaGetErrorString(e));
            return STEPS_ERR_CUDA;
        }
    }
    StepArgs b = a;
    b.window_base = nullptr;
    // the item taken about half a resident wave later: its tables into L2
    if (b.prefetch) b.prefetch = prefetch_distance(reinterpret_cast<const void *>(flow_kernel<RM, Z>), 256, smem);
    const unsigned grid = f.nwin * f.ntiles;  // one item per block
    flow_kernel<RM, Z><<<grid, 256, smem, (cudaStream_t)stream>>>(m, b, f);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("flow kernel launch: ") + cudaGetErrorString(e));
        return STEPS_ERR_CUDA;
    }
    return STEPS_OK;
}

template <bool Z>
int launch_flow_z(const ModelDev &m, const StepArgs &a, const FlowArgs &f, void *stream) {
    if (m.R <= 8) return launch_flow_t<8, Z>(m, a, f, stream);
    if (m.R <= 16) return launch_flow_t<16, Z>(m, a, f, stream);
    if (m.R <= 24) return launch_flow_t<24, Z>(m, a, f, stream);
    return launch_flow_t<32, Z>(m, a, f, stream);
}

}  // namespace

int prefetch_distance(const void *kernel, int block, size_t smem) {
    struct Entry {
        const void *k;
        size_t smem;
        int n;
    };
    static thread_local Entry cache[8] = {};
    for (const Entry &e : cache)
        if (e.k == kernel && e.smem == smem) return e.n;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
    // half a resident wave (SMs x resident blocks per SM / 2): on the 1.03M-tet
    // dendrite, 0.125 to 3 waves were timed and half a wave was fastest
    const int n = std::max(1, (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1) / 2);
    static thread_local int next = 0;
    cache[next] = Entry{kernel, smem, n};
    next = (next + 1) & 7;
    return n;
}

int launch_step(const ModelDev &m, const StepArgs &a, int block, void *stream) {
    if (a.T <= 0) return STEPS_OK;
    switch (block) {
    case 64: return launch_step_b<64>(m, a, stream);
    case 128: return launch_step_b<128>(m, a, stream);
    case 512: return launch_step_b<512>(m, a, stream);
    default: return launch_step_b<256>(m, a, stream);
    }
}

int launch_philox_test(uint64_t seed, const uint32_t *d_ctr, int64_t n, uint32_t *d_out, void *stream) {
    if (n <= 0) return STEPS_OK;
    philox_test_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        (uint32_t)seed, (uint32_t)(seed >> 32), (const uint4 *)d_ctr, n, (uint4 *)d_out);
    return cudaGetLastError() == cudaSuccess ? STEPS_OK : STEPS_ERR_CUDA;
}

int launch_flow(const ModelDev &m, const StepArgs &a, const FlowArgs &f, int block, void *stream) {
    if (a.T <= 0 || f.nwin == 0) return STEPS_OK;
    if (block != 256) {
        set_error("flow launches of the generic step kernel need 256-thread blocks");
        return STEPS_ERR_ARG;
    }
    return m.order0 ? launch_flow_z<true>(m, a, f, stream) : launch_flow_z<false>(m, a, f, stream);
}

int launch_wait_test(const void *d_src, int deliver, long long limit, uint32_t *d_status, void *stream) {
    wait_test_kernel<<<1, 32, 0, (cudaStream_t)stream>>>((const uint4 *)d_src, deliver, limit, d_status);
    return cudaGetLastError() == cudaSuccess ? STEPS_OK : STEPS_ERR_CUDA;
}

int launch_flow_wait_test(const int32_t *d_off, const int32_t *d_nb, uint32_t *d_done, long long limit,
                          uint32_t *d_status) {
    flow_wait_test_kernel<<<1, 32>>>(d_off, d_nb, d_done, limit, d_status);
    return cudaGetLastError() == cudaSuccess ? STEPS_OK : STEPS_ERR_CUDA;
}

int launch_logf_test(const float *d_x, int64_t n, float *d_out, void *stream) {
    if (n <= 0) return STEPS_OK;
    logf_test_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(d_x, n, d_out);
    return cudaGetLastError() == cudaSuccess ? STEPS_OK : STEPS_ERR_CUDA;
}

int launch_add_u64(uint64_t *p, uint64_t v, void *stream) {
    add_u64_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(p, v);
    return cudaGetLastError() == cudaSuccess ? STEPS_OK : STEPS_ERR_CUDA;
}

}  // namespace steps
