// Batched step kernel: one launch runs a window for many simulations (members
// of different sizes, seeds, time windows and models). Each block reads its
// member's model and arguments from a device table into shared memory, then
// runs the same tile body as the plain kernel; a small kernel advances every
// member's window counter and buffer parity on the device, so that the whole
// step loop can be replayed from a CUDA graph.
#include "steps_step.cuh"

namespace steps {

namespace {

template <int BLOCK, int RM, bool Z>
__global__ void __launch_bounds__(BLOCK, 2048 / BLOCK / 2)
    step_kernel_batch(const BlockWork *__restrict__ work, const RepEntry *__restrict__ reps, int32_t prefetch) {
    batch_tile<BLOCK, RM, RtModel<Z>>(work, reps, prefetch);
}

template <int BLOCK, int RM, bool Z>
int launch_batch_t(const BlockWork *work, int64_t nblocks, RepEntry *reps, int max_S, void *stream) {
    const size_t smem = (2 * (size_t)max_S + 1) * BLOCK * sizeof(int32_t);
    static size_t static_smem = [] {
        cudaFuncAttributes fa{};
        return cudaFuncGetAttributes(&fa, step_kernel_batch<BLOCK, RM, Z>) == cudaSuccess ? fa.sharedSizeBytes
                                                                                        : (size_t)0;
    }();
    if (smem + static_smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(step_kernel_batch<BLOCK, RM, Z>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            set_error(std::string("batched step kernel shared memory: ") + cudaGetErrorString(e));
            return STEPS_ERR_CUDA;
        }
    }
    // L2 prefetch about half a resident wave ahead (the work list runs through a
    // member's tiles in order)
    const int32_t prefetch = prefetch_distance(reinterpret_cast<const void *>(step_kernel_batch<BLOCK, RM, Z>), BLOCK, smem);
    step_kernel_batch<BLOCK, RM, Z><<<(unsigned)nblocks, BLOCK, smem, (cudaStream_t)stream>>>(work, reps, prefetch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("batched step kernel launch: ") + cudaGetErrorString(e));
        return STEPS_ERR_CUDA;
    }
    return STEPS_OK;
}

template <int BLOCK, bool Z>
int launch_batch_z(const BlockWork *work, int64_t nblocks, RepEntry *reps, int max_S, int max_R, void *stream) {
    if (max_R <= 8) return launch_batch_t<BLOCK, 8, Z>(work, nblocks, reps, max_S, stream);
    if (max_R <= 16) return launch_batch_t<BLOCK, 16, Z>(work, nblocks, reps, max_S, stream);
    if (max_R <= 24) return launch_batch_t<BLOCK, 24, Z>(work, nblocks, reps, max_S, stream);
    return launch_batch_t<BLOCK, 32, Z>(work, nblocks, reps, max_S, stream);
}

// Z: some member's model has order-0 reactions
template <int BLOCK>
int launch_batch_b(const BlockWork *work, int64_t nblocks, RepEntry *reps, int max_S, int max_R, bool any_order0,
                   void *stream) {
    return any_order0 ? launch_batch_z<BLOCK, true>(work, nblocks, reps, max_S, max_R, stream)
                      : launch_batch_z<BLOCK, false>(work, nblocks, reps, max_S, max_R, stream);
}

__global__ void advance_kernel(RepEntry *reps, int32_t n) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    RepEntry &e = reps[j];
    if (e.args.window < e.window_end) {
        e.args.window += 1;
        e.parity ^= 1u;
    }
}

}  // namespace

int launch_step_batch(const BlockWork *work, int64_t nblocks, RepEntry *reps, int max_S, int max_R,
                      bool any_order0, int block, void *stream) {
    if (nblocks <= 0) return STEPS_OK;
    switch (block) {
    case 64: return launch_batch_b<64>(work, nblocks, reps, max_S, max_R, any_order0, stream);
    case 128: return launch_batch_b<128>(work, nblocks, reps, max_S, max_R, any_order0, stream);
    case 512: return launch_batch_b<512>(work, nblocks, reps, max_S, max_R, any_order0, stream);
    default: return launch_batch_b<256>(work, nblocks, reps, max_S, max_R, any_order0, stream);
    }
}

int launch_advance(RepEntry *reps, int32_t n, void *stream) {
    if (n <= 0) return STEPS_OK;
    advance_kernel<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(reps, n);
    return cudaGetLastError() == cudaSuccess ? STEPS_OK : STEPS_ERR_CUDA;
}

}  // namespace steps
