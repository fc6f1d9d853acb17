// Instantiations of the fused step kernels with FP32 populations and arithmetic.
#include "launch.h"
#include "step_tma.cuh"

namespace lbfe {

namespace {
template <int S, int C, int E, bool NU, bool TMA>
void* kernel_ptr()
{
    if constexpr (TMA)
        return reinterpret_cast<void*>(&step_kernel_tma<float, kStepThreads, S, C, E, NU>);
    else
        return reinterpret_cast<void*>(&step_kernel<float, kStepThreads, S, C, E, NU>);
}

template <bool TMA>
void* pick(int scheme, int coll, int eos, bool nu)
{
#define LBFE_PICK(S, C, E)                                                                  \
    if (scheme == S && coll == C && eos == E)                                               \
        return nu ? kernel_ptr<S, C, E, true, TMA>() : kernel_ptr<S, C, E, false, TMA>();
    LBFE_PICK(0, 0, 0) LBFE_PICK(0, 0, 1) LBFE_PICK(0, 1, 0) LBFE_PICK(0, 1, 1)
    LBFE_PICK(1, 0, 0) LBFE_PICK(1, 0, 1) LBFE_PICK(1, 1, 0) LBFE_PICK(1, 1, 1)
#undef LBFE_PICK
    return nullptr;
}

constexpr size_t kTmaSmem = tma_dynamic_smem<float, kStepThreads>();

void* resolve(int scheme, int coll, int eos, bool nu, bool tma)
{
    void* k = tma ? pick<true>(scheme, coll, eos, nu) : pick<false>(scheme, coll, eos, nu);
    if (k && tma) {
        // idempotent; needed once per kernel for more than 48 KB of dynamic smem
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaSmem);
    }
    return k;
}
}  // namespace

cudaError_t launch_step_f32(int scheme, int coll, int eos, bool nu, bool tma, int nblocks, cudaStream_t s,
                            const float* fin, float* fout, const DevCase<float>* cases, const Item* items,
                            int* status)
{
    void* k = resolve(scheme, coll, eos, nu, tma);
    if (!k) return cudaErrorInvalidValue;
    void* args[] = {(void*)&fin, (void*)&fout, (void*)&cases, (void*)&items, (void*)&status};
    // the TMA kernel adds one producer warp to the kStepThreads compute threads
    return cudaLaunchKernel(k, dim3(nblocks), dim3(tma ? kStepThreads + 32 : kStepThreads), args,
                            tma ? kTmaSmem : 0, s);
}

int occupancy_step_f32(int scheme, int coll, int eos, bool nu, bool tma)
{
    void* k = resolve(scheme, coll, eos, nu, tma);
    int n = 0;
    if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, tma ? kStepThreads + 32 : kStepThreads,
                                                            tma ? kTmaSmem : 0) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

}  // namespace lbfe
