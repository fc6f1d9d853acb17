// Instantiations of the fused step kernel with FP64 populations and arithmetic
// (the variant with the per-step statistics: step_f64s.cu).
#include "launch.h"
#include "step_kernel.cuh"

namespace lbfe {

namespace {
template <int S, int C, int E, bool NU>
void* kernel_ptr()
{
    return reinterpret_cast<void*>(&step_kernel<double, kStepThreads, S, C, E, NU>);
}

void* pick(int scheme, int coll, int eos, bool nu)
{
#define LBFE_PICK(S, C, E)                                                        \
    if (scheme == S && coll == C && eos == E)                                     \
        return nu ? kernel_ptr<S, C, E, true>() : kernel_ptr<S, C, E, false>();
    LBFE_PICK(0, 0, 0) LBFE_PICK(0, 0, 1) LBFE_PICK(0, 1, 0) LBFE_PICK(0, 1, 1)
    LBFE_PICK(1, 0, 0) LBFE_PICK(1, 0, 1) LBFE_PICK(1, 1, 0) LBFE_PICK(1, 1, 1)
    LBFE_PICK(2, 0, 0) LBFE_PICK(2, 0, 1) LBFE_PICK(2, 1, 0) LBFE_PICK(2, 1, 1)
    LBFE_PICK(3, 0, 0) LBFE_PICK(3, 0, 1) LBFE_PICK(3, 1, 0) LBFE_PICK(3, 1, 1)
    LBFE_PICK(4, 0, 0) LBFE_PICK(4, 0, 1)  // Lax-Wendroff: BGK only
#undef LBFE_PICK
    return nullptr;
}
}  // namespace

cudaError_t launch_step_f64(int scheme, int coll, int eos, bool nu, int nblocks, cudaStream_t s,
                            const double* fin, double* fout, const DevCase<double>* cases,
                            const Item* items, int* status, bool stats)
{
    void* k = stats ? pick_plain_stats_f64(scheme, coll, eos, nu) : pick(scheme, coll, eos, nu);
    if (!k) return cudaErrorInvalidValue;
    void* args[] = {(void*)&fin, (void*)&fout, (void*)&cases, (void*)&items, (void*)&status};
    return cudaLaunchKernel(k, dim3(nblocks), dim3(kStepThreads), args, 0, s);
}

int occupancy_step_f64(int scheme, int coll, int eos, bool nu)
{
    void* k = pick(scheme, coll, eos, nu);
    int n = 0;
    if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kStepThreads, 0) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

}  // namespace lbfe
