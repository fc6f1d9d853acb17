// Instantiations of the persistent multi-step kernel (step_persist.cuh), both
// precisions, and its cooperative launch.
#include "step_persist.cuh"

namespace lbfe {

namespace {
template <typename T, int S, int C, int E, bool NU>
void* kernel_ptr()
{
    return reinterpret_cast<void*>(&step_kernel_persist<T, kStepThreads, S, C, E, NU>);
}

template <typename T>
void* pick(int scheme, int coll, int eos, bool nu)
{
#define LBFE_PICK(S, C, E)                                                              \
    if (scheme == S && coll == C && eos == E)                                           \
        return nu ? kernel_ptr<T, S, C, E, true>() : kernel_ptr<T, S, C, E, false>();
    LBFE_PICK(0, 0, 0) LBFE_PICK(0, 0, 1) LBFE_PICK(0, 1, 0) LBFE_PICK(0, 1, 1)
    LBFE_PICK(1, 0, 0) LBFE_PICK(1, 0, 1) LBFE_PICK(1, 1, 0) LBFE_PICK(1, 1, 1)
    LBFE_PICK(2, 0, 0) LBFE_PICK(2, 0, 1) LBFE_PICK(2, 1, 0) LBFE_PICK(2, 1, 1)
    LBFE_PICK(3, 0, 0) LBFE_PICK(3, 0, 1) LBFE_PICK(3, 1, 0) LBFE_PICK(3, 1, 1)
    LBFE_PICK(4, 0, 0) LBFE_PICK(4, 0, 1)  // Lax-Wendroff: BGK only
#undef LBFE_PICK
    return nullptr;
}

void* resolve(int prec, int scheme, int coll, int eos, bool nu)
{
    return prec == 1 ? pick<float>(scheme, coll, eos, nu) : pick<double>(scheme, coll, eos, nu);
}
}  // namespace

cudaError_t launch_persist(int prec, int scheme, int coll, int eos, bool nu, int grid, cudaStream_t s, void* buf0,
                           void* buf1, const void* cases, const Item* items, int* status, const PersistArgs& pa)
{
    void* k = resolve(prec, scheme, coll, eos, nu);
    if (!k || grid < 1) return cudaErrorInvalidValue;
    PersistArgs a = pa;
    void* args[] = {(void*)&buf0, (void*)&buf1, (void*)&cases, (void*)&items, (void*)&status, (void*)&a};
    // cooperative: every block resident at once, which the waits between
    // blocks rely on (the launch fails rather than run blocks one after another)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kStepThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, k, args);
}

int occupancy_persist(int prec, int scheme, int coll, int eos, bool nu)
{
    void* k = resolve(prec, scheme, coll, eos, nu);
    int n = 0;
    if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kStepThreads, 0) != cudaSuccess) return 0;
    return n;
}

}  // namespace lbfe
