// Instantiations of the one-column FP32 step kernels (plain loads and the TMA
// variant) and the FP32 launch; the packed kernels are instantiated per
// scheme in the step_f32_pair<S>[s].cu units and the plain-load kernel with
// the per-step statistics in step_f32s.cu (compiled in parallel).
#include "launch.h"
#include "step_pair.cuh"

namespace lbfe {

namespace {
// the packed kernel (nullptr for the Lax-Wendroff scheme, which it does not run)
template <bool ST>
void* pick_pair_st(int scheme, int coll, int eos, bool nu, bool narrow, bool walls)
{
    switch (scheme) {
    case 0: return pick_pair_scheme<0, ST>(coll, eos, nu, narrow, walls);
    case 1: return pick_pair_scheme<1, ST>(coll, eos, nu, narrow, walls);
    case 2: return pick_pair_scheme<2, ST>(coll, eos, nu, narrow, walls);
    case 3: return pick_pair_scheme<3, ST>(coll, eos, nu, narrow, walls);
    default: return nullptr;
    }
}

void* pick_pair(int scheme, int coll, int eos, bool nu, bool narrow, bool stats, bool walls)
{
    return stats ? pick_pair_st<true>(scheme, coll, eos, nu, narrow, walls)
                 : pick_pair_st<false>(scheme, coll, eos, nu, narrow, walls);
}

// NT = kPairWide / kPairNarrow select the two-columns-per-thread packed
// kernel with 128 / 64 threads (pick_pair, step_f32_pair.cu)
template <int S, int C, int E, bool NU, bool TMA, int NT>
void* kernel_ptr()
{
    if constexpr ((S == 3 || S == 4) && TMA)
        return nullptr;  // the one-column TMA kernel runs neither scheme 3 nor the Lax-Wendroff scheme
    else if constexpr (TMA)
        return reinterpret_cast<void*>(&step_kernel_tma<float, NT, S, C, E, NU>);
    else
        return reinterpret_cast<void*>(&step_kernel<float, kStepThreads, S, C, E, NU>);
}

template <bool TMA, int NT>
void* pick(int scheme, int coll, int eos, bool nu)
{
#define LBFE_PICK(S, C, E)                                                                          \
    if (scheme == S && coll == C && eos == E)                                                       \
        return nu ? kernel_ptr<S, C, E, true, TMA, NT>() : kernel_ptr<S, C, E, false, TMA, NT>();
    LBFE_PICK(0, 0, 0) LBFE_PICK(0, 0, 1) LBFE_PICK(0, 1, 0) LBFE_PICK(0, 1, 1)
    LBFE_PICK(1, 0, 0) LBFE_PICK(1, 0, 1) LBFE_PICK(1, 1, 0) LBFE_PICK(1, 1, 1)
    LBFE_PICK(2, 0, 0) LBFE_PICK(2, 0, 1) LBFE_PICK(2, 1, 0) LBFE_PICK(2, 1, 1)
    LBFE_PICK(3, 0, 0) LBFE_PICK(3, 0, 1) LBFE_PICK(3, 1, 0) LBFE_PICK(3, 1, 1)
    LBFE_PICK(4, 0, 0) LBFE_PICK(4, 0, 1)  // Lax-Wendroff: BGK only
#undef LBFE_PICK
    return nullptr;
}

// dynamic shared memory of a TMA-fed kernel (the packed kernel's scheme 3
// has a ring of its own for stage D)
size_t tma_smem(int nt, int scheme)
{
    const bool s3 = scheme == 3;
    return nt == kPairWide     ? (s3 ? pair_dynamic_smem<float, kPairThreads, 3>()
                                     : pair_dynamic_smem<float, kPairThreads, 1>())
           : nt == kPairNarrow ? (s3 ? pair_dynamic_smem<float, kPairThreadsNarrow, 3>()
                                     : pair_dynamic_smem<float, kPairThreadsNarrow, 1>())
           : nt == 128         ? tma_dynamic_smem<float, 128>()
                               : tma_dynamic_smem<float, 256>();
}

int block_threads(bool tma, int nt)
{
    return !tma ? kStepThreads : nt == kPairWide ? kPairThreads : nt == kPairNarrow ? kPairThreadsNarrow : nt + 32;
}

void* resolve(int scheme, int coll, int eos, bool nu, bool tma, int nt, bool stats = false, bool walls = false)
{
    void* k = !tma                ? (stats ? pick_plain_stats_f32(scheme, coll, eos, nu)
                                           : pick<false, kStepThreads>(scheme, coll, eos, nu))
              : nt == kPairWide   ? pick_pair(scheme, coll, eos, nu, false, stats, walls)
              : nt == kPairNarrow ? pick_pair(scheme, coll, eos, nu, true, stats, walls)
              : nt == 128    ? pick<true, 128>(scheme, coll, eos, nu)
              : nt == 256    ? pick<true, 256>(scheme, coll, eos, nu)
                             : nullptr;
    if (k && tma) {
        // idempotent; needed once per kernel for more than 48 KB of dynamic smem,
        // and the largest shared-memory carveout so that several blocks fit per SM
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem(nt, scheme));
        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    return k;
}
}  // namespace

cudaError_t launch_step_f32(int scheme, int coll, int eos, bool nu, bool tma, int nt, int nblocks,
                            cudaStream_t s, const float* fin, float* fout, const DevCase<float>* cases,
                            const Item* items, int* status, bool stats, bool walls)
{
    void* k = resolve(scheme, coll, eos, nu, tma, nt, stats, walls);
    if (!k) return cudaErrorInvalidValue;
    void* args[] = {(void*)&fin, (void*)&fout, (void*)&cases, (void*)&items, (void*)&status};
    // the TMA kernels add one producer warp to their compute threads
    return cudaLaunchKernel(k, dim3(nblocks), dim3(block_threads(tma, nt)), args, tma ? tma_smem(nt, scheme) : 0, s);
}

int occupancy_step_f32(int scheme, int coll, int eos, bool nu, bool tma, int nt, bool walls)
{
    void* k = resolve(scheme, coll, eos, nu, tma, nt, false, walls);
    int n = 0;
    if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block_threads(tma, nt),
                                                            tma ? tma_smem(nt, scheme) : 0) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

}  // namespace lbfe
