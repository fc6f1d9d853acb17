// Instantiations of the plain-load one-column step kernel with FP32
// populations that records the per-step statistics (ST = true; see
// step_kernel.cuh), in a unit of its own so that it compiles in parallel.
#include "launch.h"
#include "step_kernel.cuh"

namespace lbfe {

namespace {
template <int S, int C, int E, bool NU>
void* kernel_ptr()
{
    return reinterpret_cast<void*>(&step_kernel<float, kStepThreads, S, C, E, NU, true>);
}
}  // namespace

void* pick_plain_stats_f32(int scheme, int coll, int eos, bool nu)
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

}  // namespace lbfe
