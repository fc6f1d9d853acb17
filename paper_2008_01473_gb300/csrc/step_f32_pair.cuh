// Instantiation table of the packed two-columns-per-thread FP32 step kernel
// (step_pair.cuh) for one scheme, wide (128 threads) and narrow (64 threads);
// each step_f32_pair<scheme>.cu unit instantiates one scheme, so that the
// four compile in parallel.
#pragma once

#include "launch.h"
#include "step_pair.cuh"

namespace lbfe {

template <int S, int C, int E, bool NU>
void* pair_ptr(bool narrow)
{
    return narrow ? reinterpret_cast<void*>(&step_kernel_pair<S, C, E, NU, kPairThreadsNarrow>)
                  : reinterpret_cast<void*>(&step_kernel_pair<S, C, E, NU, kPairThreads>);
}

template <int S>
void* pick_pair_scheme(int coll, int eos, bool nu, bool narrow)
{
#define LBFE_PICK(C, E) \
    if (coll == C && eos == E) return nu ? pair_ptr<S, C, E, true>(narrow) : pair_ptr<S, C, E, false>(narrow);
    LBFE_PICK(0, 0) LBFE_PICK(0, 1) LBFE_PICK(1, 0) LBFE_PICK(1, 1)
#undef LBFE_PICK
    return nullptr;
}

}  // namespace lbfe
