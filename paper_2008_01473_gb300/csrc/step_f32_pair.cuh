// Instantiation table of the packed two-columns-per-thread FP32 step kernel
// (step_pair.cuh) for one scheme, wide (128 threads) and narrow (64 threads),
// without (ST false) or with the per-step statistics (ST true); each
// step_f32_pair<scheme>[s].cu unit instantiates one scheme and one ST, so
// that the eight compile in parallel.
#pragma once

#include "launch.h"
#include "step_pair.cuh"

namespace lbfe {

template <int S, int C, int E, bool NU, bool ST, bool WL>
void* pair_ptr_w(bool narrow)
{
    return narrow ? reinterpret_cast<void*>(&step_kernel_pair<S, C, E, NU, kPairThreadsNarrow, ST, WL>)
                  : reinterpret_cast<void*>(&step_kernel_pair<S, C, E, NU, kPairThreads, ST, WL>);
}

// lattices with walls run the WL variant
template <int S, int C, int E, bool NU, bool ST>
void* pair_ptr(bool narrow, bool walls)
{
    return walls ? pair_ptr_w<S, C, E, NU, ST, true>(narrow) : pair_ptr_w<S, C, E, NU, ST, false>(narrow);
}

template <int S, bool ST>
void* pick_pair_scheme(int coll, int eos, bool nu, bool narrow, bool walls)
{
#define LBFE_PICK(C, E)                                                                                 \
    if (coll == C && eos == E)                                                                          \
        return nu ? pair_ptr<S, C, E, true, ST>(narrow, walls) : pair_ptr<S, C, E, false, ST>(narrow, walls);
    LBFE_PICK(0, 0) LBFE_PICK(0, 1) LBFE_PICK(1, 0) LBFE_PICK(1, 1)
#undef LBFE_PICK
    return nullptr;
}

}  // namespace lbfe
