// Packed FP32 step kernels of scheme 3 (see step_f32_pair.cuh).
#include "step_f32_pair.cuh"

namespace lbfe {
template void* pick_pair_scheme<3, false>(int coll, int eos, bool nu, bool narrow, bool walls);
}  // namespace lbfe
