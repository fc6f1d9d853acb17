// Packed FP32 step kernels of scheme 0 with the per-step statistics (see
// step_f32_pair.cuh).
#include "step_f32_pair.cuh"

namespace lbfe {
template void* pick_pair_scheme<0, true>(int coll, int eos, bool nu, bool narrow, bool walls);
}  // namespace lbfe
