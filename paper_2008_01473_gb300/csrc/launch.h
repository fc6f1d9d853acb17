// Internal launch interface between the host API and the step kernels.
#pragma once

#include <cuda_runtime.h>

#include "lbfe_device.cuh"

namespace lbfe {

constexpr int kStepThreads = 256;
constexpr int kPairWide = 0, kPairNarrow = 1;  // packed-kernel shapes (nt values)

// tma: use the TMA-staged kernel (FP32 only; every case of the launch has
// nx % 4 == 0 and every item x0 % 4 == 0, wv % 4 == 0, wv + 8 <= kStepThreads).
// status: device word that a bounded wait which gave up sets to nonzero.
// nt: kernel shape on the TMA path: kPairWide = two columns per thread with
// packed FP32 arithmetic, 128 threads (256 columns per block); kPairNarrow =
// the same with 64 threads (128 columns); 128 or 256 = one column per thread.
// The plain-load kernel always uses kStepThreads.
cudaError_t launch_step_f32(int scheme, int coll, int eos, bool nu, bool tma, int nt, int nblocks,
                            cudaStream_t s, const float* fin, float* fout, const DevCase<float>* cases,
                            const Item* items, int* status);
cudaError_t launch_step_f64(int scheme, int coll, int eos, bool nu, int nblocks, cudaStream_t s,
                            const double* fin, double* fout, const DevCase<double>* cases,
                            const Item* items, int* status);
int occupancy_step_f32(int scheme, int coll, int eos, bool nu, bool tma, int nt);
int occupancy_step_f64(int scheme, int coll, int eos, bool nu);

}  // namespace lbfe
