// Internal launch interface between the host API and the step kernels.
#pragma once

#include <cuda_runtime.h>

#include "lbfe_device.cuh"

namespace lbfe {

constexpr int kStepThreads = 256;

cudaError_t launch_step_f32(int scheme, int coll, int eos, bool nu, int nblocks, cudaStream_t s,
                            const float* fin, float* fout, const DevCase<float>* cases, const Item* items);
cudaError_t launch_step_f64(int scheme, int coll, int eos, bool nu, int nblocks, cudaStream_t s,
                            const double* fin, double* fout, const DevCase<double>* cases,
                            const Item* items);
int occupancy_step_f32(int scheme, int coll, int eos, bool nu);
int occupancy_step_f64(int scheme, int coll, int eos, bool nu);

}  // namespace lbfe
