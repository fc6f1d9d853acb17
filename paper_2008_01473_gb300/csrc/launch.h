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
// The plain-load kernel always uses kStepThreads. stats: launch the variant
// that records the per-step statistics (the packed and plain-load kernels;
// the one-column TMA shapes always accumulate and check st_hist).
// walls: the group holds lattices with walls (the packed kernel's variant
// that runs them).
cudaError_t launch_step_f32(int scheme, int coll, int eos, bool nu, bool tma, int nt, int nblocks,
                            cudaStream_t s, const float* fin, float* fout, const DevCase<float>* cases,
                            const Item* items, int* status, bool stats = false, bool walls = false);
cudaError_t launch_step_f64(int scheme, int coll, int eos, bool nu, int nblocks, cudaStream_t s,
                            const double* fin, double* fout, const DevCase<double>* cases,
                            const Item* items, int* status, bool stats = false);
int occupancy_step_f32(int scheme, int coll, int eos, bool nu, bool tma, int nt, bool walls = false);
// the packed FP32 kernel of scheme S for a collision / EOS / viscosity mode,
// wide or narrow shape, without or with the per-step statistics
// (instantiated in step_f32_pair<S>.cu and step_f32_pair<S>s.cu)
template <int S, bool ST>
void* pick_pair_scheme(int coll, int eos, bool nu, bool narrow, bool walls);
extern template void* pick_pair_scheme<0, false>(int, int, bool, bool, bool);
extern template void* pick_pair_scheme<1, false>(int, int, bool, bool, bool);
extern template void* pick_pair_scheme<2, false>(int, int, bool, bool, bool);
extern template void* pick_pair_scheme<3, false>(int, int, bool, bool, bool);
extern template void* pick_pair_scheme<0, true>(int, int, bool, bool, bool);
extern template void* pick_pair_scheme<1, true>(int, int, bool, bool, bool);
extern template void* pick_pair_scheme<2, true>(int, int, bool, bool, bool);
extern template void* pick_pair_scheme<3, true>(int, int, bool, bool, bool);
// the plain-load one-column kernel with the per-step statistics (step_f32s.cu,
// step_f64s.cu); nullptr where it has no instantiation
void* pick_plain_stats_f32(int scheme, int coll, int eos, bool nu);
void* pick_plain_stats_f64(int scheme, int coll, int eos, bool nu);
int occupancy_step_f64(int scheme, int coll, int eos, bool nu);

// The row-resident kernel for short periodic lattices (step_rows.cuh):
// schemes 0-3, every case of the launch periodic with ny <= ny_max <=
// rows_max_ny(), one item per column strip of at most rows_strip_width(scheme)
// output columns spanning the whole height. prec: LB_FP32 (1) or LB_FP64 (0).
cudaError_t launch_step_rows(int prec, int scheme, int coll, int eos, bool nu, int ny_max, int nblocks,
                             cudaStream_t s, const void* fin, void* fout, const void* cases, const Item* items,
                             int* status, bool stats);
int rows_max_ny();
int rows_strip_width(int scheme);

// Arguments of the persistent multi-step kernel (step_persist.cuh).
struct PersistArgs {
    const int* nb_off;     // [nitems + 1]: CSR offsets of each item's neighbour list
    const int* nb_idx;     // neighbour item indices (the item itself excluded)
    int* progress;         // [nitems]: steps completed in this launch; [nitems]: abort word
    int nitems;
    int nsteps;
    long long spin_limit;  // clock cycles a wait may spin before it gives up
    int silent_item;       // self-test: this item never publishes its progress (-1: none)
};

// One cooperative launch of the persistent one-column kernel over `grid`
// blocks (at most occupancy_persist() x SMs, so that all are resident):
// nsteps steps starting from buf0 (see step_persist.cuh for where the state
// ends). prec: LB_FP32 (1) or LB_FP64 (0).
cudaError_t launch_persist(int prec, int scheme, int coll, int eos, bool nu, int grid, cudaStream_t s, void* buf0,
                           void* buf1, const void* cases, const Item* items, int* status, const PersistArgs& pa);
// resident blocks per SM of that kernel (0 if it has no instantiation)
int occupancy_persist(int prec, int scheme, int coll, int eos, bool nu);

}  // namespace lbfe
