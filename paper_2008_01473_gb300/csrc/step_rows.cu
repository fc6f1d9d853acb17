// Instantiations and launch of the row-resident step kernel for short
// periodic lattices (step_rows.cuh), both precisions, without and with the
// per-step statistics.
#include "launch.h"
#include "step_rows.cuh"

namespace lbfe {

namespace {
template <typename T, int RPT, bool ST>
void* pick_rows(int scheme, int coll, int eos, bool nu)
{
#define LBFE_PICK(S, C, E)                                                                               \
    if (scheme == S && coll == C && eos == E)                                                            \
        return nu ? reinterpret_cast<void*>(&step_kernel_rows<T, kRowsCols, RPT, S, C, E, true, ST>)     \
                  : reinterpret_cast<void*>(&step_kernel_rows<T, kRowsCols, RPT, S, C, E, false, ST>);
    LBFE_PICK(0, 0, 0) LBFE_PICK(0, 0, 1) LBFE_PICK(0, 1, 0) LBFE_PICK(0, 1, 1)
    LBFE_PICK(1, 0, 0) LBFE_PICK(1, 0, 1) LBFE_PICK(1, 1, 0) LBFE_PICK(1, 1, 1)
    LBFE_PICK(2, 0, 0) LBFE_PICK(2, 0, 1) LBFE_PICK(2, 1, 0) LBFE_PICK(2, 1, 1)
    LBFE_PICK(3, 0, 0) LBFE_PICK(3, 0, 1) LBFE_PICK(3, 1, 0) LBFE_PICK(3, 1, 1)
#undef LBFE_PICK
    return nullptr;
}

template <typename T, bool ST>
void* pick_rows_rpt(int rpt, int scheme, int coll, int eos, bool nu)
{
    return rpt == 1 ? pick_rows<T, 1, ST>(scheme, coll, eos, nu) : pick_rows<T, 2, ST>(scheme, coll, eos, nu);
}
}  // namespace

int rows_max_ny() { return kRowsMax; }

int rows_strip_width(int scheme)
{
    return kRowsCols - 2 * (scheme == 3 ? StepGeom<3>::HX : scheme == 1 ? StepGeom<1>::HX : StepGeom<0>::HX);  // 56, 58, 60
}

cudaError_t launch_step_rows(int prec, int scheme, int coll, int eos, bool nu, int ny_max, int nblocks,
                             cudaStream_t s, const void* fin, void* fout, const void* cases, const Item* items,
                             int* status, bool stats)
{
    if (scheme < 0 || scheme > 3 || ny_max < 1 || ny_max > kRowsMax) return cudaErrorInvalidValue;
    const int rpt = rows_per_thread(ny_max), threads = kRowsCols * rows_pass(ny_max);
    void* k;
    size_t smem;
    if (prec == 1) {  // LB_FP32
        k = stats ? pick_rows_rpt<float, true>(rpt, scheme, coll, eos, nu)
                  : pick_rows_rpt<float, false>(rpt, scheme, coll, eos, nu);
        smem = scheme != 0 ? rows_dynamic_smem<float, 1>(ny_max) : rows_dynamic_smem<float, 0>(ny_max);
    } else {
        k = stats ? pick_rows_rpt<double, true>(rpt, scheme, coll, eos, nu)
                  : pick_rows_rpt<double, false>(rpt, scheme, coll, eos, nu);
        smem = scheme != 0 ? rows_dynamic_smem<double, 1>(ny_max) : rows_dynamic_smem<double, 0>(ny_max);
    }
    if (!k) return cudaErrorInvalidValue;
    // at most 4 fields x 16 rows x 64 columns x 8 B = 32 KB: the default
    // dynamic shared-memory limit (48 KB) holds every launch
    void* args[] = {(void*)&fin, (void*)&fout, (void*)&cases, (void*)&items, (void*)&status};
    return cudaLaunchKernel(k, dim3(nblocks), dim3(threads), args, smem, s);
}

}  // namespace lbfe
