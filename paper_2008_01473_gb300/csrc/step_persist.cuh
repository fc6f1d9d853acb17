// Persistent multi-step launch of the one-column fused step (step_kernel.cuh):
// one cooperative launch advances every case of a work-list by nsteps time
// steps, so that lattices small enough to live in L2 are not bound by one
// launch per step.
//
// Block b owns the work items b, b + G, b + 2G, ... (G = gridDim.x; the
// launch is cooperative, so all G blocks are resident together) and processes
// them step after step. An item at step s reads the populations its
// neighbours wrote at step s - 1 (the pull and the stencil halo reach
// HX + 1 rows and columns beyond the item) and overwrites the buffer those
// neighbours read at step s - 1, so before step s it waits until every
// neighbour item has completed step s - 1. Each item publishes the number of
// steps it has completed (a release store after a block barrier); a waiting
// block polls its neighbours' counters with acquire loads and reads their
// populations at L2 (ld.global.cg), never through the non-coherent path.
//
// Every wait is bounded: after spin_limit cycles the block sets status[0]
// (reported by lb_reductions as LB_E_TIMEOUT) and the launch's abort word,
// and every block that waits afterwards sees the abort word and returns, so
// no launch can hang. A case flagged unstable (status[1 + case]) is skipped
// but its items still publish their progress.
#pragma once

#include "launch.h"
#include "step_kernel.cuh"

namespace lbfe {

__device__ __forceinline__ int ld_acquire_gpu(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(int* p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// buf0 holds the state at the start of the launch; after step s the state is
// in buf1 for even s, buf0 for odd s (so after nsteps steps in buf0 when
// nsteps is even).
template <typename T, int NT, int SCHEME, int COLL, int EOS, bool NU>
__global__ void __launch_bounds__(NT) step_kernel_persist(T* buf0, T* buf1, const DevCase<T>* __restrict__ cases,
                                                          const Item* __restrict__ items, int* __restrict__ status,
                                                          PersistArgs pa)
{
    __shared__ StepSmem<T, NT, SCHEME> sm;
    int* abort_word = pa.progress + pa.nitems;
    for (int s = 0; s < pa.nsteps; ++s) {
        const T* fin = (s & 1) ? buf1 : buf0;
        T* fout = (s & 1) ? buf0 : buf1;
        for (int i = blockIdx.x; i < pa.nitems; i += gridDim.x) {
            bool give_up = false;
            if (s > 0) {
                const int k1 = pa.nb_off[i + 1];
                for (int k = pa.nb_off[i] + (int)threadIdx.x; k < k1 && !give_up; k += NT) {
                    const int* p = pa.progress + pa.nb_idx[k];
                    if (ld_acquire_gpu(p) >= s) continue;
                    const long long t0 = clock64();
                    while (ld_acquire_gpu(p) < s) {
                        if (ld_acquire_gpu(abort_word)) {
                            give_up = true;
                            break;
                        }
                        if (clock64() - t0 > pa.spin_limit) {
                            atomicOr(status, 1);
                            atomicExch(abort_word, 1);
                            give_up = true;
                            break;
                        }
                    }
                }
            }
            if (__syncthreads_or(give_up)) return;
            const Item item = items[i];
            // thread 0 decides for the block (the word may change meanwhile)
            const bool skip = __syncthreads_or(threadIdx.x == 0 && *(volatile const int*)(status + 1 + item.case_id));
            if (!skip) {
                const DevCase<T> c = cases[item.case_id];
                StepAcc<T> acc;  // (handles with per-step statistics do not launch this kernel)
                const bool bad = step_item<T, NT, SCHEME, COLL, EOS, NU, true>(fin, fout, c, item, sm, acc);
                if (bad && threadIdx.x == 0) atomicOr(status + 1 + item.case_id, 1);
            }
            __syncthreads();  // every store of the item precedes the release below
            if (threadIdx.x == 0 && i != pa.silent_item) {
                __threadfence();
                st_release_gpu(pa.progress + i, s + 1);
            }
        }
    }
}

}  // namespace lbfe
