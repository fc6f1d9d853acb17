// TMA-staged variant of the fused step: the stored rows a block needs are
// copied from HBM into a shared-memory ring by bulk asynchronous copies
// (cp.async.bulk, completion on an mbarrier per ring slot), issued several
// rows ahead by one thread. Stage A then pulls its nine populations from
// shared memory, so the warps never wait on HBM latency. Stages B-D are the
// ones of step_kernel.cuh.
//
// Ring: NS slots, each holding the nine planes of one stored row over the
// block's columns [x0 - 4, x0 + wv + 4) (the rho halo of 3 plus 1 for the
// pull). A row is copied as up to three runs (periodic wrap at the lattice
// edges); every run starts on a 16-byte boundary because x0, wv and nx are
// multiples of 4 elements on this path. Stored row s (window coordinates,
// s0 = y0 - HX - 1 first) lives in slot (s - s0) % NS, phase ((s - s0) / NS) & 1.
// Stage A of iteration it reads rows s0 + it .. s0 + it + 2; after the block
// barrier that follows it, row s0 + it is dead and its slot takes row
// s0 + it + NS.
//
// Every wait is bounded (about one second of SM clock); a wait that gives up
// sets *status and the block carries on with whatever the slot holds, so no
// launch can hang. Before exiting, a block that saw a timeout waits (bounded)
// for its own copies still in flight.
#pragma once

#include "step_kernel.cuh"

namespace lbfe {

constexpr int kTmaSlots = 8;
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait on one phase of an mbarrier; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Runs of one stored row: smem column j0 .. j0 + len - 1 <- lattice columns g0 ..
struct TmaRuns {
    int n;
    int g0[3], j0[3], len[3];
};

template <typename T, int NT, int SCHEME>
struct PullTma {
    static constexpr int SW = NT;  // smem columns per plane (>= wv + 8)
    T* ring;                       // [NS][9][SW]
    uint64_t* bar;                 // [NS]
    int* flag;                     // shared: a wait of this block timed out
    int* status;                   // global status word
    const T* fin;                  // this case's stored populations
    int s0, s_last;                // first / last stored window row of the block
    int ny, pitch;
    uint32_t P;
    uint32_t row_bytes;            // bytes of one stored row over all runs and planes
    TmaRuns runs;
    int jc;                        // smem column of the thread's own lattice column

    __device__ __forceinline__ T* slot(int k) const { return ring + (size_t)k * kQ * SW; }

    // thread 0 only: copy stored window row s into its slot
    __device__ __forceinline__ void issue(int s) const
    {
        const int k = (s - s0) % kTmaSlots;
        uint64_t* b = bar + k;
        mbar_expect_tx(b, row_bytes);
        const uint32_t row = (uint32_t)wrapi(s, ny) * pitch;
        T* dst = slot(k);
#pragma unroll 1
        for (int a = 0; a < kQ; ++a) {
#pragma unroll
            for (int r = 0; r < 3; ++r)
                if (r < runs.n)
                    bulk_load(dst + a * SW + runs.j0[r], fin + (a * P + row + (uint32_t)runs.g0[r]),
                              (uint32_t)runs.len[r] * sizeof(T), b);
        }
    }

    __device__ __forceinline__ void wait_row(int s) const
    {
        const int i = s - s0;
        if (!mbar_wait(bar + i % kTmaSlots, (uint32_t)(i / kTmaSlots) & 1u)) {
            *flag = 1;
            atomicOr(status, 1);
        }
    }

    __device__ __forceinline__ void pull(int it, T* F, const T* __restrict__, const DevCase<T>&,
                                         const StepLane&, const StepRows&) const
    {
        const int s = s0 + it;  // stored window row ra - 1
        if (it == 0) {
            wait_row(s);
            wait_row(s + 1);
        }
        wait_row(s + 2);
        const T* Rm = slot(it % kTmaSlots);        // row ra - 1
        const T* R0 = slot((it + 1) % kTmaSlots);  // row ra
        const T* Rp = slot((it + 2) % kTmaSlots);  // row ra + 1
        const int j = jc;
        F[0] = R0[0 * SW + j];
        F[1] = R0[1 * SW + j - 1];
        F[2] = Rm[2 * SW + j];
        F[3] = R0[3 * SW + j + 1];
        F[4] = Rp[4 * SW + j];
        F[5] = Rm[5 * SW + j - 1];
        F[6] = Rm[6 * SW + j + 1];
        F[7] = Rp[7 * SW + j + 1];
        F[8] = Rp[8 * SW + j - 1];
    }

    __device__ __forceinline__ void after_sync(int it) const
    {
        const int s = s0 + it + kTmaSlots;
        if (threadIdx.x == 0 && s <= s_last) {
            // order the generic-proxy reads of the slot before the async-proxy refill
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(s);
        }
    }
};

template <typename T, int NT>
constexpr size_t tma_dynamic_smem()
{
    return (size_t)kTmaSlots * kQ * NT * sizeof(T) + kTmaSlots * sizeof(uint64_t);
}

// Same contract as step_kernel; every case of the launch has nx % 4 == 0 and
// every work item has x0 % 4 == 0 and wv % 4 == 0, wv + 8 <= NT.
template <typename T, int NT, int SCHEME, int COLL, int EOS, bool NU>
__global__ void __launch_bounds__(NT) step_kernel_tma(const T* __restrict__ fin, T* __restrict__ fout,
                                                      const DevCase<T>* __restrict__ cases,
                                                      const Item* __restrict__ items, int* __restrict__ status)
{
    using G = StepGeom<SCHEME>;
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ StepSmem<T, NT, SCHEME> sm;
    __shared__ int flag;
    const Item item = items[blockIdx.x];
    const DevCase<T> c = cases[item.case_id];
    fin += c.off;
    fout += c.off;

    StepLane L;
    L.t = threadIdx.x;
    const int span = item.wv + 2 * G::HX;
    const int xw = item.x0 - G::HX + L.t;
    L.xc = wrapi(xw, c.nx);
    L.xm = wrapi(xw - 1, c.nx);
    L.xp = wrapi(xw + 1, c.nx);
    L.a = L.t < span;
    L.b = L.t >= 1 && L.t < span - 1;
    L.c = L.t >= 2 && L.t < span - 2;
    L.d = L.t >= G::HX && L.t < span - G::HX;

    StepRows rows;
    rows.ra = wrapi(item.y0 - G::HX, c.ny);
    rows.rd = item.y0;
    const int niter = item.h + 2 * G::HX;

    PullTma<T, NT, SCHEME> A;
    A.ring = reinterpret_cast<T*>(dsm);
    A.bar = reinterpret_cast<uint64_t*>(dsm + (size_t)kTmaSlots * kQ * NT * sizeof(T));
    A.flag = &flag;
    A.status = status;
    A.fin = fin;
    A.s0 = item.y0 - G::HX - 1;
    A.s_last = A.s0 + niter + 1;
    A.ny = c.ny;
    A.pitch = c.pitch;
    A.P = (uint32_t)c.plane;
    A.jc = L.t + 4 - G::HX;
    {
        // runs of [x0 - 4, x0 + wv + 4) split at the periodic edges
        const int start = item.x0 - 4, end = item.x0 + item.wv + 4;
        A.runs.n = 0;
        int x = start, j = 0;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int g = wrapi(x, c.nx);
            const int len = min(end - x, c.nx - g);
            A.runs.g0[r] = g;
            A.runs.j0[r] = j;
            A.runs.len[r] = len;
            if (x < end) A.runs.n = r + 1;
            x += len;
            j += len;
        }
        A.row_bytes = (uint32_t)(kQ * (end - start) * sizeof(T));
    }
    if (L.t == 0) {
        flag = 0;
        for (int k = 0; k < kTmaSlots; ++k) mbar_init(A.bar + k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (L.t == 0)
        for (int s = A.s0; s < A.s0 + kTmaSlots && s <= A.s_last; ++s) A.issue(s);

    StepRegs<T> R;
    for (int base = 0; base < niter; base += 4) {
        step_iter<T, NT, SCHEME, COLL, EOS, NU, 0>(base, A, fin, fout, c, L, rows, sm, R);
        if (base + 1 >= niter) break;
        step_iter<T, NT, SCHEME, COLL, EOS, NU, 1>(base + 1, A, fin, fout, c, L, rows, sm, R);
        if (base + 2 >= niter) break;
        step_iter<T, NT, SCHEME, COLL, EOS, NU, 2>(base + 2, A, fin, fout, c, L, rows, sm, R);
        if (base + 3 >= niter) break;
        step_iter<T, NT, SCHEME, COLL, EOS, NU, 3>(base + 3, A, fin, fout, c, L, rows, sm, R);
    }
    // every issued row was waited on by stage A; after a timeout, drain (bounded)
    __syncthreads();
    if (L.t == 0 && flag) {
        for (int s = max(A.s0, A.s_last - kTmaSlots + 1); s <= A.s_last; ++s) {
            const int i = s - A.s0;
            mbar_wait(A.bar + i % kTmaSlots, (uint32_t)(i / kTmaSlots) & 1u);
        }
    }
}

}  // namespace lbfe
