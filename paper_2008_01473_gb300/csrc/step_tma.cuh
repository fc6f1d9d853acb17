// TMA-staged variant of the fused step: the stored rows a block needs are
// copied from HBM into a shared-memory ring by bulk asynchronous copies
// (cp.async.bulk), issued ahead of use by a dedicated producer warp. The NT
// compute threads pull their nine populations from shared memory in stage A,
// so they never wait on HBM latency; stages B-D are those of step_kernel.cuh,
// synchronised by a named barrier that the producer warp does not join.
//
// Ring: kTmaSlots slots, each holding the nine planes of one stored row over
// the block's columns [x0 - 4, x0 + wv + 4) (the rho halo of 3 plus 1 for the
// pull). A row is copied as up to three runs (periodic wrap at the lattice
// edges); every run starts on a 16-byte boundary because x0, wv and nx are
// multiples of 4 elements on this path. Stored row s (window coordinates,
// s0 = y0 - HX - 1 first) lives in slot k = (s - s0) % kTmaSlots and is the
// m-th occupant of that slot, m = (s - s0) / kTmaSlots.
//
// Two mbarriers per slot:
//   full[k]  : producer arrive.expect_tx + bulk-copy completion; the compute
//              threads wait on phase m & 1 before reading row s.
//   empty[k] : compute thread 0 arrives once stage A of iteration it = s - s0
//              (the last reader of row s) is past the block barrier; the
//              producer waits on phase (m - 1) & 1 before refilling slot k.
//
// Every wait is bounded (about one second of SM clock); a wait that gives up
// sets *status and the thread carries on, so no launch can hang. Before
// exiting, a block that saw a timeout waits (bounded) for its copies in flight.
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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
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
    T* ring;                       // [kTmaSlots][9][SW]
    uint64_t* full;                // [kTmaSlots]
    uint64_t* empty;               // [kTmaSlots]
    int* flag;                     // shared: a wait of this block timed out
    int* status;                   // global status word
    int s0, s_last;                // first / last stored window row of the block
    int jc;                        // smem column of the thread's own lattice column

    __device__ __forceinline__ T* slot(int k) const { return ring + (size_t)k * kQ * SW; }

    __device__ __forceinline__ void timed_out() const
    {
        *flag = 1;
        atomicOr(status, 1);
    }

    __device__ __forceinline__ void pull(int it, T* F, const T* __restrict__, const DevCase<T>&,
                                         const StepLane&, const StepRows&) const
    {
        if (it == 0) {
            if (!mbar_wait(full + 0, 0u)) timed_out();
            if (!mbar_wait(full + 1, 0u)) timed_out();
        }
        {
            const int i = it + 2;  // stored row s0 + it + 2 = ra + 1
            if (!mbar_wait(full + i % kTmaSlots, (uint32_t)(i / kTmaSlots) & 1u)) timed_out();
        }
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

    // after the barrier that follows stage A: row s0 + it has no reader left
    __device__ __forceinline__ void after_sync(int it) const
    {
        if (threadIdx.x == 0) mbar_arrive(empty + it % kTmaSlots);
    }

    // compute threads only (the producer warp never joins)
    __device__ __forceinline__ void sync() const { asm volatile("bar.sync 1, %0;" ::"r"(NT) : "memory"); }
};

template <typename T, int NT>
constexpr size_t tma_dynamic_smem()
{
    return (size_t)kTmaSlots * kQ * NT * sizeof(T) + 2 * kTmaSlots * sizeof(uint64_t);
}

// Producer warp, lane 0: copy stored window rows s0 .. s_last into the ring.
template <typename T, int NT, int SCHEME>
__device__ __forceinline__ void tma_produce(const PullTma<T, NT, SCHEME>& A, const T* __restrict__ fin,
                                            const DevCase<T>& c, const TmaRuns& runs, uint32_t row_bytes)
{
    const uint32_t P = (uint32_t)c.plane;
    for (int s = A.s0; s <= A.s_last; ++s) {
        const int i = s - A.s0;
        const int k = i % kTmaSlots, m = i / kTmaSlots;
        if (m > 0 && !mbar_wait(A.empty + k, (uint32_t)(m - 1) & 1u)) A.timed_out();
        // order the compute threads' generic reads of the slot before the async refill
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        uint64_t* b = A.full + k;
        mbar_expect_tx(b, row_bytes);
        const uint32_t row = (uint32_t)wrapi(s, c.ny) * c.pitch;
        T* dst = A.slot(k);
#pragma unroll 1
        for (int a = 0; a < kQ; ++a) {
#pragma unroll
            for (int r = 0; r < 3; ++r)
                if (r < runs.n)
                    bulk_load(dst + a * PullTma<T, NT, SCHEME>::SW + runs.j0[r],
                              fin + (a * P + row + (uint32_t)runs.g0[r]), (uint32_t)runs.len[r] * sizeof(T), b);
        }
    }
}

// Same contract as step_kernel, with blockDim.x == NT + 32 (NT compute
// threads and one producer warp); every case of the launch has nx % 4 == 0
// and every work item has x0 % 4 == 0, wv % 4 == 0 and wv + 8 <= NT.
template <typename T, int NT, int SCHEME, int COLL, int EOS, bool NU>
__global__ void __launch_bounds__(NT + 32) step_kernel_tma(const T* __restrict__ fin, T* __restrict__ fout,
                                                           const DevCase<T>* __restrict__ cases,
                                                           const Item* __restrict__ items,
                                                           int* __restrict__ status)
{
    static_assert(SCHEME != 3 && SCHEME != 4, "schemes 3 and 4 run on the plain-load kernel only");
    using G = StepGeom<SCHEME>;
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ StepSmem<T, NT, SCHEME> sm;
    __shared__ int flag;
    const Item item = items[blockIdx.x];
    // a case flagged unstable no longer advances (thread 0 decides for the block)
    if (__syncthreads_or(threadIdx.x == 0 && status[1 + item.case_id] != 0)) return;
    const DevCase<T> c = cases[item.case_id];
    fin += c.off;
    fout += c.off;
    const int niter = item.h + 2 * G::HX;

    PullTma<T, NT, SCHEME> A;
    A.ring = reinterpret_cast<T*>(dsm);
    A.full = reinterpret_cast<uint64_t*>(dsm + (size_t)kTmaSlots * kQ * NT * sizeof(T));
    A.empty = A.full + kTmaSlots;
    A.flag = &flag;
    A.status = status;
    A.s0 = item.y0 - G::HX - 1;
    A.s_last = A.s0 + niter + 1;
    A.jc = (int)threadIdx.x + 4 - G::HX;

    if (threadIdx.x == 0) {
        flag = 0;
        for (int k = 0; k < kTmaSlots; ++k) {
            mbar_init(A.full + k, 1);
            mbar_init(A.empty + k, 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    StepRegs<T> R;
    R.bad = false;
    R.am = R.ak = R.au = T(0);
    if (threadIdx.x >= NT) {
        // producer warp
        if (threadIdx.x == NT) {
            TmaRuns runs;
            const int start = item.x0 - 4, end = item.x0 + item.wv + 4;
            runs.n = 0;
            int x = start, j = 0;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const int g = wrapi(x, c.nx);
                const int len = min(end - x, c.nx - g);
                runs.g0[r] = g;
                runs.j0[r] = j;
                runs.len[r] = len;
                if (x < end) runs.n = r + 1;
                x += len;
                j += len;
            }
            tma_produce<T, NT, SCHEME>(A, fin, c, runs, (uint32_t)(kQ * (end - start) * sizeof(T)));
        }
    } else {
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
        rows.sa = item.y0 - G::HX;  // (this kernel never runs lattices with walls)

        using Pull = PullTma<T, NT, SCHEME>;  // (accumulating statistics; the block end reads st_hist)
        for (int base = 0; base < niter; base += 4) {
            step_iter<T, NT, SCHEME, COLL, EOS, NU, 0, Pull, false, true>(base, A, fin, fout, c, L, rows, sm, R);
            if (base + 1 >= niter) break;
            step_iter<T, NT, SCHEME, COLL, EOS, NU, 1, Pull, false, true>(base + 1, A, fin, fout, c, L, rows, sm, R);
            if (base + 2 >= niter) break;
            step_iter<T, NT, SCHEME, COLL, EOS, NU, 2, Pull, false, true>(base + 2, A, fin, fout, c, L, rows, sm, R);
            if (base + 3 >= niter) break;
            step_iter<T, NT, SCHEME, COLL, EOS, NU, 3, Pull, false, true>(base + 3, A, fin, fout, c, L, rows, sm, R);
        }
        // every issued row was waited on by stage A; after a timeout, drain (bounded)
        A.sync();
        if (L.t == 0 && flag) {
            for (int s = max(A.s0, A.s_last - kTmaSlots + 1); s <= A.s_last; ++s) {
                const int i = s - A.s0;
                mbar_wait(A.full + i % kTmaSlots, (uint32_t)(i / kTmaSlots) & 1u);
            }
        }
    }
    // the producer warp joins with R.bad == false and zero statistics
    if (__syncthreads_or(R.bad) && threadIdx.x == 0) atomicOr(status + 1 + item.case_id, 1);
    if (c.st_hist)
        stats_block(c, (double)R.am, (double)R.ak, (double)R.au,
                    (unsigned long long)item.wv * (unsigned long long)item.h);
}

}  // namespace lbfe
