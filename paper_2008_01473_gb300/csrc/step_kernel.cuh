// Fused free-energy D2Q9 time step, sliding-window form, for sm_103a.
//
// A thread block owns a strip of output columns [x0, x0 + wv) of one case and
// walks its rows [y0, y0 + h) upward, one row per iteration. Each thread owns
// one column of the strip or of a halo of HX columns on each side (HX = 3 for
// the improved scheme, 2 for the standard one). Per iteration, the stages run
// on consecutive rows, so that every field is computed once per node and only
// what neighbouring columns need passes through shared memory:
//
//   A (row r)     pull the nine populations (Eq. 10 in pull form); rho and
//                 sum e f (Eq. 12)                        -> smem rho rows
//   B (row r - 1) mu_c = E_f'(rho) - kappa lap(rho)       (Eq. 2; Eq. 30)
//                                                        -> smem mu rows
//   C (row r - 2) improved only: grad_h mu_c (Eq. 17), F (Eq. 24), u (Eq. 12),
//                 phi u with phi = rho/3 - p_m (Eq. 29)   -> smem phi-u rows
//   D (row r - 3) improved: C1, C7 (Eq. 29), collision (Eq. 28), store f*
//     (row r - 2) standard: grad mu_c, grad rho (Eq. 17), F (Eq. 13), u,
//                 collision (Eq. 9), store f*
//
// The populations of a thread's own column stay in a register ring between
// stage A and the collision. Each population is read from memory once per
// block; the only re-reads are the halo columns shared with neighbouring
// strips (L2 hits: neighbouring blocks walk the same rows at the same time)
// and the pipeline fill rows at the two ends of each row segment.
#pragma once

#include "lbfe_device.cuh"

namespace lbfe {

template <int SCHEME>
struct StepGeom {
    static constexpr int HX = SCHEME == 1 ? 3 : 2;    // column halo of rho
    static constexpr int LAG = SCHEME == 1 ? 3 : 2;   // rows between stage A and D
    static constexpr int RING = LAG + 1;              // population register ring depth
    static constexpr int NRHO = SCHEME == 1 ? 4 : 5;  // smem rows of rho
    static constexpr int NMU = 4;                     // smem rows of mu
};

template <typename T, int NT, int SCHEME>
struct StepSmem {
    T rho[StepGeom<SCHEME>::NRHO][NT];
    T mu[StepGeom<SCHEME>::NMU][NT];
    T pux[SCHEME == 1 ? 3 : 1][NT];
    T puy[SCHEME == 1 ? 3 : 1][NT];
};

template <typename T, int RING>
struct StepRegs {
    T f[RING][kQ];  // pulled populations (deviation form) of the own column
    T drho[RING];
    T jx[RING], jy[RING];
    T ux[2], uy[2], Fx[2], Fy[2];  // stage C results, two rows (improved)
};

struct StepLane {
    int t;         // thread index = window column
    int xc, xm, xp;  // lattice columns x, x-1, x+1 (periodic)
    bool a, b, c, d;  // active in stages A..D
};

template <typename T, int NT, int SCHEME, int COLL, int EOS, bool NU, int SLOT>
__device__ __forceinline__ void step_iter(int it, const T* __restrict__ fin, T* __restrict__ fout,
                                          const DevCase<T>& c, int y0, int h, const StepLane& L,
                                          StepSmem<T, NT, SCHEME>& sm,
                                          StepRegs<T, StepGeom<SCHEME>::RING>& R)
{
    using G = StepGeom<SCHEME>;
    constexpr int RING = G::RING;
    const int ny = c.ny, pitch = c.pitch, t = L.t;
    const int64_t P = c.plane;
    const int ra = y0 - G::HX + it;  // row of stage A

    // ---------------------------------------------------------------- A
    if (L.a) {
        const int r0 = wrapi(ra, ny) * pitch, rm = wrapi(ra - 1, ny) * pitch,
                  rp = wrapi(ra + 1, ny) * pitch;
        T* F = R.f[SLOT];
        F[0] = __ldg(fin + 0 * P + r0 + L.xc);
        F[1] = __ldg(fin + 1 * P + r0 + L.xm);
        F[2] = __ldg(fin + 2 * P + rm + L.xc);
        F[3] = __ldg(fin + 3 * P + r0 + L.xp);
        F[4] = __ldg(fin + 4 * P + rp + L.xc);
        F[5] = __ldg(fin + 5 * P + rm + L.xm);
        F[6] = __ldg(fin + 6 * P + rm + L.xp);
        F[7] = __ldg(fin + 7 * P + rp + L.xp);
        F[8] = __ldg(fin + 8 * P + rp + L.xm);
        const T dr = ((F[0] + (F[1] + F[3])) + (F[2] + F[4])) + ((F[5] + F[7]) + (F[6] + F[8]));
        R.drho[SLOT] = dr;
        R.jx[SLOT] = (F[1] - F[3]) + ((F[5] - F[7]) + (F[8] - F[6]));
        R.jy[SLOT] = (F[2] - F[4]) + ((F[5] - F[7]) + (F[6] - F[8]));
        sm.rho[wrapi(ra, G::NRHO)][t] = c.rho_ref + dr;
    }
    __syncthreads();

    // ---------------------------------------------------------------- B
    {
        const int rb = ra - 1;
        if (L.b && rb >= y0 - (G::HX - 1) && rb < y0 + h + G::HX - 1) {
            const T* Sm = sm.rho[wrapi(rb - 1, G::NRHO)];
            const T* S0 = sm.rho[wrapi(rb, G::NRHO)];
            const T* Sp = sm.rho[wrapi(rb + 1, G::NRHO)];
            const T rc = S0[t];
            const T lap = lap9<T>(rc, S0[t + 1], S0[t - 1], Sp[t], Sm[t], Sp[t + 1], Sp[t - 1],
                                  Sm[t + 1], Sm[t - 1]);
            sm.mu[wrapi(rb, G::NMU)][t] = dEf<EOS, T>(c, rc) - c.kappa * lap;
        }
    }
    __syncthreads();

    if constexpr (SCHEME == 1) {
        // ------------------------------------------------------------ C
        const int rcw = ra - 2;
        constexpr int S2 = (SLOT + RING - 2) % RING;  // register slot of row ra - 2
        constexpr int U2 = SLOT & 1;                  // stage C output slot of row ra - 2
        if (L.c && rcw >= y0 - 1 && rcw < y0 + h + 1) {
            const T* Mm = sm.mu[wrapi(rcw - 1, G::NMU)];
            const T* M0 = sm.mu[wrapi(rcw, G::NMU)];
            const T* Mp = sm.mu[wrapi(rcw + 1, G::NMU)];
            const T gx = gradx9<T>(M0[t + 1], M0[t - 1], Mp[t + 1], Mp[t - 1], Mm[t + 1], Mm[t - 1]);
            const T gy = grady9<T>(Mp[t], Mm[t], Mp[t + 1], Mp[t - 1], Mm[t + 1], Mm[t - 1]);
            const T rho = c.rho_ref + R.drho[S2];
            const T k = T(1.0 / 3.0) - rho;
            const T Fx = k * gx, Fy = k * gy;
            const T inv = T(1) / rho;
            const T ux = (R.jx[S2] + T(0.5) * Fx) * inv;
            const T uy = (R.jy[S2] + T(0.5) * Fy) * inv;
            const T phi = (rho - (c.c0 + M0[t])) * T(1.0 / 3.0);
            sm.pux[wrapi(rcw, 3)][t] = phi * ux;
            sm.puy[wrapi(rcw, 3)][t] = phi * uy;
            R.ux[U2] = ux;
            R.uy[U2] = uy;
            R.Fx[U2] = Fx;
            R.Fy[U2] = Fy;
        }
        __syncthreads();
        // ------------------------------------------------------------ D
        const int rd = ra - 3;
        constexpr int S3 = (SLOT + RING - 3) % RING;
        constexpr int U3 = (SLOT + 1) & 1;
        if (L.d && rd >= y0 && rd < y0 + h) {
            const T* Am = sm.pux[wrapi(rd - 1, 3)];
            const T* A0 = sm.pux[wrapi(rd, 3)];
            const T* Ap = sm.pux[wrapi(rd + 1, 3)];
            const T* Bm = sm.puy[wrapi(rd - 1, 3)];
            const T* Bp = sm.puy[wrapi(rd + 1, 3)];
            const T Ax = gradx9<T>(A0[t + 1], A0[t - 1], Ap[t + 1], Ap[t - 1], Am[t + 1], Am[t - 1]);
            const T By = grady9<T>(Bp[t], Bm[t], Bp[t + 1], Bp[t - 1], Bm[t + 1], Bm[t - 1]);
            const T C1 = Ax + By, C7 = Ax - By;
            const T drho = R.drho[S3];
            const T rho = c.rho_ref + drho;
            const T mu = sm.mu[wrapi(rd, G::NMU)][t];
            T le = c.lam_e, ls = c.lam_s, lq = c.lam_q, lv = c.lam_v;
            if (NU) {
                lv = shear_rate<SCHEME, NU, T>(c, rho, mu);
                if (COLL == 0) le = ls = lq = lv;
            }
            collide<SCHEME, T>(R.f[S3], drho, rho, R.jx[S3], R.jy[S3], R.ux[U3], R.uy[U3], R.Fx[U3],
                               R.Fy[U3], mu, C1, C7, c.rho_ref, c.c0, le, ls, lq, lv);
            const int64_t o = (int64_t)wrapi(rd, ny) * pitch + L.xc;
#pragma unroll
            for (int a = 0; a < kQ; ++a) fout[a * P + o] = R.f[S3][a];
        }
    } else {
        // ------------------------------------------------------- D (standard)
        const int rd = ra - 2;
        constexpr int S2 = (SLOT + RING - 2) % RING;
        if (L.d && rd >= y0 && rd < y0 + h) {
            const T* Mm = sm.mu[wrapi(rd - 1, G::NMU)];
            const T* M0 = sm.mu[wrapi(rd, G::NMU)];
            const T* Mp = sm.mu[wrapi(rd + 1, G::NMU)];
            const T* Rm = sm.rho[wrapi(rd - 1, G::NRHO)];
            const T* R0 = sm.rho[wrapi(rd, G::NRHO)];
            const T* Rp = sm.rho[wrapi(rd + 1, G::NRHO)];
            const T gmx = gradx9<T>(M0[t + 1], M0[t - 1], Mp[t + 1], Mp[t - 1], Mm[t + 1], Mm[t - 1]);
            const T gmy = grady9<T>(Mp[t], Mm[t], Mp[t + 1], Mp[t - 1], Mm[t + 1], Mm[t - 1]);
            const T grx = gradx9<T>(R0[t + 1], R0[t - 1], Rp[t + 1], Rp[t - 1], Rm[t + 1], Rm[t - 1]);
            const T gry = grady9<T>(Rp[t], Rm[t], Rp[t + 1], Rp[t - 1], Rm[t + 1], Rm[t - 1]);
            const T drho = R.drho[S2];
            const T rho = c.rho_ref + drho;
            const T mu = M0[t];
            const T Fx = grx * T(1.0 / 3.0) - rho * gmx;
            const T Fy = gry * T(1.0 / 3.0) - rho * gmy;
            const T inv = T(1) / rho;
            const T ux = (R.jx[S2] + T(0.5) * Fx) * inv;
            const T uy = (R.jy[S2] + T(0.5) * Fy) * inv;
            T le = c.lam_e, ls = c.lam_s, lq = c.lam_q, lv = c.lam_v;
            if (NU) {
                lv = shear_rate<SCHEME, NU, T>(c, rho, mu);
                if (COLL == 0) le = ls = lq = lv;
            }
            collide<SCHEME, T>(R.f[S2], drho, rho, R.jx[S2], R.jy[S2], ux, uy, Fx, Fy, mu, T(0), T(0),
                               c.rho_ref, c.c0, le, ls, lq, lv);
            const int64_t o = (int64_t)wrapi(rd, ny) * pitch + L.xc;
#pragma unroll
            for (int a = 0; a < kQ; ++a) fout[a * P + o] = R.f[S2][a];
        }
    }
}

// One launch advances every case listed in the work-list by one time step.
// fin/fout: population buffers (all cases, each at DevCase::off). One block
// per work item; blockDim.x == NT.
template <typename T, int NT, int SCHEME, int COLL, int EOS, bool NU>
__global__ void __launch_bounds__(NT) step_kernel(const T* __restrict__ fin, T* __restrict__ fout,
                                                  const DevCase<T>* __restrict__ cases,
                                                  const Item* __restrict__ items)
{
    using G = StepGeom<SCHEME>;
    constexpr int RING = G::RING;
    __shared__ StepSmem<T, NT, SCHEME> sm;
    const Item item = items[blockIdx.x];
    const DevCase<T> c = cases[item.case_id];
    fin += c.off;
    fout += c.off;

    StepLane L;
    L.t = threadIdx.x;
    const int span = item.wv + 2 * G::HX;  // active window width
    const int xw = item.x0 - G::HX + L.t;
    L.xc = wrapi(xw, c.nx);
    L.xm = wrapi(xw - 1, c.nx);
    L.xp = wrapi(xw + 1, c.nx);
    L.a = L.t < span;
    L.b = L.t >= 1 && L.t < span - 1;
    L.c = L.t >= 2 && L.t < span - 2;
    L.d = L.t >= G::HX && L.t < span - G::HX;

    StepRegs<T, RING> R;
    const int niter = item.h + 2 * G::HX;
    for (int base = 0; base < niter; base += RING) {
        step_iter<T, NT, SCHEME, COLL, EOS, NU, 0>(base, fin, fout, c, item.y0, item.h, L, sm, R);
        if (base + 1 >= niter) break;
        step_iter<T, NT, SCHEME, COLL, EOS, NU, 1>(base + 1, fin, fout, c, item.y0, item.h, L, sm, R);
        if (base + 2 >= niter) break;
        step_iter<T, NT, SCHEME, COLL, EOS, NU, 2>(base + 2, fin, fout, c, item.y0, item.h, L, sm, R);
        if constexpr (RING > 3) {
            if (base + 3 >= niter) break;
            step_iter<T, NT, SCHEME, COLL, EOS, NU, 3>(base + 3, fin, fout, c, item.y0, item.h, L, sm, R);
        }
    }
}

}  // namespace lbfe
