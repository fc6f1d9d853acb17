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
//                 standard only: grad_h rho of row r - 2 (Eq. 17), kept in
//                 registers
//   C (row r - 2) improved only: grad_h mu_c (Eq. 17), F (Eq. 24), u (Eq. 12),
//                 phi u with phi = rho/3 - p_m (Eq. 29)   -> smem phi-u rows
//   D (row r - 3) improved: C1, C7 (Eq. 29), collision (Eq. 28), store f*
//     (row r - 2) standard: grad mu_c (Eq. 17), F (Eq. 13), u, collision
//                 (Eq. 9), store f*
//
// Pressure-tensor form of the standard force (SCHEME 2, Eq. 13 left): stage
// B computes the tensor P of Eqs. 4-5 at row r - 1 instead of mu_c (its three
// components take the mu and phi-u rows) and stage D takes div P by Eq. 17
// applied to each component in place of rho grad mu_c.
//
// All ring buffers (shared-memory rows, the register ring of the thread's
// own populations) are four rows deep and indexed by the iteration count
// modulo 4, which the four-fold unrolled loop makes a compile-time constant.
// Periodic row indices advance incrementally. Each population is read from
// memory once per block; the only re-reads are the halo columns shared with
// neighbouring strips (L2 hits: neighbouring blocks walk the same rows at the
// same time) and the pipeline fill rows at the two ends of each row segment.
#pragma once

#include "lbfe_device.cuh"

namespace lbfe {

// Scheme 3 (the correction's derivatives of the lattice-weight average of
// phi u) reaches phi u two rows and two columns away from the node, so its
// column halo and its lag between stages A and D are one larger than the
// improved scheme's. HX == LAG for every scheme, so stage D's first row is y0.
template <int SCHEME>
struct StepGeom {
    static constexpr int HX = SCHEME == 3 ? 4 : SCHEME == 1 ? 3 : 2;   // column halo of rho
    static constexpr int LAG = SCHEME == 3 ? 4 : SCHEME == 1 ? 3 : 2;  // rows between stage A and D
    static constexpr int NB = 2;                                       // first iteration with stage B
    static constexpr int NC = 4;        // first iteration with stage C (improved schemes)
    static constexpr int ND = 2 * LAG;  // first iteration with stage D
    // rows of the phi u rings: scheme 3 reads rows ra - 6 .. ra - 2
    static constexpr int NPU = (SCHEME == 0 || SCHEME == 4) ? 1 : SCHEME == 3 ? 6 : 4;
};

template <typename T, int NT, int SCHEME>
struct StepSmem {
    T rho[4][NT];
    T mu[4][NT];
    T pux[StepGeom<SCHEME>::NPU][NT];  // phi u_x (improved) or P_xy (pressure tensor)
    T puy[StepGeom<SCHEME>::NPU][NT];  // phi u_y (improved) or P_yy (pressure tensor)
};

template <typename T>
struct StepRegs {
    T f[4][kQ];  // pulled populations (deviation form) of the own column
    T drho[4];
    T jx[4], jy[4];
    T ux[4], uy[4], Fx[4], Fy[4];  // stage C results of the last rows (improved schemes)
    T grx, gry;                    // stage B grad rho (standard)
    bool bad;                      // a stage D node had rho <= 0 or a non-finite density
    T am, ak, au;                  // statistics of the stage D nodes: sums of rho - rho_ref, rho |u|^2; max |u|^2
};

template <typename T>
__device__ __forceinline__ void node_stats(StepRegs<T>& R, T drho, T rho, T ux, T uy)
{
    const T u2 = ux * ux + uy * uy;
    R.am += drho;
    R.ak += rho * u2;
    R.au = u2 > R.au ? u2 : R.au;
}

// per-thread statistics of one work item (returned by step_item)
template <typename T>
struct StepAcc {
    T am, ak, au;
};

// rho > 0 and finite (NaN fails both comparisons)
__device__ __forceinline__ bool rho_ok(float r) { return r > 0.0f && r <= 3.402823466e38f; }
__device__ __forceinline__ bool rho_ok(double r) { return r > 0.0 && r <= 1.7976931348623157e308; }

struct StepLane {
    int t;            // thread index = window column
    int xc, xm, xp;   // lattice columns x, x-1, x+1 (periodic)
    bool a, b, c, d;  // active in stages A..D
};

// Row bookkeeping: the periodic lattice row of stage A and of stage D, and
// the window row of stage A before wrapping (walls mirror it instead).
struct StepRows {
    int ra;  // lattice row of stage A (wrapped)
    int rd;  // lattice row of stage D (wrapped)
    int sa;  // window row of stage A (may lie outside [0, ny))
};

__device__ __forceinline__ int inc_wrap(int r, int n) { return r + 1 == n ? 0 : r + 1; }
__device__ __forceinline__ int dec_wrap(int r, int n) { return r == 0 ? n - 1 : r - 1; }

template <typename T>
__device__ __forceinline__ T rcp_fast(T x);
template <>
__device__ __forceinline__ float rcp_fast<float>(float x) { return __fdividef(1.0f, x); }
template <>
__device__ __forceinline__ double rcp_fast<double>(double x) { return 1.0 / x; }

// Population load of stage A: through the read-only cache, or (COHERENT, for
// the persistent kernel, whose populations other blocks of the same launch
// write) at L2 only, so that no stale line of an earlier step is read.
template <bool COHERENT, typename T>
__device__ __forceinline__ T ld_pop(const T* p)
{
    if constexpr (COHERENT)
        return __ldcg(p);
    else
        return __ldg(p);
}

// Stage A source of the pulled populations: plain global loads.
// With walls, window rows outside the lattice pull their mirror rows, and
// the populations that reach row 0 or ny - 1 from a wall are the node's own
// outgoing ones in the opposite direction plus the moving-wall term.
template <typename T, bool COHERENT = false>
struct PullGlobal {
    __device__ __forceinline__ void pull(int, T* F, const T* __restrict__ fin, const DevCase<T>& c,
                                         const StepLane& L, const StepRows& rows) const
    {
        const int ny = c.ny, pitch = c.pitch;
        const uint32_t P = (uint32_t)c.plane;
        if (c.walls) {
            const int m = nb_row(c, rows.sa);  // mirror of a ghost row; |sa| stays well inside ny
            const uint32_t r0 = (uint32_t)m * pitch;
            F[0] = ld_pop<COHERENT>(fin + (0 * P + r0 + L.xc));
            F[1] = ld_pop<COHERENT>(fin + (1 * P + r0 + L.xm));
            F[3] = ld_pop<COHERENT>(fin + (3 * P + r0 + L.xp));
            if (m > 0) {
                const uint32_t rm = r0 - (uint32_t)pitch;
                F[2] = ld_pop<COHERENT>(fin + (2 * P + rm + L.xc));
                F[5] = ld_pop<COHERENT>(fin + (5 * P + rm + L.xm));
                F[6] = ld_pop<COHERENT>(fin + (6 * P + rm + L.xp));
            } else {  // bottom wall
                F[2] = ld_pop<COHERENT>(fin + (4 * P + r0 + L.xc));
                F[5] = ld_pop<COHERENT>(fin + (7 * P + r0 + L.xc)) + c.wall_d;
                F[6] = ld_pop<COHERENT>(fin + (8 * P + r0 + L.xc)) - c.wall_d;
            }
            if (m < ny - 1) {
                const uint32_t rp = r0 + (uint32_t)pitch;
                F[4] = ld_pop<COHERENT>(fin + (4 * P + rp + L.xc));
                F[7] = ld_pop<COHERENT>(fin + (7 * P + rp + L.xp));
                F[8] = ld_pop<COHERENT>(fin + (8 * P + rp + L.xm));
            } else {  // top wall
                F[4] = ld_pop<COHERENT>(fin + (2 * P + r0 + L.xc));
                F[7] = ld_pop<COHERENT>(fin + (5 * P + r0 + L.xc)) - c.wall_d;
                F[8] = ld_pop<COHERENT>(fin + (6 * P + r0 + L.xc)) + c.wall_d;
            }
            if (rows.sa != m) {
                // a ghost row is the mirror image of row m: its populations
                // reflected in y (2 <-> 4, 5 <-> 8, 6 <-> 7), so that rho and
                // j_x continue evenly across the wall and j_y oddly
                T t = F[2]; F[2] = F[4]; F[4] = t;
                t = F[5]; F[5] = F[8]; F[8] = t;
                t = F[6]; F[6] = F[7]; F[7] = t;
            }
            return;
        }
        const uint32_t r0 = (uint32_t)rows.ra * pitch;
        const uint32_t rm = (uint32_t)dec_wrap(rows.ra, ny) * pitch;
        const uint32_t rp = (uint32_t)inc_wrap(rows.ra, ny) * pitch;
        F[0] = ld_pop<COHERENT>(fin + (0 * P + r0 + L.xc));
        F[1] = ld_pop<COHERENT>(fin + (1 * P + r0 + L.xm));
        F[2] = ld_pop<COHERENT>(fin + (2 * P + rm + L.xc));
        F[3] = ld_pop<COHERENT>(fin + (3 * P + r0 + L.xp));
        F[4] = ld_pop<COHERENT>(fin + (4 * P + rp + L.xc));
        F[5] = ld_pop<COHERENT>(fin + (5 * P + rm + L.xm));
        F[6] = ld_pop<COHERENT>(fin + (6 * P + rm + L.xp));
        F[7] = ld_pop<COHERENT>(fin + (7 * P + rp + L.xp));
        F[8] = ld_pop<COHERENT>(fin + (8 * P + rp + L.xm));
    }
    __device__ __forceinline__ void after_sync(int) const {}
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// Stage A of the Lax-Wendroff scheme (Eq. A2 in pull form): the population
// a at node x is a_0 f*_a(x) + a_1 f*_a(x + e_a) + a_-1 f*_a(x - e_a) of
// the stored post-collision values, over the same three rows and columns
// as the plain pull; at step 0 (lw_first) the stored values are f(0)
// itself and are taken as they are. Periodic lattices only.
template <typename T, bool COHERENT>
__device__ __forceinline__ void pull_lw(T* F, const T* __restrict__ fin, const DevCase<T>& c, const StepLane& L,
                                        const StepRows& rows)
{
    constexpr int ex[kQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    constexpr int ey[kQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const int ny = c.ny, pitch = c.pitch;
    const uint32_t P = (uint32_t)c.plane;
    const uint32_t r[3] = {(uint32_t)dec_wrap(rows.ra, ny) * pitch, (uint32_t)rows.ra * pitch,
                           (uint32_t)inc_wrap(rows.ra, ny) * pitch};
    const int xs[3] = {L.xm, L.xc, L.xp};
    const T a0 = c.lw_first ? T(1) : c.lw_a0, a1 = c.lw_first ? T(0) : c.lw_a1, am1 = c.lw_first ? T(0) : c.lw_am1;
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        const T* pa = fin + a * P;
        const T f0 = ld_pop<COHERENT>(pa + r[1] + L.xc);
        const T fp = ld_pop<COHERENT>(pa + r[1 + ey[a]] + xs[1 + ex[a]]);
        const T fm = ld_pop<COHERENT>(pa + r[1 - ey[a]] + xs[1 - ex[a]]);
        F[a] = a0 * f0 + a1 * fp + am1 * fm;
    }
}

// Stage D of scheme 3 at row rd = ra - 4. The correction takes the Eq. 17
// gradient of the lattice-weight average A' = sum_a w_a A(x + e_a) of
// A = phi u_x (and of B = phi u_y). Both stencils factor into 1-D pieces
// (w = w1 x w1 with w1 = (1, 4, 1)/6, and Eq. 17's x part is half the central
// difference times w1 across y), so
//   d_x A'(x, y) = sum_dy s(dy) [ (A(x+1) - A(x-1)) / 3 + (A(x+2) - A(x-2)) / 12 ](y + dy)
// with s = (1, 8, 18, 8, 1)/36 over dy = -2..2, and d_y B' likewise with the
// roles of x and y exchanged. The populations of row rd are pulled again
// (L2-resident: stage A read them four iterations earlier) instead of being
// kept in registers for four rows.
template <typename T, int NT, int COLL, int EOS, bool NU, int SLOT, bool COHERENT, bool ST>
__device__ __forceinline__ void step_d_smooth(int it, const T* __restrict__ fin, T* __restrict__ fout,
                                              const DevCase<T>& c, const StepLane& L, const StepRows& rows,
                                              StepSmem<T, NT, 3>& sm, StepRegs<T>& R)
{
    using G = StepGeom<3>;
    constexpr int S0 = SLOT, S2 = (SLOT + 2) & 3;
    const int t = L.t;
    // phi u rows ra - 6 .. ra - 2 (dy = -2 .. 2 around rd = ra - 4)
    const T* Ar[5];
    const T* Br[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int slot = (it + 2 * G::NPU - 6 + k) % G::NPU;
        Ar[k] = sm.pux[slot];
        Br[k] = sm.puy[slot];
    }
    const T s0 = T(1.0 / 36.0), s1 = T(8.0 / 36.0), s2 = T(18.0 / 36.0);
    const T g1 = T(1.0 / 3.0), g2 = T(1.0 / 12.0);
    T hx[5];
#pragma unroll
    for (int k = 0; k < 5; ++k)
        hx[k] = g1 * (Ar[k][t + 1] - Ar[k][t - 1]) + g2 * (Ar[k][t + 2] - Ar[k][t - 2]);
    const T Ax = s0 * (hx[0] + hx[4]) + s1 * (hx[1] + hx[3]) + s2 * hx[2];
    T sb[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        if (k == 2) continue;
        const T* b = Br[k];
        sb[k] = s0 * (b[t - 2] + b[t + 2]) + s1 * (b[t - 1] + b[t + 1]) + s2 * b[t];
    }
    const T By = g1 * (sb[3] - sb[1]) + g2 * (sb[4] - sb[0]);
    const T C1 = Ax + By, C7 = Ax - By;

    T F[kQ];
    const StepRows rr{rows.rd, rows.rd, rows.rd};
    PullGlobal<T, COHERENT>().pull(it, F, fin, c, L, rr);
    const T drho = ((F[0] + (F[1] + F[3])) + (F[2] + F[4])) + ((F[5] + F[7]) + (F[6] + F[8]));
    const T jx = (F[1] - F[3]) + ((F[5] - F[7]) + (F[8] - F[6]));
    const T jy = (F[2] - F[4]) + ((F[5] - F[7]) + (F[6] - F[8]));
    const T rho = c.rho_ref + drho;
    R.bad |= !rho_ok(rho);
    const T mu = sm.mu[S0][t];  // row ra - 4
    if constexpr (ST) node_stats(R, drho, rho, R.ux[S2], R.uy[S2]);
    T le = c.lam_e, ls = c.lam_s, lq = c.lam_q, lv = c.lam_v;
    if (NU) {
        lv = shear_rate<3, NU, T>(c, rho, mu);
        if (COLL == 0) le = ls = lq = lv;
    }
    collide<3, T>(F, drho, rho, jx, jy, R.ux[S2], R.uy[S2], R.Fx[S2], R.Fy[S2], mu, C1, C7, c.rho_ref, c.c0, le,
                  ls, lq, lv);
    const uint32_t P = (uint32_t)c.plane;
    const uint32_t o = (uint32_t)rows.rd * c.pitch + L.xc;
#pragma unroll
    for (int a = 0; a < kQ; ++a) fout[a * P + o] = F[a];
}

template <typename T, int NT, int SCHEME, int COLL, int EOS, bool NU, int SLOT, class A, bool COHERENT = false,
          bool ST = false>
__device__ __forceinline__ void step_iter(int it, const A& A_, const T* __restrict__ fin, T* __restrict__ fout,
                                          const DevCase<T>& c, const StepLane& L, StepRows& rows,
                                          StepSmem<T, NT, SCHEME>& sm, StepRegs<T>& R)
{
    using G = StepGeom<SCHEME>;
    constexpr int S0 = SLOT, S1 = (SLOT + 3) & 3, S2 = (SLOT + 2) & 3, S3 = (SLOT + 1) & 3;  // rows ra - k
    const int ny = c.ny, pitch = c.pitch;
    const uint32_t P = (uint32_t)c.plane;
    const int t = L.t;

    // ---------------------------------------------------------------- A
    if (L.a) {
        T* F = R.f[S0];
        if constexpr (SCHEME == 4)
            pull_lw<T, COHERENT>(F, fin, c, L, rows);
        else
            A_.pull(it, F, fin, c, L, rows);
        const T dr = ((F[0] + (F[1] + F[3])) + (F[2] + F[4])) + ((F[5] + F[7]) + (F[6] + F[8]));
        R.drho[S0] = dr;
        R.jx[S0] = (F[1] - F[3]) + ((F[5] - F[7]) + (F[8] - F[6]));
        R.jy[S0] = (F[2] - F[4]) + ((F[5] - F[7]) + (F[6] - F[8]));
        sm.rho[S0][t] = c.rho_ref + dr;
    }
    A_.sync();
    A_.after_sync(it);  // the TMA source refills the ring slot freed by stage A

    // ---------------------------------------------------------------- B
    if (L.b && it >= G::NB) {
        const T* Sm = sm.rho[S2];
        const T* Sc = sm.rho[S1];
        const T* Sp = sm.rho[S0];
        const T rc = Sc[t];
        const T lap = lap9<T>(rc, Sc[t + 1], Sc[t - 1], Sp[t], Sm[t], Sp[t + 1], Sp[t - 1], Sm[t + 1],
                              Sm[t - 1]);
        if constexpr (SCHEME == 2) {
            // pressure tensor of row ra - 1 (P_xx in the mu rows)
            const T gx = gradx9<T>(Sc[t + 1], Sc[t - 1], Sp[t + 1], Sp[t - 1], Sm[t + 1], Sm[t - 1]);
            const T gy = grady9<T>(Sp[t], Sm[t], Sp[t + 1], Sp[t - 1], Sm[t + 1], Sm[t - 1]);
            T Pxx, Pxy, Pyy;
            pressure_tensor<T>(pEOS<EOS, T>(c, rc), rc, gx, gy, lap, c.kappa, Pxx, Pxy, Pyy);
            sm.mu[S1][t] = Pxx;
            sm.pux[S1][t] = Pxy;
            sm.puy[S1][t] = Pyy;
        } else {
            sm.mu[S1][t] = dEf<EOS, T>(c, rc) - c.kappa * lap;
        }
        if constexpr (!improved_scheme(SCHEME)) {
            // grad rho of row ra - 2 from rows ra - 3 .. ra - 1
            if (it >= G::ND) {
                const T* Qm = sm.rho[S3];
                R.grx = gradx9<T>(Sm[t + 1], Sm[t - 1], Sc[t + 1], Sc[t - 1], Qm[t + 1], Qm[t - 1]);
                R.gry = grady9<T>(Sc[t], Qm[t], Sc[t + 1], Sc[t - 1], Qm[t + 1], Qm[t - 1]);
            }
        }
    }
    A_.sync();

    if constexpr (improved_scheme(SCHEME)) {
        // ------------------------------------------------------------ C
        // stage C output slots of row ra - 2: registers (two rows deep for
        // scheme 1, four for scheme 3) and phi u rows (ring of NPU rows)
        constexpr int U2 = SCHEME == 3 ? SLOT : (SLOT & 1);
        const int P2 = SCHEME == 3 ? (it + 4) % G::NPU : S2;
        if (L.c && it >= G::NC) {
            const T* Mm = sm.mu[S3];
            const T* Mc = sm.mu[S2];
            const T* Mp = sm.mu[S1];
            const T gx = gradx9<T>(Mc[t + 1], Mc[t - 1], Mp[t + 1], Mp[t - 1], Mm[t + 1], Mm[t - 1]);
            const T gy = grady9<T>(Mp[t], Mm[t], Mp[t + 1], Mp[t - 1], Mm[t + 1], Mm[t - 1]);
            const T rho = c.rho_ref + R.drho[S2];
            const T k = T(1.0 / 3.0) - rho;
            const T Fx = k * gx, Fy = k * gy;
            const T inv = rcp_fast<T>(rho);
            const T ux = (R.jx[S2] + T(0.5) * Fx) * inv;
            const T uy = (R.jy[S2] + T(0.5) * Fy) * inv;
            const T phi = (rho - (c.c0 + Mc[t])) * T(1.0 / 3.0);
            sm.pux[P2][t] = phi * ux;
            sm.puy[P2][t] = phi * uy;
            R.ux[U2] = ux;
            R.uy[U2] = uy;
            R.Fx[U2] = Fx;
            R.Fy[U2] = Fy;
        }
        A_.sync();
        if constexpr (SCHEME == 3) {
            // -------------------------------------------------------- D (3)
            if (L.d && it >= G::ND)
                step_d_smooth<T, NT, COLL, EOS, NU, SLOT, COHERENT, ST>(it, fin, fout, c, L, rows, sm, R);
        } else {
        // ------------------------------------------------------------ D
        constexpr int U3 = (SLOT + 1) & 1;
        if (L.d && it >= G::ND) {
            const T* Am = sm.pux[S0];  // row ra - 4 shares slot S0 with row ra
            const T* Ac = sm.pux[S3];
            const T* Ap = sm.pux[S2];
            const T* Bm = sm.puy[S0];
            const T* Bp = sm.puy[S2];
            const T Ax = gradx9<T>(Ac[t + 1], Ac[t - 1], Ap[t + 1], Ap[t - 1], Am[t + 1], Am[t - 1]);
            const T By = grady9<T>(Bp[t], Bm[t], Bp[t + 1], Bp[t - 1], Bm[t + 1], Bm[t - 1]);
            const T C1 = Ax + By, C7 = Ax - By;
            const T drho = R.drho[S3];
            const T rho = c.rho_ref + drho;
            R.bad |= !rho_ok(rho);
            const T mu = sm.mu[S3][t];
            if constexpr (ST) node_stats(R, drho, rho, R.ux[U3], R.uy[U3]);
            T le = c.lam_e, ls = c.lam_s, lq = c.lam_q, lv = c.lam_v;
            if (NU) {
                lv = shear_rate<SCHEME, NU, T>(c, rho, mu);
                if (COLL == 0) le = ls = lq = lv;
            }
            collide<SCHEME, T>(R.f[S3], drho, rho, R.jx[S3], R.jy[S3], R.ux[U3], R.uy[U3], R.Fx[U3],
                               R.Fy[U3], mu, C1, C7, c.rho_ref, c.c0, le, ls, lq, lv);
            const uint32_t o = (uint32_t)rows.rd * pitch + L.xc;
#pragma unroll
            for (int a = 0; a < kQ; ++a) fout[a * P + o] = R.f[S3][a];
        }
        }
    } else {
        // ------------------------------------------------------- D (standard)
        if (L.d && it >= G::ND) {
            const T* Mm = sm.mu[S3];
            const T* Mc = sm.mu[S2];
            const T* Mp = sm.mu[S1];
            const T drho = R.drho[S2];
            const T rho = c.rho_ref + drho;
            R.bad |= !rho_ok(rho);
            T mu, Fx, Fy;
            if constexpr (SCHEME == 2) {
                // F = grad(rho/3) - div P, each component of P through Eq. 17
                const T* Xm = sm.pux[S3];
                const T* Xc = sm.pux[S2];
                const T* Xp = sm.pux[S1];
                const T* Ym = sm.puy[S3];
                const T* Yp = sm.puy[S1];
                const T divx = gradx9<T>(Mc[t + 1], Mc[t - 1], Mp[t + 1], Mp[t - 1], Mm[t + 1], Mm[t - 1]) +
                               grady9<T>(Xp[t], Xm[t], Xp[t + 1], Xp[t - 1], Xm[t + 1], Xm[t - 1]);
                const T divy = gradx9<T>(Xc[t + 1], Xc[t - 1], Xp[t + 1], Xp[t - 1], Xm[t + 1], Xm[t - 1]) +
                               grady9<T>(Yp[t], Ym[t], Yp[t + 1], Yp[t - 1], Ym[t + 1], Ym[t - 1]);
                mu = T(0);  // the standard collision does not use mu_c
                Fx = R.grx * T(1.0 / 3.0) - divx;
                Fy = R.gry * T(1.0 / 3.0) - divy;
            } else {
                const T gmx = gradx9<T>(Mc[t + 1], Mc[t - 1], Mp[t + 1], Mp[t - 1], Mm[t + 1], Mm[t - 1]);
                const T gmy = grady9<T>(Mp[t], Mm[t], Mp[t + 1], Mp[t - 1], Mm[t + 1], Mm[t - 1]);
                mu = Mc[t];
                Fx = R.grx * T(1.0 / 3.0) - rho * gmx;
                Fy = R.gry * T(1.0 / 3.0) - rho * gmy;
            }
            const T inv = rcp_fast<T>(rho);
            const T half = SCHEME == 4 ? T(0.5) * c.lw_dt : T(0.5);  // Lax-Wendroff: time step dt = A
            const T ux = (R.jx[S2] + half * Fx) * inv;
            const T uy = (R.jy[S2] + half * Fy) * inv;
            if constexpr (ST) node_stats(R, drho, rho, ux, uy);
            if constexpr (SCHEME == 4) {
                collide_lw<T>(R.f[S2], drho, rho, ux, uy, Fx, Fy, c);
            } else {
                T le = c.lam_e, ls = c.lam_s, lq = c.lam_q, lv = c.lam_v;
                if (NU) {
                    lv = shear_rate<SCHEME, NU, T>(c, rho, mu);
                    if (COLL == 0) le = ls = lq = lv;
                }
                collide<SCHEME, T>(R.f[S2], drho, rho, R.jx[S2], R.jy[S2], ux, uy, Fx, Fy, mu, T(0), T(0),
                                   c.rho_ref, c.c0, le, ls, lq, lv);
            }
            const uint32_t o = (uint32_t)rows.rd * pitch + L.xc;
#pragma unroll
            for (int a = 0; a < kQ; ++a) fout[a * P + o] = R.f[S2][a];
        }
    }
    rows.ra = inc_wrap(rows.ra, ny);
    rows.sa += 1;
    if (it >= G::ND) rows.rd = inc_wrap(rows.rd, ny);
}

// One work item of one time step (the body of step_kernel): the block walks
// the item's rows through stages A-D, reading fin and writing fout, and
// returns whether a stage D node had rho <= 0 or a non-finite density (the
// same value in every thread). COHERENT selects L2-only population loads; ST
// accumulates the thread's statistics of its stage D nodes into acc.
template <typename T, int NT, int SCHEME, int COLL, int EOS, bool NU, bool COHERENT, bool ST = false>
__device__ __forceinline__ bool step_item(const T* __restrict__ fin, T* __restrict__ fout, const DevCase<T>& c,
                                          const Item& item, StepSmem<T, NT, SCHEME>& sm, StepAcc<T>& acc)
{
    using G = StepGeom<SCHEME>;
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

    StepRows rows;
    rows.ra = wrapi(item.y0 - G::HX, c.ny);
    rows.rd = item.y0;
    rows.sa = item.y0 - G::HX;

    StepRegs<T> R;
    R.bad = false;
    R.am = R.ak = R.au = T(0);
    const int niter = item.h + 2 * G::HX;
    const PullGlobal<T, COHERENT> A;
    for (int base = 0; base < niter; base += 4) {
        step_iter<T, NT, SCHEME, COLL, EOS, NU, 0, PullGlobal<T, COHERENT>, COHERENT, ST>(base, A, fin, fout, c, L, rows,
                                                                                     sm, R);
        if (base + 1 >= niter) break;
        step_iter<T, NT, SCHEME, COLL, EOS, NU, 1, PullGlobal<T, COHERENT>, COHERENT, ST>(base + 1, A, fin, fout, c, L,
                                                                                     rows, sm, R);
        if (base + 2 >= niter) break;
        step_iter<T, NT, SCHEME, COLL, EOS, NU, 2, PullGlobal<T, COHERENT>, COHERENT, ST>(base + 2, A, fin, fout, c, L,
                                                                                     rows, sm, R);
        if (base + 3 >= niter) break;
        step_iter<T, NT, SCHEME, COLL, EOS, NU, 3, PullGlobal<T, COHERENT>, COHERENT, ST>(base + 3, A, fin, fout, c, L,
                                                                                     rows, sm, R);
    }
    acc.am = R.am;
    acc.ak = R.ak;
    acc.au = R.au;
    return __syncthreads_or(R.bad) != 0;
}

// One launch advances every case listed in the work-list by one time step.
// fin/fout: population buffers (all cases, each at DevCase::off). One block
// per work item; blockDim.x == NT. status[0]: set by a bounded wait that gave
// up (TMA variants); status[1 + case]: set when a node of the case had
// rho <= 0 or a non-finite density in stage D. The blocks of a flagged case
// return at once, so it no longer advances while the other cases go on.
// ST: the variant that also records the per-step statistics (stage D sums,
// stats_block) of the cases whose record has st_hist != 0.
template <typename T, int NT, int SCHEME, int COLL, int EOS, bool NU, bool ST = false>
__global__ void __launch_bounds__(NT) step_kernel(const T* __restrict__ fin, T* __restrict__ fout,
                                                  const DevCase<T>* __restrict__ cases,
                                                  const Item* __restrict__ items, int* __restrict__ status)
{
    __shared__ StepSmem<T, NT, SCHEME> sm;
    const Item item = items[blockIdx.x];
    // thread 0 decides for the block: another block may set the word meanwhile
    if (__syncthreads_or(threadIdx.x == 0 && status[1 + item.case_id] != 0)) return;
    const DevCase<T> c = cases[item.case_id];
    StepAcc<T> acc;
    const bool bad = step_item<T, NT, SCHEME, COLL, EOS, NU, false, ST>(fin, fout, c, item, sm, acc);
    if (bad && threadIdx.x == 0) atomicOr(status + 1 + item.case_id, 1);
    if (ST && c.st_hist)
        stats_block(c, (double)acc.am, (double)acc.ak, (double)acc.au,
                    (unsigned long long)item.wv * (unsigned long long)item.h);
}

}  // namespace lbfe
