// Fused step for short periodic lattices (ny <= kRowsMax): a block owns a
// strip of NT columns over the lattice's whole height and gives every node of
// the strip its own thread (RPT rows per thread when the strip is taller than
// one pass of threads). The stages of step_kernel.cuh (A pull, rho, j;
// B mu_c; C grad mu_c, F, u, phi u; D correction, collision, store) run one
// after the other with a block barrier between them, the fields that a
// neighbour reads (rho, mu_c, phi u) in shared memory and the rest (the
// pulled populations, j, u, F, mu_c) in the node's registers. Each node of a
// stage is computed once per step and the critical path of a step is one
// pull plus the stage arithmetic of one node; the sliding window of
// step_kernel.cuh instead walks ny + 2 HX rows as a chain of dependent row
// iterations, and with the short segments that its latency favours on small
// lattices it recomputes most rows of stages A-C several times. Schemes
// 0-3 (the chemical-potential forces, the pressure-tensor force, and scheme
// 3's Eq. 29 derivatives of the lattice-weight average of phi u), periodic
// lattices.
#pragma once

#include "step_kernel.cuh"

namespace lbfe {

constexpr int kRowsMax = 16;      // tallest lattice this kernel runs
constexpr int kRowsCols = 64;     // NT: columns per block (strip of NT - 2 HX output columns)
constexpr int kRowsPassMax = 8;   // rows of threads per block at most (blockDim.x <= NT * 8)

// Threads per block and rows per thread for a group whose tallest lattice has
// ny_max rows: one pass of ny_max rows of threads when it fits, else two rows
// per thread.
__host__ __device__ constexpr int rows_per_thread(int ny_max) { return ny_max <= kRowsPassMax ? 1 : 2; }
__host__ __device__ constexpr int rows_pass(int ny_max)
{
    return (ny_max + rows_per_thread(ny_max) - 1) / rows_per_thread(ny_max);
}

// Shared memory of a block: rho, mu_c, phi u_x, phi u_y (the last two for
// the improved schemes), or rho, P_xx, P_xy, P_yy (the pressure-tensor force),
// or rho and mu_c (the standard scheme); each [rows_pass * RPT][NT].
template <typename T, int SCHEME>
__host__ __device__ constexpr size_t rows_dynamic_smem(int ny_max)
{
    return (size_t)(SCHEME == 0 ? 2 : 4) * rows_pass(ny_max) * rows_per_thread(ny_max) * kRowsCols * sizeof(T);
}

// Same contract as step_kernel (one block per work item, status words,
// frozen cases return at once); blockDim.x == NT * RY with RY * RPT >= ny of
// every case of the launch, every item spans the whole height of its case
// (y0 == 0, h == ny <= kRowsMax) and wv + 2 HX <= NT. ST: also records the
// per-step statistics of cases with st_hist != 0.
template <typename T, int NT, int RPT, int SCHEME, int COLL, int EOS, bool NU, bool ST = false>
__global__ void __launch_bounds__(NT * kRowsPassMax, sizeof(T) == 4 ? 2 : 1)
    step_kernel_rows(const T* __restrict__ fin, T* __restrict__ fout, const DevCase<T>* __restrict__ cases,
                     const Item* __restrict__ items, int* __restrict__ status)
{
    static_assert(SCHEME >= 0 && SCHEME <= 3, "the row kernel runs schemes 0-3");
    constexpr int HX = StepGeom<SCHEME>::HX;
    extern __shared__ __align__(16) unsigned char rows_dsm[];
    const Item item = items[blockIdx.x];
    // a case flagged unstable no longer advances (thread 0 decides for the block)
    if (__syncthreads_or(threadIdx.x == 0 && status[1 + item.case_id] != 0)) return;
    const DevCase<T> c = cases[item.case_id];
    fin += c.off;
    fout += c.off;
    const int ny = c.ny;
    const int t = (int)(threadIdx.x % NT), ty = (int)(threadIdx.x / NT), RY = (int)(blockDim.x / NT);
    const int stride = RY * RPT * NT;  // words of one shared field
    T* const s_rho = reinterpret_cast<T*>(rows_dsm);
    T* const s_mu = s_rho + stride;  // mu_c, or P_xx (scheme 2)
    T* const s_ax = s_mu + stride;   // phi u_x, phi u_y (schemes 1 and 3), or P_xy, P_yy (scheme 2)
    T* const s_ay = s_ax + stride;
    const int span = item.wv + 2 * HX;  // active columns of the strip
    const int xw = item.x0 - HX + t;
    StepLane L;
    L.t = t;
    L.xc = wrapi(xw, c.nx);
    L.xm = wrapi(xw - 1, c.nx);
    L.xp = wrapi(xw + 1, c.nx);
    const bool in_a = t < span, in_b = t >= 1 && t < span - 1, in_c = t >= 2 && t < span - 2,
               in_d = t >= HX && t < span - HX;
    const PullGlobal<T> pull;

    int yk[RPT];
    bool vk[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        yk[k] = ty + k * RY;
        vk[k] = yk[k] < ny;
    }
    T F[RPT][kQ], dr[RPT], jx[RPT], jy[RPT], mu[RPT], ux[RPT], uy[RPT], fx[RPT], fy[RPT];

    // ---------------------------------------------------------------- A
#pragma unroll
    for (int k = 0; k < RPT; ++k)
        if (in_a && vk[k]) {
            const int y = yk[k];
            T* G = F[k];
            const StepRows rows{y, y, y};
            pull.pull(0, G, fin, c, L, rows);
            dr[k] = ((G[0] + (G[1] + G[3])) + (G[2] + G[4])) + ((G[5] + G[7]) + (G[6] + G[8]));
            jx[k] = (G[1] - G[3]) + ((G[5] - G[7]) + (G[8] - G[6]));
            jy[k] = (G[2] - G[4]) + ((G[5] - G[7]) + (G[6] - G[8]));
            s_rho[y * NT + t] = c.rho_ref + dr[k];
        }
    __syncthreads();

    // ---------------------------------------------------------------- B
#pragma unroll
    for (int k = 0; k < RPT; ++k)
        if (in_b && vk[k]) {
            const int y = yk[k];
            const T* Sm = s_rho + dec_wrap(y, ny) * NT;
            const T* Sc = s_rho + y * NT;
            const T* Sp = s_rho + inc_wrap(y, ny) * NT;
            const T rc = Sc[t];
            const T lap = lap9<T>(rc, Sc[t + 1], Sc[t - 1], Sp[t], Sm[t], Sp[t + 1], Sp[t - 1], Sm[t + 1],
                                  Sm[t - 1]);
            if constexpr (SCHEME == 2) {
                // the pressure tensor of Eqs. 4-5 (P_xx in the mu_c field)
                const T gx = gradx9<T>(Sc[t + 1], Sc[t - 1], Sp[t + 1], Sp[t - 1], Sm[t + 1], Sm[t - 1]);
                const T gy = grady9<T>(Sp[t], Sm[t], Sp[t + 1], Sp[t - 1], Sm[t + 1], Sm[t - 1]);
                T Pxx, Pxy, Pyy;
                pressure_tensor<T>(pEOS<EOS, T>(c, rc), rc, gx, gy, lap, c.kappa, Pxx, Pxy, Pyy);
                mu[k] = T(0);  // the standard collision does not use mu_c
                s_mu[y * NT + t] = Pxx;
                s_ax[y * NT + t] = Pxy;
                s_ay[y * NT + t] = Pyy;
            } else {
                mu[k] = dEf<EOS, T>(c, rc) - c.kappa * lap;
                s_mu[y * NT + t] = mu[k];
            }
        }
    __syncthreads();

    // ---------------------------------------------------------------- C
    // improved schemes: F = (1/3 - rho) grad mu_c, u, and phi u for the
    // correction terms of stage D; the standard scheme takes its force in D
    if constexpr (improved_scheme(SCHEME)) {
#pragma unroll
        for (int k = 0; k < RPT; ++k)
            if (in_c && vk[k]) {
                const int y = yk[k];
                const T* Mm = s_mu + dec_wrap(y, ny) * NT;
                const T* Mc = s_mu + y * NT;
                const T* Mp = s_mu + inc_wrap(y, ny) * NT;
                const T gx = gradx9<T>(Mc[t + 1], Mc[t - 1], Mp[t + 1], Mp[t - 1], Mm[t + 1], Mm[t - 1]);
                const T gy = grady9<T>(Mp[t], Mm[t], Mp[t + 1], Mp[t - 1], Mm[t + 1], Mm[t - 1]);
                const T rho = c.rho_ref + dr[k];
                const T kf = T(1.0 / 3.0) - rho;
                fx[k] = kf * gx;
                fy[k] = kf * gy;
                const T inv = rcp_fast<T>(rho);
                ux[k] = (jx[k] + T(0.5) * fx[k]) * inv;
                uy[k] = (jy[k] + T(0.5) * fy[k]) * inv;
                const T phi = (rho - (c.c0 + mu[k])) * T(1.0 / 3.0);
                s_ax[y * NT + t] = phi * ux[k];
                s_ay[y * NT + t] = phi * uy[k];
            }
        __syncthreads();
    }

    // ---------------------------------------------------------------- D
    bool bad = false;
    T am = T(0), ak = T(0), au = T(0);
    const uint32_t P = (uint32_t)c.plane;
#pragma unroll
    for (int k = 0; k < RPT; ++k)
        if (in_d && vk[k]) {
            const int y = yk[k], ym = dec_wrap(y, ny), yp = inc_wrap(y, ny);
            const T drho = dr[k];
            const T rho = c.rho_ref + drho;
            bad |= !rho_ok(rho);
            T C1 = T(0), C7 = T(0);
            if constexpr (SCHEME == 1) {
                const T* Am = s_ax + ym * NT;
                const T* Ac = s_ax + y * NT;
                const T* Ap = s_ax + yp * NT;
                const T* Bm = s_ay + ym * NT;
                const T* Bp = s_ay + yp * NT;
                const T Ax = gradx9<T>(Ac[t + 1], Ac[t - 1], Ap[t + 1], Ap[t - 1], Am[t + 1], Am[t - 1]);
                const T By = grady9<T>(Bp[t], Bm[t], Bp[t + 1], Bp[t - 1], Bm[t + 1], Bm[t - 1]);
                C1 = Ax + By;
                C7 = Ax - By;
            } else if constexpr (SCHEME == 3) {
                // the derivatives of the lattice-weight averages A' = sum_a
                // w_a (phi u_x)(x + e_a), B' likewise, through the factored
                // 5 x 5 stencil of step_d_smooth (same order of operations):
                //   d_x A' = sum_dy s(dy) [(A(x+1) - A(x-1))/3 + (A(x+2) - A(x-2))/12](y + dy)
                // with s = (1, 8, 18, 8, 1)/36, d_y B' with x and y exchanged;
                // rows y - 2 .. y + 2 wrap periodically within the strip
                const int yr[5] = {dec_wrap(ym, ny), ym, y, yp, inc_wrap(yp, ny)};
                const T s0 = T(1.0 / 36.0), s1 = T(8.0 / 36.0), s2 = T(18.0 / 36.0);
                const T g1 = T(1.0 / 3.0), g2 = T(1.0 / 12.0);
                T hx[5], sb[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    const T* a = s_ax + yr[q] * NT;
                    hx[q] = g1 * (a[t + 1] - a[t - 1]) + g2 * (a[t + 2] - a[t - 2]);
                    const T* b = s_ay + yr[q] * NT;
                    sb[q] = s0 * (b[t - 2] + b[t + 2]) + s1 * (b[t - 1] + b[t + 1]) + s2 * b[t];
                }
                const T Ax = s0 * (hx[0] + hx[4]) + s1 * (hx[1] + hx[3]) + s2 * hx[2];
                const T By = g1 * (sb[3] - sb[1]) + g2 * (sb[4] - sb[0]);
                C1 = Ax + By;
                C7 = Ax - By;
            } else {
                // standard scheme: F = grad(rho) / 3 - rho grad mu_c
                const T* Qm = s_rho + ym * NT;
                const T* Qc = s_rho + y * NT;
                const T* Qp = s_rho + yp * NT;
                const T* Mm = s_mu + ym * NT;
                const T* Mc = s_mu + y * NT;
                const T* Mp = s_mu + yp * NT;
                const T grx = gradx9<T>(Qc[t + 1], Qc[t - 1], Qp[t + 1], Qp[t - 1], Qm[t + 1], Qm[t - 1]);
                const T gry = grady9<T>(Qp[t], Qm[t], Qp[t + 1], Qp[t - 1], Qm[t + 1], Qm[t - 1]);
                if constexpr (SCHEME == 2) {
                    // F = grad(rho/3) - div P, each component of P through Eq. 17
                    const T* Xm = s_ax + ym * NT;
                    const T* Xc = s_ax + y * NT;
                    const T* Xp = s_ax + yp * NT;
                    const T* Ym = s_ay + ym * NT;
                    const T* Yp = s_ay + yp * NT;
                    const T divx = gradx9<T>(Mc[t + 1], Mc[t - 1], Mp[t + 1], Mp[t - 1], Mm[t + 1], Mm[t - 1]) +
                                   grady9<T>(Xp[t], Xm[t], Xp[t + 1], Xp[t - 1], Xm[t + 1], Xm[t - 1]);
                    const T divy = gradx9<T>(Xc[t + 1], Xc[t - 1], Xp[t + 1], Xp[t - 1], Xm[t + 1], Xm[t - 1]) +
                                   grady9<T>(Yp[t], Ym[t], Yp[t + 1], Yp[t - 1], Ym[t + 1], Ym[t - 1]);
                    fx[k] = grx * T(1.0 / 3.0) - divx;
                    fy[k] = gry * T(1.0 / 3.0) - divy;
                } else {
                    const T gmx = gradx9<T>(Mc[t + 1], Mc[t - 1], Mp[t + 1], Mp[t - 1], Mm[t + 1], Mm[t - 1]);
                    const T gmy = grady9<T>(Mp[t], Mm[t], Mp[t + 1], Mp[t - 1], Mm[t + 1], Mm[t - 1]);
                    fx[k] = grx * T(1.0 / 3.0) - rho * gmx;
                    fy[k] = gry * T(1.0 / 3.0) - rho * gmy;
                }
                const T inv = rcp_fast<T>(rho);
                ux[k] = (jx[k] + T(0.5) * fx[k]) * inv;
                uy[k] = (jy[k] + T(0.5) * fy[k]) * inv;
            }
            if constexpr (ST) {
                const T u2 = ux[k] * ux[k] + uy[k] * uy[k];
                am += drho;
                ak += rho * u2;
                au = u2 > au ? u2 : au;
            }
            T le = c.lam_e, ls = c.lam_s, lq = c.lam_q, lv = c.lam_v;
            if (NU) {
                lv = shear_rate<SCHEME, NU, T>(c, rho, mu[k]);
                if (COLL == 0) le = ls = lq = lv;
            }
            collide<SCHEME, T>(F[k], drho, rho, jx[k], jy[k], ux[k], uy[k], fx[k], fy[k], mu[k], C1, C7,
                               c.rho_ref, c.c0, le, ls, lq, lv);
            const uint32_t o = (uint32_t)y * c.pitch + L.xc;
#pragma unroll
            for (int a = 0; a < kQ; ++a) fout[a * P + o] = F[k][a];
        }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status + 1 + item.case_id, 1);
    if (ST && c.st_hist)
        stats_block(c, (double)am, (double)ak, (double)au, (unsigned long long)item.wv * (unsigned long long)ny);
}

}  // namespace lbfe
