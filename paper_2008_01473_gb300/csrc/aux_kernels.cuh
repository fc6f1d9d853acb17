// Kernels around the time step: initial populations, macroscopic-field
// export and the per-case FP64 reductions. They run once per call, not per
// step, through scratch fields of type C in the workspace: C is the storage
// precision of the populations (per-node arithmetic in C; every sum over the
// lattice in FP64).
//
// Launch shape of the per-node kernels: 256-thread blocks over
// field_grid(nx, ny); thread x of block (bx, by) handles column
// 256 bx + x of the kFieldRows rows from kFieldRows by, so that a thread
// accumulates its sums over several nodes in FP64 registers and each block
// reduces once. Neighbour rows and columns wrap by comparison, not by
// integer division.
#pragma once

#include "lbfe_device.cuh"

namespace lbfe {

constexpr int kFieldRows = 16;  // rows per block of the per-node field kernels

inline dim3 field_grid(int nx, int ny) { return dim3((nx + 255) / 256, (ny + kFieldRows - 1) / kFieldRows); }

// periodic neighbour columns, and neighbour rows (periodic, or mirrored in a wall)
__device__ __forceinline__ int col_m1(int x, int nx) { return x == 0 ? nx - 1 : x - 1; }
__device__ __forceinline__ int col_p1(int x, int nx) { return x + 1 == nx ? 0 : x + 1; }
template <typename T>
__device__ __forceinline__ int row_m1(const DevCase<T>& c, int y)
{
    return y > 0 ? y - 1 : (c.walls ? 0 : c.ny - 1);
}
template <typename T>
__device__ __forceinline__ int row_p1(const DevCase<T>& c, int y)
{
    return y + 1 < c.ny ? y + 1 : (c.walls ? c.ny - 1 : 0);
}

// Per-block partial sums: mass (or any sum), kinetic energy, max |u|^2 and a
// count of non-physical nodes.
struct Partial {
    double mass, ke, umax2, bad;
};

// Block reduction of one Partial per thread (blockDim.x == 256) into
// partials[block index]: stored, or with ADD added to the slot (its sums;
// the max is kept), so that one slot per block accumulates over many
// launches of the same grid in launch order.
template <bool ADD = false>
__device__ __forceinline__ void block_partial(double mass, double ke, double um, double bad,
                                              Partial* __restrict__ partials)
{
    __shared__ double s[4][8];
    for (int o = 16; o > 0; o >>= 1) {
        mass += __shfl_xor_sync(0xffffffffu, mass, o);
        ke += __shfl_xor_sync(0xffffffffu, ke, o);
        um = fmax(um, __shfl_xor_sync(0xffffffffu, um, o));
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s[0][w] = mass;
        s[1][w] = ke;
        s[2][w] = um;
        s[3][w] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Partial p{0.0, 0.0, 0.0, 0.0};
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            p.mass += s[0][k];
            p.ke += s[1][k];
            p.umax2 = fmax(p.umax2, s[2][k]);
            p.bad += s[3][k];
        }
        Partial& q = partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x];
        if (ADD) {
            q.mass += p.mass;
            q.ke += p.ke;
            q.umax2 = fmax(q.umax2, p.umax2);
            q.bad += p.bad;
        } else {
            q = p;
        }
    }
}

// Block reduction of per-thread accumulators (blockDim.x == 256, every
// thread calls it) into partials[block index]: sums of mass and kinetic
// energy, max |u|^2 and the count of non-physical nodes.
__device__ __forceinline__ void block_sums(double mass, double ke, double um2, int bad,
                                           Partial* __restrict__ partials)
{
    __shared__ double s[3][8];
    __shared__ int sb[8];
    for (int o = 16; o > 0; o >>= 1) {
        mass += __shfl_xor_sync(0xffffffffu, mass, o);
        ke += __shfl_xor_sync(0xffffffffu, ke, o);
        um2 = fmax(um2, __shfl_xor_sync(0xffffffffu, um2, o));
    }
    bad = __reduce_add_sync(0xffffffffu, bad);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s[0][w] = mass;
        s[1][w] = ke;
        s[2][w] = um2;
        sb[w] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Partial p{0.0, 0.0, 0.0, 0.0};
        int nb = 0;
        for (int k = 0; k < 8; ++k) {
            p.mass += s[0][k];
            p.ke += s[1][k];
            p.umax2 = fmax(p.umax2, s[2][k]);
            nb += sb[k];
        }
        p.bad = (double)nb;
        partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = p;
    }
}

// Copy the initial density (FP64, or FP32: I) into C scratch and check it:
// one Partial per block with the sum of rho0 (FP64) and the count of values
// that are not finite, not > 0, or outside the EOS domain (b rho < 1 for
// vdW, b rho / 4 < 1 for CS).
template <typename C, typename I = double>
__global__ void __launch_bounds__(256) rho0_kernel(int nx, int ny, int eos, double b,
                                                   const I* __restrict__ rho0, C* __restrict__ out,
                                                   Partial* __restrict__ partials)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y0 = blockIdx.y * kFieldRows, y1 = min(ny, y0 + kFieldRows);
    const double bl = eos == 0 ? b : 0.25 * b;
    double sum = 0.0;
    int bad = 0;
    if (x < nx)
        for (int y = y0; y < y1; ++y) {
            const int64_t i = (int64_t)y * nx + x;
            const double r = (double)rho0[i];
            const bool ok = r > 0.0 && r <= 1.7976931348623157e308 && bl * r < 1.0;
            sum += ok ? r : 0.0;
            bad += ok ? 0 : 1;
            out[i] = (C)r;
        }
    block_sums(sum, 0.0, 0.0, bad, partials);
}

// mu_c = E_f'(rho) - kappa lap(rho) on a C field (Eq. 2).
template <typename C, int EOS>
__global__ void __launch_bounds__(256) mu_field_kernel(DevCase<C> c, const C* __restrict__ rho, C* __restrict__ mu)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= c.nx) return;
    const int nx = c.nx;
    const int xm = col_m1(x, nx), xp = col_p1(x, nx);
    const int y0 = blockIdx.y * kFieldRows, y1 = min(c.ny, y0 + kFieldRows);
    for (int y = y0; y < y1; ++y) {
        const int64_t ym = (int64_t)row_m1(c, y) * nx, yc = (int64_t)y * nx, yp = (int64_t)row_p1(c, y) * nx;
        const C Cc = rho[yc + x];
        const C lap = lap9<C>(Cc, rho[yc + xp], rho[yc + xm], rho[yp + x], rho[ym + x], rho[yp + xp],
                              rho[yp + xm], rho[ym + xp], rho[ym + xm]);
        mu[yc + x] = dEf<EOS, C>(c, Cc) - c.kappa * lap;
    }
}

// Pressure tensor P of Eqs. 4-5 on C fields (pressure-tensor force form).
template <typename C, int EOS>
__global__ void __launch_bounds__(256) ptensor_kernel(DevCase<C> c, const C* __restrict__ rho, C* __restrict__ pxx,
                                                      C* __restrict__ pxy, C* __restrict__ pyy)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= c.nx) return;
    const int nx = c.nx;
    const int xm = col_m1(x, nx), xp = col_p1(x, nx);
    const int y0 = blockIdx.y * kFieldRows, y1 = min(c.ny, y0 + kFieldRows);
    for (int y = y0; y < y1; ++y) {
        const int64_t ym = (int64_t)row_m1(c, y) * nx, yc = (int64_t)y * nx, yp = (int64_t)row_p1(c, y) * nx;
        const C Cc = rho[yc + x];
        const C lap = lap9<C>(Cc, rho[yc + xp], rho[yc + xm], rho[yp + x], rho[ym + x], rho[yp + xp],
                              rho[yp + xm], rho[ym + xp], rho[ym + xm]);
        const C gx = gradx9<C>(rho[yc + xp], rho[yc + xm], rho[yp + xp], rho[yp + xm], rho[ym + xp], rho[ym + xm]);
        const C gy = grady9<C>(rho[yp + x], rho[ym + x], rho[yp + xp], rho[yp + xm], rho[ym + xp], rho[ym + xm]);
        C a, b, d;
        pressure_tensor<C>(pEOS<EOS, C>(c, Cc), Cc, gx, gy, lap, c.kappa, a, b, d);
        pxx[yc + x] = a;
        pxy[yc + x] = b;
        pyy[yc + x] = d;
    }
}

// f(0) = M^-1 m_eq(rho0, u0) with mu_c of rho0, stored as f - w rho_ref in T.
template <typename T, int SCHEME, typename C>
__device__ __forceinline__ void init_node(const DevCase<T>& c, const DevCase<C>& cc, const C* __restrict__ rho0,
                                          const double* __restrict__ ux0, const double* __restrict__ uy0,
                                          const C* __restrict__ mu0, T* __restrict__ f, int x, int y)
{
    const int64_t i = (int64_t)y * c.nx + x;
    const C rho = rho0[i];
    const C ux = ux0 ? (C)ux0[i] : C(0), uy = uy0 ? (C)uy0[i] : C(0);
    const C rr = cc.rho_ref;
    // with all deviation moments zero, the collision with rates 1 and no
    // force returns exactly M^-1 of the equilibrium (minus w rho_ref); the
    // conserved entries come from drho and rho u directly
    C d[kQ];
    for (int a = 0; a < kQ; ++a) d[a] = C(0);
    collide<SCHEME, C>(d, rho - rr, rho, rho * ux, rho * uy, ux, uy, C(0), C(0), mu0[i], C(0), C(0), rr, cc.c0,
                       C(1), C(1), C(1), C(1));
    if (c.lw_dt > T(0)) {
        // Lax-Wendroff scheme: at step 0 the storage holds f(0) at its own
        // node (the first step pulls it without Eq. A2's propagation)
        const int64_t o = (int64_t)y * c.pitch + x;
        for (int a = 0; a < kQ; ++a) f[c.off + a * c.plane + o] = (T)d[a];
        return;
    }
    // Storage holds post-collision populations before streaming (the step
    // pulls f_a(x) from x - e_a), so f_a(0) of node x is stored at x - e_a.
    constexpr int ex[kQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    constexpr int ey[kQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const int xs[3] = {col_p1(x, c.nx), x, col_m1(x, c.nx)};  // x - e for e = -1, 0, 1
    const bool wall_m = c.walls && y == 0, wall_p = c.walls && y == c.ny - 1;
    const int ysv[3] = {y + 1 == c.ny ? 0 : y + 1, y, y == 0 ? c.ny - 1 : y - 1};
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        if ((ey[a] == 1 && wall_m) || (ey[a] == -1 && wall_p)) continue;  // these arrive from a wall
        const int64_t o = (int64_t)ysv[ey[a] + 1] * c.pitch + xs[ex[a] + 1];
        f[c.off + a * c.plane + o] = (T)d[a];
    }
    if (c.walls) {
        // A population that enters from a wall is the node's own outgoing one
        // in the opposite direction plus the moving-wall term (+-wall_d on the
        // diagonals); store those outgoing slots so that the first pull
        // returns f_a(0). No other node writes them.
        const int64_t o = (int64_t)y * c.pitch + x;
        const C w = (C)cc.wall_d;
        if (y == 0) {
            f[c.off + 4 * c.plane + o] = (T)d[2];
            f[c.off + 7 * c.plane + o] = (T)(d[5] - w);
            f[c.off + 8 * c.plane + o] = (T)(d[6] + w);
        }
        if (y == c.ny - 1) {
            f[c.off + 2 * c.plane + o] = (T)d[4];
            f[c.off + 5 * c.plane + o] = (T)(d[7] + w);
            f[c.off + 6 * c.plane + o] = (T)(d[8] - w);
        }
    }
}

template <typename T, int SCHEME, typename C>
__global__ void __launch_bounds__(256) init_kernel(DevCase<T> c, DevCase<C> cc, const C* __restrict__ rho0,
                                                   const double* __restrict__ ux0, const double* __restrict__ uy0,
                                                   const C* __restrict__ mu0, T* __restrict__ f)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= c.nx) return;
    const int y0 = blockIdx.y * kFieldRows, y1 = min(c.ny, y0 + kFieldRows);
    for (int y = y0; y < y1; ++y) init_node<T, SCHEME, C>(c, cc, rho0, ux0, uy0, mu0, f, x, y);
}

// Pull the populations of the current state into C fields rho, j_x, j_y.
template <typename T, typename C>
__global__ void __launch_bounds__(256) pull_moments_kernel(DevCase<T> c, const T* __restrict__ f,
                                                           C* __restrict__ rho, C* __restrict__ jx,
                                                           C* __restrict__ jy)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= c.nx) return;
    const int nx = c.nx, ny = c.ny, pitch = c.pitch;
    const int64_t P = c.plane;
    f += c.off;
    const int xm = col_m1(x, nx), xp = col_p1(x, nx);
    const int y0 = blockIdx.y * kFieldRows, y1 = min(ny, y0 + kFieldRows);
    for (int y = y0; y < y1; ++y) {
        const int64_t rm = (int64_t)(y == 0 ? ny - 1 : y - 1) * pitch, r0 = (int64_t)y * pitch,
                      rp = (int64_t)(y + 1 == ny ? 0 : y + 1) * pitch;
        C F[kQ];
        if (c.lw_dt > T(0)) {
            // Lax-Wendroff scheme: the three-point propagation of Eq. A2 (at
            // step 0 the stored values are f(0) itself)
            constexpr int ex[kQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
            constexpr int ey[kQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
            const int64_t rr[3] = {rm, r0, rp};
            const int xs[3] = {xm, x, xp};
            const T a0 = c.lw_first ? T(1) : c.lw_a0, a1 = c.lw_first ? T(0) : c.lw_a1;
            const T am1 = c.lw_first ? T(0) : c.lw_am1;
            for (int a = 0; a < kQ; ++a)
                F[a] = (C)(a0 * f[a * P + r0 + x] + a1 * f[a * P + rr[1 + ey[a]] + xs[1 + ex[a]]] +
                           am1 * f[a * P + rr[1 - ey[a]] + xs[1 - ex[a]]]);
        } else {
            F[0] = (C)f[0 * P + r0 + x];
            F[1] = (C)f[1 * P + r0 + xm];
            F[2] = (C)f[2 * P + rm + x];
            F[3] = (C)f[3 * P + r0 + xp];
            F[4] = (C)f[4 * P + rp + x];
            F[5] = (C)f[5 * P + rm + xm];
            F[6] = (C)f[6 * P + rm + xp];
            F[7] = (C)f[7 * P + rp + xp];
            F[8] = (C)f[8 * P + rp + xm];
        }
        if (c.walls && y == 0) {  // bounce-back from the bottom wall
            F[2] = (C)f[4 * P + r0 + x];
            F[5] = (C)(f[7 * P + r0 + x] + c.wall_d);
            F[6] = (C)(f[8 * P + r0 + x] - c.wall_d);
        }
        if (c.walls && y == ny - 1) {  // and from the top wall
            F[4] = (C)f[2 * P + r0 + x];
            F[7] = (C)(f[5 * P + r0 + x] - c.wall_d);
            F[8] = (C)(f[6 * P + r0 + x] + c.wall_d);
        }
        const C dr = ((F[0] + (F[1] + F[3])) + (F[2] + F[4])) + ((F[5] + F[7]) + (F[6] + F[8]));
        const int64_t i = (int64_t)y * nx + x;
        rho[i] = (C)c.rho_ref + dr;
        jx[i] = (F[1] - F[3]) + ((F[5] - F[7]) + (F[8] - F[6]));
        jy[i] = (F[2] - F[4]) + ((F[5] - F[7]) + (F[6] - F[8]));
    }
}

// Velocity of Eq. 12 from rho, j and the force of the case's scheme; writes
// the requested outputs (FP64, or FP32: O) and one Partial per block
// (blockDim.x == 256, grid field_grid(nx, ny)): per-node arithmetic in C, the
// thread's sums over its kFieldRows nodes in FP64 registers, max |u|^2 in C,
// the bad-node count as an integer. SCHEME 2 takes its force from the
// pressure tensor P (pxx, pxy, pyy).
template <int SCHEME, typename C, typename O = double>
__global__ void __launch_bounds__(256) velocity_kernel(DevCase<C> cc, const C* __restrict__ rho,
                                                       const C* __restrict__ jx, const C* __restrict__ jy,
                                                       const C* __restrict__ mu, const C* __restrict__ pxx,
                                                       const C* __restrict__ pxy, const C* __restrict__ pyy,
                                                       O* __restrict__ out_rho, O* __restrict__ out_ux,
                                                       O* __restrict__ out_uy, O* __restrict__ out_mu,
                                                       Partial* __restrict__ partials)
{
    const int nx = cc.nx, ny = cc.ny;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y0 = blockIdx.y * kFieldRows, y1 = min(ny, y0 + kFieldRows);
    double mass = 0.0, ke = 0.0;
    C um2 = C(0);
    int bad = 0;
    if (x < nx) {
        const int xm = col_m1(x, nx), xp = col_p1(x, nx);
        for (int y = y0; y < y1; ++y) {
            const int64_t ym = (int64_t)row_m1(cc, y) * nx, yc = (int64_t)y * nx, yp = (int64_t)row_p1(cc, y) * nx;
            const int64_t i = yc + x;
            // across a wall P_xy continues oddly (the mirrored rows' y
            // gradients change sign), every other field evenly
            const C sxm = cc.walls && y == 0 ? C(-1) : C(1), sxp = cc.walls && y == ny - 1 ? C(-1) : C(1);
            const C r = rho[i];
            const C gmx = gradx9<C>(mu[yc + xp], mu[yc + xm], mu[yp + xp], mu[yp + xm], mu[ym + xp], mu[ym + xm]);
            const C gmy = grady9<C>(mu[yp + x], mu[ym + x], mu[yp + xp], mu[yp + xm], mu[ym + xp], mu[ym + xm]);
            C Fx, Fy;
            if (SCHEME == 1) {
                Fx = (C(1.0 / 3.0) - r) * gmx;
                Fy = (C(1.0 / 3.0) - r) * gmy;
            } else {
                const C grx = gradx9<C>(rho[yc + xp], rho[yc + xm], rho[yp + xp], rho[yp + xm], rho[ym + xp],
                                        rho[ym + xm]);
                const C gry = grady9<C>(rho[yp + x], rho[ym + x], rho[yp + xp], rho[yp + xm], rho[ym + xp],
                                        rho[ym + xm]);
                if (SCHEME == 2) {
                    const C divx = gradx9<C>(pxx[yc + xp], pxx[yc + xm], pxx[yp + xp], pxx[yp + xm], pxx[ym + xp],
                                             pxx[ym + xm]) +
                                   grady9<C>(sxp * pxy[yp + x], sxm * pxy[ym + x], sxp * pxy[yp + xp],
                                             sxp * pxy[yp + xm], sxm * pxy[ym + xp], sxm * pxy[ym + xm]);
                    const C divy = gradx9<C>(pxy[yc + xp], pxy[yc + xm], sxp * pxy[yp + xp], sxp * pxy[yp + xm],
                                             sxm * pxy[ym + xp], sxm * pxy[ym + xm]) +
                                   grady9<C>(pyy[yp + x], pyy[ym + x], pyy[yp + xp], pyy[yp + xm], pyy[ym + xp],
                                             pyy[ym + xm]);
                    Fx = grx * C(1.0 / 3.0) - divx;
                    Fy = gry * C(1.0 / 3.0) - divy;
                } else {
                    Fx = grx * C(1.0 / 3.0) - r * gmx;
                    Fy = gry * C(1.0 / 3.0) - r * gmy;
                }
            }
            const C half = SCHEME == 4 ? C(0.5) * cc.lw_dt : C(0.5);  // Lax-Wendroff: time step A
            const C ux = (jx[i] + half * Fx) / r;
            const C uy = (jy[i] + half * Fy) / r;
            const C m = mu[i];
            if (out_rho) out_rho[i] = (O)r;
            if (out_ux) out_ux[i] = (O)ux;
            if (out_uy) out_uy[i] = (O)uy;
            if (out_mu) out_mu[i] = (O)m;
            const C u2 = ux * ux + uy * uy;
            mass += (double)r;
            ke += (double)(C(0.5) * r * u2);
            um2 = u2 > um2 ? u2 : um2;  // a NaN leaves it (and counts as bad)
            bad += (r > C(0) && isfinite(u2) && isfinite(m)) ? 0 : 1;
        }
    }
    block_sums(mass, ke, (double)um2, bad, partials);
}

// Sum and node count of a window of a C density field [ny][nx]: the grid
// covers the window's bounding box (bw x bh nodes from (bx0, by0), indices
// periodic); disc windows keep the nodes whose periodic distance to
// (cx, cy) is below r. One Partial per block (mass = sum, bad = count).
template <typename C>
__global__ void __launch_bounds__(256) window_sum_kernel(const C* __restrict__ rho, int nx, int ny, int bx0,
                                                         int by0, int bw, int disc, double cx, double cy,
                                                         double r, Partial* __restrict__ partials)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double sum = 0.0, cnt = 0.0;
    if (i < bw) {
        const int x = wrapi(bx0 + i, nx), y = wrapi(by0 + (int)blockIdx.y, ny);
        bool in = true;
        if (disc) {
            double dx = fabs((double)x - cx), dy = fabs((double)y - cy);
            dx = fmin(dx, (double)nx - dx);
            dy = fmin(dy, (double)ny - dy);
            in = dx * dx + dy * dy < r * r;
        }
        if (in) {
            sum = (double)rho[(int64_t)y * nx + x];
            cnt = 1.0;
        }
    }
    block_partial(sum, 0.0, 0.0, cnt, partials);
}

// Fold a case's partials in a fixed order into out[0..4] =
// {mass, kinetic energy, max |u|, steps, bad-node count}.
static __global__ void finalize_kernel(const Partial* __restrict__ partials, int64_t n, double steps,
                                       double* __restrict__ out)
{
    __shared__ double s[4][256];
    double mass = 0.0, ke = 0.0, um = 0.0, bad = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
        const Partial p = partials[k];
        mass += p.mass;
        ke += p.ke;
        um = fmax(um, p.umax2);
        bad += p.bad;
    }
    s[0][threadIdx.x] = mass;
    s[1][threadIdx.x] = ke;
    s[2][threadIdx.x] = um;
    s[3][threadIdx.x] = bad;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s[0][threadIdx.x] += s[0][threadIdx.x + w];
            s[1][threadIdx.x] += s[1][threadIdx.x + w];
            s[2][threadIdx.x] = fmax(s[2][threadIdx.x], s[2][threadIdx.x + w]);
            s[3][threadIdx.x] += s[3][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = s[0][0];
        out[1] = s[1][0];
        out[2] = sqrt(s[2][0]);
        out[3] = steps;
        out[4] = s[3][0];
    }
}

}  // namespace lbfe
