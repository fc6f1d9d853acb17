// Kernels around the time step: initial populations, macroscopic-field
// export and the per-case FP64 reductions. They run once per call, not per
// step, and work through FP64 scratch fields in the workspace.
#pragma once

#include "lbfe_device.cuh"

namespace lbfe {

// Scratch layout (FP64, one case at a time): four [ny][nx] fields.
struct Scratch {
    double* s0;  // rho
    double* s1;  // j_x (moments) / u_x0 (init)
    double* s2;  // j_y (moments) / u_y0 (init)
    double* s3;  // mu_c
};

// mu_c = E_f'(rho) - kappa lap(rho) on the FP64 field s0 (Eq. 2).
template <typename T, int EOS>
__global__ void mu_field_kernel(DevCase<T> c, DevCase<double> cd, const double* __restrict__ rho,
                                double* __restrict__ mu)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= c.nx) return;
    const int nx = c.nx, ny = c.ny;
    const int xm = wrapi(x - 1, nx), xp = wrapi(x + 1, nx);
    const int ym = wrapi(y - 1, ny) * nx, y0 = y * nx, yp = wrapi(y + 1, ny) * nx;
    const double C = rho[y0 + x];
    const double lap = lap9<double>(C, rho[y0 + xp], rho[y0 + xm], rho[yp + x], rho[ym + x],
                                    rho[yp + xp], rho[yp + xm], rho[ym + xp], rho[ym + xm]);
    mu[y0 + x] = dEf<EOS, double>(cd, C) - cd.kappa * lap;
}

// f(0) = M^-1 m_eq(rho0, u0) with mu_c of rho0, stored as f - w rho_ref in T.
template <typename T, int SCHEME>
__global__ void init_kernel(DevCase<T> c, DevCase<double> cd, const double* __restrict__ rho0,
                            const double* __restrict__ ux0, const double* __restrict__ uy0,
                            const double* __restrict__ mu0, T* __restrict__ f)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= c.nx) return;
    const int i = y * c.nx + x;
    const double rho = rho0[i];
    const double ux = ux0 ? ux0[i] : 0.0, uy = uy0 ? uy0[i] : 0.0;
    const double rr = cd.rho_ref;
    // deviation moments of the equilibrium, then M^-1 (the collision with
    // all rates 1 and no force returns exactly M^-1 m_eq)
    double d[kQ];
    for (int a = 0; a < kQ; ++a) d[a] = 0.0;
    const double drho = rho - rr;
    collide<SCHEME, double>(d, drho, rho, rho * ux, rho * uy, ux, uy, 0.0, 0.0, mu0[i], 0.0, 0.0, rr,
                            cd.c0, 1.0, 1.0, 1.0, 1.0);
    // with d = 0 the moments m_e, m_s, ... of d vanish, so the rates-1 collision
    // leaves exactly the equilibrium; the conserved entries are set from
    // drho and rho u directly.
    // Storage holds post-collision populations before streaming (the step
    // pulls f_a(x) from x - e_a), so f_a(0) of node x is stored at x - e_a.
    constexpr int ex[kQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    constexpr int ey[kQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    for (int a = 0; a < kQ; ++a) {
        const int64_t o = (int64_t)wrapi(y - ey[a], c.ny) * c.pitch + wrapi(x - ex[a], c.nx);
        f[c.off + a * c.plane + o] = (T)d[a];
    }
}

// Pull the populations of the current state into FP64 rho, j_x, j_y fields.
template <typename T>
__global__ void pull_moments_kernel(DevCase<T> c, const T* __restrict__ f, double* __restrict__ rho,
                                    double* __restrict__ jx, double* __restrict__ jy)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= c.nx) return;
    const int nx = c.nx, ny = c.ny, pitch = c.pitch;
    const int64_t P = c.plane;
    f += c.off;
    const int xm = wrapi(x - 1, nx), xp = wrapi(x + 1, nx);
    const int rm = wrapi(y - 1, ny) * pitch, r0 = y * pitch, rp = wrapi(y + 1, ny) * pitch;
    double F[kQ];
    F[0] = (double)f[0 * P + r0 + x];
    F[1] = (double)f[1 * P + r0 + xm];
    F[2] = (double)f[2 * P + rm + x];
    F[3] = (double)f[3 * P + r0 + xp];
    F[4] = (double)f[4 * P + rp + x];
    F[5] = (double)f[5 * P + rm + xm];
    F[6] = (double)f[6 * P + rm + xp];
    F[7] = (double)f[7 * P + rp + xp];
    F[8] = (double)f[8 * P + rp + xm];
    const double dr = ((F[0] + (F[1] + F[3])) + (F[2] + F[4])) + ((F[5] + F[7]) + (F[6] + F[8]));
    const int i = y * nx + x;
    rho[i] = (double)c.rho_ref + dr;
    jx[i] = (F[1] - F[3]) + ((F[5] - F[7]) + (F[8] - F[6]));
    jy[i] = (F[2] - F[4]) + ((F[5] - F[7]) + (F[6] - F[8]));
}

// Per-block partial sums of a case's state: mass, kinetic energy, max |u|^2
// and a count of non-physical nodes.
struct Partial {
    double mass, ke, umax2, bad;
};

// Velocity of Eq. 12 from rho, j and the force of the case's scheme; writes
// the requested outputs and one Partial per block (blockDim.x == 256).
template <int SCHEME>
__global__ void __launch_bounds__(256) velocity_kernel(DevCase<double> cd, const double* __restrict__ rho,
                                                       const double* __restrict__ jx,
                                                       const double* __restrict__ jy,
                                                       const double* __restrict__ mu,
                                                       double* __restrict__ out_rho,
                                                       double* __restrict__ out_ux,
                                                       double* __restrict__ out_uy,
                                                       double* __restrict__ out_mu,
                                                       Partial* __restrict__ partials)
{
    const int nx = cd.nx, ny = cd.ny;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    double mass = 0.0, ke = 0.0, um = 0.0, bad = 0.0;
    if (x < nx) {
        const int xm = wrapi(x - 1, nx), xp = wrapi(x + 1, nx);
        const int ym = wrapi(y - 1, ny) * nx, y0 = y * nx, yp = wrapi(y + 1, ny) * nx;
        const int i = y0 + x;
        const double r = rho[i];
        const double gmx = gradx9<double>(mu[y0 + xp], mu[y0 + xm], mu[yp + xp], mu[yp + xm], mu[ym + xp],
                                          mu[ym + xm]);
        const double gmy = grady9<double>(mu[yp + x], mu[ym + x], mu[yp + xp], mu[yp + xm], mu[ym + xp],
                                          mu[ym + xm]);
        double Fx, Fy;
        if (SCHEME == 1) {
            Fx = (1.0 / 3.0 - r) * gmx;
            Fy = (1.0 / 3.0 - r) * gmy;
        } else {
            const double grx = gradx9<double>(rho[y0 + xp], rho[y0 + xm], rho[yp + xp], rho[yp + xm],
                                              rho[ym + xp], rho[ym + xm]);
            const double gry = grady9<double>(rho[yp + x], rho[ym + x], rho[yp + xp], rho[yp + xm],
                                              rho[ym + xp], rho[ym + xm]);
            Fx = grx * (1.0 / 3.0) - r * gmx;
            Fy = gry * (1.0 / 3.0) - r * gmy;
        }
        const double ux = (jx[i] + 0.5 * Fx) / r;
        const double uy = (jy[i] + 0.5 * Fy) / r;
        if (out_rho) out_rho[i] = r;
        if (out_ux) out_ux[i] = ux;
        if (out_uy) out_uy[i] = uy;
        if (out_mu) out_mu[i] = mu[i];
        const double u2 = ux * ux + uy * uy;
        mass = r;
        ke = 0.5 * r * u2;
        um = u2;
        bad = (r > 0.0 && isfinite(u2) && isfinite(mu[i])) ? 0.0 : 1.0;
    }
    // block reduction: warp shuffles, then one value per warp through smem
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
        partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = p;
    }
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
