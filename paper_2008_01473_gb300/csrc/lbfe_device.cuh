// Device-side definitions shared by the sm_103a kernels of the free-energy
// D2Q9 step: per-case parameter records, work items, the equations of state,
// the lattice stencils and the closed-form moment-space collision.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lbfe {

constexpr int kQ = 9;

// Scheme codes of the kernels (the lb_case codes): 0 standard, 1 improved,
// 2 standard with the pressure-tensor force, 3 improved with the derivatives
// of Eq. 29 taken on the lattice-weight average of phi u, 4 the Lax-Wendroff
// propagation scheme of Appendix A (standard force, Eqs. A1-A4). Schemes 1
// and 3 share the equilibrium, force and collision of Eqs. 24-28.
__host__ __device__ constexpr bool improved_scheme(int s) { return s == 1 || s == 3; }

struct StepStat;  // per-step statistics entry (below)

// Per-case parameters as the kernels read them (one record per case, in the
// arithmetic type T of the launch).
template <typename T>
struct DevCase {
    int32_t nx, ny, pitch;
    int32_t walls;  // 1: moving no-slip walls below y = 0 and above y = ny - 1
    int64_t off;    // element offset of the case inside a population buffer
    int64_t plane;  // elements between two velocity planes: ny * pitch
    T RT, a, b, kappa;
    T c0;           // p_m = (c0 + mu_c)/3 (Eq. 24)
    T rho_ref;      // populations are stored as f - w rho_ref
    T lam_e, lam_s, lam_q, lam_v;  // 1/tau of Eq. 8 (all 1/tau_v for BGK)
    T nu;           // > 0: tau_v from constant kinematic viscosity
    T wall_d;       // walls: moving-wall term f_eq,5 - f_eq,7 of the wall state
    // Lax-Wendroff scheme (Appendix A): time step dt = A; coefficients of
    // Eq. A2; 1/(c_s^2 dt (B - tau)), (tau - 1/2) dt and B dt / (2 c_s^2) of
    // Eqs. A3-A4; dt (1 - 1/(2 tau)) of Eq. A1
    T lw_dt, lw_a0, lw_a1, lw_am1, lw_kT, lw_fd, lw_bt, lw_g;
    int32_t lw_first;  // 1: the stored populations are the pre-collision f(0) (step 0)
    // per-step statistics (st_hist == 0: off): this case's ring of st_hist
    // entries, its counters {ticket, recorded states} and the number of work
    // items (blocks) that one step of the case launches
    int32_t st_hist;
    StepStat* st_ring;
    int32_t* st_ctr;
    int32_t st_blocks;
    int32_t pad_;
};

// One entry of the per-step statistics of a case: over the nodes of the
// state a step starts from, the sums of rho - rho_ref and of rho |u|^2, the
// largest |u|^2 (the bits of a non-negative double, which order like its
// value) and the number of nodes summed.
struct StepStat {
    double dmass, ke2;
    unsigned long long umax2;
    unsigned long long nodes;
};

// Block end of the per-step statistics (Sec. II A: mass and kinetic energy of
// the fields; the sums run in FP64 from here on). Every thread of the block
// calls it with its partial sums over its stage D nodes; thread 0 adds the
// block's sums to the case's current ring entry with FP64 atomics, and the
// case's last block of the step (a ticket over st_blocks) clears the next
// entry and advances the recorded-state counter. Kernel boundaries order the
// steps, so the next launch reads the advanced counter. blockDim.x must be a
// multiple of 32 and at most 32 W (W: the warps the block's shared partials
// hold; the packed kernel passes its own warp count so that the narrow
// shape's shared memory still fits six blocks per SM).
template <typename T, int W = 32>
__device__ __forceinline__ void stats_block(const DevCase<T>& c, double dm, double k2, double u2,
                                            unsigned long long nodes)
{
    __shared__ double s_m[W], s_k[W], s_u[W];
    constexpr unsigned kFull = 0xffffffffu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dm += __shfl_xor_sync(kFull, dm, o);
        k2 += __shfl_xor_sync(kFull, k2, o);
        u2 = fmax(u2, __shfl_xor_sync(kFull, u2, o));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    if (lane == 0) {
        s_m[w] = dm;
        s_k[w] = k2;
        s_u[w] = u2;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int i = 1; i < nw; ++i) {
        dm += s_m[i];
        k2 += s_k[i];
        u2 = fmax(u2, s_u[i]);
    }
    int32_t* ctr = c.st_ctr;
    StepStat* e = c.st_ring + (*(volatile int32_t*)(ctr + 1) % c.st_hist);
    atomicAdd(&e->dmass, dm);
    atomicAdd(&e->ke2, k2);
    atomicMax(&e->umax2, (unsigned long long)__double_as_longlong(u2 > 0.0 ? u2 : 0.0));
    atomicAdd(&e->nodes, nodes);
    __threadfence();
    if (atomicAdd(ctr, 1) == c.st_blocks - 1) {
        const int32_t n = *(volatile int32_t*)(ctr + 1) + 1;
        StepStat* nx = c.st_ring + (n % c.st_hist);
        nx->dmass = 0.0;
        nx->ke2 = 0.0;
        nx->umax2 = 0ull;
        nx->nodes = 0ull;
        *(volatile int32_t*)ctr = 0;
        __threadfence();
        *(volatile int32_t*)(ctr + 1) = n;
    }
}


// One block of work: output columns [x0, x0 + wv) and rows [y0, y0 + h) of a
// case. A block computes a halo of columns around the strip itself.
struct Item {
    int32_t case_id, x0, wv, y0, h, pad_;
};

// Elements per stored row of a population plane: nx rounded up to 32, so
// that every row starts on a 128-byte boundary. The snapshot layout of
// lb_save and the input of lb_fields_static follow it.
__host__ __device__ constexpr int pitch_of(int nx) { return (nx + 31) / 32 * 32; }

__host__ __device__ __forceinline__ int wrapi(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

// Lattice row of a neighbour row y (y may lie one row outside): periodic, or,
// with walls, the mirror image in the wall (row -1 is row 0, row ny is
// row ny - 1).
template <typename T>
__host__ __device__ __forceinline__ int nb_row(const DevCase<T>& c, int y)
{
    if (!c.walls) return wrapi(y, c.ny);
    return y < 0 ? -1 - y : (y >= c.ny ? 2 * c.ny - 1 - y : y);
}

// ---------------------------------------------------------------------- EOS
// E_f'(rho): van der Waals (Eq. 30 without the kappa term) or
// Carnahan-Starling, both written as R T h(rho) - 2 a rho.
template <int EOS, typename T>
__device__ __forceinline__ T dEf(const DevCase<T>& c, T rho);

template <>
__device__ __forceinline__ double dEf<0, double>(const DevCase<double>& c, double rho)
{
    double r = 1.0 / (1.0 - c.b * rho);
    return c.RT * (log(rho * r) + r) - 2.0 * c.a * rho;
}
template <>
__device__ __forceinline__ float dEf<0, float>(const DevCase<float>& c, float rho)
{
    float r = 1.0f / (1.0f - c.b * rho);
    return c.RT * (logf(rho * r) + r) - 2.0f * c.a * rho;
}
template <>
__device__ __forceinline__ double dEf<1, double>(const DevCase<double>& c, double rho)
{
    double n = 0.25 * c.b * rho;
    double r = 1.0 / (1.0 - n);
    double r2 = r * r;
    return c.RT * (log(rho) + 1.0 + n * (4.0 - 3.0 * n) * r2 + n * (4.0 - 2.0 * n) * r2 * r) -
           2.0 * c.a * rho;
}
template <>
__device__ __forceinline__ float dEf<1, float>(const DevCase<float>& c, float rho)
{
    float n = 0.25f * c.b * rho;
    float r = 1.0f / (1.0f - n);
    float r2 = r * r;
    return c.RT * (logf(rho) + 1.0f + n * (4.0f - 3.0f * n) * r2 + n * (4.0f - 2.0f * n) * r2 * r) -
           2.0f * c.a * rho;
}

// p_EOS = rho E_f' - E_f (below Eq. 4) in closed form: van der Waals
// rho R T / (1 - b rho) - a rho^2; Carnahan-Starling
// rho R T (1 + n + n^2 - n^3) / (1 - n)^3 - a rho^2 with n = b rho / 4.
template <int EOS, typename T>
__device__ __forceinline__ T pEOS(const DevCase<T>& c, T rho)
{
    if (EOS == 0) return rho * c.RT / (T(1) - c.b * rho) - c.a * rho * rho;
    const T n = T(0.25) * c.b * rho;
    const T r = T(1) / (T(1) - n);
    return rho * c.RT * (T(1) + n + n * n - n * n * n) * (r * r * r) - c.a * rho * rho;
}

// Thermodynamic pressure tensor at a node (Eqs. 4-5) from p_EOS, rho, the
// Eq. 17 gradient (gx, gy) and the Laplacian of rho.
template <typename T>
__device__ __forceinline__ void pressure_tensor(T p_eos, T rho, T gx, T gy, T lap, T kappa, T& Pxx, T& Pxy,
                                                T& Pyy)
{
    const T p = p_eos - kappa * (rho * lap + T(0.5) * (gx * gx + gy * gy));
    Pxx = p + kappa * gx * gx;
    Pyy = p + kappa * gy * gy;
    Pxy = kappa * gx * gy;
}

// ----------------------------------------------------------------- stencils
// Values of a field around a node: C, E(x+1), W(x-1), N(y+1), S(y-1) and corners.
// Isotropic Laplacian 6 sum_a w_a (phi(x+e_a) - phi(x)).
template <typename T>
__device__ __forceinline__ T lap9(T C, T E, T W, T N, T S, T NE, T NW, T SE, T SW)
{
    return (T(4) * ((E + W) + (N + S)) + ((NE + SW) + (NW + SE)) - T(20) * C) * T(1.0 / 6.0);
}
// Eq. 17: 3 sum_a w_a phi(x + e_a) e_a.
template <typename T>
__device__ __forceinline__ T gradx9(T E, T W, T NE, T NW, T SE, T SW)
{
    return (E - W) * T(1.0 / 3.0) + ((NE - SW) + (SE - NW)) * T(1.0 / 12.0);
}
template <typename T>
__device__ __forceinline__ T grady9(T N, T S, T NE, T NW, T SE, T SW)
{
    return (N - S) * T(1.0 / 3.0) + ((NE - SW) + (NW - SE)) * T(1.0 / 12.0);
}

// --------------------------------------------------------------- collision
// Moment-space collision of Eqs. 9 / 28 in closed form, on populations stored
// as deviations d_a = f_a - w_a rho_ref (rho_ref = 0 gives plain populations).
// Inputs: d[9] at the node, drho = sum d, rho = rho_ref + drho, jx, jy of d,
// the force F, velocity u (Eq. 12), mu_c (for p_m), C1 and C7 (Eq. 29; zero for
// the standard scheme) and the rates. Output: post-collision deviations.
// SCHEME: 0 standard, 1 improved, 2 standard with the pressure-tensor force
// (the same collision as 0), 3 improved with the averaged correction (the
// same collision as 1; only C1, C7 are computed differently).
template <int SCHEME, typename T>
__device__ __forceinline__ void collide(T (&d)[kQ], T drho, T rho, T jx, T jy, T ux, T uy, T Fx, T Fy,
                                        T mu, T C1, T C7, T rho_ref, T c0, T lam_e, T lam_s,
                                        T lam_q, T lam_v)
{
    // moments of d (rows of M)
    const T sa = (d[1] + d[3]) + (d[2] + d[4]);
    const T sd = (d[5] + d[7]) + (d[6] + d[8]);
    const T m_e = T(2) * sd - sa - T(4) * d[0];
    const T m_s = sd - T(2) * sa + T(4) * d[0];
    const T dxd = (d[5] - d[7]) + (d[8] - d[6]);
    const T dyd = (d[5] - d[7]) + (d[6] - d[8]);
    const T m_qx = dxd - T(2) * (d[1] - d[3]);
    const T m_qy = dyd - T(2) * (d[2] - d[4]);
    const T m_pxx = (d[1] + d[3]) - (d[2] + d[4]);
    const T m_pxy = (d[5] + d[7]) - (d[6] + d[8]);

    // equilibria (Eq. 11 or Eq. 27) minus the moments of w rho_ref, which are
    // rho_ref (1, -2, 1, 0, ...)
    const T uxx = ux * ux, uyy = uy * uy, u2 = uxx + uyy;
    T eq_e, eq_s, eq_qx, eq_qy;
    if (!improved_scheme(SCHEME)) {  // standard scheme, either force form: Eq. 11
        eq_e = T(3) * rho * u2 - T(2) * drho;
        eq_s = drho - T(3) * rho * u2;
        eq_qx = -rho * ux;
        eq_qy = -rho * uy;
    } else {
        const T pm3 = c0 + mu;  // 3 p_m
        eq_e = T(3) * rho * u2 - T(4) * rho + T(2) * pm3 + T(2) * rho_ref;
        eq_s = T(4) * rho - T(3) * rho * u2 - T(3) * pm3 - rho_ref;
        const T g2 = pm3 - T(2) * rho;  // rho (gamma - 2)
        eq_qx = g2 * ux;
        eq_qy = g2 * uy;
    }
    const T eq_pxx = rho * (uxx - uyy);
    const T eq_pxy = rho * ux * uy;

    // forcing moments S = M G (Eq. 14) and correction C (Eq. 29)
    const T uF = ux * Fx + uy * Fy;
    const T S_e = T(6) * uF + T(9) * C1;
    const T S_s = T(-6) * uF;
    const T S_pxx = T(2) * (ux * Fx - uy * Fy) + T(3) * C7;
    const T S_pxy = ux * Fy + uy * Fx;

    const T pe = m_e - lam_e * (m_e - eq_e) + (T(1) - T(0.5) * lam_e) * S_e;
    const T ps = m_s - lam_s * (m_s - eq_s) + (T(1) - T(0.5) * lam_s) * S_s;
    const T pqx = m_qx - lam_q * (m_qx - eq_qx) - (T(1) - T(0.5) * lam_q) * Fx;
    const T pqy = m_qy - lam_q * (m_qy - eq_qy) - (T(1) - T(0.5) * lam_q) * Fy;
    const T hv = T(1) - T(0.5) * lam_v;
    const T pxx = m_pxx - lam_v * (m_pxx - eq_pxx) + hv * S_pxx;
    const T pxy = m_pxy - lam_v * (m_pxy - eq_pxy) + hv * S_pxy;
    const T pjx = jx + Fx;  // conserved: any rate gives j + F
    const T pjy = jy + Fy;

    // f* = M^-1 m*, M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4)
    const T a0 = drho * T(1.0 / 9.0);
    const T a1 = pe * T(1.0 / 36.0);
    const T a2 = ps * T(1.0 / 36.0);
    const T a3 = pjx * T(1.0 / 6.0);
    const T a4 = pqx * T(1.0 / 12.0);
    const T a5 = pjy * T(1.0 / 6.0);
    const T a6 = pqy * T(1.0 / 12.0);
    const T a7 = pxx * T(0.25);
    const T a8 = pxy * T(0.25);
    const T b_ax = a0 - a1 - T(2) * a2;
    const T b_dg = a0 + T(2) * a1 + a2;
    const T ex = a3 - T(2) * a4, ey = a5 - T(2) * a6;
    const T X = a3 + a4, Y = a5 + a6;
    d[1] = b_ax + ex + a7;
    d[3] = b_ax - ex + a7;
    d[2] = b_ax + ey - a7;
    d[4] = b_ax - ey - a7;
    d[5] = b_dg + (X + Y) + a8;
    d[7] = b_dg - (X + Y) + a8;
    d[6] = b_dg + (Y - X) - a8;
    d[8] = b_dg + (X - Y) - a8;
    // rest population from the conserved density: equal to the M^-1 row
    // a0 - 4 (a1 - a2) in exact arithmetic, and in finite precision keeps
    // the stored density equal to the pulled one up to two rounded sums
    d[0] = drho - (((d[1] + d[3]) + (d[2] + d[4])) + ((d[5] + d[7]) + (d[6] + d[8])));
}

// BGK collision of the Lax-Wendroff scheme (Eq. A1) in population space, on
// populations stored as deviations d_a = f_a - w_a rho_ref, with the
// equilibrium of Eq. A3 (the second-order equilibrium plus
// B dt (e_a e_a - c_s^2 I) : T / (2 c_s^2)) and the tensor of Eq. A4,
//   T = [Pi - rho c_s^2 I - rho u u - (tau - 1/2) dt (u F + F u)] / (rho c_s^2 dt (B - tau)),
// Pi = sum_a e_a e_a f_a taken here as its deviation from rho c_s^2 I. The
// source is dt (1 - 1/(2 tau)) G_a with G of Eq. 14. The rest population
// is closed from the conserved density, as in collide().
template <typename T>
__device__ __forceinline__ void collide_lw(T (&d)[kQ], T drho, T rho, T ux, T uy, T Fx, T Fy, const DevCase<T>& c)
{
    constexpr int ex[kQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    constexpr int ey[kQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const T dg = (d[5] + d[7]) + (d[6] + d[8]);
    const T Pxx = (d[1] + d[3]) + dg - drho * T(1.0 / 3.0);  // Pi_xx - rho c_s^2
    const T Pyy = (d[2] + d[4]) + dg - drho * T(1.0 / 3.0);
    const T Pxy = (d[5] + d[7]) - (d[6] + d[8]);
    const T kT = c.lw_kT / rho;
    const T Txx = (Pxx - rho * ux * ux - T(2) * c.lw_fd * ux * Fx) * kT;
    const T Tyy = (Pyy - rho * uy * uy - T(2) * c.lw_fd * uy * Fy) * kT;
    const T Txy = (Pxy - rho * ux * uy - c.lw_fd * (ux * Fy + Fx * uy)) * kT;
    const T u2 = ux * ux + uy * uy;
    const T lam = c.lam_v;
    const T w[kQ] = {T(4.0 / 9.0), T(1.0 / 9.0), T(1.0 / 9.0), T(1.0 / 9.0), T(1.0 / 9.0),
                     T(1.0 / 36.0), T(1.0 / 36.0), T(1.0 / 36.0), T(1.0 / 36.0)};
#pragma unroll
    for (int a = 1; a < kQ; ++a) {
        const T eu = T(ex[a]) * ux + T(ey[a]) * uy;
        const T eeT = (T(ex[a] * ex[a]) - T(1.0 / 3.0)) * Txx + T(2 * ex[a] * ey[a]) * Txy +
                      (T(ey[a] * ey[a]) - T(1.0 / 3.0)) * Tyy;
        // f_eq,a - w_a rho_ref
        const T feq = w[a] * (drho + rho * (T(3) * eu + T(4.5) * eu * eu - T(1.5) * u2 + c.lw_bt * eeT));
        const T G = w[a] * ((T(3) * (T(ex[a]) - ux) + T(9) * eu * T(ex[a])) * Fx +
                            (T(3) * (T(ey[a]) - uy) + T(9) * eu * T(ey[a])) * Fy);
        d[a] = d[a] - lam * (d[a] - feq) + c.lw_g * G;
    }
    d[0] = drho - (((d[1] + d[3]) + (d[2] + d[4])) + ((d[5] + d[7]) + (d[6] + d[8])));
}

// Shear rate at a node: constant, or from a constant kinematic viscosity.
template <int SCHEME, bool NU, typename T>
__device__ __forceinline__ T shear_rate(const DevCase<T>& c, T rho, T mu)
{
    if (!NU) return c.lam_v;
    if (improved_scheme(SCHEME)) return T(1) / (T(0.5) + c.nu * rho * T(3) / (c.c0 + mu));
    return T(1) / (T(0.5) + T(3) * c.nu);
}

}  // namespace lbfe
