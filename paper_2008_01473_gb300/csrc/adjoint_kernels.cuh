// Kernels of the discrete adjoint (reverse-mode derivative) of one time step,
// for lb_adjoint_step, in the arithmetic type T of the handle (FP64, or FP32
// for FP32 handles; loss and parameter partials are FP64 either way). One
// thread per node, 256-thread blocks over (ceil(nx / 256), ny). Fields are
// dense [ny][nx] arrays of T; the adjoint
// of the populations (lam) is kept at the nodes, lam_a(x) = dL/df_a(x), while
// forward states are in the library's storage form (pulled on read).
//
// For the state f^n of step n the forward fields are rebuilt (rho, j, lap,
// mu_c, grad mu_c, F, u, phi, A = phi u_x, B = phi u_y, C1, C7: Eqs. 2, 12,
// 13/24, 17, 29), then the step is transposed in reverse order:
//   collision (Eqs. 9/28 in moment space, closed form)  -> adj_collide
//   correction C1/C7 and phi u (Eq. 29), velocity (Eq. 12), force
//   (Eqs. 13/24)                                          -> adj_force
//   grad mu_c (Eq. 17), mu_c = E_f' - kappa lap (Eq. 2)   -> adj_mu
//   lap and rho = sum f, j = sum e f (Eq. 12)             -> adj_lambda
// The transpose of each stencil is its own gather over x - e_a. Parameter
// derivatives (kappa, T) and the loss come out as per-block FP64 partials.
#pragma once

#include "aux_kernels.cuh"

namespace lbfe {

template <typename T>
struct AdjFields {
    // forward fields at the current state
    T *rho, *jx, *jy, *lap, *mu, *gx, *gy, *Fx, *Fy, *ux, *uy, *phi, *A, *B, *C1, *C7;
    // adjoint fields
    T *rb, *jxb, *jyb, *uxb, *uyb, *Fxb, *Fyb, *mub, *C1b, *C7b, *gxb, *gyb, *Lb;
};

__device__ constexpr int kEx[kQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__device__ constexpr int kEy[kQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
__device__ constexpr double kW[kQ] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                           1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

struct NodeIdx {
    int x, y, nx, ny;
    int64_t i;
    __device__ __forceinline__ int64_t at(int dx, int dy) const
    {
        return (int64_t)wrapi(y + dy, ny) * nx + wrapi(x + dx, nx);
    }
};

__device__ __forceinline__ bool node_of(int nx, int ny, NodeIdx& n)
{
    n.x = blockIdx.x * blockDim.x + threadIdx.x;
    n.y = blockIdx.y;
    n.nx = nx;
    n.ny = ny;
    n.i = (int64_t)n.y * nx + n.x;
    return n.x < nx;
}

// Eq. 17 at node n of field v (component d = 0: x, 1: y)
template <typename T>
__device__ __forceinline__ T grad_at(const T* v, const NodeIdx& n, int d)
{
    T s = T(0);
#pragma unroll
    for (int a = 1; a < kQ; ++a) s += T(3.0 * kW[a] * (d == 0 ? kEx[a] : kEy[a])) * v[n.at(kEx[a], kEy[a])];
    return s;
}
// transpose of the Eq. 17 component d: 3 sum_a w_a e_a v(x - e_a)
template <typename T>
__device__ __forceinline__ T gradT_at(const T* v, const NodeIdx& n, int d)
{
    T s = T(0);
#pragma unroll
    for (int a = 1; a < kQ; ++a) s += T(3.0 * kW[a] * (d == 0 ? kEx[a] : kEy[a])) * v[n.at(-kEx[a], -kEy[a])];
    return s;
}
// transpose of the Laplacian 6 sum_a w_a (v(x + e_a) - v(x)): 6 sum_a w_a (v(x - e_a) - v(x))
template <typename T>
__device__ __forceinline__ T lapT_at(const T* v, const NodeIdx& n)
{
    T s = T(0);
    const T c = v[n.i];
#pragma unroll
    for (int a = 1; a < kQ; ++a) s += T(kW[a]) * (v[n.at(-kEx[a], -kEy[a])] - c);
    return T(6) * s;
}

template <int EOS, typename T>
__device__ __forceinline__ T d2Ef_dev(const DevCase<T>& c, T rho)
{
    if (EOS == 0) {
        const T q = T(1) / (T(1) - c.b * rho);
        return c.RT * (T(1) / rho + c.b * q + c.b * q * q) - T(2) * c.a;
    }
    const T n = T(0.25) * c.b * rho, q = T(1) / (T(1) - n);
    return c.RT * (T(1) / rho + T(0.25) * c.b * (T(8) - T(2) * n) * q * q * q * q) - T(2) * c.a;
}
// R h(rho) = d E_f' / d T (R folded in: RT / T)
template <int EOS, typename T>
__device__ __forceinline__ T dEf_dT_dev(const DevCase<T>& c, T rho, T R)
{
    DevCase<T> u = c;
    u.RT = R;
    u.a = T(0);
    return dEf<EOS, T>(u, rho);
}

// ---------------------------------------------------------------- forward
// lap and mu_c of the rho field
template <typename T, int EOS>
__global__ void adj_fwd_mu(DevCase<T> c, AdjFields<T> F)
{
    NodeIdx n;
    if (!node_of(c.nx, c.ny, n)) return;
    T s = T(0);
    const T r = F.rho[n.i];
#pragma unroll
    for (int a = 1; a < kQ; ++a) s += T(kW[a]) * (F.rho[n.at(kEx[a], kEy[a])] - r);
    const T lap = T(6) * s;
    F.lap[n.i] = lap;
    F.mu[n.i] = dEf<EOS, T>(c, r) - c.kappa * lap;
}

// grad mu_c, F, u, phi, A, B; loss partials: w_u sum |u|^2 + sum s rho
template <typename T, int SCHEME>
__global__ void __launch_bounds__(256) adj_fwd_force(DevCase<T> c, AdjFields<T> F, double w_u,
                                                     const double* __restrict__ s_final, Partial* partials)
{
    NodeIdx n;
    double loss = 0.0;
    if (node_of(c.nx, c.ny, n)) {
        const T r = F.rho[n.i];
        const T gx = grad_at(F.mu, n, 0), gy = grad_at(F.mu, n, 1);
        T Fx, Fy;
        if (SCHEME == 1) {
            Fx = (T(1.0 / 3.0) - r) * gx;
            Fy = (T(1.0 / 3.0) - r) * gy;
        } else {
            Fx = grad_at(F.rho, n, 0) * T(1.0 / 3.0) - r * gx;
            Fy = grad_at(F.rho, n, 1) * T(1.0 / 3.0) - r * gy;
        }
        const T ux = (F.jx[n.i] + T(0.5) * Fx) / r, uy = (F.jy[n.i] + T(0.5) * Fy) / r;
        const T phi = (r - (c.c0 + F.mu[n.i])) * T(1.0 / 3.0);
        F.gx[n.i] = gx;
        F.gy[n.i] = gy;
        F.Fx[n.i] = Fx;
        F.Fy[n.i] = Fy;
        F.ux[n.i] = ux;
        F.uy[n.i] = uy;
        F.phi[n.i] = phi;
        F.A[n.i] = phi * ux;
        F.B[n.i] = phi * uy;
        loss = w_u * ((double)ux * ux + (double)uy * uy) + (s_final ? s_final[n.i] * (double)r : 0.0);
    }
    block_partial<true>(loss, 0.0, 0.0, 0.0, partials);
}

template <typename T>
__global__ void adj_fwd_corr(DevCase<T> c, AdjFields<T> F)
{
    NodeIdx n;
    if (!node_of(c.nx, c.ny, n)) return;
    const T Ax = grad_at(F.A, n, 0), By = grad_at(F.B, n, 1);
    F.C1[n.i] = Ax + By;
    F.C7[n.i] = Ax - By;
}

// ---------------------------------------------------------------- reverse
// Collision adjoint at each node. lam_next: adjoint of the state after the
// step (node form); has_next = 0 for the final state (no collision term).
// Writes lam_direct (the part through m = M f) and initialises every adjoint
// field, adding the |u|^2 seed when seed_u != 0.
template <typename T, int SCHEME>
__global__ void adj_collide(DevCase<T> c, AdjFields<T> F, const T* __restrict__ lam_next, int has_next,
                            int seed_u, T* __restrict__ lam_direct)
{
    NodeIdx n;
    if (!node_of(c.nx, c.ny, n)) return;
    const int64_t N = (int64_t)c.nx * c.ny;
    T rb = T(0), jxb = T(0), jyb = T(0), uxb = T(0), uyb = T(0), Fxb = T(0), Fyb = T(0), mub = T(0), C1b = T(0),
      C7b = T(0);
    T d[kQ];
    for (int a = 0; a < kQ; ++a) d[a] = T(0);
    if (has_next) {
        // lam*(x) = lam_next(x + e_a): transpose of the streaming
        T L[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) L[a] = lam_next[a * N + n.at(kEx[a], kEy[a])];
        // nu = M^-T lam* = D M lam*
        const T sa = (L[1] + L[3]) + (L[2] + L[4]), sd = (L[5] + L[7]) + (L[6] + L[8]);
        const T nr = (L[0] + sa + sd) * T(1.0 / 9.0);
        const T ne = (T(2) * sd - sa - T(4) * L[0]) * T(1.0 / 36.0);
        const T ns = (sd - T(2) * sa + T(4) * L[0]) * T(1.0 / 36.0);
        const T njx = ((L[1] - L[3]) + (L[5] - L[7]) + (L[8] - L[6])) * T(1.0 / 6.0);
        const T nqx = (T(-2) * (L[1] - L[3]) + (L[5] - L[7]) + (L[8] - L[6])) * T(1.0 / 12.0);
        const T njy = ((L[2] - L[4]) + (L[5] - L[7]) + (L[6] - L[8])) * T(1.0 / 6.0);
        const T nqy = (T(-2) * (L[2] - L[4]) + (L[5] - L[7]) + (L[6] - L[8])) * T(1.0 / 12.0);
        const T npxx = ((L[1] + L[3]) - (L[2] + L[4])) * T(0.25);
        const T npxy = ((L[5] + L[7]) - (L[6] + L[8])) * T(0.25);
        const T le = c.lam_e, ls = c.lam_s, lq = c.lam_q, lv = c.lam_v;
        // m* = m + lam (eq - m) + h S (non-conserved), rho* = rho, j* = j + F
        const T mbe = (T(1) - le) * ne, mbs = (T(1) - ls) * ns, mbqx = (T(1) - lq) * nqx, mbqy = (T(1) - lq) * nqy,
                mbxx = (T(1) - lv) * npxx, mbxy = (T(1) - lv) * npxy;
        const T qe = le * ne, qs = ls * ns, qqx = lq * nqx, qqy = lq * nqy, qxx = lv * npxx, qxy = lv * npxy;
        const T Se = (T(1) - T(0.5) * le) * ne, Ss = (T(1) - T(0.5) * ls) * ns,
                Sqx = (T(1) - T(0.5) * lq) * nqx, Sqy = (T(1) - T(0.5) * lq) * nqy,
                Sxx = (T(1) - T(0.5) * lv) * npxx, Sxy = (T(1) - T(0.5) * lv) * npxy;
        rb += nr;
        jxb += njx;
        jyb += njy;
        Fxb += njx;
        Fyb += njy;
        // direct part: M_nc^T m-bar (rows e, eps, q_x, q_y, p_xx, p_xy of M)
        d[0] = T(-4) * mbe + T(4) * mbs;
        d[1] = -mbe - T(2) * mbs - T(2) * mbqx + mbxx;
        d[2] = -mbe - T(2) * mbs - T(2) * mbqy - mbxx;
        d[3] = -mbe - T(2) * mbs + T(2) * mbqx + mbxx;
        d[4] = -mbe - T(2) * mbs + T(2) * mbqy - mbxx;
        d[5] = T(2) * mbe + mbs + mbqx + mbqy + mbxy;
        d[6] = T(2) * mbe + mbs - mbqx + mbqy - mbxy;
        d[7] = T(2) * mbe + mbs - mbqx - mbqy + mbxy;
        d[8] = T(2) * mbe + mbs + mbqx - mbqy - mbxy;
        // equilibria (Eq. 11 / Eq. 27)
        const T r = F.rho[n.i], ux = F.ux[n.i], uy = F.uy[n.i], u2 = ux * ux + uy * uy;
        if (SCHEME == 0) {
            rb += qe * (T(3) * u2 - T(2)) + qs * (T(1) - T(3) * u2) - qqx * ux - qqy * uy;
            uxb += qe * T(6) * r * ux - qs * T(6) * r * ux - qqx * r;
            uyb += qe * T(6) * r * uy - qs * T(6) * r * uy - qqy * r;
        } else {
            const T s3 = c.c0 + F.mu[n.i];
            rb += qe * (T(3) * u2 - T(4)) + qs * (T(4) - T(3) * u2) - T(2) * (qqx * ux + qqy * uy);
            uxb += qe * T(6) * r * ux - qs * T(6) * r * ux + qqx * (s3 - T(2) * r);
            uyb += qe * T(6) * r * uy - qs * T(6) * r * uy + qqy * (s3 - T(2) * r);
            mub += T(2) * qe - T(3) * qs + qqx * ux + qqy * uy;
        }
        rb += qxx * (ux * ux - uy * uy) + qxy * ux * uy;
        uxb += qxx * T(2) * r * ux + qxy * r * uy;
        uyb += -qxx * T(2) * r * uy + qxy * r * ux;
        // forcing moments S = M G (Eq. 14) and correction C (Eq. 29)
        const T Fx = F.Fx[n.i], Fy = F.Fy[n.i];
        uxb += T(6) * Fx * (Se - Ss) + T(2) * Fx * Sxx + Fy * Sxy;
        uyb += T(6) * Fy * (Se - Ss) - T(2) * Fy * Sxx + Fx * Sxy;
        Fxb += T(6) * ux * (Se - Ss) - Sqx + T(2) * ux * Sxx + uy * Sxy;
        Fyb += T(6) * uy * (Se - Ss) - Sqy - T(2) * uy * Sxx + ux * Sxy;
        if (SCHEME == 1) {
            C1b = T(9) * Se;
            C7b = T(3) * Sxx;
        }
    }
    if (seed_u) {
        uxb += T(2) * F.ux[n.i];
        uyb += T(2) * F.uy[n.i];
    }
#pragma unroll
    for (int a = 0; a < kQ; ++a) lam_direct[a * N + n.i] = d[a];
    F.rb[n.i] = rb;
    F.jxb[n.i] = jxb;
    F.jyb[n.i] = jyb;
    F.uxb[n.i] = uxb;
    F.uyb[n.i] = uyb;
    F.Fxb[n.i] = Fxb;
    F.Fyb[n.i] = Fyb;
    F.mub[n.i] = mub;
    F.C1b[n.i] = C1b;
    F.C7b[n.i] = C7b;
}

// correction (Eq. 29), velocity (Eq. 12) and force (Eqs. 13/24) transposed
template <typename T, int SCHEME>
__global__ void adj_force(DevCase<T> c, AdjFields<T> F)
{
    NodeIdx n;
    if (!node_of(c.nx, c.ny, n)) return;
    const int64_t i = n.i;
    T rb = F.rb[i], uxb = F.uxb[i], uyb = F.uyb[i], mub = F.mub[i];
    if (SCHEME == 1) {
        // A-bar = G_x^T (C1b + C7b), B-bar = G_y^T (C1b - C7b)
        T Ab = T(0), Bb = T(0);
#pragma unroll
        for (int a = 1; a < kQ; ++a) {
            const int64_t j = n.at(-kEx[a], -kEy[a]);
            Ab += T(3.0 * kW[a] * kEx[a]) * (F.C1b[j] + F.C7b[j]);
            Bb += T(3.0 * kW[a] * kEy[a]) * (F.C1b[j] - F.C7b[j]);
        }
        const T phib = Ab * F.ux[i] + Bb * F.uy[i];
        uxb += F.phi[i] * Ab;
        uyb += F.phi[i] * Bb;
        rb += phib * T(1.0 / 3.0);
        mub -= phib * T(1.0 / 3.0);
    }
    const T r = F.rho[i];
    F.jxb[i] += uxb / r;
    F.jyb[i] += uyb / r;
    const T Fxb = F.Fxb[i] + T(0.5) * uxb / r, Fyb = F.Fyb[i] + T(0.5) * uyb / r;
    rb -= (uxb * F.ux[i] + uyb * F.uy[i]) / r;
    const T k = SCHEME == 1 ? T(1.0 / 3.0) - r : -r;
    F.gxb[i] = k * Fxb;
    F.gyb[i] = k * Fyb;
    rb -= F.gx[i] * Fxb + F.gy[i] * Fyb;
    F.Fxb[i] = Fxb;
    F.Fyb[i] = Fyb;
    F.rb[i] = rb;
    F.mub[i] = mub;
}

// grad mu_c transposed, mu_c = E_f' - kappa lap transposed; parameter partials
template <typename T, int SCHEME, int EOS>
__global__ void __launch_bounds__(256) adj_mu(DevCase<T> c, T R, AdjFields<T> F, Partial* partials)
{
    NodeIdx n;
    double gk = 0.0, gT = 0.0;
    if (node_of(c.nx, c.ny, n)) {
        const int64_t i = n.i;
        const T mub = F.mub[i] + gradT_at(F.gxb, n, 0) + gradT_at(F.gyb, n, 1);
        T rb = F.rb[i];
        if (SCHEME == 0) rb += (gradT_at(F.Fxb, n, 0) + gradT_at(F.Fyb, n, 1)) * T(1.0 / 3.0);
        rb += d2Ef_dev<EOS, T>(c, F.rho[i]) * mub;
        F.rb[i] = rb;
        F.Lb[i] = -c.kappa * mub;
        gk = -(double)mub * (double)F.lap[i];
        gT = (double)mub * (double)dEf_dT_dev<EOS, T>(c, F.rho[i], R);
    }
    block_partial<true>(gk, gT, 0.0, 0.0, partials);
}

// lap transposed; lam(x)_a = lam_direct + rho-bar + e_a . j-bar (+ final density seed)
template <typename T>
__global__ void adj_lambda(DevCase<T> c, AdjFields<T> F, const T* __restrict__ lam_direct,
                           const double* __restrict__ s_final, T* __restrict__ lam)
{
    NodeIdx n;
    if (!node_of(c.nx, c.ny, n)) return;
    const int64_t N = (int64_t)c.nx * c.ny;
    const T rb = F.rb[n.i] + lapT_at(F.Lb, n) + (s_final ? (T)s_final[n.i] : T(0));
    const T jxb = F.jxb[n.i], jyb = F.jyb[n.i];
#pragma unroll
    for (int a = 0; a < kQ; ++a)
        lam[a * N + n.i] = lam_direct[a * N + n.i] + rb + T(kEx[a]) * jxb + T(kEy[a]) * jyb;
}

// Initial populations f(0) = M^-1 m_eq(rho0, 0, mu(rho0)) transposed. F.rho,
// F.lap, F.mu hold the fields of rho0.
template <typename T, int SCHEME, int EOS>
__global__ void __launch_bounds__(256) adj_init(DevCase<T> c, T R, AdjFields<T> F, const T* __restrict__ lam0,
                                                Partial* partials)
{
    NodeIdx n;
    double gk = 0.0, gT = 0.0;
    if (node_of(c.nx, c.ny, n)) {
        const int64_t N = (int64_t)c.nx * c.ny;
        T L[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) L[a] = lam0[a * N + n.i];
        const T sa = (L[1] + L[3]) + (L[2] + L[4]), sd = (L[5] + L[7]) + (L[6] + L[8]);
        const T nr = (L[0] + sa + sd) * T(1.0 / 9.0);
        const T ne = (T(2) * sd - sa - T(4) * L[0]) * T(1.0 / 36.0);
        const T ns = (sd - T(2) * sa + T(4) * L[0]) * T(1.0 / 36.0);
        // m_eq at u = 0: rho (1, -2, 1, 0...) standard; (rho, -4 rho + 2 s, 4 rho - 3 s, 0...) improved
        T rb = nr, mub = T(0);
        if (SCHEME == 0) {
            rb += T(-2) * ne + ns;
        } else {
            rb += T(-4) * ne + T(4) * ns;
            mub = T(2) * ne - T(3) * ns;
        }
        const T r = F.rho[n.i];
        F.rb[n.i] = rb + d2Ef_dev<EOS, T>(c, r) * mub;
        F.Lb[n.i] = -c.kappa * mub;
        gk = -(double)mub * (double)F.lap[n.i];
        gT = (double)mub * (double)dEf_dT_dev<EOS, T>(c, r, R);
    }
    block_partial<true>(gk, gT, 0.0, 0.0, partials);
}

template <typename T>
__global__ void adj_init_out(DevCase<T> c, AdjFields<T> F, double* __restrict__ grad_rho0)
{
    NodeIdx n;
    if (!node_of(c.nx, c.ny, n)) return;
    grad_rho0[n.i] = (double)(F.rb[n.i] + lapT_at(F.Lb, n));
}

// acc[k] += fixed-order fold of field k of the partials (k = 0: mass slot, 1: ke slot)
static __global__ void adj_accumulate(const Partial* __restrict__ partials, int64_t n, double* __restrict__ acc0,
                                      double* __restrict__ acc1)
{
    __shared__ double s[2][256];
    double a = 0.0, b = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
        a += partials[k].mass;
        b += partials[k].ke;
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s[0][threadIdx.x] += s[0][threadIdx.x + w];
            s[1][threadIdx.x] += s[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (acc0) *acc0 += s[0][0];
        if (acc1) *acc1 += s[1][0];
    }
}

}  // namespace lbfe
