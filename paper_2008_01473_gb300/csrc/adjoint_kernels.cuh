// FP64 kernels of the discrete adjoint (reverse-mode derivative) of one time
// step, for lb_adjoint_step. One thread per node, 256-thread blocks over
// (ceil(nx / 256), ny). Fields are dense [ny][nx] FP64 arrays; the adjoint
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

struct AdjFields {
    // forward fields at the current state
    double *rho, *jx, *jy, *lap, *mu, *gx, *gy, *Fx, *Fy, *ux, *uy, *phi, *A, *B, *C1, *C7;
    // adjoint fields
    double *rb, *jxb, *jyb, *uxb, *uyb, *Fxb, *Fyb, *mub, *C1b, *C7b, *gxb, *gyb, *Lb;
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
__device__ __forceinline__ double grad_at(const double* v, const NodeIdx& n, int d)
{
    double s = 0.0;
#pragma unroll
    for (int a = 1; a < kQ; ++a) s += 3.0 * kW[a] * (d == 0 ? kEx[a] : kEy[a]) * v[n.at(kEx[a], kEy[a])];
    return s;
}
// transpose of the Eq. 17 component d: 3 sum_a w_a e_a v(x - e_a)
__device__ __forceinline__ double gradT_at(const double* v, const NodeIdx& n, int d)
{
    double s = 0.0;
#pragma unroll
    for (int a = 1; a < kQ; ++a) s += 3.0 * kW[a] * (d == 0 ? kEx[a] : kEy[a]) * v[n.at(-kEx[a], -kEy[a])];
    return s;
}
// transpose of the Laplacian 6 sum_a w_a (v(x + e_a) - v(x)): 6 sum_a w_a (v(x - e_a) - v(x))
__device__ __forceinline__ double lapT_at(const double* v, const NodeIdx& n)
{
    double s = 0.0;
    const double c = v[n.i];
#pragma unroll
    for (int a = 1; a < kQ; ++a) s += kW[a] * (v[n.at(-kEx[a], -kEy[a])] - c);
    return 6.0 * s;
}

template <int EOS>
__device__ __forceinline__ double d2Ef_dev(const DevCase<double>& c, double rho)
{
    if (EOS == 0) {
        const double q = 1.0 / (1.0 - c.b * rho);
        return c.RT * (1.0 / rho + c.b * q + c.b * q * q) - 2.0 * c.a;
    }
    const double n = 0.25 * c.b * rho, q = 1.0 / (1.0 - n);
    return c.RT * (1.0 / rho + 0.25 * c.b * (8.0 - 2.0 * n) * q * q * q * q) - 2.0 * c.a;
}
// R h(rho) = d E_f' / d T (R folded in: RT / T)
template <int EOS>
__device__ __forceinline__ double dEf_dT_dev(const DevCase<double>& c, double rho, double R)
{
    DevCase<double> u = c;
    u.RT = R;
    u.a = 0.0;
    return dEf<EOS, double>(u, rho);
}

// ---------------------------------------------------------------- forward
// lap and mu_c of the rho field
template <int EOS>
__global__ void adj_fwd_mu(DevCase<double> c, AdjFields F)
{
    NodeIdx n;
    if (!node_of(c.nx, c.ny, n)) return;
    double s = 0.0;
    const double r = F.rho[n.i];
#pragma unroll
    for (int a = 1; a < kQ; ++a) s += kW[a] * (F.rho[n.at(kEx[a], kEy[a])] - r);
    const double lap = 6.0 * s;
    F.lap[n.i] = lap;
    F.mu[n.i] = dEf<EOS, double>(c, r) - c.kappa * lap;
}

// grad mu_c, F, u, phi, A, B; loss partials: w_u sum |u|^2 + sum s rho
template <int SCHEME>
__global__ void __launch_bounds__(256) adj_fwd_force(DevCase<double> c, AdjFields F, double w_u,
                                                     const double* __restrict__ s_final, Partial* partials)
{
    NodeIdx n;
    double loss = 0.0;
    if (node_of(c.nx, c.ny, n)) {
        const double r = F.rho[n.i];
        const double gx = grad_at(F.mu, n, 0), gy = grad_at(F.mu, n, 1);
        double Fx, Fy;
        if (SCHEME == 1) {
            Fx = (1.0 / 3.0 - r) * gx;
            Fy = (1.0 / 3.0 - r) * gy;
        } else {
            Fx = grad_at(F.rho, n, 0) / 3.0 - r * gx;
            Fy = grad_at(F.rho, n, 1) / 3.0 - r * gy;
        }
        const double ux = (F.jx[n.i] + 0.5 * Fx) / r, uy = (F.jy[n.i] + 0.5 * Fy) / r;
        const double phi = (r - (c.c0 + F.mu[n.i])) / 3.0;
        F.gx[n.i] = gx;
        F.gy[n.i] = gy;
        F.Fx[n.i] = Fx;
        F.Fy[n.i] = Fy;
        F.ux[n.i] = ux;
        F.uy[n.i] = uy;
        F.phi[n.i] = phi;
        F.A[n.i] = phi * ux;
        F.B[n.i] = phi * uy;
        loss = w_u * (ux * ux + uy * uy) + (s_final ? s_final[n.i] * r : 0.0);
    }
    block_partial(loss, 0.0, 0.0, 0.0, partials);
}

__global__ void adj_fwd_corr(DevCase<double> c, AdjFields F)
{
    NodeIdx n;
    if (!node_of(c.nx, c.ny, n)) return;
    const double Ax = grad_at(F.A, n, 0), By = grad_at(F.B, n, 1);
    F.C1[n.i] = Ax + By;
    F.C7[n.i] = Ax - By;
}

// ---------------------------------------------------------------- reverse
// Collision adjoint at each node. lam_next: adjoint of the state after the
// step (node form); has_next = 0 for the final state (no collision term).
// Writes lam_direct (the part through m = M f) and initialises every adjoint
// field, adding the |u|^2 seed when seed_u != 0.
template <int SCHEME>
__global__ void adj_collide(DevCase<double> c, AdjFields F, const double* __restrict__ lam_next, int has_next,
                            int seed_u, double* __restrict__ lam_direct)
{
    NodeIdx n;
    if (!node_of(c.nx, c.ny, n)) return;
    const int64_t N = (int64_t)c.nx * c.ny;
    double rb = 0.0, jxb = 0.0, jyb = 0.0, uxb = 0.0, uyb = 0.0, Fxb = 0.0, Fyb = 0.0, mub = 0.0, C1b = 0.0,
           C7b = 0.0;
    double d[kQ];
    for (int a = 0; a < kQ; ++a) d[a] = 0.0;
    if (has_next) {
        // lam*(x) = lam_next(x + e_a): transpose of the streaming
        double L[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) L[a] = lam_next[a * N + n.at(kEx[a], kEy[a])];
        // nu = M^-T lam* = D M lam*
        const double sa = (L[1] + L[3]) + (L[2] + L[4]), sd = (L[5] + L[7]) + (L[6] + L[8]);
        const double nr = (L[0] + sa + sd) / 9.0;
        const double ne = (2.0 * sd - sa - 4.0 * L[0]) / 36.0;
        const double ns = (sd - 2.0 * sa + 4.0 * L[0]) / 36.0;
        const double njx = ((L[1] - L[3]) + (L[5] - L[7]) + (L[8] - L[6])) / 6.0;
        const double nqx = (-2.0 * (L[1] - L[3]) + (L[5] - L[7]) + (L[8] - L[6])) / 12.0;
        const double njy = ((L[2] - L[4]) + (L[5] - L[7]) + (L[6] - L[8])) / 6.0;
        const double nqy = (-2.0 * (L[2] - L[4]) + (L[5] - L[7]) + (L[6] - L[8])) / 12.0;
        const double npxx = ((L[1] + L[3]) - (L[2] + L[4])) / 4.0;
        const double npxy = ((L[5] + L[7]) - (L[6] + L[8])) / 4.0;
        const double le = c.lam_e, ls = c.lam_s, lq = c.lam_q, lv = c.lam_v;
        // m* = m + lam (eq - m) + h S (non-conserved), rho* = rho, j* = j + F
        const double mbe = (1.0 - le) * ne, mbs = (1.0 - ls) * ns, mbqx = (1.0 - lq) * nqx,
                     mbqy = (1.0 - lq) * nqy, mbxx = (1.0 - lv) * npxx, mbxy = (1.0 - lv) * npxy;
        const double qe = le * ne, qs = ls * ns, qqx = lq * nqx, qqy = lq * nqy, qxx = lv * npxx, qxy = lv * npxy;
        const double Se = (1.0 - 0.5 * le) * ne, Ss = (1.0 - 0.5 * ls) * ns, Sqx = (1.0 - 0.5 * lq) * nqx,
                     Sqy = (1.0 - 0.5 * lq) * nqy, Sxx = (1.0 - 0.5 * lv) * npxx, Sxy = (1.0 - 0.5 * lv) * npxy;
        rb += nr;
        jxb += njx;
        jyb += njy;
        Fxb += njx;
        Fyb += njy;
        // direct part: M_nc^T m-bar (rows e, eps, q_x, q_y, p_xx, p_xy of M)
        d[0] = -4.0 * mbe + 4.0 * mbs;
        d[1] = -mbe - 2.0 * mbs - 2.0 * mbqx + mbxx;
        d[2] = -mbe - 2.0 * mbs - 2.0 * mbqy - mbxx;
        d[3] = -mbe - 2.0 * mbs + 2.0 * mbqx + mbxx;
        d[4] = -mbe - 2.0 * mbs + 2.0 * mbqy - mbxx;
        d[5] = 2.0 * mbe + mbs + mbqx + mbqy + mbxy;
        d[6] = 2.0 * mbe + mbs - mbqx + mbqy - mbxy;
        d[7] = 2.0 * mbe + mbs - mbqx - mbqy + mbxy;
        d[8] = 2.0 * mbe + mbs + mbqx - mbqy - mbxy;
        // equilibria (Eq. 11 / Eq. 27)
        const double r = F.rho[n.i], ux = F.ux[n.i], uy = F.uy[n.i], u2 = ux * ux + uy * uy;
        if (SCHEME == 0) {
            rb += qe * (3.0 * u2 - 2.0) + qs * (1.0 - 3.0 * u2) - qqx * ux - qqy * uy;
            uxb += qe * 6.0 * r * ux - qs * 6.0 * r * ux - qqx * r;
            uyb += qe * 6.0 * r * uy - qs * 6.0 * r * uy - qqy * r;
        } else {
            const double s3 = c.c0 + F.mu[n.i];
            rb += qe * (3.0 * u2 - 4.0) + qs * (4.0 - 3.0 * u2) - 2.0 * (qqx * ux + qqy * uy);
            uxb += qe * 6.0 * r * ux - qs * 6.0 * r * ux + qqx * (s3 - 2.0 * r);
            uyb += qe * 6.0 * r * uy - qs * 6.0 * r * uy + qqy * (s3 - 2.0 * r);
            mub += 2.0 * qe - 3.0 * qs + qqx * ux + qqy * uy;
        }
        rb += qxx * (ux * ux - uy * uy) + qxy * ux * uy;
        uxb += qxx * 2.0 * r * ux + qxy * r * uy;
        uyb += -qxx * 2.0 * r * uy + qxy * r * ux;
        // forcing moments S = M G (Eq. 14) and correction C (Eq. 29)
        const double Fx = F.Fx[n.i], Fy = F.Fy[n.i];
        uxb += 6.0 * Fx * (Se - Ss) + 2.0 * Fx * Sxx + Fy * Sxy;
        uyb += 6.0 * Fy * (Se - Ss) - 2.0 * Fy * Sxx + Fx * Sxy;
        Fxb += 6.0 * ux * (Se - Ss) - Sqx + 2.0 * ux * Sxx + uy * Sxy;
        Fyb += 6.0 * uy * (Se - Ss) - Sqy - 2.0 * uy * Sxx + ux * Sxy;
        if (SCHEME == 1) {
            C1b = 9.0 * Se;
            C7b = 3.0 * Sxx;
        }
    }
    if (seed_u) {
        uxb += 2.0 * F.ux[n.i];
        uyb += 2.0 * F.uy[n.i];
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
template <int SCHEME>
__global__ void adj_force(DevCase<double> c, AdjFields F)
{
    NodeIdx n;
    if (!node_of(c.nx, c.ny, n)) return;
    const int64_t i = n.i;
    double rb = F.rb[i], uxb = F.uxb[i], uyb = F.uyb[i], mub = F.mub[i];
    if (SCHEME == 1) {
        // A-bar = G_x^T (C1b + C7b), B-bar = G_y^T (C1b - C7b)
        double Ab = 0.0, Bb = 0.0;
#pragma unroll
        for (int a = 1; a < kQ; ++a) {
            const int64_t j = n.at(-kEx[a], -kEy[a]);
            Ab += 3.0 * kW[a] * kEx[a] * (F.C1b[j] + F.C7b[j]);
            Bb += 3.0 * kW[a] * kEy[a] * (F.C1b[j] - F.C7b[j]);
        }
        const double phib = Ab * F.ux[i] + Bb * F.uy[i];
        uxb += F.phi[i] * Ab;
        uyb += F.phi[i] * Bb;
        rb += phib / 3.0;
        mub -= phib / 3.0;
    }
    const double r = F.rho[i];
    F.jxb[i] += uxb / r;
    F.jyb[i] += uyb / r;
    const double Fxb = F.Fxb[i] + 0.5 * uxb / r, Fyb = F.Fyb[i] + 0.5 * uyb / r;
    rb -= (uxb * F.ux[i] + uyb * F.uy[i]) / r;
    const double k = SCHEME == 1 ? 1.0 / 3.0 - r : -r;
    F.gxb[i] = k * Fxb;
    F.gyb[i] = k * Fyb;
    rb -= F.gx[i] * Fxb + F.gy[i] * Fyb;
    F.Fxb[i] = Fxb;
    F.Fyb[i] = Fyb;
    F.rb[i] = rb;
    F.mub[i] = mub;
}

// grad mu_c transposed, mu_c = E_f' - kappa lap transposed; parameter partials
template <int SCHEME, int EOS>
__global__ void __launch_bounds__(256) adj_mu(DevCase<double> c, double R, AdjFields F, Partial* partials)
{
    NodeIdx n;
    double gk = 0.0, gT = 0.0;
    if (node_of(c.nx, c.ny, n)) {
        const int64_t i = n.i;
        const double mub = F.mub[i] + gradT_at(F.gxb, n, 0) + gradT_at(F.gyb, n, 1);
        double rb = F.rb[i];
        if (SCHEME == 0) rb += (gradT_at(F.Fxb, n, 0) + gradT_at(F.Fyb, n, 1)) / 3.0;
        rb += d2Ef_dev<EOS>(c, F.rho[i]) * mub;
        F.rb[i] = rb;
        F.Lb[i] = -c.kappa * mub;
        gk = -mub * F.lap[i];
        gT = mub * dEf_dT_dev<EOS>(c, F.rho[i], R);
    }
    block_partial(gk, gT, 0.0, 0.0, partials);
}

// lap transposed; lam(x)_a = lam_direct + rho-bar + e_a . j-bar (+ final density seed)
__global__ void adj_lambda(DevCase<double> c, AdjFields F, const double* __restrict__ lam_direct,
                           const double* __restrict__ s_final, double* __restrict__ lam)
{
    NodeIdx n;
    if (!node_of(c.nx, c.ny, n)) return;
    const int64_t N = (int64_t)c.nx * c.ny;
    const double rb = F.rb[n.i] + lapT_at(F.Lb, n) + (s_final ? s_final[n.i] : 0.0);
    const double jxb = F.jxb[n.i], jyb = F.jyb[n.i];
#pragma unroll
    for (int a = 0; a < kQ; ++a) lam[a * N + n.i] = lam_direct[a * N + n.i] + rb + kEx[a] * jxb + kEy[a] * jyb;
}

// Initial populations f(0) = M^-1 m_eq(rho0, 0, mu(rho0)) transposed. F.rho,
// F.lap, F.mu hold the fields of rho0.
template <int SCHEME, int EOS>
__global__ void __launch_bounds__(256) adj_init(DevCase<double> c, double R, AdjFields F,
                                                const double* __restrict__ lam0, Partial* partials)
{
    NodeIdx n;
    double gk = 0.0, gT = 0.0;
    if (node_of(c.nx, c.ny, n)) {
        const int64_t N = (int64_t)c.nx * c.ny;
        double L[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) L[a] = lam0[a * N + n.i];
        const double sa = (L[1] + L[3]) + (L[2] + L[4]), sd = (L[5] + L[7]) + (L[6] + L[8]);
        const double nr = (L[0] + sa + sd) / 9.0;
        const double ne = (2.0 * sd - sa - 4.0 * L[0]) / 36.0;
        const double ns = (sd - 2.0 * sa + 4.0 * L[0]) / 36.0;
        // m_eq at u = 0: rho (1, -2, 1, 0...) standard; (rho, -4 rho + 2 s, 4 rho - 3 s, 0...) improved
        double rb = nr, mub = 0.0;
        if (SCHEME == 0) {
            rb += -2.0 * ne + ns;
        } else {
            rb += -4.0 * ne + 4.0 * ns;
            mub = 2.0 * ne - 3.0 * ns;
        }
        const double r = F.rho[n.i];
        F.rb[n.i] = rb + d2Ef_dev<EOS>(c, r) * mub;
        F.Lb[n.i] = -c.kappa * mub;
        gk = -mub * F.lap[n.i];
        gT = mub * dEf_dT_dev<EOS>(c, r, R);
    }
    block_partial(gk, gT, 0.0, 0.0, partials);
}

__global__ void adj_init_out(DevCase<double> c, AdjFields F, double* __restrict__ grad_rho0)
{
    NodeIdx n;
    if (!node_of(c.nx, c.ny, n)) return;
    grad_rho0[n.i] = F.rb[n.i] + lapT_at(F.Lb, n);
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
