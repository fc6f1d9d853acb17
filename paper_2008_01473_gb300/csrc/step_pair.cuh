// FP32 fused step with two lattice columns per thread and packed FP32
// arithmetic (FADD2 / FMUL2 / FFMA2 of sm_100+), fed by a ring of stored rows
// that bulk asynchronous copies (cp.async.bulk, the TMA helpers of
// step_tma.cuh) fill two rows ahead of use.
//
// Same method and stage plan as step_kernel.cuh (A: pull, rho, j; B: mu_c;
// C: grad mu_c, F, u, phi u; D: correction C1/C7, collision, store), but
// thread p of the NP compute threads owns the two adjacent ring
// columns j = 2p and 2p + 1, i.e. lattice columns x0 - 4 + j and x0 - 3 + j.
// Every per-node quantity is a float2 (.x = column j, .y = column j + 1), so
// one packed instruction advances two nodes. In the five-point neighbourhoods
// of the stencils the pair's own values come from registers; only the columns
// j - 1 and j + 2 are read from the shared-memory field rows. Populations
// are stored with 64-bit stores (x0 and wv are multiples of 4).
//
// Ring: SL = 5 slots of one stored row (nine planes over the block's columns
// [x0 - 4, x0 + wv + 4)), one full-mbarrier each. Stored row i = s - s0 lives
// in slot i % SL, phase (i / SL) & 1. Stage A of iteration it reads rows
// it .. it + 2; after the block barrier that follows it, row it is dead, and
// at the end of the iteration (after stage D's stores, off the path of the
// three barrier intervals) lanes of warps 0..2 refill its slot with row
// it + SL (one lane per plane and run), so no producer warp is needed and
// three blocks fit on an SM. The slots, their
// mbarriers and phases, the refill row and the output row advance by one per
// iteration through wrapping pointer and offset updates: no row modulo or
// multiply sits on the iteration's path.
//
// Stage A reduces the pulled populations at once to the conserved sums and
// the six non-conserved moments of Eq. 9; the register rows carry those
// (12 registers per row instead of 18) until stage D relaxes them and
// transforms back.
//
// Two block shapes share the code: NP = 128 threads (256 ring columns,
// strips of up to 248 outputs; copies issued by warps 0-2, three planes
// each) for wide lattices, and NP = 64 (128 columns, strips of up to 120;
// warps 0-1 issue five and four planes) for narrow ones. A node's arithmetic
// does not depend on the shape, so both give the same bits.
//
// Column coverage per stage (ring columns; wv = strip width, halo HX):
//   A: all pairs (columns the ring does not hold give unused values)
//   B: pairs 1 .. (wv + 6)/2 - 1   -> columns [2, wv + 6)
//   C: same pairs (improved)       -> columns [2, wv + 6)
//   D: pairs 2 .. (wv + 4)/2 - 1   -> columns [4, wv + 4) = the strip
// The improved scheme needs rho on [1, wv + 7), mu_c on [2, wv + 6) and phi u
// on [3, wv + 5); the standard one rho on [2, wv + 6) and mu_c on [3, wv + 5).
//
// Scheme 3 (Eq. 29's derivatives of the lattice-weight average of phi u, a
// 5 x 5 stencil) reaches one column and one row further: the ring spans
// [x0 - 8, x0 + wv + 8) (a margin of 8 keeps the copies 16-byte aligned), phi u
// is needed on [6, wv + 10), mu_c on [5, wv + 11), rho on [3, wv + 13); stage
// D runs four rows behind stage A. The stencil factors into an x-part per
// phi u row and a y-combination of five rows: each iteration takes the
// x-part of the newest row (one shared phi u row) and keeps those of the last
// four rows in registers. Five rows of pulled populations do not fit the
// registers of three blocks per SM, so stage D reads its row's pull again,
// from a second ring of two slots: slot m & 1 holds the pull of output row
// y0 + m (plane a copied from stored row y0 + m - e_ay, so the nine planes of
// one slot come from three stored rows; with walls, a source row beyond a
// wall is taken as the mirror row's reflected plane, as in stage A's ring),
// filled by bulk copies from L2 (stage A's copies brought those rows in four
// iterations earlier) right after the first barrier that follows the
// collision of the slot's previous row, six barrier intervals before stage D
// needs it.
#pragma once

#include "step_tma.cuh"

namespace lbfe {

constexpr int kPairThreads = 128;             // compute threads per block, wide shape
constexpr int kPairCols = 2 * kPairThreads;   // ring / field columns per block, wide shape
constexpr int kPairThreadsNarrow = 64;        // the narrow shape
constexpr int kPairSlots = 5;                 // ring slots: 3 rows in use, 2 in flight

// threads that issue a stored row's bulk copies: three warps (wide), two (narrow)
__host__ __device__ constexpr int pair_issuers(int np) { return np == kPairThreads ? 96 : 64; }

// ------------------------------------------------------------ packed FP32
__device__ __forceinline__ float2 v2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return __fadd2_rn(a, b); }
// packed subtraction (sub.rn.f32x2; an FFMA2 with a (-1, -1) operand would
// need a register pair holding the constant)
__device__ __forceinline__ float2 operator-(float2 a, float2 b)
{
    unsigned long long r;
    const unsigned long long x = *reinterpret_cast<const unsigned long long*>(&a);
    const unsigned long long y = *reinterpret_cast<const unsigned long long*>(&b);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
    return *reinterpret_cast<const float2*>(&r);
}
__device__ __forceinline__ float2 operator*(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ void st2(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }

// Row of a field around the pair: own (x = col j, y = col j + 1) plus the
// neighbours at j - 1 (l) and j + 2 (r). The stencils below combine the
// shifted neighbours with scalar adds that write each half of a pair
// directly (a packed operation on the shifted pair (c.y, r) would first
// have to assemble it in an aligned register pair), then go on packed.
struct Row2 {
    float2 c;
    float l, r;
};

// neighbours through aligned 64-bit loads (a stride-2 scalar pattern would
// hit each shared-memory bank twice); needs 2 <= j <= (ring columns) - 4
__device__ __forceinline__ Row2 row2(const float* row, int j, float2 own)
{
    Row2 q;
    q.c = own;
    q.l = ld2(row + j - 2).y;
    q.r = ld2(row + j + 2).x;
    return q;
}

// 6 sum_a w_a (phi(x + e_a) - phi(x)) with rows S (y-1), C (y), N (y+1)
__device__ __forceinline__ float2 lap2(const Row2& S, const Row2& C, const Row2& N)
{
    const float2 ew = make_float2(C.c.y + C.l, C.r + C.c.x);      // E + W
    const float2 nesw = make_float2(N.c.y + S.l, N.r + S.c.x);    // NE + SW
    const float2 nwse = make_float2(N.l + S.c.y, N.c.x + S.r);    // NW + SE
    const float2 edges = ew + (N.c + S.c);
    const float2 corners = nesw + nwse;
    return fma2(edges, v2(4.0f / 6.0f), fma2(corners, v2(1.0f / 6.0f), C.c * v2(-20.0f / 6.0f)));
}

// Eq. 17 components
__device__ __forceinline__ float2 gx2(const Row2& S, const Row2& C, const Row2& N)
{
    const float2 d = make_float2(C.c.y - C.l, C.r - C.c.x);       // E - W
    const float2 a = make_float2(N.c.y - S.l, N.r - S.c.x);       // NE - SW
    const float2 b = make_float2(S.c.y - N.l, S.r - N.c.x);       // SE - NW
    return fma2(d, v2(1.0f / 3.0f), (a + b) * v2(1.0f / 12.0f));
}
__device__ __forceinline__ float2 gy2(const Row2& S, const Row2& N)
{
    const float2 a = make_float2(N.c.y - S.l, N.r - S.c.x);       // NE - SW
    const float2 b = make_float2(N.l - S.c.y, N.c.x - S.r);       // NW - SE
    return fma2(N.c - S.c, v2(1.0f / 3.0f), (a + b) * v2(1.0f / 12.0f));
}

template <int EOS>
__device__ __forceinline__ float2 dEf2(const DevCase<float>& c, float2 rho)
{
    float2 out;
    if (EOS == 0) {
        const float2 r = make_float2(__fdividef(1.0f, fmaf(-c.b, rho.x, 1.0f)),
                                     __fdividef(1.0f, fmaf(-c.b, rho.y, 1.0f)));
        const float2 lg = make_float2(__logf(rho.x * r.x), __logf(rho.y * r.y));
        out = fma2(v2(c.RT), lg + r, rho * v2(-2.0f * c.a));
    } else {
        const float2 n = rho * v2(0.25f * c.b);
        const float2 r = make_float2(__fdividef(1.0f, 1.0f - n.x), __fdividef(1.0f, 1.0f - n.y));
        const float2 r2 = r * r;
        const float2 lg = make_float2(__logf(rho.x), __logf(rho.y));
        const float2 t1 = n * (v2(4.0f) - v2(3.0f) * n) * r2;
        const float2 t2 = n * (v2(4.0f) - v2(2.0f) * n) * r2 * r;
        out = fma2(v2(c.RT), lg + v2(1.0f) + t1 + t2, rho * v2(-2.0f * c.a));
    }
    return out;
}

// The six non-conserved moments (e, eps, q_x, q_y, p_xx, p_xy of the
// Lallemand-Luo basis, Eq. 9) of the pair's deviation populations. Stage A
// takes them right after the pull and the register rows carry these six
// instead of the nine populations until stage D collides.
__device__ __forceinline__ void moments2(const float2 (&d)[kQ], float2 (&m)[6])
{
    const float2 sa = (d[1] + d[3]) + (d[2] + d[4]);
    const float2 sd = (d[5] + d[7]) + (d[6] + d[8]);
    m[0] = fma2(v2(2.0f), sd, fma2(v2(-4.0f), d[0], v2(0.0f) - sa));
    m[1] = fma2(v2(-2.0f), sa, fma2(v2(4.0f), d[0], sd));
    const float2 d57 = d[5] - d[7];
    const float2 dxd = d57 + (d[8] - d[6]);
    const float2 dyd = d57 + (d[6] - d[8]);
    m[2] = fma2(v2(-2.0f), d[1] - d[3], dxd);
    m[3] = fma2(v2(-2.0f), d[2] - d[4], dyd);
    m[4] = (d[1] + d[3]) - (d[2] + d[4]);
    m[5] = (d[5] + d[7]) - (d[6] + d[8]);
}

// Moment-space collision (Eqs. 9 / 28) on deviation populations, packed:
// post-collision deviation populations d from the conserved (drho, jx, jy)
// and the non-conserved moments m. Same algebra as collide() in
// lbfe_device.cuh.
template <int SCHEME>
__device__ __forceinline__ void collide2m(float2 (&d)[kQ], const float2 (&m)[6], float2 drho, float2 rho,
                                          float2 jx, float2 jy, float2 ux, float2 uy, float2 Fx, float2 Fy,
                                          float2 mu, float2 C1, float2 C7, const DevCase<float>& c, float2 le,
                                          float2 ls, float2 lq, float2 lv)
{
    const float2 m_e = m[0], m_s = m[1], m_qx = m[2], m_qy = m[3], m_pxx = m[4], m_pxy = m[5];

    const float2 uxx = ux * ux, uyy = uy * uy;
    const float2 ru2 = rho * (uxx + uyy);
    float2 eq_e, eq_s, eq_qx, eq_qy;
    if (!improved_scheme(SCHEME)) {  // standard equilibrium (Eq. 11), either force form
        eq_e = fma2(v2(3.0f), ru2, v2(-2.0f) * drho);
        eq_s = fma2(v2(-3.0f), ru2, drho);
        eq_qx = v2(0.0f) - rho * ux;
        eq_qy = v2(0.0f) - rho * uy;
    } else {
        const float2 pm3 = v2(c.c0) + mu;  // 3 p_m
        eq_e = fma2(v2(3.0f), ru2, fma2(v2(-4.0f), rho, fma2(v2(2.0f), pm3, v2(2.0f * c.rho_ref))));
        eq_s = fma2(v2(-3.0f), ru2, fma2(v2(4.0f), rho, fma2(v2(-3.0f), pm3, v2(-c.rho_ref))));
        const float2 g2 = fma2(v2(-2.0f), rho, pm3);  // rho (gamma - 2)
        eq_qx = g2 * ux;
        eq_qy = g2 * uy;
    }
    const float2 eq_pxx = rho * (uxx - uyy);
    const float2 eq_pxy = rho * ux * uy;

    const float2 uF = fma2(ux, Fx, uy * Fy);
    const float2 S_e = fma2(v2(6.0f), uF, v2(9.0f) * C1);
    const float2 S_pxx = fma2(v2(2.0f), fma2(ux, Fx, v2(0.0f) - uy * Fy), v2(3.0f) * C7);
    const float2 S_pxy = fma2(ux, Fy, uy * Fx);

    // m* = m - lam (m - eq) + (1 - lam/2) S
    const float2 he = fma2(v2(-0.5f), le, v2(1.0f)), hs = fma2(v2(-0.5f), ls, v2(1.0f));
    const float2 hq = fma2(v2(-0.5f), lq, v2(1.0f)), hv = fma2(v2(-0.5f), lv, v2(1.0f));
    const float2 pe = fma2(he, S_e, fma2(le, eq_e - m_e, m_e));
    const float2 ps = fma2(hs, v2(-6.0f) * uF, fma2(ls, eq_s - m_s, m_s));
    const float2 pqx = fma2(v2(0.0f) - hq, Fx, fma2(lq, eq_qx - m_qx, m_qx));
    const float2 pqy = fma2(v2(0.0f) - hq, Fy, fma2(lq, eq_qy - m_qy, m_qy));
    const float2 pxx = fma2(hv, S_pxx, fma2(lv, eq_pxx - m_pxx, m_pxx));
    const float2 pxy = fma2(hv, S_pxy, fma2(lv, eq_pxy - m_pxy, m_pxy));

    // f* = M^-1 m*
    const float2 a0 = drho * v2(1.0f / 9.0f);
    const float2 a1 = pe * v2(1.0f / 36.0f);
    const float2 a2 = ps * v2(1.0f / 36.0f);
    const float2 a3 = (jx + Fx) * v2(1.0f / 6.0f);
    const float2 a4 = pqx * v2(1.0f / 12.0f);
    const float2 a5 = (jy + Fy) * v2(1.0f / 6.0f);
    const float2 a6 = pqy * v2(1.0f / 12.0f);
    const float2 a7 = pxx * v2(0.25f);
    const float2 a8 = pxy * v2(0.25f);
    const float2 b_ax = fma2(v2(-2.0f), a2, a0 - a1);
    const float2 b_dg = fma2(v2(2.0f), a1, a0 + a2);
    const float2 ex = fma2(v2(-2.0f), a4, a3), ey = fma2(v2(-2.0f), a6, a5);
    const float2 X = a3 + a4, Y = a5 + a6;
    d[1] = (b_ax + ex) + a7;
    d[3] = (b_ax - ex) + a7;
    d[2] = (b_ax + ey) - a7;
    d[4] = (b_ax - ey) - a7;
    d[5] = (b_dg + (X + Y)) + a8;
    d[7] = (b_dg - (X + Y)) + a8;
    d[6] = (b_dg + (Y - X)) - a8;
    d[8] = (b_dg + (X - Y)) - a8;
    // Rest population last, from the conserved density (m*_rho = drho):
    // d0 = drho - the sum of the eight moving ones. In exact arithmetic this
    // is the M^-1 row a0 - 4 (a1 - a2); in FP32 it keeps the stored density
    // equal to the pulled one up to the rounding of two sums, where nine
    // independently rounded rows of magnitude |drho| drift the mass
    // systematically once the flow is steady (the same rounding every step).
    d[0] = drho - (((d[1] + d[3]) + (d[2] + d[4])) + ((d[5] + d[7]) + (d[6] + d[8])));
}

// the same collision from the populations (in place)
template <int SCHEME>
__device__ __forceinline__ void collide2(float2 (&d)[kQ], float2 drho, float2 rho, float2 jx, float2 jy,
                                         float2 ux, float2 uy, float2 Fx, float2 Fy, float2 mu, float2 C1,
                                         float2 C7, const DevCase<float>& c, float2 le, float2 ls, float2 lq,
                                         float2 lv)
{
    float2 m[6];
    moments2(d, m);
    collide2m<SCHEME>(d, m, drho, rho, jx, jy, ux, uy, Fx, Fy, mu, C1, C7, c, le, ls, lq, lv);
}

// Ring columns on each side of a strip (a multiple of 4, for 16-byte aligned
// bulk copies): the stencil chain's column halo plus one for the pull.
template <int SCHEME>
struct PairGeom {
    static constexpr int M = SCHEME == 3 ? 8 : 4;
    static constexpr int NPU = SCHEME == 0 || SCHEME == 3 ? 1 : 4;  // rows of the phi u rings
    static constexpr int SL = kPairSlots;                           // slots of stage A's ring
    static constexpr int SD = SCHEME == 3 ? 2 : 0;                  // slots of stage D's ring
};

template <int SCHEME, int COLS>
struct PairSmem {
    float rho[4][COLS];
    float mu[4][COLS];
    float pux[PairGeom<SCHEME>::NPU][COLS];  // phi u_x (improved) or P_xy (pressure tensor)
    float puy[PairGeom<SCHEME>::NPU][COLS];  // phi u_y (improved) or P_yy (pressure tensor)
};

template <int SCHEME>
struct PairRegs {
    float2 m[SCHEME == 3 ? 1 : 4][6];  // non-conserved moments of the pulled pair (scheme 3 pulls again in D)
    float2 drho[4], jx[4], jy[4];
    float2 mu[4];
    float2 ux[SCHEME == 3 ? 4 : 2], uy[SCHEME == 3 ? 4 : 2];  // stage C results (improved)
    float2 Fx[SCHEME == 3 ? 4 : 2], Fy[SCHEME == 3 ? 4 : 2];
    float2 grx, gry;  // stage B grad rho (standard)
    // scheme 3: x-parts of the correction's stencil of phi u rows ra - 6 .. ra - 3;
    // row ra - 2 - d (taken d iterations ago) in slot (SLOT - d) & 3
    float2 hx[SCHEME == 3 ? 4 : 1], sb[SCHEME == 3 ? 4 : 1];
    float2 am, ak;    // statistics of the stage D nodes: sums of rho - rho_ref and rho |u|^2
    float au;         // and the largest |u|^2
};

template <int SCHEME>
__device__ __forceinline__ void pair_stats(PairRegs<SCHEME>& R, float2 drho, float2 rho, float2 ux, float2 uy)
{
    const float2 u2 = fma2(ux, ux, uy * uy);
    R.am = R.am + drho;
    R.ak = fma2(rho, u2, R.ak);
    R.au = fmaxf(R.au, fmaxf(u2.x, u2.y));
}

struct PairCtx {
    float* ring;        // [SL][9][ring columns], then scheme 3's [SD][9][ring columns]
    uint64_t* full;
    int* flag;
    int* status;
    const float* fin;   // this case's stored populations
    int s0, s_last;     // first / last stored window row of the block
    TmaRuns runs;       // column runs of one stored row (periodic split)
    uint32_t row_bytes;
    int j;              // ring column of the pair's first node
    int jm, jq;         // ring columns j - 1 and j + 2, clamped to the ring
    bool b, c, d;       // pair active in stages B/C, D
    // ring slots advance by pointer: the slots of stored rows it, it + 1,
    // it + 2 (stage A's three rows; the first is refilled at the end of the
    // iteration), the mbarriers of the slots of rows it and it + 2, and the
    // phase parity that row it + 2 completes
    float *pRm, *pR0, *pRp;
    uint64_t *fm, *f2;
    uint32_t par2;
    uint32_t irow;      // row offset (row * pitch) of the next refill, stored row it + SL
    uint32_t plane_rows; // ny * pitch
    int rd;             // lattice row of stage D
    float* out;         // fout + column of the pair's first node (stage D pairs)
    float* orow;        // out + rd * pitch
    int* bad;           // shared: a stage D node had rho <= 0 or a non-finite density
    uint32_t drow;      // scheme 3: row offset of this lane's plane for the next stage D copy
    // this thread's share of a row refill: one (plane, run) copy, or none
    const float* iss_src;  // source of the copy in row 0
    uint32_t iss_dst;      // ring offset of the copy within a slot (floats)
    uint32_t iss_dst_refl; // the same for a ghost row beyond a wall (plane reflected in y)
    uint32_t iss_bytes;
    int iss_ey;            // e_ay of the copy's plane (stage D's ring of scheme 3, with walls)
    bool iss_on;
};

// The pull of Eq. 10 for the pair from ring rows holding stored rows y - 1
// (Rm), y (R0) and y + 1 (Rp), or from one slot of stage D's ring that holds
// each plane's source row already (Rm = R0 = Rp): plane a from the row of
// y - e_ay, column x - e_ax. The planes that shift in x take one scalar load
// per node, straight into its half of the pair (the outermost pairs of the
// block read clamped columns jm, jq and produce unused values).
template <int SW>
__device__ __forceinline__ void pull_ring(float2 (&F)[kQ], const float* Rm, const float* R0, const float* Rp, int j,
                                          int jm, int jq)
{
    F[0] = ld2(R0 + 0 * SW + j);
    F[1] = make_float2(R0[1 * SW + jm], R0[1 * SW + j]);
    F[2] = ld2(Rm + 2 * SW + j);
    F[3] = make_float2(R0[3 * SW + j + 1], R0[3 * SW + jq]);
    F[4] = ld2(Rp + 4 * SW + j);
    F[5] = make_float2(Rm[5 * SW + jm], Rm[5 * SW + j]);
    F[6] = make_float2(Rm[6 * SW + j + 1], Rm[6 * SW + jq]);
    F[7] = make_float2(Rp[7 * SW + j + 1], Rp[7 * SW + jq]);
    F[8] = make_float2(Rp[8 * SW + jm], Rp[8 * SW + j]);
}

// rho > 0 and finite for both nodes of a pair (NaN fails both comparisons)
__device__ __forceinline__ bool pair_ok(float2 rho)
{
    return rho.x > 0.0f && rho.x <= 3.402823466e38f && rho.y > 0.0f && rho.y <= 3.402823466e38f;
}

__device__ __forceinline__ void pair_timeout(const PairCtx& X)
{
    *X.flag = 1;
    atomicOr(X.status, 1);
}

// This thread's share of every row copy, fixed for the block: thread 0 arms
// a slot's mbarrier with the row's byte count, and each lane of an issuing
// warp copies one (plane, run) pair: wide shape, warp w < 3 takes planes
// 3w .. 3w + 2; narrow shape, warp 0 planes 0-4, warp 1 planes 5-8. Returns
// e_ay of the thread's plane (stage D's ring copies plane a from row y - e_ay).
template <int NP>
__device__ __forceinline__ int pair_issue_setup(PairCtx& X, const DevCase<float>& c)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int pw = NP == kPairThreads ? 3 : (w == 0 ? 5 : 4);  // planes of this warp
    const int a0 = NP == kPairThreads ? 3 * w : (w == 0 ? 0 : 5);
    X.iss_on = threadIdx.x < pair_issuers(NP) && lane < pw * X.runs.n;
    const int a = X.iss_on ? a0 + lane % pw : 0, r = X.iss_on ? lane / pw : 0;
    const int g0 = r == 0 ? X.runs.g0[0] : (r == 1 ? X.runs.g0[1] : X.runs.g0[2]);
    const int j0 = r == 0 ? X.runs.j0[0] : (r == 1 ? X.runs.j0[1] : X.runs.j0[2]);
    const int len = r == 0 ? X.runs.len[0] : (r == 1 ? X.runs.len[1] : X.runs.len[2]);
    constexpr int refl[kQ] = {0, 1, 4, 3, 2, 8, 7, 6, 5};  // e_a with e_y negated
    X.iss_src = X.fin + ((uint32_t)a * (uint32_t)c.plane + (uint32_t)g0);
    X.iss_dst = (uint32_t)(a * 2 * NP + j0);
    X.iss_dst_refl = (uint32_t)(refl[a] * 2 * NP + j0);
    X.iss_bytes = (uint32_t)len * sizeof(float);
    return (a == 2 || a == 5 || a == 6) ? 1 : (a == 4 || a == 7 || a == 8) ? -1 : 0;
}

// Row offset of the stored row that fills window row s, and whether the slot
// takes its planes reflected in y: periodic lattices wrap; with walls, a
// ghost row beyond a wall is the mirror image of row nb_row(s) (R19), whose
// populations the slot holds reflected (2 <-> 4, 5 <-> 8, 6 <-> 7), so that
// the plain pull of stage A reads the mirrored state.
__device__ __forceinline__ uint32_t window_row(const DevCase<float>& c, int s, bool& reflected)
{
    const int m = c.walls ? nb_row(c, s) : wrapi(s, c.ny);
    reflected = c.walls && m != s;
    return (uint32_t)m * c.pitch;
}

// Copy the stored row at row offset `row` (row * pitch) into a slot whose
// mbarrier is `bar`, its planes reflected in y if `refl`. (A copy may
// complete before the arming arrive; the phase cannot complete before it,
// since that arrive is the phase's only one.) Called by the first
// pair_issuers(NP) threads only.
__device__ __forceinline__ void pair_issue(const PairCtx& X, float* slot, uint64_t* bar, uint32_t row,
                                           bool refl = false)
{
    if (threadIdx.x == 0) mbar_expect_tx(bar, X.row_bytes);
    if (X.iss_on) {
        // order earlier generic-proxy reads of the slot before the async refill
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        bulk_load(slot + (refl ? X.iss_dst_refl : X.iss_dst), X.iss_src + row, X.iss_bytes, bar);
    }
}

// With walls, a plane whose source row y - e_ay lies beyond a wall is the
// mirror row's reflected plane (R19): the thread of plane b copies it, from
// row nb_row(y + e_by), into the position of refl(b), where the plain pull
// reads it; it copies its own plane only when y - e_by is inside. Every
// position gets one copy, so the row's byte count is the periodic one.
// Called by the first pair_issuers(NP) threads only; lattice row y, not
// wrapped (walled items lie inside [0, ny)).
__device__ __forceinline__ void pair_issue_walls(const PairCtx& X, const DevCase<float>& c, float* slot,
                                                 uint64_t* bar, int y)
{
    if (threadIdx.x == 0) mbar_expect_tx(bar, X.row_bytes);
    if (X.iss_on) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const int sn = y - X.iss_ey, sg = y + X.iss_ey;
        if (sn >= 0 && sn < c.ny)
            bulk_load(slot + X.iss_dst, X.iss_src + (uint32_t)sn * c.pitch, X.iss_bytes, bar);
        if (sg < 0 || sg >= c.ny)
            bulk_load(slot + X.iss_dst_refl, X.iss_src + (uint32_t)nb_row(c, sg) * c.pitch, X.iss_bytes, bar);
    }
}

// Scheme 3: refill stage D's ring, right after stage A's barrier. Output row
// m = it - ND + 1 goes to the slot of row m - 2, which stage D collided in the
// last iteration and no thread has read since that barrier (rows 0 and 1 were
// issued at the start; m < h, i.e. it <= niter - 2). The copy has six stage
// intervals of lead (issued at the end of the iteration, three, it arrived
// late: 56.5 k instead of 59.7 k MLUPS at 4096^2).
template <int SCHEME, int NP, int SLOT, bool WL>
__device__ __forceinline__ void pair_issue_d(int it, PairCtx& X, const DevCase<float>& c)
{
    if constexpr (SCHEME == 3) {
        using G = StepGeom<SCHEME>;
        constexpr int SLN = PairGeom<SCHEME>::SL + ((SLOT + 1) & 1);
        if (threadIdx.x < pair_issuers(NP) && it >= G::ND + 1 && X.s0 + it + 3 <= X.s_last) {
            float* const slot = X.ring + SLN * (kQ * 2 * NP);
            if (WL && c.walls) {
                pair_issue_walls(X, c, slot, X.full + SLN, X.rd + 1);  // X.rd: the row of this iteration's D
            } else {
                pair_issue(X, slot, X.full + SLN, X.drow);
                X.drow = X.drow + c.pitch == X.plane_rows ? 0u : X.drow + c.pitch;
            }
        }
    }
}

template <int SCHEME, int COLL, int EOS, bool NU, int NP, int SLOT, bool ST, bool WL>
__device__ __forceinline__ void pair_iter(int it, PairCtx& X, const DevCase<float>& c, PairSmem<SCHEME, 2 * NP>& sm,
                                          PairRegs<SCHEME>& R)
{
    using G = StepGeom<SCHEME>;
    constexpr int S0 = SLOT, S1 = (SLOT + 3) & 3, S2 = (SLOT + 2) & 3, S3 = (SLOT + 1) & 3;
    constexpr int SW = 2 * NP;
    const int j = X.j;

    // ---------------------------------------------------------------- A
    {
        if (it == 0) {
            if (!mbar_wait(X.full + 0, 0u)) pair_timeout(X);
            if (!mbar_wait(X.full + 1, 0u)) pair_timeout(X);
        }
        if (!mbar_wait(X.f2, X.par2)) pair_timeout(X);  // stored row it + 2 (ra + 1)
        const float* Rm = X.pRm;
        const float* R0 = X.pR0;
        const float* Rp = X.pRp;
        float2 F[kQ];
        pull_ring<SW>(F, Rm, R0, Rp, j, X.jm, X.jq);
        if (WL && c.walls) {
            // With ghost rows held reflected, the plain pull above is the
            // wall reading everywhere but for the diagonals that cross a wall
            // (halfway bounce-back with the moving-wall term): on the wall
            // rows themselves and, mirrored, on the ghost rows next to them.
            // They are the wall row's own outgoing populations.
            const int sa = X.s0 + it + 1;  // window row of stage A
            const float2 wd = v2(c.wall_d);
            if (sa == 0 || sa == -1) {
                const float* W = sa == 0 ? R0 : Rp;  // slot of row 0
                const float2 f7 = ld2(W + 7 * SW + j), f8 = ld2(W + 8 * SW + j);
                if (sa == 0) {
                    F[5] = f7 + wd;
                    F[6] = f8 - wd;
                } else {
                    F[8] = f7 + wd;
                    F[7] = f8 - wd;
                }
            } else if (sa == c.ny - 1 || sa == c.ny) {
                const float* W = sa == c.ny - 1 ? R0 : Rm;  // slot of row ny - 1
                const float2 f5 = ld2(W + 5 * SW + j), f6 = ld2(W + 6 * SW + j);
                if (sa == c.ny - 1) {
                    F[7] = f5 - wd;
                    F[8] = f6 + wd;
                } else {
                    F[5] = f6 + wd;
                    F[6] = f5 - wd;
                }
            }
        }
        const float2 dr = ((F[0] + (F[1] + F[3])) + (F[2] + F[4])) + ((F[5] + F[7]) + (F[6] + F[8]));
        R.drho[S0] = dr;
        R.jx[S0] = (F[1] - F[3]) + ((F[5] - F[7]) + (F[8] - F[6]));
        R.jy[S0] = (F[2] - F[4]) + ((F[5] - F[7]) + (F[6] - F[8]));
        st2(sm.rho[S0] + j, v2(c.rho_ref) + dr);
        if constexpr (SCHEME != 3) moments2(F, R.m[S0]);  // scheme 3 keeps only the sums
    }
    __syncthreads();
    pair_issue_d<SCHEME, NP, SLOT, WL>(it, X, c);

    // ---------------------------------------------------------------- B
    if (X.b && it >= G::NB) {
        const float2 rr = v2(c.rho_ref);
        const Row2 Sm = row2(sm.rho[S2], j, rr + R.drho[S2]);
        const Row2 Sc = row2(sm.rho[S1], j, rr + R.drho[S1]);
        const Row2 Sp = row2(sm.rho[S0], j, rr + R.drho[S0]);
        if constexpr (SCHEME == 2) {
            // pressure tensor of row ra - 1 (Eqs. 4-5; P_xx in the mu rows)
            const float2 gx = gx2(Sm, Sc, Sp), gy = gy2(Sm, Sp);
            const float2 lap = lap2(Sm, Sc, Sp);
            const float2 r = Sc.c;
            const float2 pe = make_float2(pEOS<EOS, float>(c, r.x), pEOS<EOS, float>(c, r.y));
            const float2 p = pe - v2(c.kappa) * fma2(r, lap, v2(0.5f) * fma2(gx, gx, gy * gy));
            st2(sm.mu[S1] + j, fma2(v2(c.kappa) * gx, gx, p));
            st2(sm.pux[S1] + j, v2(c.kappa) * gx * gy);
            st2(sm.puy[S1] + j, fma2(v2(c.kappa) * gy, gy, p));
        } else {
            const float2 mu = fma2(v2(-c.kappa), lap2(Sm, Sc, Sp), dEf2<EOS>(c, Sc.c));
            R.mu[S1] = mu;
            st2(sm.mu[S1] + j, mu);
        }
        if constexpr (!improved_scheme(SCHEME)) {
            if (it >= G::ND) {  // grad rho of row ra - 2 from rows ra - 3 .. ra - 1
                const Row2 Qm = row2(sm.rho[S3], j, rr + R.drho[S3]);
                R.grx = gx2(Qm, Sm, Sc);
                R.gry = gy2(Qm, Sc);
            }
        }
    }
    __syncthreads();

    if constexpr (improved_scheme(SCHEME)) {
        // ------------------------------------------------------------ C
        // results of row ra - 2: u, F in registers (two rows deep; four for
        // scheme 3, whose stage D is two rows further behind) and phi u in
        // the shared rows (scheme 3: one row, read by stage D of the same
        // iteration)
        constexpr int U2 = SCHEME == 3 ? SLOT : (SLOT & 1);
        float* const pux_w = SCHEME == 3 ? sm.pux[0] : sm.pux[S2];
        float* const puy_w = SCHEME == 3 ? sm.puy[0] : sm.puy[S2];
        if (X.c && it >= G::NC) {
            const Row2 Mm = row2(sm.mu[S3], j, R.mu[S3]);
            const Row2 Mc = row2(sm.mu[S2], j, R.mu[S2]);
            const Row2 Mp = row2(sm.mu[S1], j, R.mu[S1]);
            const float2 gx = gx2(Mm, Mc, Mp), gy = gy2(Mm, Mp);
            const float2 rho = v2(c.rho_ref) + R.drho[S2];
            const float2 k = v2(1.0f / 3.0f) - rho;
            const float2 Fx = k * gx, Fy = k * gy;
            const float2 inv = make_float2(__fdividef(1.0f, rho.x), __fdividef(1.0f, rho.y));
            const float2 ux = fma2(v2(0.5f), Fx, R.jx[S2]) * inv;
            const float2 uy = fma2(v2(0.5f), Fy, R.jy[S2]) * inv;
            const float2 phi = (rho - (v2(c.c0) + Mc.c)) * v2(1.0f / 3.0f);
            st2(pux_w + j, phi * ux);
            st2(puy_w + j, phi * uy);
            R.ux[U2] = ux;
            R.uy[U2] = uy;
            R.Fx[U2] = Fx;
            R.Fy[U2] = Fy;
        }
        __syncthreads();
        if constexpr (SCHEME == 3) {
            // -------------------------------------------------------- D (3)
            // row rd = ra - 4. C1 = d_x A' + d_y B', C7 = d_x A' - d_y B' with
            // A' = sum_a w_a (phi u_x)(x + e_a), B' likewise: the Eq. 17
            // gradient of the averages factors into
            //   d_x A' = sum_dy s(dy) [(A(x+1) - A(x-1))/3 + (A(x+2) - A(x-2))/12](y + dy)
            // with s = (1, 8, 18, 8, 1)/36 over dy = -2 .. 2, and d_y B' with
            // the roles of x and y exchanged. The x-parts (the bracket for A,
            // the s-weighted sum over x for B) of row ra - 2 are taken here
            // once; those of rows ra - 6 .. ra - 3 are in a register ring of
            // four, row ra - 2 - d in slot (SLOT - d) & 3, so row ra - 2 takes
            // the slot of row ra - 6 once that is read.
            const float2 g1 = v2(1.0f / 3.0f), g2 = v2(1.0f / 12.0f);
            const float2 s0 = v2(1.0f / 36.0f), s1 = v2(8.0f / 36.0f), s2 = v2(18.0f / 36.0f);
            if (X.d && it >= G::NC) {
                constexpr int K6 = SLOT, K5 = (SLOT + 1) & 3, K4 = (SLOT + 2) & 3, K3 = (SLOT + 3) & 3;
                const float* a = sm.pux[0] + j;
                const float2 aL = ld2(a - 2), aO = ld2(a), aR = ld2(a + 2);
                // the shifted differences and sums as scalar halves (no pair assembly)
                const float2 hx4 = fma2(g1, make_float2(aO.y - aL.y, aR.x - aO.x), g2 * (aR - aL));
                const float* b = sm.puy[0] + j;
                const float2 bL = ld2(b - 2), bO = ld2(b), bR = ld2(b + 2);
                const float2 sb4 = fma2(s0, bL + bR, fma2(s1, make_float2(bL.y + bO.y, bO.x + bR.x), s2 * bO));
                if (it >= G::ND) {
                    const float2 Ax = fma2(s0, R.hx[K6] + hx4, fma2(s1, R.hx[K5] + R.hx[K3], s2 * R.hx[K4]));
                    const float2 By = fma2(g1, R.sb[K3] - R.sb[K5], g2 * (sb4 - R.sb[K6]));
                    const float2 C1 = Ax + By, C7 = Ax - By;
                    // the pull of row rd from stage D's ring: output row m = it - ND
                    // of the item in slot m & 1, phase (m / 2) & 1 (both fixed by
                    // SLOT, since ND is a multiple of 4)
                    constexpr int SLD = PairGeom<SCHEME>::SL + (SLOT & 1);
                    if (!mbar_wait(X.full + SLD, (uint32_t)(SLOT >> 1) & 1u)) pair_timeout(X);
                    const float* Dr = X.ring + SLD * (kQ * SW);
                    float2 F[kQ];
                    pull_ring<SW>(F, Dr, Dr, Dr, j, X.jm, X.jq);
                    if (WL && c.walls) {
                        // the diagonals that cross a wall (as in stage A): the
                        // wall row's own outgoing populations, which the slot
                        // holds at the reflected positions (7 -> 6, 8 -> 5 at
                        // row 0; 5 -> 8, 6 -> 7 at row ny - 1)
                        const float2 wd = v2(c.wall_d);
                        if (X.rd == 0) {
                            F[5] = ld2(Dr + 6 * SW + j) + wd;
                            F[6] = ld2(Dr + 5 * SW + j) - wd;
                        } else if (X.rd == c.ny - 1) {
                            F[7] = ld2(Dr + 8 * SW + j) - wd;
                            F[8] = ld2(Dr + 7 * SW + j) + wd;
                        }
                    }
                    const float2 drho = ((F[0] + (F[1] + F[3])) + (F[2] + F[4])) + ((F[5] + F[7]) + (F[6] + F[8]));
                    const float2 jx = (F[1] - F[3]) + ((F[5] - F[7]) + (F[8] - F[6]));
                    const float2 jy = (F[2] - F[4]) + ((F[5] - F[7]) + (F[6] - F[8]));
                    const float2 rho = v2(c.rho_ref) + drho;
                    if (!pair_ok(rho)) *X.bad = 1;
                    const float2 mu = R.mu[S0];  // row ra - 4
                    float2 le = v2(c.lam_e), ls = v2(c.lam_s), lq = v2(c.lam_q), lv = v2(c.lam_v);
                    if (NU) {
                        lv = make_float2(shear_rate<SCHEME, NU, float>(c, rho.x, mu.x),
                                         shear_rate<SCHEME, NU, float>(c, rho.y, mu.y));
                        if (COLL == 0) le = ls = lq = lv;
                    }
                    if constexpr (ST) pair_stats(R, drho, rho, R.ux[S2], R.uy[S2]);
                    collide2<SCHEME>(F, drho, rho, jx, jy, R.ux[S2], R.uy[S2], R.Fx[S2], R.Fy[S2], mu, C1, C7, c, le,
                                     ls, lq, lv);
                    float* o = X.orow;
                    const uint32_t P = (uint32_t)c.plane;
#pragma unroll
                    for (int a = 0; a < kQ; ++a) st2(o + a * P, F[a]);
                }
                R.hx[K6] = hx4;
                R.sb[K6] = sb4;
            }
        } else {
        // ------------------------------------------------------------ D
        constexpr int U3 = (SLOT + 1) & 1;
        if (X.d && it >= G::ND) {
            const Row2 Am = row2(sm.pux[S0], j, ld2(sm.pux[S0] + j));  // row ra - 4
            const Row2 Ac = row2(sm.pux[S3], j, ld2(sm.pux[S3] + j));  // row ra - 3
            const Row2 Ap = row2(sm.pux[S2], j, ld2(sm.pux[S2] + j));  // row ra - 2
            const Row2 Bm = row2(sm.puy[S0], j, ld2(sm.puy[S0] + j));
            const Row2 Bp = row2(sm.puy[S2], j, ld2(sm.puy[S2] + j));
            const float2 Ax = gx2(Am, Ac, Ap), By = gy2(Bm, Bp);
            const float2 C1 = Ax + By, C7 = Ax - By;
            const float2 drho = R.drho[S3];
            const float2 rho = v2(c.rho_ref) + drho;
            if (!pair_ok(rho)) *X.bad = 1;
            const float2 mu = R.mu[S3];
            float2 le = v2(c.lam_e), ls = v2(c.lam_s), lq = v2(c.lam_q), lv = v2(c.lam_v);
            if (NU) {
                lv = make_float2(shear_rate<SCHEME, NU, float>(c, rho.x, mu.x),
                                 shear_rate<SCHEME, NU, float>(c, rho.y, mu.y));
                if (COLL == 0) le = ls = lq = lv;
            }
            if constexpr (ST) pair_stats(R, drho, rho, R.ux[U3], R.uy[U3]);
            float2 d[kQ];
            collide2m<SCHEME>(d, R.m[S3], drho, rho, R.jx[S3], R.jy[S3], R.ux[U3], R.uy[U3], R.Fx[U3], R.Fy[U3],
                              mu, C1, C7, c, le, ls, lq, lv);
            float* o = X.orow;
            const uint32_t P = (uint32_t)c.plane;
#pragma unroll
            for (int a = 0; a < kQ; ++a) st2(o + a * P, d[a]);
        }
        }
    } else {
        // ------------------------------------------------------- D (standard)
        if (X.d && it >= G::ND) {
            const float2 drho = R.drho[S2];
            const float2 rho = v2(c.rho_ref) + drho;
            if (!pair_ok(rho)) *X.bad = 1;
            float2 mu, Fx, Fy;
            if constexpr (SCHEME == 2) {
                // F = grad(rho/3) - div P, each component of P through Eq. 17
                const Row2 Pm = row2(sm.mu[S3], j, ld2(sm.mu[S3] + j));
                const Row2 Pc = row2(sm.mu[S2], j, ld2(sm.mu[S2] + j));
                const Row2 Pp = row2(sm.mu[S1], j, ld2(sm.mu[S1] + j));
                const Row2 Xm = row2(sm.pux[S3], j, ld2(sm.pux[S3] + j));
                const Row2 Xc = row2(sm.pux[S2], j, ld2(sm.pux[S2] + j));
                const Row2 Xp = row2(sm.pux[S1], j, ld2(sm.pux[S1] + j));
                const Row2 Ym = row2(sm.puy[S3], j, ld2(sm.puy[S3] + j));
                const Row2 Yp = row2(sm.puy[S1], j, ld2(sm.puy[S1] + j));
                const float2 divx = gx2(Pm, Pc, Pp) + gy2(Xm, Xp);
                const float2 divy = gx2(Xm, Xc, Xp) + gy2(Ym, Yp);
                mu = v2(0.0f);  // the standard collision does not use mu_c
                Fx = fma2(R.grx, v2(1.0f / 3.0f), v2(0.0f) - divx);
                Fy = fma2(R.gry, v2(1.0f / 3.0f), v2(0.0f) - divy);
            } else {
                const Row2 Mm = row2(sm.mu[S3], j, R.mu[S3]);
                const Row2 Mc = row2(sm.mu[S2], j, R.mu[S2]);
                const Row2 Mp = row2(sm.mu[S1], j, R.mu[S1]);
                const float2 gmx = gx2(Mm, Mc, Mp), gmy = gy2(Mm, Mp);
                mu = Mc.c;
                Fx = fma2(R.grx, v2(1.0f / 3.0f), v2(0.0f) - rho * gmx);
                Fy = fma2(R.gry, v2(1.0f / 3.0f), v2(0.0f) - rho * gmy);
            }
            const float2 inv = make_float2(__fdividef(1.0f, rho.x), __fdividef(1.0f, rho.y));
            const float2 ux = fma2(v2(0.5f), Fx, R.jx[S2]) * inv;
            const float2 uy = fma2(v2(0.5f), Fy, R.jy[S2]) * inv;
            float2 le = v2(c.lam_e), ls = v2(c.lam_s), lq = v2(c.lam_q), lv = v2(c.lam_v);
            if (NU) {
                lv = make_float2(shear_rate<SCHEME, NU, float>(c, rho.x, mu.x),
                                 shear_rate<SCHEME, NU, float>(c, rho.y, mu.y));
                if (COLL == 0) le = ls = lq = lv;
            }
            if constexpr (ST) pair_stats(R, drho, rho, ux, uy);
            float2 d[kQ];
            collide2m<SCHEME>(d, R.m[S2], drho, rho, R.jx[S2], R.jy[S2], ux, uy, Fx, Fy, mu, v2(0.0f), v2(0.0f), c,
                              le, ls, lq, lv);
            float* o = X.orow;
            const uint32_t P = (uint32_t)c.plane;
#pragma unroll
            for (int a = 0; a < kQ; ++a) st2(o + a * P, d[a]);
        }
    }
    // stored row it (ra - 1) has had no reader since stage A's barrier: refill
    // its slot now, with the iteration's arithmetic issued (the copy still has
    // two iterations of lead before stage A needs it)
    constexpr int SL = PairGeom<SCHEME>::SL;
    if (threadIdx.x < pair_issuers(NP) && X.s0 + it + SL <= X.s_last) {
        if (WL && c.walls) {
            bool refl;
            const uint32_t row = window_row(c, X.s0 + it + SL, refl);
            pair_issue(X, X.pRm, X.fm, row, refl);
        } else {
            pair_issue(X, X.pRm, X.fm, X.irow);
        }
    }
    // advance the ring, the refill row and the output row by one (wrapping
    // compares instead of row modulos and multiplies)
    X.irow = X.irow + c.pitch == X.plane_rows ? 0u : X.irow + c.pitch;
    {
        constexpr int SLOTF = kQ * SW;
        float* const ring_end = X.ring + SL * SLOTF;
        X.fm = X.fm + 1 == X.full + SL ? X.full : X.fm + 1;
        const bool wrap = X.f2 + 1 == X.full + SL;
        X.f2 = wrap ? X.full : X.f2 + 1;
        X.par2 ^= wrap ? 1u : 0u;
        X.pRm = X.pR0;
        X.pR0 = X.pRp;
        X.pRp = X.pRp + SLOTF == ring_end ? X.ring : X.pRp + SLOTF;
    }
    if (it >= G::ND) {
        const bool w = X.rd + 1 == c.ny;
        X.rd = w ? 0 : X.rd + 1;
        X.orow = w ? X.out : X.orow + c.pitch;
    }
}

// stage A's ring, scheme 3's stage D ring, and one mbarrier per slot
template <typename T, int NP, int SCHEME>
constexpr size_t pair_dynamic_smem()
{
    constexpr int slots = PairGeom<SCHEME>::SL + PairGeom<SCHEME>::SD;
    return (size_t)slots * kQ * (2 * NP) * sizeof(T) + slots * sizeof(uint64_t);
}

// FP32 step with NP threads of two columns each: blockDim.x == NP (128 or
// 64). Every case of the launch has nx % 4 == 0 (and nx >= 8 for scheme 3,
// so that each margin of the ring is one copy run); every item x0 % 4 == 0,
// wv % 4 == 0, wv + 2 M <= 2 NP with M = PairGeom<SCHEME>::M (4, or 8 for
// scheme 3). ST: the variant that also records the per-step statistics
// (stats_block) of the cases whose record has st_hist != 0. WL: the variant
// that also runs lattices with walls.
template <int SCHEME, int COLL, int EOS, bool NU, int NP, bool ST = false, bool WL = false>
__global__ void __launch_bounds__(NP, NP == kPairThreads ? 3 : 6) step_kernel_pair(const float* __restrict__ fin,
                                                                    float* __restrict__ fout,
                                                                    const DevCase<float>* __restrict__ cases,
                                                                    const Item* __restrict__ items,
                                                                    int* __restrict__ status)
{
    using G = StepGeom<SCHEME>;
    static_assert(SCHEME != 4, "scheme 4 runs on the plain-load kernel only");
    constexpr int M = PairGeom<SCHEME>::M;
    constexpr int SL = PairGeom<SCHEME>::SL, SD = PairGeom<SCHEME>::SD;
    constexpr int SLOTF = kQ * (2 * NP);
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ __align__(16) PairSmem<SCHEME, 2 * NP> sm;
    __shared__ int flag, bad;
    const Item item = items[blockIdx.x];
    // a case flagged unstable by an earlier step no longer advances (thread 0
    // decides for the block: another block may set the word meanwhile)
    if (__syncthreads_or(threadIdx.x == 0 && status[1 + item.case_id] != 0)) return;
    const DevCase<float> c = cases[item.case_id];
    fin += c.off;
    fout += c.off;
    const int niter = item.h + 2 * G::HX;

    PairCtx X;
    X.ring = reinterpret_cast<float*>(dsm);
    X.full = reinterpret_cast<uint64_t*>(dsm + (size_t)(SL + SD) * SLOTF * sizeof(float));
    X.flag = &flag;
    X.status = status;
    X.fin = fin;
    X.s0 = item.y0 - G::HX - 1;
    X.s_last = X.s0 + niter + 1;
    {
        // runs of [x0 - 4, x0 + wv + 4) split at the periodic edges
        const int start = item.x0 - M, end = item.x0 + item.wv + M;
        X.runs.n = 0;
        int x = start, jj = 0;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int g = wrapi(x, c.nx);
            const int len = min(end - x, c.nx - g);
            X.runs.g0[r] = g;
            X.runs.j0[r] = jj;
            X.runs.len[r] = len;
            if (x < end) X.runs.n = r + 1;
            x += len;
            jj += len;
        }
        X.row_bytes = (uint32_t)(kQ * (end - start) * sizeof(float));
    }
    const int ey = pair_issue_setup<NP>(X, c);
    if constexpr (WL) X.iss_ey = ey;
    if (threadIdx.x == 0) {
        flag = 0;
        bad = 0;
        for (int k = 0; k < SL + SD; ++k) mbar_init(X.full + k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x < pair_issuers(NP)) {
        for (int i = 0; i < SL && X.s0 + i <= X.s_last; ++i) {
            bool refl;
            const uint32_t row = window_row(c, X.s0 + i, refl);
            pair_issue(X, X.ring + i * SLOTF, X.full + i, row, refl);
        }
        if constexpr (SCHEME == 3) {
            // stage D's ring: the pulls of output rows y0 and y0 + 1 (this
            // thread's plane from stored row y - e_ay), then row y0 + 2's
            // source row for the first refill
            for (int m = 0; m < SD && m < item.h; ++m) {
                if (WL && c.walls)
                    pair_issue_walls(X, c, X.ring + (SL + m) * SLOTF, X.full + SL + m, item.y0 + m);
                else
                    pair_issue(X, X.ring + (SL + m) * SLOTF, X.full + SL + m,
                               (uint32_t)wrapi(item.y0 + m - ey, c.ny) * c.pitch);
            }
            X.drow = (uint32_t)wrapi(item.y0 + SD - ey, c.ny) * c.pitch;
        }
    }

    const int p = threadIdx.x;
    X.j = 2 * p;
    if constexpr (SCHEME == 3) {  // ring columns: mu [4, wv + 12), phi u [6, wv + 10), strip [8, wv + 8)
        X.b = p >= 2 && 2 * p < item.wv + 12;
        X.c = p >= 3 && 2 * p < item.wv + 10;
        X.d = p >= 4 && 2 * p < item.wv + 8;
    } else {
        X.b = p >= 1 && 2 * p < item.wv + 6;
        X.d = p >= 2 && 2 * p < item.wv + 4;
        X.c = X.b;
    }
    X.jm = X.j > 0 ? X.j - 1 : 0;
    X.jq = X.j + 2 < 2 * NP ? X.j + 2 : 2 * NP - 1;
    X.pRm = X.ring;
    X.pR0 = X.ring + SLOTF;
    X.pRp = X.ring + 2 * SLOTF;
    X.fm = X.full;
    X.f2 = X.full + 2;
    X.par2 = 0;
    X.plane_rows = (uint32_t)c.ny * c.pitch;
    X.irow = (uint32_t)wrapi(X.s0 + SL, c.ny) * c.pitch;
    X.rd = item.y0;
    X.out = fout + (X.d ? item.x0 - M + 2 * p : 0);
    X.orow = X.out + (uint32_t)X.rd * c.pitch;
    X.bad = &bad;

    PairRegs<SCHEME> R;
    R.am = R.ak = v2(0.0f);
    R.au = 0.0f;
    for (int base = 0; base < niter; base += 4) {
        pair_iter<SCHEME, COLL, EOS, NU, NP, 0, ST, WL>(base, X, c, sm, R);
        if (base + 1 >= niter) break;
        pair_iter<SCHEME, COLL, EOS, NU, NP, 1, ST, WL>(base + 1, X, c, sm, R);
        if (base + 2 >= niter) break;
        pair_iter<SCHEME, COLL, EOS, NU, NP, 2, ST, WL>(base + 2, X, c, sm, R);
        if (base + 3 >= niter) break;
        pair_iter<SCHEME, COLL, EOS, NU, NP, 3, ST, WL>(base + 3, X, c, sm, R);
    }
    // every issued row was waited on by stage A; after a timeout, drain (bounded)
    __syncthreads();
    if (threadIdx.x == 0 && bad) atomicOr(status + 1 + item.case_id, 1);
    if (ST && c.st_hist)
        stats_block<float, NP / 32>(c, (double)R.am.x + (double)R.am.y, (double)R.ak.x + (double)R.ak.y, (double)R.au,
                    (unsigned long long)item.wv * (unsigned long long)item.h);
    if (threadIdx.x == 0 && flag) {
        for (int s = max(X.s0, X.s_last - SL + 1); s <= X.s_last; ++s) {
            const int i = s - X.s0;
            mbar_wait(X.full + i % SL, (uint32_t)(i / SL) & 1u);
        }
        for (int m = max(0, item.h - SD); m < item.h; ++m)  // scheme 3: stage D's ring
            mbar_wait(X.full + SL + (m & 1), (uint32_t)(m >> 1) & 1u);
    }
}

}  // namespace lbfe
