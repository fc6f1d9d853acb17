// C-ABI entry points of liblbfe (declared and documented in include/lbfe.h):
// validation, workspace layout, work-list construction and the launches of
// the step, initialisation, field-export and reduction kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbfe.h"
#include "adjoint_kernels.cuh"
#include "aux_kernels.cuh"
#include "launch.h"
#include "step_tma.cuh"

using namespace lbfe;

namespace {

constexpr size_t kAlign = 256;
constexpr int kMinRows = 8;     // smallest row segment of the slot-share rules
constexpr int kMinSegRows = 2;  // smallest explicit row segment (latency-bound small lattices)
// scratch fields: rho, j_x, j_y, mu (0-3), host staging of outputs / init
// inputs (4-7), pressure tensor P_xx, P_xy, P_yy (8-10)
constexpr int kScratchFields = 11;
constexpr int kPairCols256 = 256, kPairCols128 = 128;  // ring columns of the wide / narrow packed blocks

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int halo_of(int scheme) { return scheme == LB_IMPROVED_SMOOTH ? 4 : scheme == LB_IMPROVED ? 3 : 2; }

// cases that only the one-column plain-load kernel runs: the Lax-Wendroff
// scheme, and the averaged correction on lattices narrower than its 8-column
// ring margin
bool one_column_only(const lb_case& c)
{
    return c.scheme == LB_LAX_WENDROFF || (c.scheme == LB_IMPROVED_SMOOTH && c.nx < 8);
}

// Widest strip of output columns a block of nt threads can own. Lattices with
// nx % 4 == 0 get strips of a multiple of 4 columns, at most nt - 8 wide, as
// the TMA-staged kernel needs (16-byte aligned runs of [x0 - 4, x0 + wv + 4)).
int strip_width(const lb_case& c, int nt)
{
    if (c.nx % 4 != 0) return nt - 2 * halo_of(c.scheme);
    return nt - (c.scheme == LB_IMPROVED_SMOOTH ? 16 : 8);  // the packed kernel's ring margins (4 or 8)
}

int strips_of(const lb_case& c, int nt) { return (c.nx + strip_width(c, nt) - 1) / strip_width(c, nt); }

constexpr int kMinBlockThreads = 128;  // narrowest block any path uses

int64_t max_items_of(const lb_case& c)
{
    // (the row kernel's whole-height strips: at least rows_strip_width(3) wide)
    return std::max<int64_t>((int64_t)strips_of(c, kMinBlockThreads) * ((c.ny + kMinSegRows - 1) / kMinSegRows),
                             (c.nx + rows_strip_width(LB_IMPROVED_SMOOTH) - 1) / rows_strip_width(LB_IMPROVED_SMOOTH));
}

// periodic lattices of schemes 0-3 short enough for the row kernel
bool rows_eligible(const lb_case& c)
{
    return !c.walls && c.scheme != LB_LAX_WENDROFF && c.ny <= rows_max_ny();
}

constexpr int kMaxNeighbours = 32;  // neighbour items per item that the persistent launch tracks

struct Layout {
    size_t cases32, cases64, items, f[2], scratch, partials, red, status, nb_off, nb_idx, progress, total;
    std::vector<int64_t> off;  // element offset of each case in a population buffer
    int64_t max_items = 0, max_nodes = 0, max_parts = 0;
};

Layout layout_of(const lb_case* cs, int n, int prec)
{
    Layout L;
    const size_t es = prec == LB_FP32 ? 4 : 8;
    size_t p = 0;
    L.cases32 = p;
    p = align_up(p + n * sizeof(DevCase<float>), kAlign);
    L.cases64 = p;
    p = align_up(p + n * sizeof(DevCase<double>), kAlign);
    int64_t elems = 0;
    for (int i = 0; i < n; ++i) {
        L.max_items += max_items_of(cs[i]);
        L.max_nodes = std::max<int64_t>(L.max_nodes, (int64_t)cs[i].nx * cs[i].ny);
        L.max_parts = std::max<int64_t>(L.max_parts, (int64_t)((cs[i].nx + 255) / 256) * cs[i].ny);
        L.off.push_back(elems);
        elems += (int64_t)align_up((size_t)kQ * cs[i].ny * pitch_of(cs[i].nx) * es, kAlign) / es;
    }
    L.items = p;
    p = align_up(p + L.max_items * sizeof(Item), kAlign);
    for (int b = 0; b < 2; ++b) {
        L.f[b] = p;
        p = align_up(p + elems * es, kAlign);
    }
    L.scratch = p;  // kScratchFields FP64 fields of the largest case
    p = align_up(p + kScratchFields * align_up(L.max_nodes * sizeof(double), kAlign), kAlign);
    L.partials = p;
    p = align_up(p + L.max_parts * sizeof(Partial), kAlign);
    L.red = p;
    p = align_up(p + n * 8 * sizeof(double), kAlign);
    L.status = p;  // [0]: a bounded wait gave up; [1 + case]: the case went unstable
    p = align_up(p + (1 + n) * sizeof(int), kAlign);
    // persistent launch: neighbour lists (CSR) and per-item progress + abort word
    L.nb_off = p;
    p = align_up(p + (L.max_items + 1) * sizeof(int), kAlign);
    L.nb_idx = p;
    p = align_up(p + L.max_items * kMaxNeighbours * sizeof(int), kAlign);
    L.progress = p;
    p = align_up(p + (L.max_items + 1) * sizeof(int), kAlign);
    L.total = p;
    return L;
}

std::string check_case(const lb_case& c, int i)
{
    char buf[160];
    auto bad = [&](const char* what) {
        snprintf(buf, sizeof buf, "case %d: %s", i, what);
        return std::string(buf);
    };
    if (c.nx < 3 || c.ny < 3) return bad("nx and ny must be >= 3");
    // the step kernel addresses a case's nine planes with 32-bit offsets
    if ((int64_t)kQ * c.ny * pitch_of(c.nx) >= (int64_t)1 << 31) return bad("lattice too large");
    if (c.scheme != LB_STANDARD && c.scheme != LB_IMPROVED && c.scheme != LB_STANDARD_PT &&
        c.scheme != LB_IMPROVED_SMOOTH && c.scheme != LB_LAX_WENDROFF)
        return bad("unknown scheme");
    if (c.collision != LB_BGK && c.collision != LB_MRT) return bad("unknown collision");
    if (c.eos != LB_VDW && c.eos != LB_CS) return bad("unknown eos");
    if (c.walls != 0 && c.walls != 1) return bad("walls must be 0 or 1");
    const double v[] = {c.a, c.b, c.R, c.T, c.kappa, c.tau_v, c.tau_e, c.tau_s, c.tau_q, c.pm_c0,
                        c.nu, c.rho_ref, c.wall_u, c.rho_wall, c.lw_A, c.lw_B};
    for (double x : v)
        if (!std::isfinite(x)) return bad("non-finite parameter");
    if (!(c.a > 0 && c.b > 0 && c.R > 0 && c.T > 0 && c.kappa > 0)) return bad("a, b, R, T, kappa must be > 0");
    if (!(c.tau_v > 0.5 && c.tau_e > 0.5 && c.tau_s > 0.5 && c.tau_q > 0.5))
        return bad("relaxation times must be > 1/2");
    if (c.nu < 0 || c.rho_ref < 0) return bad("nu and rho_ref must be >= 0");
    if (c.scheme == LB_LAX_WENDROFF) {
        if (c.collision != LB_BGK || c.walls || c.nu != 0.0)
            return bad("the Lax-Wendroff scheme is BGK, periodic and has nu = 0");
        if (!(c.lw_A > 0.0 && c.lw_A <= 1.0) || !(c.lw_B < c.tau_v - 0.5))
            return bad("Lax-Wendroff needs 0 < lw_A <= 1 and lw_B < tau_v - 1/2");
    }
    if (c.walls) {
        // the row pipeline mirrors up to four rows across each wall
        if (c.ny < 8) return bad("walls need ny >= 8");
        if (!(c.rho_wall > 0) || !(std::fabs(c.wall_u) <= 0.3))
            return bad("walls need rho_wall > 0 and |wall_u| <= 0.3");
    }
    return std::string();
}

// E_f'(rho) on the host (Eq. 30 without the kappa term; Carnahan-Starling)
double host_dEf(const lb_case& c, double rho)
{
    if (c.eos == LB_VDW) {
        const double q = 1.0 / (1.0 - c.b * rho);
        return c.R * c.T * (std::log(rho * q) + q) - 2.0 * c.a * rho;
    }
    const double n = 0.25 * c.b * rho, q = 1.0 / (1.0 - n);
    return c.R * c.T * (std::log(rho) + 1.0 + n * (4.0 - 3.0 * n) * q * q + n * (4.0 - 2.0 * n) * q * q * q) -
           2.0 * c.a * rho;
}

// Moving-wall term of the diagonal directions: f_eq,5 - f_eq,7 of the running
// scheme at the wall state (rho_wall, (wall_u, 0), E_f'(rho_wall)), which is
// P u_wall / 2 with P = rho_wall / 3 (standard equilibrium, Eq. 11) or the
// modified pressure p_m = (c0 + mu_c) / 3 (Eq. 27); the axis directions normal
// to the walls get no term.
double wall_delta(const lb_case& c)
{
    if (!c.walls) return 0.0;
    const double P = improved_scheme(c.scheme) ? (c.pm_c0 + host_dEf(c, c.rho_wall)) / 3.0 : c.rho_wall / 3.0;
    return 0.5 * P * c.wall_u;
}

template <typename T>
DevCase<T> dev_case(const lb_case& c, int64_t off, double rho_ref)
{
    DevCase<T> d{};
    d.nx = c.nx;
    d.ny = c.ny;
    d.pitch = pitch_of(c.nx);
    d.off = off;
    d.plane = (int64_t)c.ny * d.pitch;
    d.RT = (T)(c.R * c.T);
    d.a = (T)c.a;
    d.b = (T)c.b;
    d.kappa = (T)c.kappa;
    d.c0 = (T)c.pm_c0;
    d.rho_ref = (T)rho_ref;
    d.walls = c.walls;
    d.wall_d = (T)wall_delta(c);
    const bool bgk = c.collision == LB_BGK;
    d.lam_v = (T)(1.0 / c.tau_v);
    d.lam_e = (T)(1.0 / (bgk ? c.tau_v : c.tau_e));
    d.lam_s = (T)(1.0 / (bgk ? c.tau_v : c.tau_s));
    d.lam_q = (T)(1.0 / (bgk ? c.tau_v : c.tau_q));
    d.nu = (T)c.nu;
    if (c.scheme == LB_LAX_WENDROFF) {
        const double A = c.lw_A, B = c.lw_B, tau = c.tau_v;
        d.lw_dt = (T)A;
        d.lw_a0 = (T)(1.0 - A * A);
        d.lw_a1 = (T)(A * (A - 1.0) / 2.0);
        d.lw_am1 = (T)(A * (A + 1.0) / 2.0);
        d.lw_kT = (T)(1.0 / ((1.0 / 3.0) * A * (B - tau)));
        d.lw_fd = (T)((tau - 0.5) * A);
        d.lw_bt = (T)(B * A * 1.5);
        d.lw_g = (T)(A * (1.0 - 0.5 / tau));
    }
    return d;
}

struct Group {
    int scheme, coll, eos;
    bool nu;
    bool tma;              // TMA-staged kernel (FP32, every nx % 4 == 0)
    int nt;                // compute threads per block
    int64_t first, count;  // slice of the item array
    bool walls = false;    // lattices with walls (the packed kernel's variant for them)
    bool rows = false;     // the row kernel (short periodic lattices, whole-height strips)
    int ny_max = 0;        // row kernel: tallest lattice of the group
};

}  // namespace

struct lb_handle {
    std::vector<lb_case> cases;
    int prec = LB_FP32;
    cudaStream_t stream = nullptr;
    uint8_t* ws = nullptr;
    Layout L;
    int cur = 0;
    std::vector<double> rho_ref;
    std::vector<int64_t> steps;
    std::vector<char> inited;
    std::vector<Group> groups;
    std::vector<Item> items;
    int path = 0;           // 0: TMA-staged kernel where eligible, 1: plain-load kernel only
    bool use_graph = true;  // replay lb_step through captured CUDA graphs
    cudaStream_t cap_stream = nullptr;              // private stream used only for graph capture
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // kGraphSteps steps starting from buffer 0 / 1
    int tma_threads = 0;    // TMA kernel shape: 0 packed two-column, 128 or 256 one-column
    int seg_rows = 0;       // work-list rows per segment, 0: share of the block slots
    bool autotune = true;   // pick seg_rows (and narrow) by timing on the first lb_step
    bool narrow = false;    // narrow packed blocks for the lattices that prefer them
    bool rows_on = true;    // the row kernel runs the lattices it can (LBFE_ROWS=0: never)
    bool narrow_fixed = false;  // narrow set by LBFE_PAIR_NARROW, not tuned
    std::vector<cudaStream_t> aux;       // capture branches for groups after the first
    std::vector<cudaEvent_t> fork_join;  // [2 * branch]: fork, join
    bool tuned = false;
    // persistent multi-step launch (step_persist.cuh): 0 never, 1 always (a
    // one-group handle; its group runs the one-column kernel), 2 timed
    // against graph replay on the first long enough lb_step and kept if faster
    int persist_mode = 2;
    bool persist = false;        // in use
    bool persist_tuned = false;  // the choice of mode 2 has been made
    bool nb_ok = false;          // neighbour lists built for the current work-list
    int persist_grid = 0;
    long long spin_limit = kWaitCycles;
    // per-step statistics (lb_step_stats_attach): the caller's device buffer
    // ([ncases][2] int32 counters {ticket, recorded states}, then
    // [ncases][st_hist] StepStat entries), whether the kernels see it (off
    // while the autotuner times trial launches), the state index of each
    // case's first recorded entry, and the work items per case of the list
    uint8_t* st_buf = nullptr;
    int st_hist = 0;
    bool st_live = false;
    std::vector<int64_t> st_base;
    std::vector<int32_t> case_items;
    std::string err;

    void* fbuf(int b) const { return ws + L.f[b]; }
    DevCase<float>* dc32() const { return reinterpret_cast<DevCase<float>*>(ws + L.cases32); }
    DevCase<double>* dc64() const { return reinterpret_cast<DevCase<double>*>(ws + L.cases64); }
    Item* ditems() const { return reinterpret_cast<Item*>(ws + L.items); }
    double* scratch(int k) const
    {
        return reinterpret_cast<double*>(ws + L.scratch +
                                         k * align_up(L.max_nodes * sizeof(double), kAlign));
    }
    Partial* partials() const { return reinterpret_cast<Partial*>(ws + L.partials); }
    int* status() const { return reinterpret_cast<int*>(ws + L.status); }
    int* nb_off() const { return reinterpret_cast<int*>(ws + L.nb_off); }
    int* nb_idx() const { return reinterpret_cast<int*>(ws + L.nb_idx); }
    int* progress() const { return reinterpret_cast<int*>(ws + L.progress); }
    double* red() const { return reinterpret_cast<double*>(ws + L.red); }

    lb_status fail(lb_status s, const std::string& m)
    {
        err = m;
        return s;
    }
    lb_status cuda(cudaError_t e, const char* where)
    {
        if (e == cudaSuccess) return LB_OK;
        err = std::string(where) + ": " + cudaGetErrorString(e);
        return LB_E_CUDA;
    }
    int32_t* st_ctr() const { return reinterpret_cast<int32_t*>(st_buf); }
    StepStat* st_ring() const
    {
        return reinterpret_cast<StepStat*>(st_buf + align_up(2 * sizeof(int32_t) * cases.size(), kAlign));
    }
    template <typename T>
    void set_stats(DevCase<T>& c, int i) const
    {
        if (!st_live || !st_buf) return;
        c.st_hist = st_hist;
        c.st_ring = st_ring() + (size_t)i * st_hist;
        c.st_ctr = st_ctr() + 2 * i;
        c.st_blocks = i < (int)case_items.size() ? case_items[i] : 0;
    }
    lb_status upload_case(int i)
    {
        DevCase<float> c32 = dev_case<float>(cases[i], L.off[i], rho_ref[i]);
        DevCase<double> c64 = dev_case<double>(cases[i], L.off[i], rho_ref[i]);
        // a Lax-Wendroff case at step 0 holds f(0) itself (see pull_lw)
        c32.lw_first = c64.lw_first = cases[i].scheme == LB_LAX_WENDROFF && steps[i] == 0;
        set_stats(c32, i);
        set_stats(c64, i);
        lb_status s = cuda(cudaMemcpyAsync(dc32() + i, &c32, sizeof c32, cudaMemcpyHostToDevice, stream),
                           "upload case");
        if (s != LB_OK) return s;
        s = cuda(cudaMemcpyAsync(dc64() + i, &c64, sizeof c64, cudaMemcpyHostToDevice, stream), "upload case");
        if (s != LB_OK) return s;
        return cuda(cudaStreamSynchronize(stream), "upload case");
    }
};

namespace {

constexpr int kGraphSteps = 8;  // steps per captured graph (even: buffer parity returns)

// Split every case into column strips and row segments. seg_rows == 0: each
// case gets a share of the resident block slots proportional to its node
// count, so that one launch fills the GPU about once; seg_rows > 0: segments
// of about seg_rows rows (at least kMinSegRows). Within a group the items run
// longest first, so the block scheduler hands the short ones to the slots
// that free up last. The decomposition changes no result: every node's
// update is the same arithmetic on the same inputs whichever item owns it.
// Packed-kernel shape of an FP32 lattice with nx % 4 == 0: the narrow
// (64-thread, 128-column) blocks when they cover the lattice's columns with
// fewer idle lanes than the wide (128-thread, 256-column) ones.
bool prefers_narrow(const lb_case& c)
{
    // block columns each shape spends on the lattice (its strips are at most
    // strip_width: ring margins of 4, or 8 for the averaged correction)
    const int ww = strip_width(c, kPairCols256), wn = strip_width(c, kPairCols128);
    const int wide = (c.nx + ww - 1) / ww * kPairCols256;
    const int narrow = (c.nx + wn - 1) / wn * kPairCols128;
    return narrow < wide;
}

void build_items(lb_handle* h)
{
    const int seg_rows = h->seg_rows;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int n = (int)h->cases.size();
    h->items.clear();
    h->groups.clear();
    // one group (one launch per step) per kernel variant and block shape
    auto emit = [&](const std::vector<int>& members, int s, int co, int e, int nu, bool tma, int nt, bool walls) {
        if (members.empty()) return;
        double nodes = 0;
        for (int i : members) nodes += (double)h->cases[i].nx * h->cases[i].ny;
        const int width = !tma ? kStepThreads
                          : nt == kPairWide   ? kPairCols256
                          : nt == kPairNarrow ? kPairCols128
                                              : nt;  // columns per block
        const int occ = h->prec == LB_FP32 ? occupancy_step_f32(s, co, e, nu == 1, tma, nt, walls && tma)
                                           : occupancy_step_f64(s, co, e, nu == 1);
        const double slots = (double)sms * occ;
        Group g{s, co, e, nu == 1, tma, nt, (int64_t)h->items.size(), 0};
        g.walls = walls && tma;
        for (int i : members) {
            const lb_case& c = h->cases[i];
            int ns = strips_of(c, width);
            const int q = c.nx % 4 == 0 ? 4 : 1;  // strip edges on multiples of q
            // the case's share of the block slots, over one wave of blocks
            // (seg_rows 0, -1) or two and four waves (-2, -3), whose later
            // waves fill the slots that short items free
            const double waves = seg_rows == -2 ? 2.0 : seg_rows == -3 ? 4.0 : 1.0;
            const double share = slots * waves * ((double)c.nx * c.ny) / nodes;
            const int min_rows = seg_rows > 0 ? std::max(kMinSegRows, std::min(kMinRows, seg_rows)) : kMinRows;
            const int max_seg = std::max(1, c.ny / min_rows);
            int nseg = seg_rows > 0 ? (c.ny + seg_rows / 2) / seg_rows : (int)std::floor(share / ns);
            if (seg_rows == -1) {
                // slot share, filled: up to four more (narrower) strips when
                // strips x segments then comes closer to the case's share
                int best = std::min(std::max(1, nseg), max_seg) * ns;
                // never more strips than the workspace's item table allows
                // for the case (strips of the narrowest block, see max_items_of)
                const int m_max = std::min({ns + 4, c.nx / q, strips_of(c, kMinBlockThreads)});
                for (int m = ns + 1; m <= m_max; ++m) {
                    const int sm = std::min(std::max(1, (int)std::floor(share / m)), max_seg);
                    if (sm * m > best && sm * m <= std::max(share, (double)ns)) {
                        best = sm * m;
                        ns = m;
                        nseg = sm;
                    }
                }
            }
            nseg = std::min(std::max(1, nseg), max_seg);
            for (int k = 0; k < ns; ++k) {
                const int x0 = q * (int)((int64_t)(c.nx / q) * k / ns);
                const int x1 = q * (int)((int64_t)(c.nx / q) * (k + 1) / ns);
                for (int r = 0; r < nseg; ++r) {
                    const int y0 = (int)((int64_t)c.ny * r / nseg);
                    const int y1 = (int)((int64_t)c.ny * (r + 1) / nseg);
                    h->items.push_back(Item{i, x0, x1 - x0, y0, y1 - y0, 0});
                }
            }
        }
        g.count = (int64_t)h->items.size() - g.first;
        std::stable_sort(h->items.begin() + g.first, h->items.end(),
                         [](const Item& a, const Item& b) { return a.h > b.h; });
        h->groups.push_back(g);
    };

    // short periodic lattices of schemes 0-3 run on the row kernel,
    // except under the persistent launch (whose kernel runs every item)
    const bool rows_ok = h->rows_on && h->persist_mode != 1;
    for (int s = 0; s < 5; ++s)
        for (int co = 0; co < 2; ++co)
            for (int e = 0; e < 2; ++e)
                for (int nu = 0; nu < 2; ++nu)
                    for (int al = 0; al < 4; ++al) {
                        // al: 0 lattices with nx % 4 != 0; 1 with nx % 4 == 0 (TMA-eligible);
                        // 2 the cases only the plain-load kernel runs; 3 with nx % 4 == 0
                        // and walls (the packed kernel's variant for walls)
                        // (the one-column TMA shapes of LBFE_STEP_THREADS do not run scheme 3)
                        const bool tma = h->prec == LB_FP32 && h->path != 1 && (al == 1 || al == 3) &&
                                         !(s == LB_IMPROVED_SMOOTH && h->tma_threads != 0);
                        const bool pair = tma && h->tma_threads == 0;
                        std::vector<int> members, narrow;
                        for (int i = 0; i < n; ++i) {
                            const lb_case& c = h->cases[i];
                            if (rows_ok && rows_eligible(c)) continue;  // the row kernel's groups below
                            // (the one-column TMA shapes pull no walls)
                            const bool plain = one_column_only(c) || (c.walls && h->tma_threads != 0);
                            const int kind = plain ? 2 : c.nx % 4 != 0 ? 0 : c.walls ? 3 : 1;
                            if (c.scheme == s && c.collision == co && c.eos == e && (c.nu > 0) == (nu == 1) &&
                                kind == al)
                                (pair && h->narrow && prefers_narrow(c) ? narrow : members).push_back(i);
                        }
                        emit(members, s, co, e, nu, tma, !tma ? kStepThreads : pair ? kPairWide : h->tma_threads,
                             al == 3);
                        emit(narrow, s, co, e, nu, tma, kPairNarrow, al == 3);
                    }
    // the row kernel: one item per strip of at most rows_strip_width columns
    // over the lattice's whole height, whatever the segment rule
    for (int s = 0; rows_ok && s < 4; ++s)
        for (int co = 0; co < 2; ++co)
            for (int e = 0; e < 2; ++e)
                for (int nu = 0; nu < 2; ++nu) {
                    Group g{s, co, e, nu == 1, false, 0, (int64_t)h->items.size(), 0};
                    g.rows = true;
                    const int w = rows_strip_width(s);
                    for (int i = 0; i < n; ++i) {
                        const lb_case& c = h->cases[i];
                        if (!rows_eligible(c) || c.scheme != s || c.collision != co || c.eos != e ||
                            (c.nu > 0) != (nu == 1))
                            continue;
                        g.ny_max = std::max(g.ny_max, c.ny);
                        const int ns = (c.nx + w - 1) / w;
                        for (int k = 0; k < ns; ++k) {
                            const int x0 = (int)((int64_t)c.nx * k / ns), x1 = (int)((int64_t)c.nx * (k + 1) / ns);
                            h->items.push_back(Item{i, x0, x1 - x0, 0, c.ny, 0});
                        }
                    }
                    g.count = (int64_t)h->items.size() - g.first;
                    if (g.count > 0) h->groups.push_back(g);
                }
    // work items per case (the blocks one step of the case launches)
    h->case_items.assign(h->cases.size(), 0);
    for (const Item& it : h->items) ++h->case_items[it.case_id];
}

lb_status upload_items(lb_handle* h)
{
    h->nb_ok = false;
    if ((int64_t)h->items.size() > h->L.max_items)
        return h->fail(LB_E_STATE, "work-list larger than the workspace's item table");
    lb_status s = h->cuda(cudaMemcpyAsync(h->ditems(), h->items.data(), h->items.size() * sizeof(Item),
                                          cudaMemcpyHostToDevice, h->stream),
                          "upload items");
    // the statistics' tickets count the items of each case
    for (int i = 0; s == LB_OK && h->st_live && i < (int)h->cases.size(); ++i) s = h->upload_case(i);
    return s;
}

// Statistics recorded by the step launches or not: the case table is
// uploaded again, and the captured graphs, whose launches name the kernel
// variants without or with statistics, are dropped (captured again by the
// next lb_step).
lb_status stats_live(lb_handle* h, bool on)
{
    const bool want = on && h->st_buf;
    if (h->st_live == want) return LB_OK;
    h->st_live = want;
    lb_status s = h->cuda(cudaStreamSynchronize(h->stream), "stats sync");
    for (cudaGraphExec_t& g : h->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    for (int i = 0; s == LB_OK && i < (int)h->cases.size(); ++i) s = h->upload_case(i);
    return s;
}

// Restart case i's statistics at its current state (a new or loaded state).
lb_status stats_restart(lb_handle* h, int i)
{
    if (!h->st_buf) return LB_OK;
    h->st_base[i] = h->steps[i];
    lb_status s = h->cuda(cudaMemsetAsync(h->st_ctr() + 2 * i, 0, 2 * sizeof(int32_t), h->stream), "stats reset");
    if (s == LB_OK)
        s = h->cuda(cudaMemsetAsync(h->st_ring() + (size_t)i * h->st_hist, 0, sizeof(StepStat), h->stream),
                    "stats reset");
    return s;
}

lb_status check_handle(lb_handle* h) { return h ? LB_OK : LB_E_INVALID; }

// The device address of host memory that kernels can read and write
// directly (page-locked and mapped, as cudaHostAlloc memory is under unified
// addressing), or nullptr for pageable memory. Kernels then move the data
// over the host link themselves, overlapping it with their arithmetic,
// instead of a copy before or after them.
template <typename P>
P* mapped_view(P* p)
{
    cudaPointerAttributes a{};
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // a pageable pointer may leave an error behind on older runtimes
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost && a.devicePointer ? static_cast<P*>(a.devicePointer) : nullptr;
}

// Failure-detection self-test: one thread waits, bounded like every wait of
// the step kernels, on an mbarrier phase that nothing completes (no copy is
// issued, no other thread arrives), then records the give-up in the status
// word the way the step kernels do.
__global__ void wait_selftest_kernel(int* status)
{
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(&bar, 0u)) atomicOr(status, 1);
}

// Pull-moment, chemical-potential and velocity passes for one case, in the
// storage precision C per node (FP64 sums); outputs may be device pointers
// or NULL. Partials of the case land in h->partials().
template <typename T, typename C, typename O>
lb_status fields_pass_t(lb_handle* h, int i, O* o_rho, O* o_ux, O* o_uy, O* o_mu)
{
    const lb_case& c = h->cases[i];
    DevCase<T> ct = dev_case<T>(c, h->L.off[i], h->rho_ref[i]);
    const DevCase<C> cc = dev_case<C>(c, h->L.off[i], h->rho_ref[i]);
    ct.lw_first = c.scheme == LB_LAX_WENDROFF && h->steps[i] == 0;  // f(0) stored unpropagated
    const dim3 blk(256), grd = field_grid(c.nx, c.ny);
    C* s0 = reinterpret_cast<C*>(h->scratch(0));
    C* s1 = reinterpret_cast<C*>(h->scratch(1));
    C* s2 = reinterpret_cast<C*>(h->scratch(2));
    C* s3 = reinterpret_cast<C*>(h->scratch(3));
    pull_moments_kernel<T, C><<<grd, blk, 0, h->stream>>>(ct, (const T*)h->fbuf(h->cur), s0, s1, s2);
    if (c.eos == LB_VDW)
        mu_field_kernel<C, 0><<<grd, blk, 0, h->stream>>>(cc, s0, s3);
    else
        mu_field_kernel<C, 1><<<grd, blk, 0, h->stream>>>(cc, s0, s3);
    if (improved_scheme(c.scheme)) {
        velocity_kernel<1, C, O><<<grd, blk, 0, h->stream>>>(cc, s0, s1, s2, s3, nullptr, nullptr, nullptr, o_rho, o_ux,
                                                          o_uy, o_mu, h->partials());
    } else if (c.scheme == LB_STANDARD_PT) {
        C* p0 = reinterpret_cast<C*>(h->scratch(8));
        C* p1 = reinterpret_cast<C*>(h->scratch(9));
        C* p2 = reinterpret_cast<C*>(h->scratch(10));
        if (c.eos == LB_VDW)
            ptensor_kernel<C, 0><<<grd, blk, 0, h->stream>>>(cc, s0, p0, p1, p2);
        else
            ptensor_kernel<C, 1><<<grd, blk, 0, h->stream>>>(cc, s0, p0, p1, p2);
        velocity_kernel<2, C, O><<<grd, blk, 0, h->stream>>>(cc, s0, s1, s2, s3, p0, p1, p2, o_rho, o_ux, o_uy, o_mu,
                                                          h->partials());
    } else if (c.scheme == LB_LAX_WENDROFF) {
        velocity_kernel<4, C, O><<<grd, blk, 0, h->stream>>>(cc, s0, s1, s2, s3, nullptr, nullptr, nullptr, o_rho, o_ux,
                                                          o_uy, o_mu, h->partials());
    } else {
        velocity_kernel<0, C, O><<<grd, blk, 0, h->stream>>>(cc, s0, s1, s2, s3, nullptr, nullptr, nullptr, o_rho, o_ux,
                                                          o_uy, o_mu, h->partials());
    }
    return h->cuda(cudaGetLastError(), "fields pass");
}

// outputs of the field type O: double, or float (lb_moments_f32)
template <typename O>
lb_status fields_pass(lb_handle* h, int i, O* o_rho, O* o_ux, O* o_uy, O* o_mu)
{
    return h->prec == LB_FP32 ? fields_pass_t<float, float, O>(h, i, o_rho, o_ux, o_uy, o_mu)
                              : fields_pass_t<double, double, O>(h, i, o_rho, o_ux, o_uy, o_mu);
}

// FP32 field -> FP64 field (n values), for the FP32 initial velocities.
__global__ void __launch_bounds__(256) widen_kernel(const float* __restrict__ in, double* __restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

// Initial populations of case i from rho0 (FP64 or FP32, I) on the device or
// in mapped host memory and the FP64 u0 fields in scratch 1, 2 when given:
// rho0 -> C scratch 4 with a device-side check, mu_c of rho0, then the
// equilibrium.
template <typename T, typename C, typename I>
lb_status init_pass_t(lb_handle* h, int i, const I* d_rho0, const double* pux, const double* puy)
{
    const lb_case& c = h->cases[i];
    const int64_t N = (int64_t)c.nx * c.ny;
    const dim3 blk(256), grd = field_grid(c.nx, c.ny);
    C* r0 = reinterpret_cast<C*>(h->scratch(4));
    C* mu = reinterpret_cast<C*>(h->scratch(5));
    rho0_kernel<C, I><<<grd, blk, 0, h->stream>>>(c.nx, c.ny, c.eos, c.b, d_rho0, r0, h->partials());
    finalize_kernel<<<1, 256, 0, h->stream>>>(h->partials(), (int64_t)grd.x * grd.y, 0.0, h->red() + 8 * i);
    double chk[5];
    lb_status s = h->cuda(cudaMemcpyAsync(chk, h->red() + 8 * i, sizeof chk, cudaMemcpyDeviceToHost, h->stream),
                          "check rho0");
    if (s == LB_OK) s = h->cuda(cudaStreamSynchronize(h->stream), "check rho0");
    if (s != LB_OK) return s;
    if (chk[4] != 0.0) return h->fail(LB_E_INVALID, "rho0 must be finite, > 0 and inside the EOS domain");
    if (h->prec == LB_FP32) h->rho_ref[i] = c.rho_ref > 0 ? c.rho_ref : chk[0] / (double)N;
    if ((s = h->upload_case(i)) != LB_OK) return s;
    const DevCase<T> ct = dev_case<T>(c, h->L.off[i], h->rho_ref[i]);
    const DevCase<C> cc = dev_case<C>(c, h->L.off[i], h->rho_ref[i]);
    if (c.eos == LB_VDW)
        mu_field_kernel<C, 0><<<grd, blk, 0, h->stream>>>(cc, r0, mu);
    else
        mu_field_kernel<C, 1><<<grd, blk, 0, h->stream>>>(cc, r0, mu);
    if (improved_scheme(c.scheme))
        init_kernel<T, 1, C><<<grd, blk, 0, h->stream>>>(ct, cc, r0, pux, puy, mu, (T*)h->fbuf(h->cur));
    else
        init_kernel<T, 0, C><<<grd, blk, 0, h->stream>>>(ct, cc, r0, pux, puy, mu, (T*)h->fbuf(h->cur));
    return h->cuda(cudaGetLastError(), "init kernels");
}

}  // namespace

extern "C" {

lb_status lb_workspace_bytes(const lb_case* cases, int32_t ncases, int32_t precision, size_t* bytes)
{
    if (!cases || ncases <= 0 || !bytes || (precision != LB_FP32 && precision != LB_FP64))
        return LB_E_INVALID;
    for (int i = 0; i < ncases; ++i)
        if (!check_case(cases[i], i).empty()) return LB_E_INVALID;
    *bytes = layout_of(cases, ncases, precision).total;
    return LB_OK;
}

lb_status lb_create(const lb_case* cases, int32_t ncases, int32_t precision, void* d_workspace,
                    size_t ws_bytes, void* cuda_stream, lb_handle** out)
{
    if (!out) return LB_E_INVALID;
    *out = nullptr;
    if (!cases || ncases <= 0 || (precision != LB_FP32 && precision != LB_FP64)) return LB_E_INVALID;
    for (int i = 0; i < ncases; ++i)
        if (!check_case(cases[i], i).empty()) return LB_E_INVALID;
    Layout L = layout_of(cases, ncases, precision);
    if (!d_workspace || ((uintptr_t)d_workspace % kAlign) != 0 || ws_bytes < L.total) return LB_E_WORKSPACE;
    lb_handle* h = new lb_handle();
    h->cases.assign(cases, cases + ncases);
    h->prec = precision;
    h->stream = (cudaStream_t)cuda_stream;
    h->ws = (uint8_t*)d_workspace;
    h->L = L;
    h->rho_ref.assign(ncases, 0.0);
    for (int i = 0; i < ncases; ++i) h->rho_ref[i] = precision == LB_FP32 ? cases[i].rho_ref : 0.0;
    h->steps.assign(ncases, 0);
    h->inited.assign(ncases, 0);
    if (const char* p = std::getenv("LBFE_STEP_PATH")) h->path = std::strcmp(p, "ldg") == 0 ? 1 : 0;
    if (const char* p = std::getenv("LBFE_GRAPH")) h->use_graph = std::strcmp(p, "0") != 0;
    if (const char* p = std::getenv("LBFE_STEP_THREADS")) {
        const int v = std::atoi(p);
        h->tma_threads = (v == 128 || v == 256) ? v : 0;
    }
    if (const char* p = std::getenv("LBFE_SEG_ROWS")) {
        h->seg_rows = std::max(-3, std::atoi(p));
        h->autotune = false;
    }
    if (const char* p = std::getenv("LBFE_ROWS")) h->rows_on = std::strcmp(p, "0") != 0;
    if (const char* p = std::getenv("LBFE_PAIR_NARROW")) {
        h->narrow = std::strcmp(p, "0") != 0;
        h->narrow_fixed = true;
    }
    build_items(h);
    lb_status s = upload_items(h);
    if (s == LB_OK)
        s = h->cuda(cudaMemsetAsync(h->status(), 0, (1 + ncases) * sizeof(int), h->stream), "clear status");
    for (int i = 0; i < ncases && s == LB_OK; ++i) s = h->upload_case(i);
    if (s != LB_OK) {
        delete h;
        return s;
    }
    *out = h;
    return LB_OK;
}

extern "C++" {
// lb_init_fields and lb_init_fields_f32 (field type I)
template <typename I>
static lb_status init_fields_t(lb_handle* h, int32_t case_id, const I* rho0, const I* ux0, const I* uy0,
                               int32_t on_device)
{
    if (check_handle(h) != LB_OK) return LB_E_INVALID;
    if (case_id < 0 || case_id >= (int)h->cases.size() || !rho0)
        return h->fail(LB_E_INVALID, "lb_init_fields: bad case id or null rho0");
    const lb_case& c = h->cases[case_id];
    const int64_t N = (int64_t)c.nx * c.ny;
    const size_t bytes = N * sizeof(I);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    double *s0 = h->scratch(0), *s1 = h->scratch(1), *s2 = h->scratch(2);
    h->steps[case_id] = 0;  // before the case table is uploaded (Lax-Wendroff step-0 flag)
    lb_status s = LB_OK;
    const I* d_rho0 = rho0;
    if (!on_device) {
        // page-locked host rho0 is read by rho0_kernel itself
        const I* m = mapped_view(rho0);
        if (m)
            d_rho0 = m;
        else
            s = h->cuda(cudaMemcpyAsync(s0, rho0, bytes, kind, h->stream), "copy rho0");
        if (!m) d_rho0 = reinterpret_cast<const I*>(s0);
    }
    // u0 as FP64 in scratch 1, 2 (FP32 u0 is copied to scratch 6, 7, which
    // the init pass does not use, and widened from there)
    const double* pu[2] = {nullptr, nullptr};
    const I* u0[2] = {ux0, uy0};
    double* su[2] = {s1, s2};
    for (int k = 0; k < 2 && s == LB_OK; ++k) {
        if (!u0[k]) continue;
        if constexpr (sizeof(I) == sizeof(double)) {
            s = h->cuda(cudaMemcpyAsync(su[k], u0[k], bytes, kind, h->stream), "copy u0");
        } else {
            float* tmp = reinterpret_cast<float*>(h->scratch(6 + k));
            s = h->cuda(cudaMemcpyAsync(tmp, u0[k], bytes, kind, h->stream), "copy u0");
            if (s == LB_OK) {
                widen_kernel<<<(unsigned)std::min<int64_t>((N + 255) / 256, 4096), 256, 0, h->stream>>>(tmp, su[k], N);
                s = h->cuda(cudaGetLastError(), "widen u0");
            }
        }
        pu[k] = su[k];
    }
    if (s != LB_OK) return s;
    s = h->prec == LB_FP32 ? init_pass_t<float, float, I>(h, case_id, d_rho0, pu[0], pu[1])
                           : init_pass_t<double, double, I>(h, case_id, d_rho0, pu[0], pu[1]);
    if (s == LB_OK)  // a fresh state clears the case's instability flag
        s = h->cuda(cudaMemsetAsync(h->status() + 1 + case_id, 0, sizeof(int), h->stream), "clear case flag");
    if (s != LB_OK) return s;
    h->steps[case_id] = 0;
    h->inited[case_id] = 1;
    return stats_restart(h, case_id);
}
}  // extern "C++"

lb_status lb_init_fields(lb_handle* h, int32_t case_id, const double* rho0, const double* ux0,
                         const double* uy0, int32_t on_device)
{
    return init_fields_t<double>(h, case_id, rho0, ux0, uy0, on_device);
}

lb_status lb_init_fields_f32(lb_handle* h, int32_t case_id, const float* rho0, const float* ux0, const float* uy0,
                             int32_t on_device)
{
    return init_fields_t<float>(h, case_id, rho0, ux0, uy0, on_device);
}

// Enqueue one time step (every group) on stream st, reading buffer cur.
// With several groups, the groups after the first run on branch streams that
// fork from st and join it again, so their launches can overlap on the GPU
// (they write disjoint cases); inside a capture this makes them parallel
// graph nodes.
static lb_status enqueue_step(lb_handle* h, int cur, cudaStream_t st)
{
    const int nb = (int)h->groups.size() - 1;
    lb_status s = LB_OK;
    while ((int)h->aux.size() < nb && s == LB_OK) {
        cudaStream_t a = nullptr;
        cudaEvent_t f = nullptr, j = nullptr;
        s = h->cuda(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking), "branch stream");
        if (s == LB_OK) s = h->cuda(cudaEventCreateWithFlags(&f, cudaEventDisableTiming), "branch event");
        if (s == LB_OK) s = h->cuda(cudaEventCreateWithFlags(&j, cudaEventDisableTiming), "branch event");
        if (a) h->aux.push_back(a);
        if (f) h->fork_join.push_back(f);
        if (j) h->fork_join.push_back(j);
    }
    if (s != LB_OK) return s;
    for (int b = 0; b < nb && s == LB_OK; ++b) {
        s = h->cuda(cudaEventRecord(h->fork_join[2 * b], st), "fork");
        if (s == LB_OK) s = h->cuda(cudaStreamWaitEvent(h->aux[b], h->fork_join[2 * b], 0), "fork");
    }
    for (int k = 0; k <= nb && s == LB_OK; ++k) {
        const Group& g = h->groups[k];
        const cudaStream_t gs = k == 0 ? st : h->aux[k - 1];
        cudaError_t e;
        if (g.rows)
            e = launch_step_rows(h->prec, g.scheme, g.coll, g.eos, g.nu, g.ny_max, (int)g.count, gs, h->fbuf(cur),
                                 h->fbuf(cur ^ 1),
                                 h->prec == LB_FP32 ? (const void*)h->dc32() : (const void*)h->dc64(),
                                 h->ditems() + g.first, h->status(), h->st_live);
        else if (h->prec == LB_FP32)
            e = launch_step_f32(g.scheme, g.coll, g.eos, g.nu, g.tma, g.nt, (int)g.count, gs,
                                (const float*)h->fbuf(cur), (float*)h->fbuf(cur ^ 1), h->dc32(),
                                h->ditems() + g.first, h->status(), h->st_live, g.walls);
        else
            e = launch_step_f64(g.scheme, g.coll, g.eos, g.nu, (int)g.count, gs, (const double*)h->fbuf(cur),
                                (double*)h->fbuf(cur ^ 1), h->dc64(), h->ditems() + g.first, h->status(),
                                h->st_live);
        if (e != cudaSuccess) s = h->cuda(e, "step launch");
    }
    for (int b = 0; b < nb; ++b) {  // join every branch, even after a failed launch
        lb_status t = h->cuda(cudaEventRecord(h->fork_join[2 * b + 1], h->aux[b]), "join");
        if (t == LB_OK) t = h->cuda(cudaStreamWaitEvent(st, h->fork_join[2 * b + 1], 0), "join");
        if (s == LB_OK) s = t;
    }
    return s;
}

// Capture kGraphSteps steps starting from buffer cur into h->graph[cur].
static lb_status capture_graph(lb_handle* h, int cur)
{
    if (!h->cap_stream) {
        lb_status s = h->cuda(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), "capture stream");
        if (s != LB_OK) return s;
    }
    lb_status s = h->cuda(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (s != LB_OK) return s;
    lb_status ls = LB_OK;
    for (int k = 0; k < kGraphSteps && ls == LB_OK; ++k) ls = enqueue_step(h, cur ^ (k & 1), h->cap_stream);
    cudaGraph_t g = nullptr;
    s = h->cuda(cudaStreamEndCapture(h->cap_stream, &g), "end capture");
    if (ls != LB_OK || s != LB_OK) {
        if (g) cudaGraphDestroy(g);
        return ls != LB_OK ? ls : s;
    }
    s = h->cuda(cudaGraphInstantiate(&h->graph[cur], g, 0), "instantiate graph");
    cudaGraphDestroy(g);
    return s;
}

// Time one step under each candidate work-list and keep the fastest. Every
// trial launch reads the current buffer and writes the other one, which the
// next real step overwrites, so the state is untouched. Each candidate runs
// for about 1 ms per pass (3 to 64 launches) in two interleaved passes, its
// time is the better pass, and a candidate replaces the slot-share rule only
// if it is at least 2 % faster.
static lb_status tune_time(lb_handle* h, cudaEvent_t e0, cudaEvent_t e1, int reps, float* ms)
{
    lb_status s = h->cuda(cudaEventRecord(e0, h->stream), "tune record");
    for (int r = 0; r < reps && s == LB_OK; ++r) s = enqueue_step(h, h->cur, h->stream);
    if (s == LB_OK) s = h->cuda(cudaEventRecord(e1, h->stream), "tune record");
    if (s == LB_OK) s = h->cuda(cudaEventSynchronize(e1), "tune sync");
    if (s == LB_OK) s = h->cuda(cudaEventElapsedTime(ms, e0, e1), "tune time");
    if (s == LB_OK) *ms /= (float)reps;
    return s;
}

static lb_status autotune(lb_handle* h)
{
    // the row kernel's work-lists do not depend on the segment rule
    bool all_rows = true;
    for (const Group& g : h->groups) all_rows = all_rows && g.rows;
    if (all_rows) {
        h->tuned = true;
        return LB_OK;
    }
    // candidates: row-segment rule x (narrow packed blocks off, on); the
    // second half only when some lattice prefers narrow blocks
    // (short segments serve lattices small enough that a step is bound by the
    // latency of its row pipeline: fewer rows per item, more items at once)
    static const int segs[] = {0, -1, -2, -3, 256, 128, 64, 32, 16, 8, 4, 2};
    constexpr int kSegs = (int)(sizeof segs / sizeof segs[0]);
    bool any_narrow = false;
    if (h->prec == LB_FP32 && h->path != 1 && h->tma_threads == 0 && !h->narrow_fixed)
        for (const lb_case& c : h->cases) any_narrow = any_narrow || (c.nx % 4 == 0 && prefers_narrow(c));
    const bool narrow0 = h->narrow;
    const int kCands = any_narrow ? 2 * kSegs : kSegs;
    auto apply = [&](int k) {
        h->seg_rows = segs[k % kSegs];
        h->narrow = any_narrow ? k >= kSegs : narrow0;
    };
    // trial launches record no statistics
    const bool st_was = h->st_live;
    lb_status s = stats_live(h, false);
    if (s != LB_OK) return s;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    s = h->cuda(cudaEventCreate(&e0), "tune event");
    if (s == LB_OK) s = h->cuda(cudaEventCreate(&e1), "tune event");
    float best_ms[2 * kSegs];
    for (float& b : best_ms) b = 1e30f;
    int reps = 3;
    // candidate 0 (the current list) sets the launch count: two warm-up
    // launches, then one timed
    if (s == LB_OK) {
        float t1 = 0.f;
        for (int r = 0; r < 2 && s == LB_OK; ++r) s = enqueue_step(h, h->cur, h->stream);
        if (s == LB_OK) s = tune_time(h, e0, e1, 1, &t1);
        if (s == LB_OK) reps = std::max(3, std::min(64, (int)(1.0f / std::max(t1, 1e-3f))));
    }
    for (int pass = 0; pass < 2 && s == LB_OK; ++pass)
        for (int k = 0; k < kCands && s == LB_OK; ++k) {
            apply(k);
            build_items(h);
            if ((int64_t)h->items.size() > h->L.max_items) continue;
            if ((s = upload_items(h)) != LB_OK) break;
            if ((s = enqueue_step(h, h->cur, h->stream)) != LB_OK) break;
            float ms = 0.f;
            if ((s = tune_time(h, e0, e1, reps, &ms)) != LB_OK) break;
            best_ms[k] = std::min(best_ms[k], ms);
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    int best = 0;
    for (int k = 1; k < kCands; ++k)
        if (best_ms[k] < 0.98f * best_ms[0] && best_ms[k] < best_ms[best]) best = k;
    apply(best);
    build_items(h);
    lb_status u = upload_items(h);
    if (u == LB_OK) u = stats_live(h, st_was);
    h->tuned = true;
    return s != LB_OK ? s : u;
}

// Work-list built again after a change of the rules that shape it (the
// captured graphs name the old groups and are dropped).
static lb_status rebuild_worklist(lb_handle* h)
{
    lb_status s = h->cuda(cudaStreamSynchronize(h->stream), "work-list sync");
    for (cudaGraphExec_t& g : h->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    build_items(h);
    return s == LB_OK ? upload_items(h) : s;
}

// ------------------------------------------------------ persistent launch
constexpr int kPersistChunk = 1024;  // steps per persistent launch

// Column / row halo around an item that its step reads: the pull and the
// stencil halo (HX + 1 either side).
static int persist_reach(const lb_case& c) { return halo_of(c.scheme) + 1; }

// circular intervals [a0, a0 + la) and [b0, b0 + lb) modulo n intersect
static bool circ_overlap(int a0, int la, int b0, int lb, int n)
{
    if (la >= n || lb >= n) return true;
    const int d1 = ((b0 - a0) % n + n) % n, d2 = ((a0 - b0) % n + n) % n;
    return d1 < la || d2 < lb;
}

// A one-group handle can use the persistent kernel (mode 2 only where its
// group already runs the one-column kernel, so that results do not change).
static bool persist_possible(const lb_handle* h, bool strict)
{
    if (h->groups.size() != 1 || h->st_buf) return false;  // (per-step statistics need one launch per step)
    const Group& g = h->groups[0];
    if (strict && (g.tma || g.rows)) return false;
    return occupancy_persist(h->prec, g.scheme, g.coll, g.eos, g.nu) > 0;
}

// Neighbour lists of the group's items (every other item of the same case
// whose output overlaps the item's input), uploaded as CSR; false if an item
// has more than kMaxNeighbours of them.
static lb_status build_neighbours(lb_handle* h, bool* ok)
{
    *ok = false;
    const Group& g = h->groups[0];
    std::vector<int> off(1, 0), idx;
    for (int64_t i = 0; i < g.count; ++i) {
        const Item& a = h->items[g.first + i];
        const lb_case& c = h->cases[a.case_id];
        const int r = persist_reach(c);
        int cnt = 0;
        for (int64_t j = 0; j < g.count; ++j) {
            if (j == i) continue;
            const Item& b = h->items[g.first + j];
            if (b.case_id != a.case_id) continue;
            if (circ_overlap(a.x0 - r, a.wv + 2 * r, b.x0, b.wv, c.nx) &&
                circ_overlap(a.y0 - r, a.h + 2 * r, b.y0, b.h, c.ny)) {
                idx.push_back((int)j);
                if (++cnt > kMaxNeighbours) return LB_OK;
            }
        }
        off.push_back((int)idx.size());
    }
    lb_status s = h->cuda(cudaMemcpyAsync(h->nb_off(), off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice,
                                          h->stream),
                          "upload neighbours");
    if (s == LB_OK && !idx.empty())
        s = h->cuda(cudaMemcpyAsync(h->nb_idx(), idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice,
                                    h->stream),
                    "upload neighbours");
    if (s == LB_OK) s = h->cuda(cudaStreamSynchronize(h->stream), "upload neighbours");
    if (s != LB_OK) return s;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int occ = occupancy_persist(h->prec, g.scheme, g.coll, g.eos, g.nu);
    h->persist_grid = (int)std::min<int64_t>(g.count, (int64_t)occ * sms);
    h->nb_ok = *ok = true;
    return LB_OK;
}

// nsteps steps of the single group by persistent launches of up to
// kPersistChunk steps; silent_item >= 0 is the self-test (that item never
// publishes its progress, so its neighbours' waits give up after spin).
static lb_status enqueue_persist(lb_handle* h, int64_t nsteps, int silent_item, long long spin)
{
    const Group& g = h->groups[0];
    for (int64_t done = 0; done < nsteps;) {
        const int chunk = (int)std::min<int64_t>(kPersistChunk, nsteps - done);
        lb_status s = h->cuda(cudaMemsetAsync(h->progress(), 0, (g.count + 1) * sizeof(int), h->stream),
                              "clear progress");
        if (s != LB_OK) return s;
        PersistArgs pa;
        pa.nb_off = h->nb_off();
        pa.nb_idx = h->nb_idx();
        pa.progress = h->progress();
        pa.nitems = (int)g.count;
        pa.nsteps = chunk;
        pa.spin_limit = spin;
        pa.silent_item = silent_item;
        const void* cases = h->prec == LB_FP32 ? (const void*)h->dc32() : (const void*)h->dc64();
        s = h->cuda(launch_persist(h->prec, g.scheme, g.coll, g.eos, g.nu, h->persist_grid, h->stream,
                                   h->fbuf(h->cur), h->fbuf(h->cur ^ 1), cases, h->ditems() + g.first, h->status(),
                                   pa),
                    "persistent launch");
        if (s != LB_OK) return s;
        if (chunk & 1) h->cur ^= 1;
        done += chunk;
    }
    return LB_OK;
}

// Mode 2: time 16 steps of graph replay against 16 steps of the persistent
// launch (after 8 untimed persistent steps that load the kernel), with the
// call's own steps, and keep the faster mode. Both modes run the same
// per-node arithmetic, so the choice changes no result. Consumes 40 steps.
static lb_status tune_persist(lb_handle* h)
{
    h->persist_tuned = true;
    if (!h->graph[h->cur]) {
        lb_status s = capture_graph(h, h->cur);
        if (s != LB_OK) return s;
    }
    cudaEvent_t e[4] = {};
    lb_status s = LB_OK;
    for (auto& x : e)
        if (s == LB_OK) s = h->cuda(cudaEventCreate(&x), "tune event");
    if (s == LB_OK) s = enqueue_persist(h, kGraphSteps, -1, h->spin_limit);
    if (s == LB_OK) s = h->cuda(cudaEventRecord(e[0], h->stream), "tune record");
    for (int k = 0; k < 2 && s == LB_OK; ++k)
        s = h->cuda(cudaGraphLaunch(h->graph[h->cur], h->stream), "graph launch");
    if (s == LB_OK) s = h->cuda(cudaEventRecord(e[1], h->stream), "tune record");
    if (s == LB_OK) s = h->cuda(cudaEventRecord(e[2], h->stream), "tune record");
    if (s == LB_OK) s = enqueue_persist(h, 2 * kGraphSteps, -1, h->spin_limit);
    if (s == LB_OK) s = h->cuda(cudaEventRecord(e[3], h->stream), "tune record");
    if (s == LB_OK) s = h->cuda(cudaEventSynchronize(e[3]), "tune sync");
    float tg = 0.f, tp = 0.f;
    if (s == LB_OK) s = h->cuda(cudaEventElapsedTime(&tg, e[0], e[1]), "tune time");
    if (s == LB_OK) s = h->cuda(cudaEventElapsedTime(&tp, e[2], e[3]), "tune time");
    for (auto& x : e)
        if (x) cudaEventDestroy(x);
    if (s == LB_OK) h->persist = tp < 0.98f * tg;
    return s;
}

lb_status lb_step(lb_handle* h, int64_t nsteps)
{
    if (check_handle(h) != LB_OK) return LB_E_INVALID;
    if (nsteps < 0) return h->fail(LB_E_INVALID, "lb_step: nsteps < 0");
    for (size_t i = 0; i < h->cases.size(); ++i)
        if (!h->inited[i]) return h->fail(LB_E_STATE, "lb_step: every case needs lb_init_fields first");
    if (h->autotune && !h->tuned && nsteps > 0) {
        lb_status s = autotune(h);
        if (s != LB_OK) return s;
    }
    int64_t n = nsteps;
    // a Lax-Wendroff case at step 0 holds f(0) unpropagated: run that step on
    // its own, then mark the case's populations as post-collision
    bool lw0 = false;
    for (size_t i = 0; i < h->cases.size(); ++i)
        lw0 = lw0 || (h->cases[i].scheme == LB_LAX_WENDROFF && h->steps[i] == 0);
    if (lw0 && n > 0) {
        lb_status s = enqueue_step(h, h->cur, h->stream);
        if (s != LB_OK) return s;
        h->cur ^= 1;
        for (auto& st : h->steps) st += 1;
        for (size_t i = 0; i < h->cases.size() && s == LB_OK; ++i)
            if (h->cases[i].scheme == LB_LAX_WENDROFF) s = h->upload_case((int)i);
        if (s != LB_OK) return s;
        --n;
        nsteps = n;
    }
    if (h->persist_mode != 0 && n > 0 && persist_possible(h, h->persist_mode == 2)) {
        if (!h->nb_ok) {
            bool ok = false;
            lb_status s = build_neighbours(h, &ok);
            if (s != LB_OK) return s;
            if (!ok) h->persist = false, h->persist_tuned = true;
        }
        if (h->nb_ok && h->persist_mode == 1) h->persist = true;
        if (h->nb_ok && h->persist_mode == 2 && !h->persist_tuned && n >= 5 * kGraphSteps) {
            lb_status s = tune_persist(h);
            if (s != LB_OK) return s;
            n -= 5 * kGraphSteps;
        }
        if (h->persist && h->nb_ok) {
            lb_status s = enqueue_persist(h, n, -1, h->spin_limit);
            if (s != LB_OK) return s;
            n = 0;
        }
    }
    if (h->use_graph && n >= kGraphSteps) {
        if (!h->graph[h->cur]) {
            lb_status s = capture_graph(h, h->cur);
            if (s != LB_OK) return s;
        }
        for (; n >= kGraphSteps; n -= kGraphSteps) {
            lb_status s = h->cuda(cudaGraphLaunch(h->graph[h->cur], h->stream), "graph launch");
            if (s != LB_OK) return s;
        }
    }
    for (; n > 0; --n) {
        lb_status s = enqueue_step(h, h->cur, h->stream);
        if (s != LB_OK) return s;
        h->cur ^= 1;
    }
    for (auto& st : h->steps) st += nsteps;
    return LB_OK;
}

lb_status lb_launch_mode(lb_handle* h, int32_t mode, int32_t* persistent)
{
    if (check_handle(h) != LB_OK) return LB_E_INVALID;
    if (mode < -1 || mode > 2) return h->fail(LB_E_INVALID, "lb_launch_mode: mode must be -1, 0, 1 or 2");
    if (mode >= 0) {
        // the row kernel's groups exist outside the persistent launch only:
        // entering or leaving it rebuilds the work-list
        bool any_rows = false;
        for (const lb_case& c : h->cases) any_rows = any_rows || (h->rows_on && rows_eligible(c));
        const int old = h->persist_mode;
        h->persist_mode = mode;
        lb_status s = any_rows && (old == 1) != (mode == 1) ? rebuild_worklist(h) : LB_OK;
        if (s == LB_OK && mode == 1 && !persist_possible(h, false)) {
            h->persist_mode = old;
            if (any_rows && old != 1) rebuild_worklist(h);
            return h->fail(LB_E_INVALID, "lb_launch_mode: the persistent launch needs a handle whose cases all "
                                         "share one kernel group and no per-step statistics attached");
        }
        if (s != LB_OK) return s;
        h->persist = mode == 1;
        h->persist_tuned = mode != 2;
    }
    if (persistent) *persistent = h->persist ? 1 : 0;
    return LB_OK;
}

lb_status lb_persistent_selftest(lb_handle* h, int64_t nsteps)
{
    if (check_handle(h) != LB_OK) return LB_E_INVALID;
    if (nsteps < 2 || !persist_possible(h, false))
        return h->fail(LB_E_INVALID, "lb_persistent_selftest: needs nsteps >= 2 and a one-group handle");
    for (size_t i = 0; i < h->cases.size(); ++i)
        if (!h->inited[i]) return h->fail(LB_E_STATE, "lb_persistent_selftest: every case needs lb_init_fields");
    if (!h->nb_ok) {
        bool ok = false;
        lb_status s = build_neighbours(h, &ok);
        if (s != LB_OK) return s;
        if (!ok) return h->fail(LB_E_INVALID, "lb_persistent_selftest: an item has too many neighbours");
    }
    if (h->groups[0].count < 2) return h->fail(LB_E_INVALID, "lb_persistent_selftest: needs at least two items");
    // about 10 ms of SM clock per wait; item 0 never publishes, so the first
    // neighbour that waits for it gives up, and every block then returns
    lb_status s = enqueue_persist(h, std::min<int64_t>(nsteps, kPersistChunk), 0, 20000000LL);
    for (auto& st : h->steps) st += std::min<int64_t>(nsteps, kPersistChunk);
    return s;
}

lb_status lb_worklist(const lb_handle* h, int32_t* seg_rows, int64_t* n_items, int32_t* narrow)
{
    if (!h) return LB_E_INVALID;
    if (seg_rows) *seg_rows = h->seg_rows;
    if (n_items) *n_items = (int64_t)h->items.size();
    if (narrow) {
        *narrow = 0;
        for (const Group& g : h->groups) *narrow |= g.tma && g.nt == kPairNarrow;
    }
    return LB_OK;
}

extern "C++" {
// lb_moments and lb_moments_f32 (field type O)
template <typename O>
static lb_status moments_t(lb_handle* h, int32_t case_id, O* rho, O* ux, O* uy, O* mu, int32_t on_device)
{
    if (check_handle(h) != LB_OK) return LB_E_INVALID;
    if (case_id < 0 || case_id >= (int)h->cases.size()) return h->fail(LB_E_INVALID, "lb_moments: bad case id");
    if (!h->inited[case_id]) return h->fail(LB_E_STATE, "lb_moments: case not initialised");
    const lb_case& c = h->cases[case_id];
    const size_t bytes = (size_t)c.nx * c.ny * sizeof(O);
    O* outs[4] = {rho, ux, uy, mu};
    O* dst[4];
    bool staged[4] = {false, false, false, false};
    for (int k = 0; k < 4; ++k) {
        dst[k] = outs[k];
        if (outs[k] && !on_device) {
            // page-locked host outputs are written by the export kernel itself
            O* m = mapped_view(outs[k]);
            staged[k] = m == nullptr;
            dst[k] = m ? m : reinterpret_cast<O*>(h->scratch(4 + k));
        }
    }
    lb_status s = fields_pass<O>(h, case_id, dst[0], dst[1], dst[2], dst[3]);
    if (s != LB_OK) return s;
    if (!on_device) {
        for (int k = 0; k < 4 && s == LB_OK; ++k)
            if (staged[k])
                s = h->cuda(cudaMemcpyAsync(outs[k], dst[k], bytes, cudaMemcpyDeviceToHost, h->stream), "copy out");
        if (s == LB_OK) s = h->cuda(cudaStreamSynchronize(h->stream), "moments sync");
    }
    return s;
}
}  // extern "C++"

lb_status lb_moments(lb_handle* h, int32_t case_id, double* rho, double* ux, double* uy, double* mu,
                     int32_t on_device)
{
    return moments_t<double>(h, case_id, rho, ux, uy, mu, on_device);
}

lb_status lb_moments_f32(lb_handle* h, int32_t case_id, float* rho, float* ux, float* uy, float* mu,
                         int32_t on_device)
{
    return moments_t<float>(h, case_id, rho, ux, uy, mu, on_device);
}

lb_status lb_reductions(lb_handle* h, double* out, int32_t* case_status)
{
    if (check_handle(h) != LB_OK) return LB_E_INVALID;
    if (!out) return h->fail(LB_E_INVALID, "lb_reductions: null out");
    const int n = (int)h->cases.size();
    for (int i = 0; i < n; ++i)
        if (!h->inited[i]) return h->fail(LB_E_STATE, "lb_reductions: case not initialised");
    for (int i = 0; i < n; ++i) {
        lb_status s = fields_pass<double>(h, i, nullptr, nullptr, nullptr, nullptr);
        if (s != LB_OK) return s;
        const lb_case& c = h->cases[i];
        const dim3 g = field_grid(c.nx, c.ny);
        finalize_kernel<<<1, 256, 0, h->stream>>>(h->partials(), (int64_t)g.x * g.y, (double)h->steps[i],
                                                  h->red() + 8 * i);
        if ((s = h->cuda(cudaGetLastError(), "finalize")) != LB_OK) return s;
    }
    std::vector<double> red((size_t)n * 8);
    std::vector<int> flags((size_t)n + 1);
    lb_status s = h->cuda(cudaMemcpyAsync(red.data(), h->red(), red.size() * sizeof(double),
                                          cudaMemcpyDeviceToHost, h->stream),
                          "copy reductions");
    if (s == LB_OK)
        s = h->cuda(cudaMemcpyAsync(flags.data(), h->status(), flags.size() * sizeof(int), cudaMemcpyDeviceToHost,
                                    h->stream),
                    "copy status");
    if (s == LB_OK) s = h->cuda(cudaStreamSynchronize(h->stream), "reductions sync");
    if (s != LB_OK) return s;
    const int timeout = flags[0];
    bool unstable = false;
    for (int i = 0; i < n; ++i) {
        for (int k = 0; k < 5; ++k) out[5 * i + k] = red[8 * i + k];
        // flagged by a step kernel (and since then frozen), or non-physical now
        const bool bad = flags[1 + i] != 0 || red[8 * i + 4] != 0.0 || !std::isfinite(red[8 * i]);
        out[5 * i + 4] = 0.0;
        if (case_status) case_status[i] = bad ? LB_E_UNSTABLE : LB_OK;
        unstable |= bad;
    }
    if (timeout) {
        if (h->cuda(cudaMemsetAsync(h->status(), 0, sizeof(int), h->stream), "clear status") != LB_OK)
            return LB_E_CUDA;
        return h->fail(LB_E_TIMEOUT, "a bounded wait for a bulk copy gave up; results since the last "
                                     "lb_reductions are unreliable");
    }
    if (unstable) return h->fail(LB_E_UNSTABLE, "a case has rho <= 0 or non-finite values");
    return LB_OK;
}

constexpr int32_t kMaxStatHistory = 1 << 20;

lb_status lb_step_stats_bytes(const lb_handle* h, int32_t history, size_t* bytes)
{
    if (!h || !bytes || history < 1 || history > kMaxStatHistory) return LB_E_INVALID;
    *bytes = align_up(2 * sizeof(int32_t) * h->cases.size(), kAlign) +
             (size_t)history * h->cases.size() * sizeof(StepStat);
    return LB_OK;
}

lb_status lb_step_stats_attach(lb_handle* h, void* d_buf, size_t bytes, int32_t history)
{
    if (check_handle(h) != LB_OK) return LB_E_INVALID;
    lb_status s = stats_live(h, false);  // the kernels stop seeing the previous buffer
    if (s != LB_OK) return s;
    h->st_buf = nullptr;
    h->st_hist = 0;
    if (!d_buf) return LB_OK;
    size_t need = 0;
    if (lb_step_stats_bytes(h, history, &need) != LB_OK)
        return h->fail(LB_E_INVALID, "lb_step_stats_attach: history must be in [1, 2^20]");
    if (bytes < need || (uintptr_t)d_buf % 16 != 0)
        return h->fail(LB_E_INVALID, "lb_step_stats_attach: buffer smaller than lb_step_stats_bytes or not "
                                     "16-byte aligned");
    s = h->cuda(cudaMemsetAsync(d_buf, 0, need, h->stream), "stats clear");
    if (s != LB_OK) return s;
    h->st_buf = (uint8_t*)d_buf;
    h->st_hist = history;
    h->st_base.assign(h->steps.begin(), h->steps.end());
    return stats_live(h, true);
}

// recorded states of case i still in the ring: [first, first + count)
static lb_status stats_range(lb_handle* h, int32_t i, int64_t* first, int64_t* count, int32_t* recorded)
{
    int32_t n = 0;
    lb_status s = h->cuda(cudaMemcpyAsync(&n, h->st_ctr() + 2 * i + 1, sizeof n, cudaMemcpyDeviceToHost, h->stream),
                          "stats counter");
    if (s == LB_OK) s = h->cuda(cudaStreamSynchronize(h->stream), "stats sync");
    if (s != LB_OK) return s;
    const int64_t kept = std::min<int64_t>(n, h->st_hist);
    *first = h->st_base[i] + n - kept;
    *count = kept;
    if (recorded) *recorded = n;
    return LB_OK;
}

lb_status lb_step_stats_range(lb_handle* h, int32_t case_id, int64_t* first_state, int64_t* count)
{
    if (check_handle(h) != LB_OK) return LB_E_INVALID;
    if (case_id < 0 || case_id >= (int)h->cases.size() || !first_state || !count)
        return h->fail(LB_E_INVALID, "lb_step_stats_range: bad case id or null output");
    if (!h->st_buf) return h->fail(LB_E_STATE, "lb_step_stats_range: no statistics buffer attached");
    return stats_range(h, case_id, first_state, count, nullptr);
}

lb_status lb_step_stats_read(lb_handle* h, int32_t case_id, int64_t first_state, int32_t count, double* out)
{
    if (check_handle(h) != LB_OK) return LB_E_INVALID;
    if (case_id < 0 || case_id >= (int)h->cases.size() || count < 0 || (count > 0 && !out))
        return h->fail(LB_E_INVALID, "lb_step_stats_read: bad case id, count or output");
    if (!h->st_buf) return h->fail(LB_E_STATE, "lb_step_stats_read: no statistics buffer attached");
    int64_t first = 0, kept = 0;
    int32_t n = 0;
    lb_status s = stats_range(h, case_id, &first, &kept, &n);
    if (s != LB_OK) return s;
    if (first_state < first || first_state + count > first + kept)
        return h->fail(LB_E_INVALID, "lb_step_stats_read: states outside the recorded range (lb_step_stats_range)");
    if (count == 0) return LB_OK;
    std::vector<StepStat> e((size_t)count);
    const StepStat* ring = h->st_ring() + (size_t)case_id * h->st_hist;
    // entry k of the case (k-th recorded state since the restart) is at ring[k % history]
    const int64_t k0 = first_state - h->st_base[case_id];
    const int64_t r0 = k0 % h->st_hist;
    const int64_t n1 = std::min<int64_t>(count, h->st_hist - r0);
    s = h->cuda(cudaMemcpyAsync(e.data(), ring + r0, n1 * sizeof(StepStat), cudaMemcpyDeviceToHost, h->stream),
                "stats read");
    if (s == LB_OK && n1 < count)
        s = h->cuda(cudaMemcpyAsync(e.data() + n1, ring, (count - n1) * sizeof(StepStat), cudaMemcpyDeviceToHost,
                                    h->stream),
                    "stats read");
    if (s == LB_OK) s = h->cuda(cudaStreamSynchronize(h->stream), "stats sync");
    if (s != LB_OK) return s;
    const lb_case& c = h->cases[case_id];
    // the share of rho_ref in the mass, with rho_ref as the kernels hold it
    const double rr = h->prec == LB_FP32 ? (double)(float)h->rho_ref[case_id] : h->rho_ref[case_id];
    const double base = (double)c.nx * c.ny * rr;
    for (int32_t k = 0; k < count; ++k) {
        double u2;
        memcpy(&u2, &e[k].umax2, sizeof u2);
        out[4 * k + 0] = base + e[k].dmass;
        out[4 * k + 1] = 0.5 * e[k].ke2;
        out[4 * k + 2] = std::sqrt(u2);
        out[4 * k + 3] = (double)e[k].nodes;
    }
    return LB_OK;
}

lb_status lb_window_means(lb_handle* h, int32_t case_id, int32_t nwin, const lb_window* win, double* mean)
{
    if (check_handle(h) != LB_OK) return LB_E_INVALID;
    if (case_id < 0 || case_id >= (int)h->cases.size() || nwin < 0 || (nwin > 0 && (!win || !mean)))
        return h->fail(LB_E_INVALID, "lb_window_means: bad arguments");
    if (!h->inited[case_id]) return h->fail(LB_E_STATE, "lb_window_means: case not initialised");
    const lb_case& c = h->cases[case_id];
    // bounding boxes first, so that nothing is enqueued for a bad window
    std::vector<int> bx(nwin), by(nwin), bw(nwin), bh(nwin);
    for (int k = 0; k < nwin; ++k) {
        const lb_window& w = win[k];
        const double v[] = {w.a, w.b, w.c, w.d};
        for (double x : v)
            if (!std::isfinite(x)) return h->fail(LB_E_INVALID, "lb_window_means: non-finite window");
        if (w.kind == LB_WIN_RECT) {
            if (!(w.c >= 1 && w.c <= c.nx && w.d >= 1 && w.d <= c.ny))
                return h->fail(LB_E_INVALID, "lb_window_means: rectangle larger than the lattice or empty");
            bx[k] = (int)std::floor(w.a);
            by[k] = (int)std::floor(w.b);
            bw[k] = (int)w.c;
            bh[k] = (int)w.d;
        } else if (w.kind == LB_WIN_DISC) {
            if (!(w.c > 0 && 2 * w.c <= std::min(c.nx, c.ny)))
                return h->fail(LB_E_INVALID, "lb_window_means: disc radius outside (0, min(nx, ny) / 2]");
            bx[k] = (int)std::floor(w.a - w.c);
            by[k] = (int)std::floor(w.b - w.c);
            bw[k] = std::min(c.nx, (int)std::ceil(2 * w.c) + 2);
            bh[k] = std::min(c.ny, (int)std::ceil(2 * w.c) + 2);
        } else {
            return h->fail(LB_E_INVALID, "lb_window_means: unknown window kind");
        }
        bx[k] = ((bx[k] % c.nx) + c.nx) % c.nx;
        by[k] = ((by[k] % c.ny) + c.ny) % c.ny;
    }
    lb_status s = fields_pass<double>(h, case_id, nullptr, nullptr, nullptr, nullptr);  // rho -> scratch 0
    if (s != LB_OK) return s;
    double* res = h->red() + 8 * case_id;  // the case's reduction slot, rewritten by lb_reductions
    std::vector<double> out(5);
    for (int k = 0; k < nwin && s == LB_OK; ++k) {
        const dim3 blk(256), grd((bw[k] + 255) / 256, bh[k]);
        const bool disc = win[k].kind == LB_WIN_DISC;
        // disc centre in [0, nx) x [0, ny), so that periodic distances are min(d, n - d)
        const double cx = win[k].a - c.nx * std::floor(win[k].a / c.nx);
        const double cy = win[k].b - c.ny * std::floor(win[k].b / c.ny);
        if (h->prec == LB_FP32)
            window_sum_kernel<float><<<grd, blk, 0, h->stream>>>(reinterpret_cast<const float*>(h->scratch(0)), c.nx,
                                                                c.ny, bx[k], by[k], bw[k], disc, cx, cy, win[k].c,
                                                                h->partials());
        else
            window_sum_kernel<double><<<grd, blk, 0, h->stream>>>(h->scratch(0), c.nx, c.ny, bx[k], by[k], bw[k],
                                                                 disc, cx, cy, win[k].c, h->partials());
        finalize_kernel<<<1, 256, 0, h->stream>>>(h->partials(), (int64_t)grd.x * grd.y, 0.0, res);
        s = h->cuda(cudaGetLastError(), "window sums");
        if (s == LB_OK)
            s = h->cuda(cudaMemcpyAsync(out.data(), res, 5 * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
                        "copy window sums");
        if (s == LB_OK) s = h->cuda(cudaStreamSynchronize(h->stream), "window sync");
        if (s == LB_OK) mean[k] = out[4] > 0 ? out[0] / out[4] : std::nan("");
    }
    return s;
}

lb_status lb_wait_selftest(lb_handle* h)
{
    if (check_handle(h) != LB_OK) return LB_E_INVALID;
    wait_selftest_kernel<<<1, 32, 0, h->stream>>>(h->status());
    return h->cuda(cudaGetLastError(), "wait self-test");
}

lb_status lb_snapshot_bytes(const lb_handle* h, int32_t case_id, size_t* bytes)
{
    if (!h || !bytes || case_id < 0 || case_id >= (int)h->cases.size()) return LB_E_INVALID;
    const lb_case& c = h->cases[case_id];
    const size_t es = h->prec == LB_FP32 ? 4 : 8;
    *bytes = 16 + (size_t)kQ * c.ny * pitch_of(c.nx) * es;
    return LB_OK;
}

lb_status lb_save(lb_handle* h, int32_t case_id, void* host_buf, size_t bytes)
{
    size_t need = 0;
    if (lb_snapshot_bytes(h, case_id, &need) != LB_OK || !host_buf || bytes < need) {
        if (h) h->err = "lb_save: bad arguments";
        return LB_E_INVALID;
    }
    if (!h->inited[case_id]) return h->fail(LB_E_STATE, "lb_save: case not initialised");
    const size_t es = h->prec == LB_FP32 ? 4 : 8;
    uint8_t* p = (uint8_t*)host_buf;
    int64_t st = h->steps[case_id];
    memcpy(p, &st, 8);
    memcpy(p + 8, &h->rho_ref[case_id], 8);
    lb_status s = h->cuda(cudaMemcpyAsync(p + 16, (uint8_t*)h->fbuf(h->cur) + h->L.off[case_id] * es, need - 16,
                                          cudaMemcpyDeviceToHost, h->stream),
                          "save");
    if (s == LB_OK) s = h->cuda(cudaStreamSynchronize(h->stream), "save sync");
    return s;
}

lb_status lb_load(lb_handle* h, int32_t case_id, const void* host_buf, size_t bytes)
{
    size_t need = 0;
    if (lb_snapshot_bytes(h, case_id, &need) != LB_OK || !host_buf || bytes < need) {
        if (h) h->err = "lb_load: bad arguments";
        return LB_E_INVALID;
    }
    const size_t es = h->prec == LB_FP32 ? 4 : 8;
    const uint8_t* p = (const uint8_t*)host_buf;
    int64_t st;
    double rr;
    memcpy(&st, p, 8);
    memcpy(&rr, p + 8, 8);
    if (st < 0 || !std::isfinite(rr) || rr < 0) return h->fail(LB_E_INVALID, "lb_load: corrupt snapshot header");
    h->rho_ref[case_id] = h->prec == LB_FP32 ? rr : 0.0;
    h->steps[case_id] = st;  // before the case table is uploaded (Lax-Wendroff step-0 flag)
    lb_status s = h->upload_case(case_id);
    if (s == LB_OK)
        s = h->cuda(cudaMemcpyAsync((uint8_t*)h->fbuf(h->cur) + h->L.off[case_id] * es, p + 16, need - 16,
                                    cudaMemcpyHostToDevice, h->stream),
                    "load");
    if (s == LB_OK)
        s = h->cuda(cudaMemsetAsync(h->status() + 1 + case_id, 0, sizeof(int), h->stream), "clear case flag");
    if (s == LB_OK) s = h->cuda(cudaStreamSynchronize(h->stream), "load sync");
    if (s != LB_OK) return s;
    h->steps[case_id] = st;
    h->inited[case_id] = 1;
    return stats_restart(h, case_id);
}

}  // extern "C"

// ------------------------------------------------------------------ adjoint
namespace {

struct AdjLayout {
    size_t cases, items, ckpt, seg, lam, lamd, fields, partials, partials2, acc, rho0, sfin, grad, status, total;
    int64_t K, ncp, state, nitems, N, parts;
};

constexpr int kAdjFields = 29;

// es: bytes of the handle's arithmetic type (states, adjoint populations and
// fields); rho0, s_final and the density gradient stay FP64.
AdjLayout adj_layout(const lb_case& c, int64_t nsteps, int64_t K, size_t es)
{
    AdjLayout L;
    L.K = K;
    L.ncp = nsteps / K + 1;
    L.N = (int64_t)c.nx * c.ny;
    L.state = (int64_t)kQ * c.ny * pitch_of(c.nx);
    L.nitems = max_items_of(c);
    L.parts = (int64_t)((c.nx + 255) / 256) * c.ny;
    size_t p = 0;
    auto take = [&](size_t bytes) {
        const size_t at = p;
        p = align_up(p + bytes, kAlign);
        return at;
    };
    L.cases = take(sizeof(DevCase<double>));
    L.items = take(L.nitems * sizeof(Item));
    L.ckpt = take((size_t)L.ncp * L.state * es);
    L.seg = take((size_t)(K + 1) * L.state * es);
    L.lam = take((size_t)kQ * L.N * es);
    L.lamd = take((size_t)kQ * L.N * es);
    L.fields = take((size_t)kAdjFields * align_up(L.N * es, kAlign));
    L.partials = take(L.parts * sizeof(Partial));
    L.partials2 = take(L.parts * sizeof(Partial));
    L.acc = take(8 * sizeof(double));
    L.rho0 = take(L.N * sizeof(double));
    L.sfin = take(L.N * sizeof(double));
    L.grad = take(L.N * sizeof(double));
    L.status = take(2 * sizeof(int));  // step-kernel status words of the one-case work-list
    L.total = p;
    return L;
}

int64_t adj_default_K(int64_t nsteps)
{
    int64_t K = 1;
    while (K * K < nsteps) ++K;
    return K;
}

// T: the handle's arithmetic type. FP32 runs the forward and the recompute
// with the FP32 step kernel (plain loads, deviation storage about rho_ref)
// and the reverse sweep in FP32; the loss and the kappa / T partials are
// summed in FP64 either way.
template <typename T, int SCHEME, int EOS>
lb_status adjoint_run(lb_handle* h, const lb_case& c, const AdjLayout& L, uint8_t* ws, const double* s_fin,
                      int64_t nsteps, int64_t u_from, double rho_ref)
{
    cudaStream_t st = h->stream;
    const DevCase<T> cd = dev_case<T>(c, 0, rho_ref);
    const DevCase<T>* dcase = reinterpret_cast<const DevCase<T>*>(ws + L.cases);
    const Item* items = reinterpret_cast<const Item*>(ws + L.items);
    int* status = reinterpret_cast<int*>(ws + L.status);
    T* ckpt = reinterpret_cast<T*>(ws + L.ckpt);
    T* seg = reinterpret_cast<T*>(ws + L.seg);
    T* lam = reinterpret_cast<T*>(ws + L.lam);
    T* lamd = reinterpret_cast<T*>(ws + L.lamd);
    // per-block slots that accumulate over the whole reverse sweep: the loss
    // (parts) and the kappa / T gradients (parts2); folded once at the end
    Partial* parts = reinterpret_cast<Partial*>(ws + L.partials);
    Partial* parts2 = reinterpret_cast<Partial*>(ws + L.partials2);
    double* acc = reinterpret_cast<double*>(ws + L.acc);
    const double* rho0 = reinterpret_cast<const double*>(ws + L.rho0);
    double* grad = reinterpret_cast<double*>(ws + L.grad);
    AdjFields<T> F;
    T** fp = reinterpret_cast<T**>(&F);
    for (int k = 0; k < kAdjFields; ++k)
        fp[k] = reinterpret_cast<T*>(ws + L.fields + k * align_up(L.N * sizeof(T), kAlign));
    const dim3 blk(256), grd((c.nx + 255) / 256, c.ny);  // the adj_* kernels: one node per thread
    const dim3 fgrd = field_grid(c.nx, c.ny);             // the field kernels of aux_kernels.cuh
    const int nitems = (int)L.nitems;
    const T R = (T)c.R;
    auto state = [&](int64_t k) { return ckpt + k * L.state; };
    auto step = [&](const T* in, T* out) {
        if constexpr (sizeof(T) == 4)
            return launch_step_f32(SCHEME, c.collision, EOS, false, false, kStepThreads, nitems, st, in, out, dcase,
                                   items, status);
        else
            return launch_step_f64(SCHEME, c.collision, EOS, false, nitems, st, in, out, dcase, items, status);
    };
    // rho0 in T (the check partials land in parts and are not used)
    auto load_rho0 = [&]() { rho0_kernel<T><<<fgrd, blk, 0, st>>>(c.nx, c.ny, c.eos, c.b, rho0, F.rho, parts); };
    lb_status cs0 = h->cuda(cudaMemsetAsync(status, 0, 2 * sizeof(int), st), "adjoint status");
    if (cs0 != LB_OK) return cs0;
    // forward: f(0), then the checkpoints every K steps
    load_rho0();
    mu_field_kernel<T, EOS><<<fgrd, blk, 0, st>>>(cd, F.rho, F.mu);
    init_kernel<T, SCHEME, T><<<fgrd, blk, 0, st>>>(cd, cd, F.rho, nullptr, nullptr, F.mu, state(0));
    const T* cur = state(0);
    for (int64_t n = 0; n < nsteps; ++n) {
        T* out = ((n + 1) % L.K == 0) ? state((n + 1) / L.K) : (cur == seg ? seg + L.state : seg);
        if (step(cur, out) != cudaSuccess) return h->cuda(cudaGetLastError(), "adjoint forward");
        cur = out;
    }
    lb_status ms = h->cuda(cudaMemsetAsync(acc, 0, 4 * sizeof(double), st), "adjoint clear");
    if (ms == LB_OK) ms = h->cuda(cudaMemsetAsync(lam, 0, (size_t)kQ * L.N * sizeof(T), st), "adjoint clear");
    if (ms == LB_OK) ms = h->cuda(cudaMemsetAsync(parts, 0, L.parts * sizeof(Partial), st), "adjoint clear");
    if (ms == LB_OK) ms = h->cuda(cudaMemsetAsync(parts2, 0, L.parts * sizeof(Partial), st), "adjoint clear");
    if (ms != LB_OK) return ms;
    // reverse sweep over segments [s, e], states s+1..e rebuilt into seg
    for (int64_t s = (nsteps / L.K) * L.K, e = nsteps; s >= 0; e = s - 1, s -= L.K) {
        for (int64_t n = s + 1; n <= e; ++n) {
            const T* in = n - 1 == s ? state(s / L.K) : seg + (n - 1 - s) * L.state;
            if (step(in, seg + (n - s) * L.state) != cudaSuccess)
                return h->cuda(cudaGetLastError(), "adjoint recompute");
        }
        for (int64_t n = e; n >= s; --n) {
            const T* fn = n == s ? state(s / L.K) : seg + (n - s) * L.state;
            pull_moments_kernel<T, T><<<fgrd, blk, 0, st>>>(cd, fn, F.rho, F.jx, F.jy);
            adj_fwd_mu<T, EOS><<<grd, blk, 0, st>>>(cd, F);
            adj_fwd_force<T, SCHEME><<<grd, blk, 0, st>>>(cd, F, n >= u_from ? 1.0 : 0.0,
                                                          n == nsteps ? s_fin : nullptr, parts);
            if (SCHEME == 1) adj_fwd_corr<T><<<grd, blk, 0, st>>>(cd, F);
            adj_collide<T, SCHEME><<<grd, blk, 0, st>>>(cd, F, lam, n < nsteps, n >= u_from, lamd);
            adj_force<T, SCHEME><<<grd, blk, 0, st>>>(cd, F);
            adj_mu<T, SCHEME, EOS><<<grd, blk, 0, st>>>(cd, R, F, parts2);
            adj_lambda<T><<<grd, blk, 0, st>>>(cd, F, lamd, n == nsteps ? s_fin : nullptr, lam);
        }
        if (s == 0) break;
    }
    // the loss, before load_rho0's check partials overwrite parts
    adj_accumulate<<<1, 256, 0, st>>>(parts, L.parts, acc + 0, nullptr);
    // initial populations
    load_rho0();
    adj_fwd_mu<T, EOS><<<grd, blk, 0, st>>>(cd, F);
    adj_init<T, SCHEME, EOS><<<grd, blk, 0, st>>>(cd, R, F, lam, parts2);
    adj_accumulate<<<1, 256, 0, st>>>(parts2, L.parts, acc + 1, acc + 2);
    adj_init_out<T><<<grd, blk, 0, st>>>(cd, F, grad);
    return h->cuda(cudaGetLastError(), "adjoint kernels");
}

}  // namespace

extern "C" {

lb_status lb_adjoint_workspace_bytes(const lb_handle* h, int32_t case_id, int64_t nsteps, int32_t ckpt_every,
                                     size_t* bytes)
{
    if (!h || !bytes || case_id < 0 || case_id >= (int)h->cases.size() || nsteps < 0 || ckpt_every < 0)
        return LB_E_INVALID;
    const int64_t K = ckpt_every > 0 ? ckpt_every : adj_default_K(nsteps);
    *bytes = adj_layout(h->cases[case_id], nsteps, K, h->prec == LB_FP32 ? sizeof(float) : sizeof(double)).total;
    return LB_OK;
}

lb_status lb_adjoint_step(lb_handle* h, int32_t case_id, const double* rho0, int64_t nsteps, int64_t u_from,
                     const double* s_final, int32_t on_device, int32_t ckpt_every, void* d_ws, size_t ws_bytes,
                     double* loss, double* grad_rho0, double* grad_kappa, double* grad_T)
{
    if (check_handle(h) != LB_OK) return LB_E_INVALID;
    if (case_id < 0 || case_id >= (int)h->cases.size() || !rho0 || nsteps < 0 || u_from < 0 || ckpt_every < 0 ||
        !loss || !grad_kappa || !grad_T)
        return h->fail(LB_E_INVALID, "lb_adjoint_step: bad arguments");
    const lb_case& c = h->cases[case_id];
    if (c.nu > 0) return h->fail(LB_E_INVALID, "lb_adjoint_step: constant relaxation times only (nu = 0)");
    if (c.scheme == LB_STANDARD_PT)
        return h->fail(LB_E_INVALID, "lb_adjoint_step: no adjoint of the pressure-tensor force form");
    if (c.scheme == LB_IMPROVED_SMOOTH || c.scheme == LB_LAX_WENDROFF)
        return h->fail(LB_E_INVALID, "lb_adjoint_step: no adjoint of LB_IMPROVED_SMOOTH or LB_LAX_WENDROFF");
    if (c.walls) return h->fail(LB_E_INVALID, "lb_adjoint_step: periodic lattices only (no walls)");
    const int64_t K = ckpt_every > 0 ? ckpt_every : adj_default_K(nsteps);
    const bool f32 = h->prec == LB_FP32;
    const AdjLayout L = adj_layout(c, nsteps, K, f32 ? sizeof(float) : sizeof(double));
    if (!d_ws || ((uintptr_t)d_ws % kAlign) != 0 || ws_bytes < L.total)
        return h->fail(LB_E_WORKSPACE, "lb_adjoint_step: workspace misaligned or smaller than lb_adjoint_workspace_bytes");
    uint8_t* ws = static_cast<uint8_t*>(d_ws);
    cudaStream_t st = h->stream;
    // one-case step tables at offset 0 of the workspace's state buffers
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    std::vector<Item> items;
    {
        const int ns = strips_of(c, kStepThreads);
        int nseg = std::max(1, std::min(c.ny / kMinRows, (2 * sms) / ns));
        for (int k = 0; k < ns; ++k) {
            const int q = c.nx % 4 == 0 ? 4 : 1;
            const int x0 = q * (int)((int64_t)(c.nx / q) * k / ns), x1 = q * (int)((int64_t)(c.nx / q) * (k + 1) / ns);
            for (int g = 0; g < nseg; ++g) {
                const int y0 = (int)((int64_t)c.ny * g / nseg), y1 = (int)((int64_t)c.ny * (g + 1) / nseg);
                items.push_back(Item{0, x0, x1 - x0, y0, y1 - y0, 0});
            }
        }
    }
    AdjLayout Lr = L;
    Lr.nitems = (int64_t)items.size();
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    lb_status s = h->cuda(cudaMemcpyAsync(ws + L.items, items.data(), items.size() * sizeof(Item),
                                          cudaMemcpyHostToDevice, st),
                          "adjoint items");
    if (s == LB_OK) s = h->cuda(cudaMemcpyAsync(ws + L.rho0, rho0, L.N * sizeof(double), kind, st), "adjoint rho0");
    const double* sfin = nullptr;
    if (s == LB_OK && s_final) {
        s = h->cuda(cudaMemcpyAsync(ws + L.sfin, s_final, L.N * sizeof(double), kind, st), "adjoint s_final");
        sfin = reinterpret_cast<const double*>(ws + L.sfin);
    }
    if (s != LB_OK) return s;
    // validate rho0 on the device (its sum gives the FP32 deviation reference)
    double rho_ref = 0.0;
    {
        Partial* parts = reinterpret_cast<Partial*>(ws + L.partials);
        double* acc = reinterpret_cast<double*>(ws + L.acc);
        double* scratch = reinterpret_cast<double*>(ws + L.grad);
        const dim3 blk(256), grd = field_grid(c.nx, c.ny);
        rho0_kernel<double><<<grd, blk, 0, st>>>(c.nx, c.ny, c.eos, c.b,
                                                 reinterpret_cast<const double*>(ws + L.rho0), scratch, parts);
        finalize_kernel<<<1, 256, 0, st>>>(parts, (int64_t)grd.x * grd.y, 0.0, acc);
        double chk[5];
        s = h->cuda(cudaMemcpyAsync(chk, acc, sizeof chk, cudaMemcpyDeviceToHost, st), "adjoint check");
        if (s == LB_OK) s = h->cuda(cudaStreamSynchronize(st), "adjoint check");
        if (s != LB_OK) return s;
        if (chk[4] != 0.0) return h->fail(LB_E_INVALID, "lb_adjoint_step: rho0 must be finite, > 0 and inside the EOS domain");
        rho_ref = c.rho_ref > 0 ? c.rho_ref : chk[0] / (double)L.N;  // FP32 deviation reference
    }
    // the one-case parameter record in the handle's type
    if (f32) {
        const DevCase<float> cd = dev_case<float>(c, 0, rho_ref);
        s = h->cuda(cudaMemcpyAsync(ws + L.cases, &cd, sizeof cd, cudaMemcpyHostToDevice, st), "adjoint case");
    } else {
        const DevCase<double> cd = dev_case<double>(c, 0, 0.0);
        s = h->cuda(cudaMemcpyAsync(ws + L.cases, &cd, sizeof cd, cudaMemcpyHostToDevice, st), "adjoint case");
    }
    if (s != LB_OK) return s;
#define LBFE_ADJ(T, S, E) adjoint_run<T, S, E>(h, c, Lr, ws, sfin, nsteps, u_from, f32 ? rho_ref : 0.0)
    if (c.scheme == LB_IMPROVED)
        s = f32 ? (c.eos == LB_VDW ? LBFE_ADJ(float, 1, 0) : LBFE_ADJ(float, 1, 1))
                : (c.eos == LB_VDW ? LBFE_ADJ(double, 1, 0) : LBFE_ADJ(double, 1, 1));
    else
        s = f32 ? (c.eos == LB_VDW ? LBFE_ADJ(float, 0, 0) : LBFE_ADJ(float, 0, 1))
                : (c.eos == LB_VDW ? LBFE_ADJ(double, 0, 0) : LBFE_ADJ(double, 0, 1));
#undef LBFE_ADJ
    if (s != LB_OK) return s;
    double acc[4];
    int stw[2] = {0, 0};
    s = h->cuda(cudaMemcpyAsync(acc, ws + L.acc, sizeof acc, cudaMemcpyDeviceToHost, st), "adjoint results");
    if (s == LB_OK)
        s = h->cuda(cudaMemcpyAsync(stw, ws + L.status, sizeof stw, cudaMemcpyDeviceToHost, st), "adjoint status");
    if (s == LB_OK && grad_rho0)
        s = h->cuda(cudaMemcpyAsync(grad_rho0, ws + L.grad, L.N * sizeof(double),
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st),
                    "adjoint grad");
    if (s == LB_OK) s = h->cuda(cudaStreamSynchronize(st), "adjoint sync");
    if (s != LB_OK) return s;
    *loss = acc[0];
    *grad_kappa = acc[1];
    *grad_T = acc[2];
    if (stw[0]) return h->fail(LB_E_TIMEOUT, "lb_adjoint_step: a bounded wait of a step kernel gave up");
    if (stw[1] || !std::isfinite(acc[0]) || !std::isfinite(acc[1]) || !std::isfinite(acc[2]))
        return h->fail(LB_E_UNSTABLE, "lb_adjoint_step: unstable forward run, or non-finite loss or gradient");
    return LB_OK;
}

const char* lb_last_error(const lb_handle* h) { return h ? h->err.c_str() : "null handle"; }

void lb_destroy(lb_handle* h)
{
    if (!h) return;
    for (cudaGraphExec_t& g : h->graph)
        if (g) cudaGraphExecDestroy(g);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (cudaStream_t a : h->aux) cudaStreamDestroy(a);
    for (cudaEvent_t e : h->fork_join) cudaEventDestroy(e);
    delete h;
}

}  // extern "C"
