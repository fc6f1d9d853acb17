/*
 * lbfe.h - C ABI of the GB300 (sm_103a) forcing-based free-energy D2Q9
 * lattice Boltzmann library (Li, Yu & Huang, "Achieving thermodynamic
 * consistency in a class of free-energy multiphase lattice Boltzmann models").
 *
 * One time step of one periodic case is, per node:
 *   rho = sum_a f_a, rho u = sum_a e_a f_a + F/2                 (Eq. 12)
 *   mu_c = E_f'(rho) - kappa lap(rho)                            (Eq. 2; vdW Eq. 30)
 *   F = grad_h(rho/3) - rho grad_h mu_c   (standard scheme,       Eq. 13 right)
 *   F = (1/3 - rho) grad_h mu_c           (improved scheme,       Eq. 24)
 *   grad_h = isotropic gradient                                  (Eq. 17)
 *   m* = m - Lambda (m - m_eq) + (I - Lambda/2)(S + C)           (Eqs. 9, 28)
 *   m_eq from Eq. 11 (standard) or Eq. 27 (improved), S = M G with G of Eq. 14,
 *   C = (0, 9 C1, 0, 0, 0, 0, 0, 3 C7, 0) of Eq. 29 (improved only),
 *   Lambda from Eq. 8 (MRT) or 1/tau_v on every moment (BGK),
 *   f* = M^-1 m*, streamed f_a(x + e_a, t + 1) = f*_a(x, t)      (Eq. 10).
 * M is the Lallemand-Luo D2Q9 matrix, moments ordered (rho, e, eps, j_x, q_x,
 * j_y, q_y, p_xx, p_xy); velocities e0=(0,0), e1=(1,0), e2=(0,1), e3=(-1,0),
 * e4=(0,-1), e5=(1,1), e6=(-1,1), e7=(-1,-1), e8=(1,-1).
 *
 * Conventions for every entry point:
 *  - Ownership: the caller allocates the device workspace (size from
 *    lb_workspace_bytes) and every input/output buffer, and frees them after
 *    lb_destroy. The library allocates host memory only (handle, tables,
 *    captured graphs) and never frees caller memory.
 *  - Streams: all device work is enqueued on the stream given to lb_create
 *    (a cudaStream_t passed as void*; NULL = legacy default stream). Calls
 *    that return data to host memory synchronise that stream before
 *    returning.
 *  - Fields: FP64, row-major [ny][nx], x fastest. A pointer flagged
 *    on_device = 1 is a device address, otherwise a host address.
 *  - Errors: every call returns an lb_status; nothing throws, exits or traps.
 *    lb_last_error() gives a one-line description of the handle's last failure.
 *  - A handle is not thread-safe; separate handles are independent.
 */
#ifndef LBFE_H
#define LBFE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LB_OK = 0,
    LB_E_INVALID = 1,   /* bad argument or parameter set (nothing was enqueued) */
    LB_E_CUDA = 2,      /* a CUDA runtime call failed; see lb_last_error */
    LB_E_UNSTABLE = 3,  /* a case produced rho <= 0 or a non-finite value */
    LB_E_TIMEOUT = 4,   /* a bounded device-side wait gave up (see lb_wait_selftest) */
    LB_E_WORKSPACE = 5, /* workspace pointer misaligned or too small */
    LB_E_STATE = 6      /* call out of order (e.g. step before init) */
} lb_status;

/* LB_STANDARD: standard scheme, chemical-potential force (Eq. 13 right);
 * LB_IMPROVED: the improved scheme (Eqs. 24-29), the derivatives of Eq. 29
 * by the Eq. 17 gradient of phi u_x and phi u_y; LB_STANDARD_PT: standard
 * scheme with the pressure-tensor force F = grad(rho c_s^2) - div P (Eq. 13
 * left), P of Eqs. 4-5 built from the Eq. 17 gradient and the isotropic
 * Laplacian of rho, div P by Eq. 17 on each component.
 * LB_IMPROVED_SMOOTH: the improved scheme with Eq. 29's derivatives taken as
 * the Eq. 17 gradient of the lattice-weight average sum_a w_a (phi u)(x + e_a)
 * (a 5 x 5 stencil). The paper does not state its discretisation of these
 * derivatives (Sec. III). With the plain Eq. 17 difference the improved
 * scheme's vapour is linearly unstable at 0.7 T_c (vdW set of Sec. IV, any
 * relaxation times); the averaged form damps the grid-scale modes that drive
 * that instability and keeps 0.7 T_c stable for tau_v >= 0.8, or with MRT at
 * the constant kinematic viscosity 0.04 of Table II. Same steady states as
 * LB_IMPROVED (C vanishes at u = 0). FP32 cases with nx % 4 == 0 and
 * nx >= 8 run on the packed kernel (its stage D reads the row's pull a
 * second time, from a shared-memory ring that bulk copies fill out of L2),
 * the others on the one-column plain-load kernel;
 * no lb_adjoint_step. */
/* LB_LAX_WENDROFF: the comparison scheme of Appendix A (Lou and Guo's
 * Lax-Wendroff propagation): the standard force (Eq. 13 right), velocity
 * u = (sum_a e_a f_a + A F / 2) / rho, the BGK collision of Eq. A1 (rate
 * 1 / tau_v, source A (1 - 1/(2 tau_v)) G of Eq. 14) with the equilibrium of
 * Eq. A3 and its tensor T of Eq. A4, and the three-point propagation of
 * Eq. A2, a_0 = 1 - A^2, a_1 = A (A - 1)/2, a_-1 = A (A + 1)/2, over a time
 * step A (lw_A, the CFL number; lw_B is B of Eq. A3, kinematic viscosity
 * c_s^2 (tau_v - 1/2 - B) A). A step advances time by A, so it takes 1/A
 * steps per unit of the other schemes' time. BGK only, periodic, nu = 0; the
 * one-column kernel; no adjoint and no lb_fields_static. Storage: at step 0
 * the populations are f(0) (pre-collision, unshifted), after that the
 * post-collision values before Eq. A2's propagation. */
enum { LB_STANDARD = 0, LB_IMPROVED = 1, LB_STANDARD_PT = 2, LB_IMPROVED_SMOOTH = 3, LB_LAX_WENDROFF = 4 };
enum { LB_BGK = 0, LB_MRT = 1 };            /* single rate 1/tau_v / Eq. 8 */
enum { LB_VDW = 0, LB_CS = 1 };             /* Eq. 30 / Carnahan-Starling */
enum { LB_FP64 = 0, LB_FP32 = 1 };          /* population storage and arithmetic */

/* One independent periodic case. Eq. 30 (vdW):
 *   E_f = rho R T ln[rho/(1 - b rho)] - a rho^2;
 * Carnahan-Starling (not in the paper):
 *   E_f = R T rho ln rho + R T rho (4n - 3n^2)/(1 - n)^2 - a rho^2, n = b rho/4.
 * tau_e, tau_s, tau_q are the free MRT times of Eq. 8 (tau_c = 1); BGK uses
 * tau_v alone. nu > 0 selects constant kinematic viscosity: tau_v at each
 * node follows from eta = nu rho with eta = p_m (tau_v - 1/2) (improved,
 * below Eq. 29) or rho c_s^2 (tau_v - 1/2) (standard, below Eq. 8).
 * p_m = (pm_c0 + mu_c)/3 (Eq. 24 uses pm_c0 = 1). rho_ref is the reference
 * density of FP32 storage (populations are stored as f_a - w_a rho_ref);
 * rho_ref = 0 asks lb_init_fields to use the mean of the initial density.
 *
 * walls = 1 (Sec. IV C: a droplet carried between moving plates): periodic in
 * x, no-slip walls half a node below y = 0 and above y = ny - 1, both moving
 * at (wall_u, 0). A population that streams into a wall returns to its node
 * in the opposite direction (halfway bounce-back) plus the difference of the
 * running scheme's equilibria in the two directions at the wall state
 * (rho_wall, velocity (wall_u, 0), mu_c = E_f'(rho_wall)). The stencils
 * (Laplacian, Eq. 17 gradients) see the lattice continued across each wall
 * by its mirror image: ghost row -k holds row k - 1 reflected in the wall
 * (the same density and j_x, j_y with its sign changed) and every field is
 * computed there by the same formulas, so that scalar fields continue evenly
 * and the y components of vector fields oddly. The wall term carries momentum in proportion
 * to the wall state's pressure (rho_wall / 3, or p_m of Eq. 24), so rho_wall
 * is the density of the fluid that touches the walls (rho_g for a droplet in
 * its vapour): another value drives that fluid at wall_u times the ratio of
 * the two pressures. Needs ny >= 8. FP32 cases with nx % 4 == 0 (and
 * nx >= 8 for LB_IMPROVED_SMOOTH) run on the packed kernel, whose row rings
 * hold the ghost rows with their planes reflected; the others on the
 * one-column step kernel. No adjoint and no lb_fields_static. */
typedef struct {
    int32_t nx, ny;      /* >= 3 each */
    int32_t scheme;      /* LB_STANDARD, LB_IMPROVED, LB_STANDARD_PT, LB_IMPROVED_SMOOTH or LB_LAX_WENDROFF */
    int32_t collision;   /* LB_BGK or LB_MRT */
    int32_t eos;         /* LB_VDW or LB_CS */
    int32_t walls;       /* 0: periodic in y; 1: moving no-slip walls (below) */
    double a, b, R, T;   /* EOS parameters; T absolute */
    double kappa;        /* > 0, Eq. 1 */
    double tau_v, tau_e, tau_s, tau_q; /* each > 1/2 */
    double pm_c0;        /* Eq. 24 constant */
    double nu;           /* 0 or > 0 */
    double rho_ref;      /* FP32 storage reference, >= 0 */
    double wall_u;       /* walls: x velocity of both walls, |wall_u| <= 0.3 */
    double rho_wall;     /* walls: density of the wall state, > 0 */
    double lw_A;         /* LB_LAX_WENDROFF: CFL number A, 0 < A <= 1 (unused otherwise) */
    double lw_B;         /* LB_LAX_WENDROFF: B of Eq. A3, B < tau_v - 1/2 (unused otherwise) */
} lb_case;

typedef struct lb_handle lb_handle;

/* Bytes of device workspace that lb_create needs for these cases at this
 * precision (LB_FP64 or LB_FP32). The workspace must be 256-byte aligned. */
lb_status lb_workspace_bytes(const lb_case* cases, int32_t ncases, int32_t precision,
                             size_t* bytes);

/* Validate the cases, lay the workspace out and build the launch work-lists.
 * d_workspace: device memory of at least lb_workspace_bytes bytes, owned by
 * the caller and not touched by anyone else until lb_destroy. cuda_stream:
 * cudaStream_t (void*). On LB_OK *out holds a new handle.
 * Kernel selection (results are bit-identical either way): FP32 groups whose
 * lattices all have nx % 4 == 0 use the TMA-staged step kernel, others the
 * plain-load one. Environment overrides read here, for tuning:
 * LBFE_STEP_PATH=ldg forces the plain-load kernel; LBFE_STEP_THREADS=128|256
 * sets the compute threads per block of the TMA kernel (default 128);
 * LBFE_ROWS=0 keeps short periodic lattices off the row kernel (lb_step). */
lb_status lb_create(const lb_case* cases, int32_t ncases, int32_t precision, void* d_workspace,
                    size_t ws_bytes, void* cuda_stream, lb_handle** out);

/* Set case case_id to f(0) = M^-1 m_eq(rho0, u0) of its scheme, with mu_c of
 * Eq. 2 evaluated on rho0 (the paper gives no initialisation rule).
 * rho0 [ny][nx] must be > 0; ux0/uy0 may be NULL (fluid at rest). Pointers
 * are device addresses if on_device, else host (copied synchronously;
 * page-locked host memory, as from cudaHostAlloc, is read by the first init
 * kernel directly over the host link). */
lb_status lb_init_fields(lb_handle* h, int32_t case_id, const double* rho0, const double* ux0,
                         const double* uy0, int32_t on_device);
/* The same with FP32 fields: the state equals lb_init_fields' from the same
 * values widened to FP64 (rho0 is checked and summed in FP64 all the same).
 * For FP32 handles, whose per-node arithmetic is FP32 anyway (the precision
 * pattern keeps FP64 for the global sums only), it halves the bytes that
 * cross the host link. */
lb_status lb_init_fields_f32(lb_handle* h, int32_t case_id, const float* rho0, const float* ux0,
                             const float* uy0, int32_t on_device);

/* Advance every case by nsteps time steps (Eqs. 9-14, 24-29, pull form of
 * Eq. 10): one fused kernel launch per step and per group of cases that
 * share scheme, collision, EOS, viscosity mode, nx % 4 == 0 and walls; each launch
 * runs a work-list of (case, column strip, row segment) items. FP32 cases
 * with nx % 4 == 0 run the packed two-column kernel fed by bulk copies;
 * FP64 cases, other widths, Lax-Wendroff cases and LB_IMPROVED_SMOOTH cases
 * narrower than 8 run the one-column plain-load kernel.
 * Periodic cases with ny <= 16 (every scheme but LB_LAX_WENDROFF), in
 * either precision, run the row kernel instead (one thread per node of a
 * whole-height strip of 64 columns, 56, 58 or 60 of them output, the stages
 * separated by block barriers), except under the persistent launch: on
 * lattices that short the sliding-window kernels are bound by the latency
 * of their chain of row iterations. Its results agree with the other
 * kernels' to rounding (FP64: the oracle's 1e-11; FP32: the storage's
 * rounding), and are bit-identical between runs. The
 * first
 * call with nsteps > 0 autotunes the work-list: it times one step under
 * several row-segment sizes, with and without narrow blocks for the lattices
 * that fit them better, and keeps the fastest (these trial launches read
 * the current populations and write only the buffer the next step
 * overwrites, so the state and every result are unchanged; the choice
 * affects speed only). LBFE_SEG_ROWS=n before lb_create fixes the segment
 * size instead (0: a share of the GPU's block slots per case; -1: the same
 * share, filled with up to four narrower strips per case), and
 * LBFE_PAIR_NARROW=0|1 the narrow-block choice. Groups run as parallel
 * branches that fork from and join the handle's stream. Runs of 8
 * steps replay a CUDA graph captured on the first such call (on a private
 * stream, then launched on the handle's stream; set LBFE_GRAPH=0 before
 * lb_create to launch every step directly). Enqueued asynchronously, except
 * that the autotuning call synchronises the stream.
 * Instability: a step kernel that meets a node with rho <= 0 or a
 * non-finite density flags the case on the device; from the next launch on
 * the case's blocks return at once, so it stops advancing (its buffers keep
 * its last two states) while the other cases of the handle go on, with no
 * host round trip. lb_reductions reports the case as LB_E_UNSTABLE until
 * lb_init_fields or lb_load gives it a new state. */
lb_status lb_step(lb_handle* h, int64_t nsteps);

/* Persistent multi-step launch. For a handle whose cases all share one
 * kernel group (same scheme, collision, EOS and viscosity mode), lb_step can
 * run n steps as cooperative launches of a persistent kernel (up to 1024
 * steps each) instead of one launch per step: the blocks stay resident,
 * each owning items of the work-list, and an item's step waits (bounded)
 * until the neighbouring items have completed the step before. It serves
 * lattices small enough to live in L2, where one launch per step is bound
 * by launch latency. The persistent kernel is the one-column kernel.
 * mode: 0 never; 1 always (an FP32 group with nx % 4 == 0 then leaves the
 * packed kernel for the one-column one, whose FP32 rounding differs in the
 * last bits; cases of the row kernel leave it too: entering or leaving mode
 * 1 rebuilds the work-list, synchronising the stream); 2 (default) automatic: for a handle whose group already runs
 * the one-column kernel (FP64; FP32 with nx % 4 != 0, Lax-Wendroff or
 * LB_IMPROVED_SMOOTH with walls or narrower than 8), the first lb_step of at least 40 steps times 16 steps
 * of graph replay against 16 persistent steps (its own steps: results are
 * identical either way) and keeps the faster; -1 leaves the mode unchanged.
 * *persistent (may be NULL) tells whether the persistent launch is in use.
 * A wait that gives up (about one second) sets the status word that
 * lb_reductions reports as LB_E_TIMEOUT, and the launch returns. */
lb_status lb_launch_mode(lb_handle* h, int32_t mode, int32_t* persistent);

/* Failure-detection self-test of the persistent launch (the paper has no
 * counterpart): runs nsteps (2 .. 1024) persistent steps in which work item
 * 0 never publishes its progress and every wait gives up after about 10 ms
 * of SM clock. The first block that waits for item 0 gives up and sets the
 * launch's abort word, every other waiting block returns, and the next
 * lb_reductions reports LB_E_TIMEOUT. The handle's populations are then
 * unreliable (reinitialise them); the GPU context stays usable. Needs a
 * one-group handle whose work-list has at least two items. */
lb_status lb_persistent_selftest(lb_handle* h, int64_t nsteps);

/* The work-list in use: rows per segment (0: slot-share rule over one wave
 * of blocks, -1: the filled slot-share rule, -2 / -3: the slot-share rule
 * over two / four waves), item count,
 * and whether narrow blocks (64 threads, 128 columns) run the lattices that
 * fit them with fewer idle lanes. Before the first lb_step it is the untuned
 * default. Any pointer may be NULL. */
lb_status lb_worklist(const lb_handle* h, int32_t* seg_rows, int64_t* n_items, int32_t* narrow);

/* Macroscopic fields of case case_id at the current step: rho and u of
 * Eq. 12 (u includes the F/2 shift) and mu_c of Eq. 2, computed per node in
 * the storage precision and returned as FP64; any output may be NULL.
 * Device outputs if on_device, else host (stream synchronised; the export
 * kernel writes page-locked host outputs, as from cudaHostAlloc, directly
 * over the host link, pageable ones are staged in the workspace). */
lb_status lb_moments(lb_handle* h, int32_t case_id, double* rho, double* ux, double* uy,
                     double* mu, int32_t on_device);
/* The same with FP32 outputs: each value is lb_moments' rounded to FP32 (for
 * FP32 handles the exact per-node FP32 value), at half the bytes. */
lb_status lb_moments_f32(lb_handle* h, int32_t case_id, float* rho, float* ux, float* uy, float* mu,
                         int32_t on_device);

/* Reductions of every case's current state, FP64 sums in a fixed order:
 * out[5*c + {0,1,2,3,4}] = {mass sum rho, kinetic energy sum rho|u|^2/2,
 * max |u|, step count, 0} with rho, u of Eq. 12; case_status[c] = LB_OK or
 * LB_E_UNSTABLE (rho <= 0 or a non-finite value at some node now, or the
 * case was flagged by a step kernel and frozen, see lb_step). Host
 * pointers (case_status may be NULL); synchronises the stream. Returns
 * LB_E_UNSTABLE if any case is unstable; every entry is still written. */
lb_status lb_reductions(lb_handle* h, double* out, int32_t* case_status);

/* Per-step statistics fused into the step kernels: the mass and kinetic
 * energy of the macroscopic fields of Eq. 12, recorded every step instead of
 * on demand. With a buffer attached, each step of lb_step records, for
 * every case, the state the step starts from (the fields lb_moments would
 * return just before it): {mass sum rho, kinetic energy sum rho|u|^2/2,
 * max |u|, node count}. Stage D of the step kernels sums rho - rho_ref and
 * rho|u|^2 per thread in the storage precision (FP32 for FP32 handles, over
 * at most one work item's rows); each block reduces its sums in FP64 with
 * warp shuffles and adds them to the case's entry with FP64 atomics, and
 * the case's last block advances a ring of `history` entries. The sums
 * agree with lb_reductions to FP64 rounding for FP64 handles and to about
 * 1e-6 relative for FP32 ones. The order of the atomics is not fixed, so
 * the last bits can differ between runs. While a buffer is attached,
 * lb_step does not use the persistent launch and the autotuner's trial
 * launches record nothing. lb_init_fields and lb_load restart a case's
 * record at its new state. A case frozen by the instability flag (lb_step)
 * stops recording.
 *
 * lb_step_stats_bytes: device bytes of a buffer with `history` entries per
 *   case (1 <= history <= 2^20).
 * lb_step_stats_attach: attach a caller-owned device buffer of at least that
 *   size, 16-byte aligned. It is cleared here and never freed by the
 *   library. d_buf NULL detaches. Recording starts at each case's current
 *   state.
 * lb_step_stats_range: the recorded states of case_id still held in the
 *   ring: [*first_state, *first_state + *count). Synchronises the stream;
 *   LB_E_STATE without a buffer.
 * lb_step_stats_read: out[4*k + {0,1,2,3}] for state first_state + k,
 *   0 <= k < count, all inside that range (else LB_E_INVALID). Host output;
 *   synchronises the stream. */
lb_status lb_step_stats_bytes(const lb_handle* h, int32_t history, size_t* bytes);
lb_status lb_step_stats_attach(lb_handle* h, void* d_buf, size_t bytes, int32_t history);
lb_status lb_step_stats_range(lb_handle* h, int32_t case_id, int64_t* first_state, int64_t* count);
lb_status lb_step_stats_read(lb_handle* h, int32_t case_id, int64_t first_state, int32_t count, double* out);

/* Coexistence-density averages (the rho_g / rho_l measurements of Sec. IV):
 * the mean of rho (Eq. 12) at the current step over each of nwin windows of
 * case case_id, with the node values in the storage precision and the sums
 * in FP64 on the GPU, in a fixed order. A window is
 *   kind LB_WIN_RECT: nodes x0 <= x < x0 + w, y0 <= y < y0 + h, indices
 *     taken modulo nx, ny (a = x0, b = y0, c = w, d = h; 1 <= w <= nx,
 *     1 <= h <= ny), or
 *   kind LB_WIN_DISC: nodes whose periodic distance to (a, b) is below c
 *     (0 < c <= min(nx, ny) / 2; d unused).
 * mean[k] = (sum of rho over window k) / (its node count), NaN for a disc
 * that holds no node. Host outputs; synchronises the handle's stream. */
enum { LB_WIN_RECT = 0, LB_WIN_DISC = 1 };
typedef struct {
    int32_t kind, reserved;
    double a, b, c, d;
} lb_window;
lb_status lb_window_means(lb_handle* h, int32_t case_id, int32_t nwin, const lb_window* win, double* mean);

/* Failure-detection self-test (the paper has no counterpart): enqueues on the
 * handle's stream one kernel whose single thread waits, with the bound of the
 * step kernels' waits (about one second of SM clock), on an mbarrier phase
 * that nothing completes, and then records the give-up in the handle's
 * status word as a step kernel would. The next lb_reductions returns
 * LB_E_TIMEOUT and clears the word. Nothing else is written; the GPU context
 * stays usable. */
lb_status lb_wait_selftest(lb_handle* h);

/* Bytes of one case's snapshot (populations + step counter) for lb_save. */
lb_status lb_snapshot_bytes(const lb_handle* h, int32_t case_id, size_t* bytes);

/* Copy case case_id's populations and step counter to / from host memory
 * (bit-exact resume). host_buf must hold lb_snapshot_bytes bytes. Layout:
 * int64 step counter, double rho_ref, then the stored populations
 * [9][ny][pitch] (pitch = nx rounded up to a multiple of 32) in the storage
 * form of the library: post-collision values before streaming, so that
 * f_a(x) at the current step is element x - e_a of plane a (periodic);
 * FP32 planes hold f_a - w_a rho_ref. */
lb_status lb_save(lb_handle* h, int32_t case_id, void* host_buf, size_t bytes);
lb_status lb_load(lb_handle* h, int32_t case_id, const void* host_buf, size_t bytes);

/* Reverse-mode gradient of a trajectory of case case_id (either precision,
 * constant relaxation times, LB_STANDARD or LB_IMPROVED), the discrete
 * adjoint of the step above, in the handle's precision: an LB_FP32 handle
 * runs the forward pass, the recompute and the reverse sweep in FP32 (the
 * FP32 step kernel; loss and parameter sums in FP64), an LB_FP64 handle all
 * in FP64:
 *   f(0) = M^-1 m_eq(rho0, 0) as lb_init_fields, then nsteps steps;
 *   L = sum_{n = u_from}^{nsteps} sum_x |u^n(x)|^2 + sum_x s_final(x) rho^N(x)
 * (u^n, rho^n of Eq. 12 after n steps; s_final may be NULL). Outputs the loss,
 * dL/drho0 [ny][nx] (may be NULL), dL/dkappa and dL/dT (T absolute). The
 * forward trajectory is recomputed from checkpoints taken every ckpt_every
 * steps (0: about sqrt(nsteps)). d_ws: caller-owned device memory of at least
 * lb_adjoint_workspace_bytes, 256-byte aligned. rho0, s_final and grad_rho0
 * are device pointers if on_device, else host. Runs on the handle's stream,
 * synchronises it, and leaves the handle's own state untouched. It is the
 * reverse-time counterpart of lb_init_fields followed by lb_step(nsteps): one
 * call runs all nsteps adjoint steps, newest first. LB_STANDARD_PT and
 * LB_IMPROVED_SMOOTH cases, walls and nu > 0 give LB_E_INVALID. */
lb_status lb_adjoint_workspace_bytes(const lb_handle* h, int32_t case_id, int64_t nsteps, int32_t ckpt_every,
                                     size_t* bytes);
lb_status lb_adjoint_step(lb_handle* h, int32_t case_id, const double* rho0, int64_t nsteps, int64_t u_from,
                     const double* s_final, int32_t on_device, int32_t ckpt_every, void* d_ws, size_t ws_bytes,
                     double* loss, double* grad_rho0, double* grad_kappa, double* grad_T);

/* Host thermodynamics for set-up (FP64, Newton): critical point and the
 * Maxwell equal-area coexistence densities rho_g < rho_l (Sec. IV A; Table II
 * lists the vdW values). eos = LB_VDW or LB_CS. */
lb_status lb_critical(int32_t eos, double a, double b, double R, double* Tc, double* rho_c);

/* Flat-interface surface tension of the square-gradient free energy (Eq. 1)
 * at coexistence: sigma = integral over rho_g..rho_l of
 * sqrt(2 kappa (E_f(rho) - mu rho + p)), FP64 quadrature. Needs T < T_c. */
lb_status lb_surface_tension(int32_t eos, double a, double b, double R, double T, double kappa, double* sigma);

/* Eq. 32: gas and liquid densities around a circular droplet of radius r
 * from the Young-Laplace pressures p_sat + rho_sat / (rho_l_sat - rho_g_sat)
 * sigma / r inverted on each branch of p_EOS. LB_E_INVALID if T >= T_c or
 * the gas pressure exceeds the gas spinodal (droplet too small). */
lb_status lb_young_laplace(int32_t eos, double a, double b, double R, double T, double sigma, double r,
                           double* rho_g, double* rho_l);
lb_status lb_maxwell(int32_t eos, double a, double b, double R, double T, double* rho_g,
                     double* rho_l);

/* lb_fields_static: the field-export and reduction pass of lb_moments and
 * lb_reductions without any device allocation and without a handle. The
 * paper has no counterpart; this exists for callers that cannot call
 * cudaMalloc or hand the library a workspace: plug-ins running inside an
 * application or framework that owns all device memory through its own
 * pool, and code on paths where an allocation would synchronise the device
 * or is forbidden (real-time loops, restricted embedding environments).
 *
 * Inputs: one case c (nx, ny, scheme, eos, a, b, R, T, kappa, pm_c0 are used)
 * and d_pops, a device array of its populations in the snapshot layout of
 * lb_save ([9][ny][pitch], pitch = nx rounded up to 32, storage form of the
 * library; FP32 planes hold f_a - w_a rho_ref). Outputs (device pointers):
 * (LB_STANDARD, LB_IMPROVED or LB_IMPROVED_SMOOTH cases; LB_STANDARD_PT is
 * rejected with LB_E_INVALID) d_rho, d_ux, d_uy, d_mu [ny][nx] as in lb_moments (each may
 * be NULL) and
 * d_red[5] = {mass, kinetic energy, max |u|, 0, count of nodes with rho <= 0
 * or non-finite values}. Work is enqueued on cuda_stream; nothing is
 * synchronised.
 *
 * Scratch: a fixed device array inside the library, sized for
 * nx, ny <= LB_STATIC_MAX_SIDE and nx * ny <= LB_STATIC_MAX_NODES (about
 * 8.5 MB, held on every GPU that loads the library until the process exits).
 * Larger cases are rejected with LB_E_INVALID before anything is enqueued.
 * The first call on a device looks up the array's device address (a CUDA
 * runtime call); make that first call before any stream capture. Every call
 * on a device shares the one array: calls whose work may overlap on the GPU
 * (different streams without ordering, or concurrent host threads) race and
 * must be serialised by the caller. A CUDA error already pending on the
 * calling thread when the call starts gives LB_E_CUDA with nothing enqueued
 * and the error left in place for its owner. */
#define LB_STATIC_MAX_SIDE 4096
#define LB_STATIC_MAX_NODES 262144
lb_status lb_fields_static(const lb_case* c, int32_t precision, const void* d_pops, double rho_ref,
                           double* d_rho, double* d_ux, double* d_uy, double* d_mu, double* d_red,
                           void* cuda_stream);

const char* lb_last_error(const lb_handle* h);
void lb_destroy(lb_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* LBFE_H */
