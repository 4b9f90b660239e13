/*
 * sbi.h - C ABI of the GB300 (sm_103a) enhanced spectral boundary integral
 * (ESBI) hot path: the surface vertical velocity of a periodic free surface over
 * variable depth, and fixed-step RK4 time stepping of the free-surface
 * equations that use it.
 *
 * Method: Wang, "An enhanced spectral boundary integral method for modeling
 * highly nonlinear water waves in variable depth" (arXiv 2310.19840).
 *   - Governing problem: Laplace equation in -h0+delta(x) <= z <= eta(x) with
 *     the free-surface and impermeable-seabed conditions (Sec. 2.1).
 *   - Prognostic equations: Zakharov form of the kinematic and dynamic surface
 *     conditions, Eq. (prognostic) (Sec. 2.2).
 *   - Diagnostic: V = sum_{l=1..M} V_l by the successive approximation of
 *     Sec. 2.4 (recursions app-V-scs / app-phi-scs, explicit forms in
 *     Appendix C), dealiased by the 2/(l+1) rule (end of Sec. 2.4).
 *   - Energy: Eq. (energy) (Sec. 3.1).  Low-pass filter: Eq. (filter).
 *     Damping pressure: Eq. (pd).
 *
 * Conventions shared by every call:
 *   - A grid is nx x ny points on a periodic Lx x Ly box; ny = 1 is a 1-D
 *     problem (Ly is then a unit width).  nx is a power of two in [16, 4096];
 *     ny is 1 or a power of two in [8, 2048].
 *   - Fields are row-major, index = iy * nx + ix (x fastest), double precision
 *     on the host side of the ABI.  Pointers flagged on_device = 1 are CUDA
 *     device pointers (for example a torch tensor's data_ptr()); otherwise they
 *     are host pointers.
 *   - The library copies every input; callers keep ownership of their buffers.
 *     A context owns all the device memory it allocates and frees it in
 *     sbi_destroy.
 *   - Every int-returning call returns SBI_OK or one of the SBI_E* codes below
 *     and never aborts the process or traps the device; sbi_last_error() gives
 *     the message of the last failure on that context.
 *   - Calls on one context are not thread-safe; different contexts are
 *     independent.  Work is enqueued on opt.cuda_stream (NULL: the legacy
 *     default stream).
 */
#ifndef SBI_H
#define SBI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SBI_OK             0
#define SBI_EINVAL         1   /* bad grid, size, order, pointer or member index */
#define SBI_ENOMEM         2   /* device allocation failed */
#define SBI_ECUDA          3   /* a CUDA runtime call failed */
#define SBI_ENONFINITE     4   /* NaN or Inf appeared in the state */
#define SBI_ENOTCONVERGED  5   /* adaptive order reached M without meeting adapt_tol */
#define SBI_ETIMEOUT       6   /* a bounded device-side wait expired: a column pass whose inputs
                                    * arrive by bulk copies gave up waiting for one (reported by
                                    * sbi_step / sbi_step_streamed with check_finite = 1) */

#define SBI_FP32 0             /* FFTs, multipliers, products in FP32; FP64 state, RK4 sums, invariants */
#define SBI_FP64 1             /* everything in FP64 (the plain path) */

#define SBI_DIAG_ESBI 0        /* V by the ESBI successive approximation (Sec. 2.4) */
#define SBI_DIAG_HOS 1         /* V by the HOS perturbation expansion (flat bottom) */

#define SBI_RK4 0              /* classical RK4 on (eta, phi~) */
#define SBI_LAWSON_RK4 1       /* integrating factor (Sec. 2.2) with RK4 stages (Lawson) */
#define SBI_IF_RK45 2          /* integrating factor with the six-stage 5(4) pair of Sec. 2.2
                                  (Cash-Karp): fixed steps in sbi_step, adaptive ones in
                                  sbi_step_adaptive */

typedef struct sbi_ctx sbi_ctx;   /* opaque */

typedef struct {
    int nx, ny;                   /* points; ny = 1 for 1-D */
    double Lx, Ly;                /* periodic box [m]; Ly ignored when ny = 1 */
} sbi_grid;

typedef struct {
    int    order;        /* M, highest order of the successive approximation, 1..7 (default 7; Sec. 2.4) */
    double alias_frac;   /* kept fraction alpha of each axis' modes: |m| < alpha n/2 (default 0.5; Sec. 2.4) */
    double h0;           /* reference depth h0 [m], delta = h0 - h; NAN: mean of h (default NAN).
                            INFINITY selects deep water (only with h == NULL) */
    int    precision;    /* SBI_FP32 (default) or SBI_FP64 */
    double adapt_tol;    /* 0: fixed order M (default).  > 0: stop at the first l with
                            ||F{V_l}|| <= adapt_tol ||sum_{m<=l} F{V_m}|| (per member) */
    double filt_beta1;   /* low-pass filter Lambda = exp(-|k/(beta1 k_ref)|^beta2) applied to the */
    double filt_beta2;   /* state after every step, Eq. (filter); beta1 <= 0 disables (default) */
    double k_ref;        /* reference wavenumber of the filter [rad/m] */
    const double* sponge_w; /* damping weight w(x, y) (nx*ny host doubles, same for every member) or NULL */
    double sponge_nu;    /* damping strength nu [1/s]: p_d = nu F^-1{ ik/(-k^2) . F{w grad phi~} }, Eq. (pd) */
    void*  cuda_stream;  /* cudaStream_t used for all work (NULL: legacy default stream) */
    int    check_finite; /* 1 (default): sbi_step synchronizes and checks the state for NaN/Inf;
                            0: sbi_step only enqueues work */
    int    set_state_dealias; /* 1 (default): sbi_set_state removes the modes outside the dealias
                            mask; 0: the fields are stored exactly as given (for bit-exact
                            checkpoint/restart of states read with sbi_get_state) */
    void* (*dev_alloc)(size_t bytes, void* user);  /* optional device allocator (NULL: cudaMalloc) */
    void  (*dev_free)(void* ptr, void* user);      /* matching free (NULL: cudaFree) */
    void*  alloc_user;   /* passed to dev_alloc / dev_free */
    int    autotune;     /* 1 (default): before a step graph is captured (and on the first
                            diagnostic), time each row and column pass at a few block shapes
                            (rows per block, columns per block) and keep the fastest.  The
                            shapes change only how the work is split into blocks, never the
                            arithmetic, so results are identical with any choice.  0: use
                            the largest shape that fits (no timing runs). */
    int    integrator;   /* SBI_RK4 (default): classical RK4 with a fixed step.
                            SBI_LAWSON_RK4: the integrating factor of Sec. 2.2, e^{-A(t-t0)}
                            with A the linearisation d/dt (eta^, phi^) = [[0, k tanh(k h0)],
                            [-g, 0]] (eta^, phi^), applied exactly per mode, and classical RK4
                            stages for the nonlinear part (Lawson's scheme); the paper uses an
                            adaptive embedded RK5(4) for that part, which SBI_IF_RK45
                            provides.  The integrating factors are not combined with
                            adapt_tol > 0, SBI_IF_RK45 not with the wavemaker. */
    int    diagnostic;   /* SBI_DIAG_ESBI (default): V by the successive approximation of
                            Sec. 2.4.  SBI_DIAG_HOS: V by the HOS perturbation expansion of
                            the section comparing ESBI and HOS (its Eqs. HOS to HOSZ) on a flat
                            bottom at h0: phi^(m) = -sum_n eta^n/n! d^n_z phi^(m-n), W =
                            sum_{m+n<=M} eta^n/n! d^{n+1}_z phi^(m), V = W (1 + |grad eta|^2)
                            - grad eta . grad phi~, all dealiased; order = M.  Variable depth
                            or adapt_tol > 0 give SBI_EINVAL. */
    int    state_fp64;   /* SBI_FP32 only.  0 (default): the state (eta, phi~) and the RK sums
                            are kept as double-single float pairs (about 48 bits), updated with
                            error-free float transformations; dt/6 and the stage offsets c dt
                            enter as double-single pairs too.  1: they are kept and updated
                            in FP64 (the transforms, multipliers and products stay FP32).
                            Both use 8 bytes per value; results differ only in the last bits
                            of the state.  Ignored by SBI_FP64, whose state is FP64. */
    int    schedule;     /* how a step's launches are split into graph branches (see
                            sbi_schedule_report); the results are the same bits for every
                            value.  0 (default): chosen by timing on the first step when
                            autotune = 1, else B = 3.  B > 0: units of at most total/B
                            points (member ranges of one group), run as concurrent
                            branches; 1 gives one branch per group.  -1: one branch per
                            group, the branches one after another. */
    int    col_staging;  /* inputs of the column passes: 0 (default): direct loads, or bulk
                            copies (TMA) into shared memory where the autotuner times that form
                            faster; 1: bulk copies wherever a column holds at least 32 points
                            (the autotuner then times block shapes of that form only); -1:
                            direct loads only.  The arithmetic is the same either way. */
} sbi_options;

/* Fill *opt with the defaults listed above. */
void sbi_default_options(sbi_options* opt);

/* Create a context for one problem.
 *   g        grid (see conventions).
 *   gravity  g [m/s^2], > 0.
 *   h        still-water depth h(x, y) > 0, nx*ny host doubles, or NULL for a
 *            flat bottom of depth opt->h0 (which must then be given).  The
 *            bottom variation delta = h0 - h enters the recursion of Sec. 2.4.
 *   opt      options or NULL for the defaults.
 *   out      receives the context; NULL on failure.
 * The state is zero after creation.  SBI_EINVAL for a bad grid, order,
 * alias_frac, depth or pointer; SBI_ENOMEM / SBI_ECUDA on device failures. */
int sbi_create(const sbi_grid* g, double gravity, const double* h,
               const sbi_options* opt, sbi_ctx** out);

/* Create one context holding n independent problems ("members"), possibly on
 * different grids; every member is advanced by each sbi_step.  grids[i] and
 * h[i] (h may be NULL, or h[i] NULL for a flat member) as in sbi_create; one
 * option set (and one h0 rule) for all members. */
int sbi_create_batch(int n, const sbi_grid* grids, double gravity,
                     const double* const* h, const sbi_options* opt, sbi_ctx** out);

/* Number of members of a context (1 for sbi_create). */
int sbi_num_members(const sbi_ctx* ctx);

/* Set the state (eta, phi~) of one member: nx*ny doubles each.  Unless
 * opt.set_state_dealias = 0 the modes outside the dealias mask of Sec. 2.4 are
 * removed on entry, so the stored state is band-limited (in the FP32 path the
 * removal is computed in FP32 and added to the FP64 state).  Other members are
 * not touched.  Synchronizes the stream. */
int sbi_set_state(sbi_ctx* ctx, int member, const double* eta, const double* phi,
                  int on_device);

/* Copy the state of one member out (nx*ny doubles each).  Synchronizes the stream. */
int sbi_get_state(sbi_ctx* ctx, int member, double* eta, double* phi, int on_device);

/* Set / copy out the state of every member at once.  eta and phi each hold
 * sum over members of nx*ny doubles: member 0's field (row-major), then
 * member 1's, and so on, in member order.  The result is the same as one
 * sbi_set_state / sbi_get_state per member; the work is batched per member
 * group (one conversion launch per run of members that are consecutive in
 * the buffer, one dealias pass per group) and the stream is synchronized
 * once.  Device buffers (on_device = 1) and host buffers that the device can
 * address (pinned, mapped memory) are read and written by the conversion
 * kernels themselves; other host buffers go through a staging buffer of the
 * group's size (allocated on first use and kept) by copies.  The paper has
 * no counterpart (the calls batch its per-problem initial condition and
 * output). */
int sbi_set_state_all(sbi_ctx* ctx, const double* eta, const double* phi, int on_device);
int sbi_get_state_all(sbi_ctx* ctx, double* eta, double* phi, int on_device);

/* Surface vertical velocity V = sqrt(1+|grad eta|^2) dphi/dn at the current
 * state (Sec. 2.2-2.4), nx*ny doubles.  With eulerian_w = 1 the Eulerian
 * vertical velocity at the surface, w = (V + grad eta . grad phi~)/(1+|grad eta|^2),
 * is returned instead.  Synchronizes the stream. */
int sbi_vertical_velocity(sbi_ctx* ctx, int member, double* V_out, int on_device,
                          int eulerian_w);

/* V of one member from the implicit convolution equations of Appendix A (the
 * "iterative approach" that the successive scheme of Sec. 2.4 replaces), by
 * `iterations` fixed-point iterations
 *   F{V_{n+1}} = G + L(V_n),  V_0 = V^(1) = F^{-1}{k tanh(k h0) F{phi~}},
 * where G holds V^(1) and the grad phi~ terms of V^(2..M) and L the terms in
 * V, every term C_h k c F{eta^a F^{-1}{mult F{eta^b X}}} with the
 * coefficients of Appendix A (e_h = e^{-2 k h0}, C_h = 1/(1 + e_h),
 * D_h = 1/(1 - e_h); the remaining integrals I^(S), I^(B) are left out) and
 * every forward transform dealiased.  M is the context's order.  Over a
 * variable bottom the bottom potential varphi~ of Appendix B is iterated
 * with V (its delta grad varphi~ terms enter V^(j)), from
 * varphi~_0 = F^{-1}{sech(k h0) F{phi~}}.
 *   iterations  1..64.
 *   V_out       nx*ny doubles (host or device as on_device), V after the last
 *               iteration.
 *   increments  NULL or `iterations` host doubles: the relative L2 change
 *               ||V_{n+1} - V_n|| / ||V_{n+1}|| of each iteration (FP64).
 * The iteration diverges when the steepness makes L expansive (roughly
 * k H / 2 > 0.1 on one wavelength of 64 points); the call still returns the
 * last iterate and SBI_OK unless a value is non-finite.  Every member of the
 * member's group is iterated.  Synchronizes the stream.  SBI_EINVAL for
 * iterations outside 1..64. */
int sbi_vertical_velocity_implicit(sbi_ctx* ctx, int member, int iterations, double* V_out,
                                   int on_device, double* increments);

/* Advance every member by n classical RK4 steps of size dt [s] (Sec. 2.2 with
 * a fixed step); after each step the state is dealiased and, when enabled,
 * low-pass filtered.  The step is replayed from a CUDA graph. */
int sbi_step(sbi_ctx* ctx, double dt, int n);

/* The state of every member streamed through the device for n steps: the
 * same result, bit for bit, as
 *   sbi_set_state_all(ctx, eta_in, phi_in, 0); sbi_step(ctx, dt, n);
 *   sbi_get_state_all(ctx, eta_out, phi_out, 0);
 * (Sec. 2.2 steps between the copies), with the copies of one unit
 * overlapping the steps of the others.  The units are those of the step
 * schedule (member ranges of one group, see sbi_schedule_report), each cut
 * into k member ranges.  Each unit runs on a stream of its own: copy of its
 * eta and phi~ in (copy engine, into a device staging buffer), conversion,
 * the entry pass of sbi_set_state_all, n replays of the unit's step graph,
 * conversion out and copy out; the first unit's stream has the highest
 * priority, so the units finish one after another and the last copies out
 * overlap the remaining steps.  With opt.autotune = 1, the first call whose
 * n > 0 and whose outputs overlap no input times k = 1, 2, 3, 4 and 6 on whole
 * one-step calls (these write eta_out and phi_out, which the call then
 * overwrites with its result) and keeps the fastest (k = 1 unless another is
 * 3 % faster; sbi_schedule_report lists the "streamed-" times).  The paper
 * has no counterpart (it holds one problem's state on one device).
 *   eta_in, phi_in    sum over members of nx*ny doubles each, member order as
 *                     in sbi_set_state_all; host (pinned memory for the
 *                     overlap; pageable memory works but its copies block) or
 *                     device memory.
 *   eta_out, phi_out  the same sizes, written after the n steps; they may be
 *                     eta_in, phi_in themselves (k is then not timed).
 *   dt, n             as in sbi_step; n = 0 copies the entry state out.
 * Contexts whose schedule has one unit, the adaptive pair (SBI_IF_RK45), a
 * wavemaker or profiling on run the three calls one after another.  Two
 * device staging buffers per group (the group's points x 8 bytes each) are
 * allocated on first use and kept.  Synchronizes the stream.  SBI_EINVAL for
 * a NULL buffer, dt <= 0 or n < 0; SBI_ENONFINITE as sbi_step. */
int sbi_step_streamed(sbi_ctx* ctx, const double* eta_in, const double* phi_in, double dt, int n,
                      double* eta_out, double* phi_out);

/* Mass int eta dA and total energy 1/2 int (V phi~ + g eta^2) dA (Eq. energy,
 * dimensional, unit density) of one member, reduced in FP64 in a fixed order.
 * Synchronizes the stream. */
int sbi_invariants(sbi_ctx* ctx, int member, double* mass, double* energy);

/* Crest of one member's current surface (the crest position and speed of the
 * solitary-wave runs, Sec. 3.1): the largest sample of eta (the first in
 * row-major order among equal samples) and its position refined along each
 * axis by the parabola through the sample and its two periodic neighbours,
 * x = (i + (f_- - f_+) / (2 (f_- - 2 f_0 + f_+))) dx (no shift where the
 * denominator vanishes); y = 0 for a 1-D member.  *height is the sample.
 * The crest speed is the change of x over time.  Computed in FP64 on the
 * device in a fixed order.  NaN results for a non-finite state.
 * Synchronizes the stream.  SBI_EINVAL for a NULL pointer. */
int sbi_crest(sbi_ctx* ctx, int member, double* x, double* y, double* height);

/* Simulation time t [s] of the context: 0 after creation, advanced by dt for
 * every step of sbi_step.  It sets the phase of the wavemaker pressure. */
int sbi_set_time(sbi_ctx* ctx, double t);
int sbi_get_time(const sbi_ctx* ctx, double* t);

/* Pneumatic wavemaker of the submerged-bar section (Sec. 3, its Eq. for p_g):
 * a surface pressure subtracted in the dynamic condition, as the damping
 * pressure of Eq. (pd) is,
 *   p_g / rho = g sum_j a_j sqrt(e/2pi) [1 + 2 k_j h0 / sinh(2 k_j h0)]
 *                 exp(-(k_j d)^2 / 2) sin(omega_j t + theta_j),
 * with omega_j^2 = g k_j tanh(k_j h0) (h0 of each member group; deep water:
 * the bracket is 1), d the periodic distance in x from x0 and no dependence on
 * y (a line source in 2-D).  In linear theory it radiates waves of amplitude
 * a_j on both sides.  The printed pressure is nondimensional (g = 1); the
 * factor g is this library's dimensional reading.
 *   ncomp  number of components J, 0..256 (0 removes the wavemaker)
 *   amp, omega, phase   J host doubles each: a_j [m], omega_j [rad/s] > 0, theta_j
 *   x0     centre of the bell [m] (0: split in halves at both ends of the box)
 * The pressure of each RK4 stage is evaluated at the stage's time.  The step
 * graph is re-captured.  SBI_EINVAL for bad arguments. */
int sbi_set_wavemaker(sbi_ctx* ctx, int ncomp, const double* amp, const double* omega,
                      const double* phase, double x0);

/* Orders used by the last diagnostic of a member (M unless adapt_tol > 0). */
int sbi_orders_used(sbi_ctx* ctx, int member, int* orders);

/* Per-kernel-family timing of the step (for measurement).  sbi_profile_enable
 * turns on CUDA-event pairs around every pass of the captured step (the graph
 * is re-captured).  While it is on, the member groups of a batch run one after
 * the other instead of concurrently, so that each pair times one launch that
 * has the GPU to itself.  sbi_profile_read returns, for family i < *count (at most
 * cap entries), its name, the number of timed launches and their total device
 * milliseconds since the last enable, and synchronizes the stream. */
int sbi_profile_enable(sbi_ctx* ctx, int on);
int sbi_profile_read(sbi_ctx* ctx, int cap, const char** names, long long* launches,
                     double* total_ms, int* count);

/* Algorithmic device-memory traffic of one step, in bytes, summed over all
 * kernels of the step: each kernel counted as reading its inputs once and
 * writing its outputs once.  family < 0 gives the whole step. */
int sbi_step_bytes(const sbi_ctx* ctx, int family, double* bytes);

/* Transform work of one step: the number of one-dimensional transform
 * passes over a whole field (along x or along y) times the field's points,
 * summed over the kernels of a family (family < 0: the whole step).  A 2-D
 * FFT of a field counts twice.  Column passes count the whole field although
 * they transform only the kept x-modes.  This is the unit of the
 * bandwidth model in which every transform pass streams its field once in
 * and once out. */
int sbi_step_transforms(const sbi_ctx* ctx, int family, double* point_transforms);

/* Adaptive integrating-factor steps (integrator = SBI_IF_RK45) from the
 * context time to t_end (Sec. 2.2: six-stage fifth-order RK with an embedded
 * fourth-order solution, step size from their difference).  Each attempt
 * computes both solutions; its error is the largest over members and over
 * eta, phi~ of ||u5 - u4|| / ||u_n|| (L2 over the member's kept modes).  The
 * step is accepted (the order-5 solution kept) when the error is at most
 * tol; the next step is h min(5, max(0.2, 0.9 (tol/err)^(1/5))), the last one
 * cut to end at t_end.  A batch shares one step size.
 *   t_end     end time [s]; nothing happens when it is not after the context time
 *   tol       > 0, relative error per step
 *   h_inout   in: the first trial step [s]; out: the proposed next step
 *   accepted, rejected   out (may be NULL): attempts taken
 * Synchronizes once per attempt (the error is read on the host).
 * SBI_EINVAL for bad arguments or another integrator; SBI_ENOTCONVERGED when
 * the step underflows; SBI_ENONFINITE when the error or the state is not
 * finite. */
int sbi_step_adaptive(sbi_ctx* ctx, double t_end, double tol, double* h_inout, int* accepted,
                      int* rejected);

/* Number of kernel launches in one captured step. */
int sbi_step_launches(const sbi_ctx* ctx, int* launches);

/* Choices of the autotuner (opt.autotune), one line per distinct pass shape:
 *   "<pass shape>: rpc|cpb <chosen>/<default> <ms per launch> ms", e.g.
 *   "row nx=512 rows=16384 slots=1 ops=21 CPPPPPPCPPPPPPCPPPPPP: rpc 8/16 0.0910 ms"
 * A column choice with the suffix "s" (e.g. "cpb 4s/8") is the staged form:
 * each column's inputs arrive in shared memory by bulk copies (TMA,
 * cp.async.bulk), the next input in flight while the current one is
 * transformed; the arithmetic is the same.
 * (ms is -1 for a shape that was not timed: one candidate only, or a pass
 * that is not re-run because its outputs alias its inputs).
 * Writes at most cap bytes (NUL-terminated) into buf and the full length
 * (without the NUL) into *needed; buf may be NULL when cap is 0.  The paper
 * has no counterpart. */
int sbi_autotune_report(const sbi_ctx* ctx, char* buf, size_t cap, size_t* needed);

/* The step schedule: how the members are split into the branches of a step
 * graph.  A branch (unit) is a range of members of one group (members on the
 * same grid); the units run as concurrent graph branches, or one after another
 * ("serial").  Any split gives the same results bit for bit, since every
 * member's arithmetic is the same; only how the launches fill the GPU changes.
 * With opt.autotune = 1 the first step of the classical RK4 or Lawson scheme
 * captures and times each candidate (one branch per group, the serial order,
 * and splits into member ranges of at most total/B points for B = 2, 3, 4, 6)
 * on the real buffers, the state saved before and restored exactly after, and
 * keeps the fastest (the default, B = 3, unless another is 3 % faster).  The
 * saved copy (the state, its working copies, the time and the device flags:
 * about 24 bytes per point in FP32) is a temporary device allocation through
 * opt.dev_alloc or cudaMalloc, freed before the call returns; when it cannot
 * be made, nothing is timed and the default is kept.
 * Report lines:
 *   "chosen|default|tried <ms> ms per step: <name> [serial|concurrent] <U> units: <nx>x<ny>[m0:m1] ..."
 * ("default ..." alone, without a time, when nothing was timed).  Empty before
 * the first step.  Buffer conventions as sbi_autotune_report.  The paper has
 * no counterpart (its runs are one problem at a time). */
int sbi_schedule_report(const sbi_ctx* ctx, char* buf, size_t cap, size_t* needed);

/* Test hook for the bounded waits of the staged column pass (col_staging =
 * 1): with on = 1, each column's mbarrier is armed for 16 bytes more than its
 * bulk copy delivers, so every wait runs out (after about a second), the
 * device flag is set and the next sbi_step returns SBI_ETIMEOUT; the copies
 * themselves complete normally.  on = 0 restores normal operation; the
 * context stays usable.  Drops the captured step graphs.  The paper has no
 * counterpart. */
int sbi_test_stall_staged_copies(sbi_ctx* ctx, int on);

/* Mass and energy of one state without any device allocation.  (This entry
 * point has no counterpart in the paper; it serves callers that may not
 * allocate device memory.)
 *
 * Some callers cannot call cudaMalloc or cudaFree: code running inside
 * another framework's memory pool or a fixed arena, plugins that are handed
 * device buffers only, and hosts that forbid allocation (and the device
 * synchronisation it implies) once they are running.  This call computes the
 * same reductions as sbi_invariants, mass = int eta dA and energy =
 * 1/2 int (V phi~ + g eta^2) dA in FP64, from caller-owned DEVICE arrays eta,
 * phi and V (nx*ny doubles each, row-major; V as returned by
 * sbi_vertical_velocity with on_device = 1), on the caller's stream
 * (cuda_stream, NULL: legacy default stream), and writes the two host doubles
 * *mass and *energy (it synchronises that stream).  It needs no context.
 *
 * Its partial sums live in one file-scope device array of 64 KB (room for
 * 4096 chunks of 8192 points): grids of more than 33,554,432 points are
 * rejected with SBI_EINVAL.  Every device that loads the library holds the
 * array until the process exits.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  All calls share the array:
 * calls whose work overlaps on the GPU race and must be serialised by the
 * caller.  Nothing in the array needs to start at zero (each call writes every
 * partial sum before reading it).  No cudaMalloc, cudaFree or other allocating
 * routine is called.  Errors: SBI_EINVAL (NULL pointer, bad grid, too large),
 * SBI_ECUDA; the message is returned by sbi_noalloc_last_error(). */
int sbi_invariants_noalloc(const sbi_grid* g, double gravity, const double* eta,
                           const double* phi, const double* V, void* cuda_stream,
                           double* mass, double* energy);

/* Message of the last failing sbi_invariants_noalloc call on this thread. */
const char* sbi_noalloc_last_error(void);

/* Message of the last failing call on ctx (or of the last failing create when
 * ctx is NULL).  Never NULL. */
const char* sbi_last_error(const sbi_ctx* ctx);

/* Free every device buffer, graph and stream of the context.  NULL is ignored. */
void sbi_destroy(sbi_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SBI_H */
