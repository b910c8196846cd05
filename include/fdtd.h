/*
 * fdtd.h -- C ABI of the GB300 Bessel-antenna FDTD library (libfdtd_gb300.so).
 *
 * Method (Ardaneh, Giust, Morel, Courvoisier, "Generation of a Bessel beam in
 * FDTD using a cylindrical antenna", arXiv:2102.12978):
 *   - standard second-order Yee leapfrog of E and H (Section 4);
 *   - z periodic (Section 1 and Section 4: the box spans whole axial periods),
 *     CPML on the transverse x/y faces (Section 4, Roden-Gedney CPML),
 *     PEC behind the CPML;
 *   - a hollow cylindrical annulus ("Bessel antenna", Fig. 3) that adds, after
 *     each curl update, the analytic order-m vector Bessel field of Eq. 12 built
 *     from the Hertz-potential solutions Eq. 5-9 (soft source, Eq. 13);
 *   - the time-integrated fluence, integral of |S| dt (Section 2), which per
 *     window of whole periods gives the intensity of Section 5.
 *
 * Units: c = eps0 = mu0 = 1 (eta = 1); lengths in source wavelengths
 * (lambda = 1), times in optical periods (omega = 2 pi).  The paper's SI
 * setup has lambda = 0.8 um.
 *
 * Conventions for every call:
 *   - No call aborts or exits; every failure is a status code, and
 *     fdtd_last_error() gives a one-line reason (thread-local).
 *   - Device memory is owned by the caller: fdtd_required_bytes() gives the
 *     size of one device arena that the caller allocates (e.g. a torch uint8
 *     tensor) and passes to fdtd_create_grid(); the library carves fields,
 *     CPML auxiliaries, fluence and source tables out of it, and allocates no
 *     device memory of its own.  The arena must stay alive until
 *     fdtd_destroy_grid().
 *   - Work is queued on the caller's CUDA stream (a cudaStream_t passed as
 *     void*; NULL = legacy default stream).  Calls that return data to the host
 *     synchronise that stream and report asynchronous CUDA errors.
 *   - A grid belongs to the device that was current at fdtd_create_grid.
 *     Every call that queues work for a grid, or reads or writes its memory,
 *     returns FDTD_EINVAL and queues nothing while another device is current.
 *   - Field storage: structure of arrays, one array per component, x fastest,
 *     rows padded to a pitch of 32 elements; two copies of E, H and the
 *     H-side CPML auxiliaries are kept (ping-pong), because the fused step
 *     reads step n from one copy while writing step n+1 into the other.
 *   - Yee positions (in cells, from the box corner): Ex (i+1/2, j, k),
 *     Ey (i, j+1/2, k), Ez (i, j, k+1/2), Hx (i, j+1/2, k+1/2),
 *     Hy (i+1/2, j, k+1/2), Hz (i+1/2, j+1/2, k); E at t = n dt and H at
 *     (n - 1/2) dt.  The beam axis is at (nx/2, ny/2).  Tangential E on the
 *     planes i = 0 and j = 0 (and on the virtual walls i = nx, j = ny) is zero.
 */
#ifndef FDTD_GB300_H
#define FDTD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FDTD_OK = 0,
    FDTD_EINVAL = 1,   /* invalid argument or descriptor                     */
    FDTD_ENOMEM = 2,   /* arena too small / host allocation failed           */
    FDTD_ECUDA = 3,    /* a CUDA runtime call or kernel failed               */
    FDTD_ETIMEOUT = 4, /* a bounded device-side wait expired                 */
    FDTD_ESTATE = 5    /* call not valid in the grid's current state         */
} fdtd_status;

typedef enum { FDTD_F32 = 0, FDTD_F64 = 1 } fdtd_precision;

/* Field components for get/set calls. */
enum { FDTD_EX = 0, FDTD_EY = 1, FDTD_EZ = 2, FDTD_HX = 3, FDTD_HY = 4, FDTD_HZ = 5 };

/* Polarisation of the injected beam: which Hertz potential of Eq. 5 drives it. */
enum {
    FDTD_POL_Y = 0,          /* Pi_x (Eq. 6): linear, y-polarised (paper default)  */
    FDTD_POL_X = 1,          /* Pi_y (Eq. 7): linear, x-polarised                  */
    FDTD_POL_CIRC_PLUS = 2,  /* (Pi_x + i Pi_y)/sqrt 2                             */
    FDTD_POL_CIRC_MINUS = 3, /* (Pi_x - i Pi_y)/sqrt 2                             */
    FDTD_POL_Z = 4           /* Pi_z (Eq. 8): for m = 0 azimuthal (TE), radial (TM) */
};
enum { FDTD_TE = 0, FDTD_TM = 1 };                    /* Eq. 9a / Eq. 9b       */
enum { FDTD_ENV_CW_SIN2 = 0, FDTD_ENV_GAUSS = 1 };     /* CW ramp / Eq. 12 f(t) */
enum { FDTD_INJECT_ALL = 0, FDTD_INJECT_TANGENTIAL = 1 };

/* Grid descriptor.  Section 4 fixes a cubic mesh and z-periodicity; the CPML
 * constants are not given by the paper and are exposed here (defaults in
 * brackets: order 3, sigma scale 0.8, kappa_max 1, alpha_max 0.05 * 2 pi). */
typedef struct {
    int nx, ny, nz;          /* cells; nx, ny >= 2*npml + 2, nz >= 1               */
    int npml;                /* CPML cells on each transverse face (0 = PEC box)   */
    double dx, dy, dz;       /* cell sizes in wavelengths                          */
    double dt;               /* time step in periods; 0 => courant * Yee limit     */
    double courant;          /* used when dt == 0, must be in (0, 1]               */
    double pml_order;        /* sigma = sigma_max u^order                          */
    double pml_sigma_scale;  /* sigma_max = scale (order+1) / (eta d)              */
    double pml_kappa_max;    /* kappa = 1 + (kappa_max - 1) u^order                */
    double pml_alpha_max;    /* alpha = alpha_max (1 - u)                          */
    int precision;           /* fdtd_precision of the field arithmetic             */
    int fluence;             /* 1: accumulate the fluence (FP64 accumulator)       */
    int z_boundary;          /* FDTD_Z_PERIODIC (the antenna boxes of Section 4) or
                                FDTD_Z_WALLS (the Bessel-Gauss box of Section 2)   */
    int npml_z;              /* FDTD_Z_WALLS: CPML cells inside each z wall (same
                                constants as x/y; 2*npml_z + 2 <= nz); else 0      */
} fdtd_grid_desc;

/* z boundary.  FDTD_Z_WALLS puts PEC walls at z = 0 and z = nz dz (tangential
 * E_x, E_y zero on the plane k = 0; fields past the last plane read as the
 * wall) with npml_z CPML cells inside each.  A z-walled grid runs on tile
 * variant 5 and the cell batch engines only
 * (EINVAL elsewhere), takes no antenna (the antenna boxes are z-periodic,
 * Section 4) and has no adjoint (EINVAL). */
enum { FDTD_Z_PERIODIC = 0, FDTD_Z_WALLS = 1 };

/* Bessel-antenna descriptor (Section 4, Fig. 3, Eq. 12-13).  The antenna is
 * every Yee point of each component whose distance r from the beam axis, in
 * cells, satisfies r_center - thickness/2 <= r < r_center + thickness/2,
 * along the whole z length.  The value added after the curl update at such a
 * point p of component c, at that component's own time t, is
 *     f(t) * Re{ w_amp[col] e^{i w_phase[col]} A_c(p) e^{-i omega t'} }
 * with A the complex E (or H) amplitude of the TE/TM order-m beam (Eq. 6-9,
 * e^{+i beta z} carried in A), t' = t (CW) or t - T0 (Gaussian), and col the
 * point's column j*nx + i.  Both weight arrays are host arrays of nx*ny
 * doubles, copied by the call; NULL means amplitude 1 / phase 0. */
typedef struct {
    int m;                   /* Bessel order                                       */
    double theta;            /* cone angle, radians (K = k sin, beta = k cos)      */
    int pol;                 /* FDTD_POL_*                                         */
    int mode;                /* FDTD_TE / FDTD_TM                                  */
    double E0;               /* field amplitude of Eq. 9                           */
    double r_center;         /* ring centre radius, cells of dx                    */
    double thickness;        /* ring thickness, cells of dx                        */
    int envelope;            /* FDTD_ENV_*                                         */
    double ramp;             /* CW: f = sin^2(pi t / (2 ramp)) for t < ramp, else 1 */
    double T, T0;            /* Gaussian: f = exp(-(t-T0)^2 / T^2)                 */
    int inject;              /* FDTD_INJECT_ALL (Eq. 13) or _TANGENTIAL (drop the
                                radial x/y projection at each point)               */
    const double* w_amp;     /* host, nx*ny, or NULL                               */
    const double* w_phase;   /* host, nx*ny, or NULL                               */
} fdtd_annulus_desc;

/* Wall source: the Bessel-Gauss reference beam of Section 2, a Gaussian beam
 * polarised along x with the axicon phase Phi(r) = -k r sin(theta), injected
 * as a soft E_x sheet on the E plane k = plane.  After each E update (time
 * t = (n+1) dt, after the antenna's E terms) every E_x point of that plane
 * with j >= 1 gets
 *     f(t) Re{ E0 exp(-r^2 / w0^2) e^{-i k r sin(theta)} e^{-i omega t'} }
 * with r the distance of the E_x point (i+1/2, j) from the beam axis
 * (nx/2, ny/2) in wavelengths, and f, t' as in fdtd_annulus_desc.  The sheet
 * radiates to both sides; put it on the first plane past the low-z CPML
 * of a z-walled grid (plane = npml_z), so that the backward half is
 * absorbed.  The column coefficients are evaluated on the host in FP64. */
typedef struct {
    double theta;            /* cone angle of the axicon, radians                  */
    double w0;               /* Gaussian waist, wavelengths (> 0)                  */
    double E0;               /* amplitude                                          */
    int envelope;            /* FDTD_ENV_*                                         */
    double ramp;             /* CW ramp length, periods                            */
    double T, T0;            /* Gaussian envelope, periods                         */
    int plane;               /* E plane k of the sheet; 0 <= plane < nz, and not
                                0 on a z-walled grid (the z = 0 PEC wall)          */
} fdtd_wall_desc;

typedef struct fdtd_grid fdtd_grid;
typedef struct fdtd_batch fdtd_batch;
typedef struct fdtd_adjoint fdtd_adjoint;

/* Fill *d with the defaults (courant 0.95, CPML constants above, F32, fluence on). */
void fdtd_grid_desc_default(fdtd_grid_desc* d);

/* Bytes of device arena a grid with this descriptor needs (0 if invalid). */
size_t fdtd_required_bytes(const fdtd_grid_desc* d);

/* Create a grid on the current CUDA device.  `arena` is a device pointer to
 * at least fdtd_required_bytes(d) bytes, 256-byte aligned, owned by the caller;
 * `stream` is a cudaStream_t (or NULL).  Zeroes the fields, CPML auxiliaries
 * and fluence, uploads the CPML profiles (Section 4), and sets the step
 * counter to 0.  Also makes the fixed staging array of fdtd_fluence_noalloc
 * resident on the device (16 MiB, once per device; see that call).  Returns
 * EINVAL on a bad descriptor (Courant > 1, CPML wider than a quarter of the
 * box, ...), ENOMEM if arena_bytes is too small. */
fdtd_status fdtd_create_grid(const fdtd_grid_desc* d, void* arena, size_t arena_bytes,
                             void* stream, fdtd_grid** out);

/* Build the antenna (Fig. 3) and its FP64 coefficients A_c (Eq. 6-9, Eq. 12)
 * on the host and upload them into the arena.  Replaces any earlier source.
 * EINVAL if the ring reaches into the CPML or outside the box. */
fdtd_status fdtd_set_annulus_source(fdtd_grid* g, const fdtd_annulus_desc* s);

/* Remove the source (source-free runs). */
fdtd_status fdtd_clear_source(fdtd_grid* g);

/* Set (w != NULL) or remove (w == NULL) the wall source of fdtd_wall_desc:
 * its column coefficients are evaluated on the host in FP64 and uploaded into
 * the arena.  It adds to the antenna, if any.  Set it before the grid joins
 * a batch.  EINVAL on a bad descriptor or if the grid's tile variant is not
 * 5. */
fdtd_status fdtd_set_wall_source(fdtd_grid* g, const fdtd_wall_desc* w);

/* Host-only: the wall source's complex column coefficients
 * E0 exp(-r^2/w0^2) e^{-i k r sin(theta)} into out[ny][nx] (re, im
 * interleaved: 2*nx*ny doubles; the row j = 0 is zero).  Runs no GPU code.
 * EINVAL on a bad descriptor. */
fdtd_status fdtd_wall_coefficients(const fdtd_grid_desc* d, const fdtd_wall_desc* w, double* out);

/* Advance nsteps full Yee steps (asynchronous on the grid's stream).  Each
 * step n: H^{n+1/2} (with CPML psi) -> H soft source at (n+1/2) dt ->
 * fluence += |E^n x (H^{n-1/2}+H^{n+1/2})/2| dt at cell centres ->
 * E^{n+1} (with CPML psi) -> E soft source at (n+1) dt (Eq. 13) -> wall
 * source at (n+1) dt.  One or two kernel launches per step (tile variant).
 * Small grids, whose passes take a few microseconds, are bound by the cost
 * of those launches; a batch of one grid (fdtd_batch_create with n = 1)
 * replays 64 steps from one CUDA graph instead, with the same results
 * (64 x 64 x 32 cells on GB300: 10.3 us per step alone, 6.0 in a batch). */
fdtd_status fdtd_step(fdtd_grid* g, int nsteps);

/* Copy the fluence (nz*ny*nx doubles, x fastest, dense) to dst (device if
 * on_device, else host), then zero the accumulator if reset.  Synchronises
 * the stream.  Cell (i,j,k) is centred at (i+1/2, j+1/2, k+1/2).  FP64 grids
 * accumulate in FP64; FP32 grids keep an FP32 sum plus a Kahan compensation
 * term, which the export kernel combines in FP64. */
fdtd_status fdtd_fluence(fdtd_grid* g, void* dst, int on_device, int reset);

/* Copy one field component (FDTD_EX..FDTD_HZ) as a dense nz*ny*nx array of the
 * grid's precision (float or double) to / from dst (device if on_device).
 * fdtd_get_field synchronises the stream. */
fdtd_status fdtd_get_field(fdtd_grid* g, int component, void* dst, int on_device);
fdtd_status fdtd_set_field(fdtd_grid* g, int component, const void* src, int on_device);

/* Full state (fields, CPML auxiliaries, fluence, step counter): its size in
 * bytes, and device-to-device save / load (dst/src are device pointers of at
 * least fdtd_state_bytes bytes).  Used for checkpoints and resume. */
size_t fdtd_state_bytes(const fdtd_grid* g);
fdtd_status fdtd_save_state(fdtd_grid* g, void* dev_dst);
fdtd_status fdtd_load_state(fdtd_grid* g, const void* dev_src);

/* Step counter, time step and antenna point count of component c. */
int64_t fdtd_get_step(const fdtd_grid* g);
fdtd_status fdtd_set_step(fdtd_grid* g, int64_t n);
double fdtd_get_dt(const fdtd_grid* g);
int64_t fdtd_antenna_points(const fdtd_grid* g, int component);

/* Tile configuration of the step.  A CTA owns a 32 x ty block of columns
 * (ty in {4, 8, 16}); variants 0-4 march lz planes of z per CTA:
 *   0  one pass, plain coalesced loads into a shared-memory ring;
 *   1  one pass, every z plane staged by TMA bulk-tensor copies into a
 *      multi-stage shared-memory ring (mbarrier completion);
 *   2  variant 1 with two rows of the tile per thread;
 *   3  two passes (H, then E with the fluence term), plain loads;
 *   4  two passes, a TMA-staged H pass with the fluence term, then E;
 *   5  two cell-parallel passes, one thread per cell (lz unused; grids
 *      of more than 65535 planes are launched in chunks of planes);
 *   6  one cell-parallel pass, the neighbouring H recomputed per cell
 *      (needs nz <= 65535, else EINVAL);
 *   7  two steps per launch (temporal blocking; FP32 grids, ty 8 or 16,
 *      else EINVAL; lz 2 interleaves the window rows in the CTAs' work so
 *      that x-neighbouring windows march side by side, any other lz takes
 *      the windows row by row): windows of 32 x ty columns march along z,
 *      recomputing two rings of halo columns, so that fields, psi and the
 *      fluence cross HBM once per two steps.  An odd step count ends with
 *      one step of variant 5.  The CTAs' shares of the work are balanced on
 *      per-window costs (fdtd_set_balance).
 * The TMA variants (1, 2, 4) have no FP64 32x16 tile (EINVAL).  A z-walled
 * grid or one with a wall source takes variant 5 only (EINVAL otherwise;
 * fdtd_autotune then times the ty of variant 5 only).
 * fdtd_create_grid picks a default (variant 5, ty 4); fdtd_autotune times
 * the candidates on this grid (running `steps` steps for each, then
 * restoring the state) and keeps the fastest.  Results agree to rounding
 * for every configuration. */
fdtd_status fdtd_set_tile(fdtd_grid* g, int variant, int ty, int lz);

/* Work-split weights of tile variant 7 (the paper has no counterpart): a
 * window's plane is estimated to cost 1, plus w_shell if the window holds
 * CPML shell columns, plus w_antenna if it holds antenna columns, and each
 * CTA takes a contiguous range of (window, plane) work of equal estimated
 * cost; a window also costs three planes at its start (the two-step
 * wavefront refills there).  Weights in [0, 16] (else EINVAL); defaults 0.25
 * and 0.2.  fdtd_autotune times a few pairs, then refines the fastest pair's
 * ranges on measured times (fdtd_measure_balance), with the windows row by
 * row and interleaved (lz 1 and 2), and times those; it keeps the fastest.
 * While refined ranges are in use, fdtd_get_balance returns -1 for both
 * weights; fdtd_set_balance returns to the weights.  The results do not
 * depend on the balance, only the time does. */
fdtd_status fdtd_set_balance(fdtd_grid* g, float w_shell, float w_antenna);
fdtd_status fdtd_get_balance(const fdtd_grid* g, float* w_shell, float* w_antenna);
/* Refine the CTAs' work ranges of the grid's variant-7 tile on measured
 * times (the paper has no counterpart): in four rounds, three launches record
 * the SM cycles every CTA takes, and the ranges' boundaries move toward equal
 * shares of the measured time (all the way in the first round, three
 * quarters of the way after it).  The 24 steps run from a copy of the state
 * and are undone (the state is saved to
 * `scratch_state`, fdtd_state_bytes bytes of device memory the caller owns,
 * and restored).  The refined ranges are used from then on (fdtd_autotune
 * does the same for its fastest weights).  EINVAL unless the tile is variant
 * 7; the ranges are dropped when the antenna's columns change, and hold for
 * single-grid steps only (a batch's two-step launches use the weights). */
fdtd_status fdtd_measure_balance(fdtd_grid* g, void* scratch_state);

/* Test hooks of tile variant 7's host logic (no device work; the paper has
 * no counterpart).
 * fdtd_debug_tb2_order writes to out[m] the window (wy * t + wx) that the
 * CTAs take at flattened position m = 0 .. t*u - 1, for windows t along x by
 * u along y, nz planes, `slots` CTAs and window order `order` (the lz of
 * fdtd_set_tile: 2 interleaves the window rows, anything else takes them row
 * by row).  out holds t*u ints.  Returns the interleave stride D (1: row by
 * row), or -1 for an invalid argument.
 * fdtd_debug_tb2_refine runs one refinement step of fdtd_measure_balance on
 * host data: from the ranges' starts (slots + 1 items, starts[0] = 0, not
 * decreasing, the last the item count) and each CTA's measured cycles, it
 * writes the new starts to out (slots + 1 items), each boundary moved `step`
 * (in (0, 1]) of the way to where every CTA's share of the total, spread
 * evenly over the items it ran, is equal.  EINVAL for invalid arguments. */
int fdtd_debug_tb2_order(int t, int u, int nz, int slots, int order, int* out);
fdtd_status fdtd_debug_tb2_refine(int slots, const long long* starts, const unsigned long long* cycles, double step,
                                  long long* out);

/* Measurement (the paper has no counterpart): advance `nsteps` steps like
 * fdtd_step and time every kernel launch of a step with CUDA events recorded
 * on the grid's stream.  pass_ms[p] (host array of max_passes floats) gets
 * the total milliseconds of kernel p of a step summed over the steps;
 * *n_passes = kernels per step (1 for variants 0-2; 2 for variants 3-5:
 * [0] H pass, [1] E pass with the fluence term, or for variant 4 [0] H pass
 * with the fluence term, [1] E pass).  Synchronizes the stream.  EINVAL if
 * max_passes is smaller than the kernels per step. */
fdtd_status fdtd_step_timed(fdtd_grid* g, int nsteps, float* pass_ms, int max_passes, int* n_passes);

/* Test hook (the paper has no counterpart): fault injection on the host side
 * of a device wait.  kind 1 makes the next step of a TMA variant (tile
 * variants 1 and 2) withhold one plane's bulk copies in its first CTA: that
 * CTA's bounded mbarrier wait (about 2^32 SM cycles) expires, it raises the
 * grid's error word, drains its other copies and returns, and the next
 * synchronising call (fdtd_sync, fdtd_fluence, ...) returns FDTD_ETIMEOUT;
 * the device context stays usable.  kind 0 clears a pending fault; a fault
 * applies to one step only.  EINVAL for another kind. */
fdtd_status fdtd_debug_inject_fault(fdtd_grid* g, int kind);

/* Test hook: record `device` as the device the grid lives on, so that a test
 * on one GPU can check that every entry point refuses (FDTD_EINVAL, nothing
 * queued) a grid whose device is not the current one.  The grid is unusable
 * until its own device is recorded again.  EINVAL for device < 0. */
fdtd_status fdtd_debug_set_device(fdtd_grid* g, int device);
fdtd_status fdtd_get_tile(const fdtd_grid* g, int* variant, int* ty, int* lz);
fdtd_status fdtd_autotune(fdtd_grid* g, int steps, void* scratch_state);

/* Synchronise the grid's stream and report any pending CUDA error; returns
 * FDTD_ETIMEOUT (and clears the word) if a kernel's bounded wait expired. */
fdtd_status fdtd_sync(fdtd_grid* g);

void fdtd_destroy_grid(fdtd_grid* g);

/* ---- Batched stepping of many independent grids --------------------------
 * Several grids (any sizes, sources, cone angles; one precision; all created
 * on the current device and at the same step parity) advance together, K =
 * 64 consecutive steps per CUDA-graph replay or per persistent launch.
 * Two engines:
 *   FDTD_BATCH_CELL (default): a CUDA graph of K steps with one branch per
 *     grid (up to 16 concurrent streams, shared round-robin).  Each grid
 *     steps in its own mode (fdtd_batch_set_grid_mode): the cell passes of
 *     tile variant 5 on 32 x 4, 32 x 8 or 32 x 16 blocks (the arithmetic of
 *     variant 5, bit for bit), or, for FP32 z-periodic grids without a wall
 *     source, the two-step kernel of tile variant 7 on a share of the SMs
 *     proportional to the grid's cells (the arithmetic of variant 7, bit for
 *     bit).  Steps that do not fill a replay run one by one with the cell
 *     passes.
 *   FDTD_BATCH_PERSISTENT_CELL: one cooperative kernel launch per 64 steps
 *     and per group of up to 24 grids (no graph): every CTA stays resident
 *     and takes runs of cell blocks of all grids in order from a counter,
 *     H pass, grid barrier, E pass, barrier, step after step (the
 *     arithmetic of tile variant 5, bit for bit; every grid kind; no limit
 *     on nz).  Its barrier waits are bounded: an expired wait raises
 *     the batch's error word and every CTA returns (ETIMEOUT from
 *     fdtd_batch_sync).
 * FDTD_BATCH_PERSISTENT (a persistent TMA engine of earlier versions, which
 * ran slower than the grids stepped one by one) is no longer built:
 * fdtd_batch_set_engine refuses it with EINVAL.
 * `dev_table` is a device buffer of fdtd_batch_required_bytes bytes
 * (256-byte aligned), owned by the caller and alive until
 * fdtd_batch_destroy; `stream` is a cudaStream_t.  While a grid belongs to
 * a batch (until fdtd_batch_destroy), fdtd_step, fdtd_step_timed,
 * fdtd_autotune and the source calls (fdtd_set_annulus_source,
 * fdtd_clear_source, fdtd_set_wall_source) on it return ESTATE: the batch
 * holds copies of its arguments.  A grid must outlive its batches.  A grid
 * whose copy parity no longer matches the batch's (fdtd_load_state of
 * another parity) makes fdtd_batch_step return ESTATE.
 * fdtd_batch_set_engine switches engines between steps (EINVAL for an
 * unknown engine).  fdtd_batch_sync waits for the stream and reports CUDA
 * errors or an expired device wait (ETIMEOUT).  fdtd_batch_work_items: cell
 * blocks per step and pass. */
enum { FDTD_BATCH_PERSISTENT = 0, FDTD_BATCH_CELL = 1, FDTD_BATCH_PERSISTENT_CELL = 2 };
/* Grid modes of the graph engine. */
enum { FDTD_BATCH_MODE_CELL4 = 0, FDTD_BATCH_MODE_CELL8 = 1, FDTD_BATCH_MODE_CELL16 = 2,
       FDTD_BATCH_MODE_TWO_STEP = 3 };
size_t fdtd_batch_required_bytes(int n_grids, int precision);
fdtd_status fdtd_batch_create(fdtd_grid* const* grids, int n, void* dev_table, size_t table_bytes, void* stream,
                              fdtd_batch** out);
fdtd_status fdtd_batch_set_engine(fdtd_batch* b, int engine);
int fdtd_batch_get_engine(const fdtd_batch* b);
/* Mode of grid q (0-based, creation order) in the graph engine; EINVAL for
 * an unknown mode or the two-step mode on a grid that cannot take it.  The
 * default is FDTD_BATCH_MODE_CELL4.  -1 from the getter for a bad index. */
fdtd_status fdtd_batch_set_grid_mode(fdtd_batch* b, int q, int mode);
int fdtd_batch_get_grid_mode(const fdtd_batch* b, int q);
/* CTAs of grid q's two-step launches in the graph engine (-1 for a bad index). */
int fdtd_batch_get_grid_ctas(const fdtd_batch* b, int q);
/* Autotuner of the batch (the paper has no counterpart).  Saves every grid's
 * state into `scratch` (a device buffer of at least
 * fdtd_batch_autotune_bytes bytes, owned by the caller; ENOMEM if smaller).
 * Times each grid alone on the cell passes of each block height (32 x 4, 8,
 * 16) over `steps` steps (rounded up to even) and keeps the fastest as its
 * cell mode.  Then times, over 64 steps of the whole batch (the better of two
 * replays): the graph engine with every grid of at least N cells on the
 * two-step kernel, for N over the sizes of the grids that can take it (and
 * with none), each with the two-step launches on shares of the SMs
 * proportional to the grids' cells or on every SM; and the persistent cell
 * engine.  Keeps the fastest, and restores every grid's state and step
 * counter.  The results of later steps do not depend on the choices beyond
 * the rounding of the chosen kernels. */
size_t fdtd_batch_autotune_bytes(const fdtd_batch* b);
fdtd_status fdtd_batch_autotune(fdtd_batch* b, int steps, void* scratch, size_t scratch_bytes);
/* Test hook (the paper has no counterpart): kind 1 makes CTA 0 of the next
 * FDTD_BATCH_PERSISTENT_CELL launch return without arriving at the grid
 * barrier, so that the other CTAs' bounded waits (about 2^32 SM cycles)
 * expire: they raise the batch's error word and return, and the next
 * fdtd_batch_sync returns FDTD_ETIMEOUT (and resets the error word and the
 * barrier); the device context stays usable.  kind 0 clears a pending
 * fault.  EINVAL for another kind. */
fdtd_status fdtd_batch_debug_inject_fault(fdtd_batch* b, int kind);
fdtd_status fdtd_batch_step(fdtd_batch* b, int nsteps);
fdtd_status fdtd_batch_sync(fdtd_batch* b);
int fdtd_batch_work_items(const fdtd_batch* b);
void fdtd_batch_destroy(fdtd_batch* b);

/* ---- Reverse-time adjoint -------------------------------------------------
 * Gradient of a loss L(E) with respect to the antenna's per-column amplitude
 * and phase weights (fdtd_annulus_desc.w_amp / w_phase).  The forward step is
 * linear in the state and in the weighted source coefficients; the adjoint
 * applies the exact transpose of the discrete step (CPML and PEC included)
 * backwards in time.  The paper computes no gradients: this is the transpose
 * of the method's discrete update.
 *
 * Grids with z walls or a wall source have no adjoint (EINVAL).
 *
 * The adjoint holds its own state (adjoints of E, H and of the CPML psi, two
 * copies each) and a per-(component, column) accumulator in a caller-owned
 * device arena of fdtd_adjoint_required_bytes bytes.  `probe_cells` (host,
 * n_probes linear cell indices (k*ny + j)*nx + i) are the points of E
 * component `component` (FDTD_EX..FDTD_EZ) at which the loss reads E.
 *
 *   fdtd_probe_read     forward field at the probes from the grid's current
 *                       state (device buffer of n_probes field-precision
 *                       values); asynchronous.
 *   fdtd_adjoint_reset  zero the adjoint state and gradient and place the
 *                       adjoint at forward step n_end (the adjoint of
 *                       E^{n_end}, H^{n_end - 1/2}).
 *   fdtd_adjoint_step   nsteps reverse steps.  Before reversing forward step
 *                       m -> m+1 (m = position - 1 - r), row r of dLdE (device,
 *                       field precision, row stride ld elements, n_probes
 *                       values) is added at the probes as dL/dE^{m+1}; NULL
 *                       injects nothing.  The source terms of every reversed
 *                       step enter the weight gradient.
 *   fdtd_adjoint_gradient  dL/dw_amp and dL/dw_phase per column (nx*ny
 *                       doubles each, host or device); synchronises.
 *   fdtd_adjoint_get    copy one adjoint component (0..2 E, 3..5 H) to a
 *                       dense device array; synchronises. */
size_t fdtd_adjoint_required_bytes(const fdtd_grid* g, int64_t n_probes);
fdtd_status fdtd_adjoint_create(fdtd_grid* g, int component, const int64_t* probe_cells, int64_t n_probes,
                                void* arena, size_t bytes, fdtd_adjoint** out);
fdtd_status fdtd_adjoint_reset(fdtd_adjoint* a, int64_t n_end);
fdtd_status fdtd_probe_read(fdtd_adjoint* a, void* dev_out);
/* Advance the adjoint's grid by nsteps single steps (the grid's tile, or one
 * step of variant 5 when the grid runs variant 7) and after step s copy the
 * probe values (as fdtd_probe_read) into row s of dev_rows (device, rows of
 * ld >= n_probes elements of the field precision), all queued on the grid's
 * stream with no host synchronisation: the forward pass of a gradient
 * records its loss window in one call.  EINVAL for a bad argument, ESTATE
 * while the grid belongs to a batch. */
fdtd_status fdtd_probe_record(fdtd_adjoint* a, int nsteps, void* dev_rows, int64_t ld);
fdtd_status fdtd_adjoint_step(fdtd_adjoint* a, int nsteps, const void* dLdE, int64_t ld);
int64_t fdtd_adjoint_position(const fdtd_adjoint* a);
fdtd_status fdtd_adjoint_get(fdtd_adjoint* a, int component, void* dst);
fdtd_status fdtd_adjoint_gradient(fdtd_adjoint* a, double* dLdw_amp, double* dLdw_phase, int on_device);
void fdtd_adjoint_destroy(fdtd_adjoint* a);

/* ---- Fluence read-out without device allocation --------------------------
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory at the moment they read the result (for
 * example inside a hook that must not grow a caching allocator, or on a
 * system whose device memory is reserved up front).  It returns exactly what
 * fdtd_fluence returns, but stages the export in a fixed 16 MiB array
 * compiled into the library (2^21 doubles) instead of the grid's arena,
 * and calls no cudaMalloc, cudaFree or other allocating routine.
 *   - The array becomes resident on a device when the first grid is created
 *     there: fdtd_create_grid looks up its device address (under lazy module
 *     loading that lookup loads the array's module, which takes the 16 MiB),
 *     and it stays resident until the process exits.  The read-out itself
 *     loads nothing and only uses the address cached by fdtd_create_grid.
 *     Every grid creation on the device refreshes that address, so after a
 *     cudaDeviceReset (which ends every grid of the device) the library is
 *     used again by creating new grids.
 *   - Grids with more than fdtd_fluence_noalloc_max_cells() cells are
 *     rejected with FDTD_EINVAL, as is a call made while a device other than
 *     the grid's is current.
 *   - All calls share the one array, which keeps the last call's contents
 *     (every element read back is written by the call itself, so nothing has
 *     to be cleared first); calls that overlap on the GPU (different streams
 *     or threads at once) race on it and must be serialised by the caller.
 *   - dst, on_device and reset as for fdtd_fluence; synchronises the stream. */
size_t fdtd_fluence_noalloc_max_cells(void);
fdtd_status fdtd_fluence_noalloc(fdtd_grid* g, void* dst, int on_device, int reset);

/* ---- Measurement of the FP64 pipe (the paper has no counterpart) ---------
 * The FP64 cell passes are bound by the device's FP64 FMA rate, not by HBM.
 * fdtd_measure_fp64_rate times one launch of a kernel in which every thread
 * (2048 per SM) runs `chains` independent (8) or dependent (1) chains of
 * `iters` FP64 fused multiply-adds, with CUDA events on `stream`, and returns
 * the FMAs per second over all threads (*fma_per_s, thread-level: one FMA is
 * one FP64 instruction of one thread) and the kernel time in ms.  dev_sink is
 * a device buffer of at least 8 bytes owned by the caller (written only in a
 * case that does not occur).  Synchronises the stream.  EINVAL for chains
 * other than 1 or 8, or iters < 1. */
fdtd_status fdtd_measure_fp64_rate(void* dev_sink, void* stream, int chains, int iters, double* fma_per_s,
                                   double* ms);

/* fdtd_debug_vec_norm: out[i] = |S| from x[i] = |S|^2 >= 0 for n FP64 values,
 * computed by the device function every FP64 fluence term uses (Section 2's
 * |E x Hbar|: one Newton step on s^2 = x from the single-precision reciprocal
 * square root; relative error below 2.5e-13 for x in [2^-126, 2^128), the
 * correctly rounded square root elsewhere, 0 for x = 0).  dev_x and dev_out
 * are device arrays of n doubles owned by the caller; the kernel runs on
 * `stream` and the call synchronises it; n = 0 does nothing.  EINVAL for
 * n < 0, or for a null pointer with n > 0. */
fdtd_status fdtd_debug_vec_norm(const void* dev_x, void* dev_out, int64_t n, void* stream);

/* Host-only: the per-column source coefficients A_c (see fdtd_annulus_desc)
 * without weights, evaluated at z = 0 and at z = dz/2 as appropriate for the
 * component, into out[6][ny][nx] complex doubles (re, im interleaved:
 * 12*nx*ny doubles), plus the antenna mask out_mask[ny][nx] (bit c set when
 * column (i,j) holds a point of component c).  Runs no GPU code; exposed so
 * that the FP64 precompute can be checked on a host without a GPU.  The
 * descriptor is checked as by fdtd_set_annulus_source (EINVAL). */
fdtd_status fdtd_source_coefficients(const fdtd_grid_desc* d, const fdtd_annulus_desc* s,
                                     double* out, uint8_t* out_mask);

/* Host-only: the Bessel function J_n(x) the precompute uses (Miller backward
 * recurrence with the Neumann-series normalisation). */
double fdtd_bessel_j(int n, double x);

const char* fdtd_status_string(fdtd_status s);
const char* fdtd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FDTD_GB300_H */
