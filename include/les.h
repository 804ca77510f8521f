/*
 * les.h — C ABI of libles.so, a single-GPU (sm_103a) implementation of the
 * per-stage residual evaluation and Runge-Kutta update of the filtered
 * compressible Navier-Stokes LES of Junqueira-Junior, Yamouni, Azevedo &
 * Wolf, "Large Eddy Simulations of Supersonic Jet Flows for Aeroacoustic
 * Applications" (AIAA 2015, arXiv:2212.12365).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Jet units (Sec. "Dimensionless Formulation"): lengths in jet diameters
 *   D, velocities in jet sound speed a_j, density in rho_j, temperature in
 *   T_j; hence p = rho T / gamma, c^2 = T, Cp = 1/(gamma-1).
 * - Grids are structured with ni x nj x nk points; host arrays are dense,
 *   point (i,j,k) at linear index (k*nj + j)*ni + i (i = xi = axial fastest).
 *   Field arrays of 5 variables are [field][point] (5*N doubles).
 * - The scheme advances Qhat = J^-1 [rho, rho u, rho v, rho w, e]
 *   (Eq. hat_Q_vec).  FP64 handles store Qhat; FP32 handles store the
 *   unscaled Q and advance it by the same update times J (a uniform flow is
 *   then stored exactly alike at every point).  The API exchanges the
 *   unscaled Q, primitives (rho, u, v, w, p), or the raw stored state.
 * - Every function returns LES_OK (0) or a negative LES_ERR_* code; the text
 *   of the last error of a handle is returned by les_last_error().  A
 *   NULL handle or pointer where one is required gives LES_ERR_ARG.  CUDA
 *   failures give LES_ERR_CUDA and leave the handle usable only for
 *   les_destroy().  No entry point waits on the device without bound.
 * - Ownership: host arrays passed in are read (or written) during the call
 *   only; the library copies what it keeps.  Device buffers passed in
 *   (workspace, probe output) are borrowed: the caller keeps them alive
 *   until les_destroy() (workspace) or until the probe is re-registered.
 * - Streams: all device work of a handle runs on the cudaStream_t given at
 *   creation (NULL = legacy default stream).  les_step() is asynchronous;
 *   functions returning host data synchronise that stream.
 */
#ifndef LES_H
#define LES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define LES_OK 0
#define LES_ERR_ARG (-1)       /* invalid argument or unsupported combination */
#define LES_ERR_OOM (-2)       /* device allocation failed / workspace too small */
#define LES_ERR_CUDA (-3)      /* a CUDA runtime call failed */
#define LES_ERR_NONFINITE (-4) /* diagnostics found NaN/Inf in the state or residual */
#define LES_ERR_TIMEOUT (-5)   /* a bounded device-side wait gave up (fused FP32 stage staging copy) */
#define LES_ERR_STATE (-6)     /* call out of order (e.g. step before set_state) */

/* Face boundary conditions (Sec. "Boundary Conditions").  Faces are ordered
 * i-, i+, j-, j+, k-, k+.  PERIODIC must be set on both faces of an axis
 * declared periodic and nowhere else; a periodic axis lists its unique planes
 * (the paper's overlapping last plane, equal to the first plus the period
 * shift, is rejected: drop it).  INFLOW_JET is allowed on the i- face
 * only (jet axis along x at y = z = 0). */
#define LES_BC_PERIODIC 0   /* Sec. "Periodic Boundary Condition", modulo indexing */
#define LES_BC_FARFIELD 1   /* Sec. "Far Field Boundary", Riemann invariants */
#define LES_BC_INFLOW_JET 2 /* Sec. "Entrance Boundary": jet (supersonic: all variables
                               imposed; subsonic: u imposed, v and w from the interior,
                               T and p from the jet's total conditions) + far field */
#define LES_BC_EXIT 3       /* Sec. "Exit Boundary Condition" */
#define LES_BC_CENTERLINE 4 /* Sec. "Centerline Boundary Condition": the j- face is the
                               degenerate axis of a polar mesh (J^-1 = 0 allowed there; k
                               must be periodic): its state is the azimuthal mean of the
                               ring j = 1, stored unscaled */

/* Storage / arithmetic precision of the stencil path. Metrics and the
 * Jacobian are always computed in FP64; diagnostics sum in FP64. */
#define LES_FP64 0
#define LES_FP32 1
/* FP32 with the separable-metric stage: only for a Cartesian-product grid
 * (x depends on i only, y on j only, z on k only; LES_ERR_ARG otherwise).
 * The cofactors are then diagonal products of the three 1-D spacings
 * dx/dxi, dy/deta, dz/dzeta (Sec. "Transformation of Coordinates"), which the
 * stage kernel reads from three 1-D tables instead of nine stored fields;
 * everything else behaves as LES_FP32 (state kinds, probe, diagnostics). */
#define LES_FP32_SEPARABLE 2

/* State kinds for les_set_state / les_get_state. */
#define LES_STATE_CONSERVED 0 /* unscaled Q = [rho, rho u, rho v, rho w, e] */
#define LES_STATE_PRIMITIVE 1 /* [rho, u, v, w, p] */
#define LES_STATE_RAW 2       /* the stored state, for bit-exact checkpoints: Qhat = J^-1 Q
                                 (FP64 handles) or Q (FP32 handles) */

/* Point fields for les_debug_field. */
#define LES_FIELD_MU_SGS 0   /* Smagorinsky mu_sgs (Sec. "Subgrid Scale Viscosity") */
#define LES_FIELD_MU 1       /* Sutherland mu/mu_j (Eq. sutherland) */
#define LES_FIELD_P 2        /* pressure */
#define LES_FIELD_T 3        /* temperature T/T_j */
#define LES_FIELD_LAMBDA_XI 4   /* lambda-bar along xi (Turkel-Vatsa scaling) */
#define LES_FIELD_LAMBDA_ETA 5
#define LES_FIELD_LAMBDA_ZETA 6
#define LES_FIELD_METRICS 7  /* 10 x N: J^-1 xi_x ... J^-1 zeta_z, J^-1 (FP64) */

typedef struct les_grid_desc {
    int ni, nj, nk;          /* points per axis; each >= 4 */
    const double *x, *y, *z; /* host coordinates, ni*nj*nk each */
    int periodic[3];         /* 1 if the axis is periodic (no duplicated point) */
    double period_shift[3][3]; /* [axis][x,y,z]: coordinate offset of one period */
    int face_bc[6];          /* LES_BC_* for faces i-, i+, j-, j+, k-, k+ */
    int precision;           /* LES_FP64 or LES_FP32 */
    void *workspace;         /* optional device memory for all buffers (NULL: the
                                library allocates); borrowed, 256-byte aligned */
    size_t workspace_bytes;  /* size of workspace (>= les_workspace_bytes()) */
} les_grid_desc;

typedef struct les_params {
    double gamma;     /* specific heat ratio (1.4) */
    double Pr;        /* Prandtl number (0.72) */
    double Pr_sgs;    /* SGS Prandtl number (0.6, Eidson model) */
    double Cs;        /* Smagorinsky constant (0.17) */
    double k2, k4;    /* Turkel-Vatsa constants (0.25, 0.016) */
    double Re;        /* rho_j a_j D / mu_j; INFINITY = inviscid */
    double mach_j;    /* jet Mach number (> 0; < 1 selects the subsonic entrance) */
    double TR;        /* T_j / T_inf (PR = 1: p_j = p_inf) */
    double T_inf_dim; /* ambient temperature in K for Sutherland (288.15) */
    double S1_dim;    /* Sutherland constant in K (110.4) */
    double theta;     /* inflow momentum thickness in D (0.05) */
    double noise_amp; /* inflow velocity noise amplitude / U_j (1e-3) */
    double cfl;       /* CFL number for the time step (0.5) */
    double dt;        /* fixed time step; 0 = from cfl at the first les_set_state */
    uint64_t seed;    /* SplitMix64 seed of the inflow noise */
} les_params;

typedef struct les_diag {
    double dt;                /* time step in use */
    int64_t step;             /* completed steps (time level) */
    double max_abs_rhs_rho;   /* L-inf of the continuity residual, interior points */
    double l2_rhs[5];         /* sqrt(sum RHS_f^2) over interior points */
    double sum_qhat[5];       /* sum of Qhat_f over all points (compensated FP64) */
    int64_t nonfinite;        /* number of non-finite state/residual values */
} les_diag;

typedef struct les_handle les_handle;

/* Bytes of device workspace les_create_grid needs for this grid (caller-
 * provided workspace mode).  Returns 0 on invalid dimensions. */
size_t les_workspace_bytes(const les_grid_desc *g);

/* Create a solver for one grid (Secs. "Transformation of Coordinates",
 * "Boundary Conditions").  Copies the coordinates to the device and computes
 * the nine metric cofactors J^-1 d(xi,eta,zeta)/d(x,y,z) in conservative
 * form and J^-1 in FP64.  stream: a cudaStream_t (NULL = default stream).
 * On success *out owns all device memory of the solver until les_destroy.
 * Errors: LES_ERR_ARG (dims < 4, inconsistent periodic/BC flags, a periodic
 * axis in the overlapping form, INFLOW_JET
 * off the i- face, mach_j <= 0 with INFLOW_JET, non-positive J^-1, an FP32
 * grid of 2^31 / 5 or more padded points: nk x nj x ni rounded up to 32),
 * LES_ERR_OOM, LES_ERR_CUDA. */
int les_create_grid(const les_grid_desc *g, const les_params *p, void *stream, les_handle **out);

/* Batched form: njets independent grids/parameter sets in one handle; every
 * les_step advances all of them with one persistent launch per kernel of a
 * stage.  Jet results are bit-identical to single-grid handles of the same
 * precision.  Per-jet state access through les_set_state_jet etc. */
int les_create_batch(const les_grid_desc *g, const les_params *p, int njets, void *stream,
                     les_handle **out);

/* Set the state of jet 0 (or of jet `jet`).  q: host array 5*N of `kind`
 * (LES_STATE_*).  Applies the boundary conditions of the current time level
 * (level 0 carries no inflow noise) and, if no time step is fixed yet,
 * sets dt = cfl / max(lambda_xi + lambda_eta + lambda_zeta) over the state
 * (Sec. "Numerical Formulation", spectral radii).  Synchronises the stream.
 * Errors: LES_ERR_ARG (bad kind/jet), LES_ERR_CUDA. */
int les_set_state(les_handle *h, const double *q, int kind);
int les_set_state_jet(les_handle *h, int jet, const double *q, int kind);

/* Advance every jet by nsteps steps of the 5-stage Runge-Kutta scheme
 * (Eq. localdt, alpha = 1/4, 1/6, 3/8, 1/2, 1); after each stage of step
 * n -> n+1 the boundary conditions of level n+1 are applied (faces y, z, x).
 * One step is captured once as a CUDA graph and replayed.  Asynchronous on
 * the handle's stream.  Errors: LES_ERR_STATE (no state set), LES_ERR_CUDA. */
int les_step(les_handle *h, int nsteps);

/* Copy the state of jet 0 / jet `jet` to the host array q (5*N, `kind`).
 * Synchronises the stream.  Errors: LES_ERR_ARG, LES_ERR_CUDA, and, for FP32
 * handles, LES_ERR_TIMEOUT once a staging wait of the fused stage (the
 * bounded wait for the TMA copy of the next plane's state) has given up since
 * the handle was created.  The stage then reads that plane, and every later
 * one of the launch, directly from global memory, so q is still written and
 * holds the state a normal step gives; the handle keeps reporting the
 * timeout (it points to a stalled copy engine).  If the stage's final,
 * bounded wait for such an abandoned copy gives up as well, the copy may
 * still land in shared memory another CTA uses: the call then returns
 * LES_ERR_CUDA, q is still written but the state is unreliable. */
int les_get_state(les_handle *h, double *q, int kind);
int les_get_state_jet(les_handle *h, int jet, double *q, int kind);

/* Time level and time step (checkpoint/resume): les_set_time fixes both;
 * a following les_set_state with LES_STATE_RAW resumes bit-identically. */
int les_set_time(les_handle *h, int64_t step, double dt);
int les_get_time(les_handle *h, int64_t *step, double *dt);

/* Register a surface probe on jet 0 (FW-H input surface): npts points xyz
 * (host, 3*npts: all x, then all y, then all z).  After every step whose
 * time level is a multiple of every_n, rho, u, v, w, p at the points are
 * interpolated trilinearly from the 8 surrounding grid points and written to
 * frame f = (count % capacity) of dev_out, a device array of
 * out_capacity_frames * 5 * npts elements of the state precision (float or
 * double), layout [frame][field][point]; count counts frames from
 * registration.  The grid must be a Cartesian product (x = x(i), y = y(j),
 * z = z(k)).  npts = 0 removes the probe.  Errors: LES_ERR_ARG (non-product
 * grid, point outside the grid, every_n < 1). */
int les_probe_surface(les_handle *h, const double *xyz, int npts, int every_n, void *dev_out,
                      int out_capacity_frames);
/* Frames written since registration. */
int les_probe_frames(les_handle *h, int64_t *frames);

/* Residual monitor of jet 0 / jet `jet` (Sec. "Computational Performance
 * Assessment": max |RHS| of continuity) and conservation sums, computed from
 * the current state.  Returns LES_ERR_NONFINITE if any state or residual
 * value is NaN/Inf, LES_ERR_TIMEOUT as les_get_state does (d is still filled
 * in both cases).  Synchronises the stream. */
int les_get_diagnostics(les_handle *h, les_diag *d);
int les_get_diagnostics_jet(les_handle *h, int jet, les_diag *d);

/* Test access: RHS (5*N doubles, zero at boundary points) of the current
 * state (Eq. spatial_discret), and point fields LES_FIELD_* (N doubles; 10*N
 * for LES_FIELD_METRICS). */
int les_debug_rhs(les_handle *h, int jet, double *rhs);
int les_debug_field(les_handle *h, int jet, int field, double *out);

/* Tracing: run nsteps steps eagerly (not from the graph) with CUDA events
 * around every kernel launch on the handle's stream, and accumulate the
 * device time per kernel kind into ms_out[LES_KERNEL_KINDS] (milliseconds,
 * summed over launches) and the launch counts into counts (may be NULL).
 * The state advances exactly as with les_step.  Synchronises the stream. */
#define LES_KERNEL_POINT 0  /* primitives, Sutherland, lambda-bar, point fluxes */
#define LES_KERNEL_GRADS 1  /* derivatives, Smagorinsky/Eidson, pressure sensor */
#define LES_KERNEL_IFACE 2  /* interface fluxes (inviscid, dissipation, viscous) */
#define LES_KERNEL_UPDATE 3 /* flux differences and stage update */
#define LES_KERNEL_BC 4     /* boundary faces */
#define LES_KERNEL_OTHER 5  /* time-level counter, probe */
#define LES_KERNEL_KINDS 6
int les_profile_step(les_handle *h, int nsteps, double *ms_out, int64_t *counts);

/* Work decomposition of the fused FP32 stage (LES_FP32, LES_FP32_SEPARABLE
 * handles): ty = 8 or 16 grid rows per CTA tile (32 x ty/2 threads, two rows
 * each), kc >= 1
 * planes per k-chunk item, kc = 0 for the balanced form (every CTA of the
 * persistent grid takes one contiguous, equal share of all tile-planes), or
 * kc = -1 for the lockstep form (whole columns in waves of one tile per CTA,
 * so that neighbouring tiles share their halo planes through L2, then the
 * remaining tile-planes shared out as in the balanced form).  By default the
 * first les_step picks the fastest choice by timing them (autotuner); this
 * call sets it instead and disables the tuning for the handle.  Results are
 * bit-identical for every choice.  Errors: LES_ERR_ARG (FP64 handle, bad ty,
 * kc < -1). */
int les_set_fused_tiling(les_handle *h, int ty, int kc);

/* Test access to the timeout path of the fused FP32 stage: max_polls >= 0
 * bounds every staging wait to that many polls of its mbarrier (0: the first
 * wait of each CTA gives up at once, while its copy is still in flight, so
 * that the fallback to direct loads and the LES_ERR_TIMEOUT report run on a
 * healthy device); -1 restores the default (2^22 polls).  The copy a wait
 * gave up on is still waited for, with the default bound, before the CTA
 * exits.  Errors: LES_ERR_ARG (FP64 handle, max_polls < -1). */
int les_debug_stage_wait(les_handle *h, int max_polls);

/* Kernel launches issued by the most recent les_step call (all steps). */
int64_t les_last_launch_count(les_handle *h);

/* Index-bounds checking, the debug build that stands in for a memory
 * checker.  A library compiled with -DLES_BOUNDS_CHECK checks, in every
 * kernel, each point index against its grid (i, j, k within the axes) and,
 * in the fused FP32 stage, every global offset against the padded point
 * count and every shared-memory slot against its table; the first index out
 * of range is recorded and that access is redirected to index 0 instead of
 * faulting.  Results are otherwise those of the normal build.
 * les_bounds_checking() returns 1 for such a library, 0 for a normal one.
 * les_bounds_violation(h, out) writes the first violation of the kernels run
 * for handle h since its creation: 0 if none, else (site << 48) | value with
 * site 1 a point index (value = k << 32 | j << 16 | i, 16 bits each), 2-4 a
 * fused-stage global offset (state, static record, update), 5-7 a fused-stage
 * shared-memory slot (point ring, plane tables, eta-flux rows).  In every
 * build, site 8 records a staging wait of the fused stage that gave up and
 * site 9 an abandoned staging copy that did not complete before its CTA
 * exited (see les_get_state); in a normal build no other site is recorded.
 * Synchronises the stream.  Errors: LES_ERR_ARG. */
int les_bounds_checking(void);
int les_bounds_violation(les_handle *h, uint64_t *out);

/* Residual / conservation sums without any device allocation.  The paper
 * has no counterpart: this is a library service for callers that must not
 * allocate device memory — code inside a framework whose caching allocator
 * holds (nearly) all device memory, and per-step monitoring hooks that
 * cannot afford cudaMalloc/cudaFree latency or their device-wide
 * synchronisation.  It computes what les_get_diagnostics reports from the
 * caller's own buffers:
 *   qhat, rhs : device arrays of 5*npoints doubles, [field][point] (dense
 *               layout of les_get_state and les_debug_rhs; qhat = J^-1 Q,
 *               the raw state of an FP64 handle);
 *               rhs should be zero at boundary points;
 *   out       : device array of 12 doubles: [0] max |rhs_rho|,
 *               [1..5] sqrt(sum rhs_f^2), [6..10] compensated sum of qhat_f,
 *               [11] count of non-finite values;
 *   stream    : cudaStream_t the two kernels are launched on (NULL allowed).
 * Asynchronous; allocates nothing.  Its scratch is one file-scope device
 * array of LES_NOALLOC_MAX_POINTS/65536 x 17 doubles (557 KB), held by every
 * GPU that loads the library until exit; the first call on a device looks up
 * that array's device address (make it before any stream capture).  All calls
 * share the array: calls that overlap on the GPU (different streams without
 * ordering) race and give wrong sums.  Errors: LES_ERR_ARG for null pointers,
 * npoints < 1 or npoints > LES_NOALLOC_MAX_POINTS (with a message on stderr),
 * LES_ERR_CUDA if the address lookup or a launch fails. */
#define LES_NOALLOC_MAX_POINTS 268435456LL
int les_diag_sums_noalloc(const double *qhat, const double *rhs, int64_t npoints, double *out,
                          void *stream);

/* Measured arithmetic throughput of the current device, for the compute-bound
 * roofline fractions reported beside the stage timings (the paper has no
 * counterpart: it is a measurement utility).  kind 0: FP64 fused multiply-add
 * (DFMA); 1: FP32 fused multiply-add (FFMA); 2: paired FP32 fused multiply-add
 * (fma.rn.f32x2, two lanes per instruction).  Launches a short loop of
 * independent multiply-add chains on the legacy default stream (timed with
 * CUDA events, best of five after a warm-up; tens of milliseconds) and writes
 * the achieved rate in TFLOP/s (FMA = 2 FLOP) to *tflops.  Synchronises the
 * device's default stream.  Errors: LES_ERR_ARG (null pointer, unknown kind),
 * LES_ERR_CUDA. */
#define LES_PEAK_FP64_FMA 0
#define LES_PEAK_FP32_FMA 1
#define LES_PEAK_FP32X2_FMA 2
int les_measure_peak(int kind, double *tflops);

/* Far-field acoustic pressure from the probe surface's frames by the Ffowcs
 * Williams-Hawkings equation (the paper names FW-H as the far-field step fed
 * by its probe surface, Secs. "Introduction" and "Concluding Remarks", but
 * gives no formulation).  Adopted: Farassat's Formulation 1A (NASA
 * TM-2007-214853, 2007) with the permeable-surface source terms of
 * di Francescantonio (J. Sound Vib. 202, 1997) for a surface at rest in a
 * medium at rest (ambient pressure p0, sound speed c0):
 *   Q = rho u.n, L_i = (p - p0) n_i + rho u_i u.n,
 *   4 pi p'(x, t) = sum over panels of A [dQ/dtau / r + (dL_r/dtau)/(c0 r) + L_r/r^2]
 * at the emission time tau = t - r/c0 (r = |x - y|, L_r = L.(x - y)/r);
 * d/dtau by second-order differences between frames (central; one-sided at
 * the first and last frame), values at tau by linear interpolation between
 * frames.
 * ring: device array [capacity][5][npts] of (rho, u, v, w, p), double for
 *   precision LES_FP64, float for LES_FP32 / LES_FP32_SEPARABLE, as
 *   les_probe_surface fills it; frames_written: frames written so far
 *   (les_probe_frames).  The last min(frames_written, capacity) frames are
 *   used in time order, the oldest of them at tau = 0, frame m at m dtau.
 * xyz, nrm: host, 3*npts each (all x, then y, then z): panel centres (the
 *   probe points, in the ring's point order) and unit outward normals;
 *   area: host, npts panel areas.
 * obs: host, 3*nobs observer positions; observer times t_k = t0 + k dt_obs,
 *   k < nt, on the tau axis.  Every emission time t_k - r/c0 must lie within
 *   [0, (frames - 1) dtau] for every panel and observer.
 * p_out: host, nobs*nt doubles, layout [observer][time]: p' = p - p0.
 * ms_out: NULL, or 2 doubles receiving the device time (ms) of the source
 *   pass and of the observer pass.
 * Allocates device scratch (32 bytes per panel and frame, plus partial sums)
 * for the call and frees it; runs on `stream`, synchronises it.  The sums
 * have a fixed order: the same inputs give the same bits.  Errors:
 * LES_ERR_ARG (null pointer, fewer than 3 frames, an emission time outside
 * the frames, an observer on a panel; text in les_last_error(NULL)),
 * LES_ERR_OOM, LES_ERR_CUDA. */
int les_fwh(const void *ring, int precision, int capacity, int64_t frames_written, int npts, const double *xyz,
            const double *nrm, const double *area, double dtau, double p0, double c0, int nobs, const double *obs,
            double t0, double dt_obs, int nt, double *p_out, void *stream, double *ms_out);

/* Human-readable description of a handle: precision, jets, device bytes and
 * the stage kernel configuration chosen by the autotuner (FP32: fused tile
 * height and k-chunk; FP64: four-kernel stage).  Valid until the next call
 * on the handle. */
const char *les_describe(les_handle *h);

/* Text of the last error of handle h; with h = NULL, the text of the last
 * failed les_create_grid / les_create_batch of the calling thread ("" if
 * none).  The pointer stays valid until the next call on the handle (or the
 * next creation on the thread). */
const char *les_last_error(les_handle *h);
int les_destroy(les_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* LES_H */
