/*
 * stencil.h -- C ABI of the GB300 stencil engine (libstencil.so).
 *
 * The engine sweeps stencil functions over padded 1D/3D arrays on one NVIDIA GB300 GPU
 * (sm_103a).  It implements the computations of "Stencil Computations on AMD and Nvidia
 * Graphics Processors: Performance and Tuning Strategies" (Pekkila et al., arXiv 2406.08923):
 *
 *   STENCIL_XCORR      1D cross-correlation f'_i = sum_{j=-r..r} g_j f^_{i+j}       (Sec. 3.1, Eq. 3)
 *   STENCIL_DIFFUSION  forward-Euler step of df/dt = alpha lap f with the central
 *                      2nd-derivative stencil of order 2r per axis (r = 1..4; r = 3 is
 *                      the 6th-order case) in 1, 2 or 3 dimensions, folded into one
 *                      star-shaped cross-correlation                               (Sec. 3.2, Eqs. 4-7;
 *                                                                                   radius sweep, Sec. 5.3)
 *   STENCIL_MHD8       one 3-stage Runge-Kutta step of the 8-field non-ideal MHD system
 *                      in non-conservative form, 6th-order central 1st, 2nd and mixed
 *                      derivatives fused with the nonlinear right-hand side          (Sec. 3.3, Eqs. 8-9,
 *                                                                                   Appendix A, Eqs. A1-A4)
 *   STENCIL_MAXFILTER  1D max filter f'_i = max_{j=-r..r} f^_{i+j}, the nonlinear
 *                      stencil example                                             (Sec. 2.1)
 *
 * Arrays are "augmented" arrays f^ (Sec. 2.4, Eq. 2): the interior is surrounded by a halo of
 * width r whose values are the boundary function beta.  With STENCIL_BC_PERIODIC the library
 * fills the halo with the periodic image of the interior; with STENCIL_BC_CALLER the caller
 * fills it and the library only reads it.
 *
 * Conventions for every entry point:
 *   - Device pointers are plain CUDA device addresses (e.g. torch tensor data_ptr()), owned
 *     by the caller and at least 16-byte aligned.  `stream` is a cudaStream_t passed as
 *     void* (NULL = the legacy default stream).  Work is enqueued on `stream` and returns
 *     before it completes unless stated otherwise.
 *   - Host pointers are owned by the caller and only read/written during the call.
 *   - Errors are returned as stencil_status; nothing aborts, exits or throws across the ABI.
 *     stencil_last_error_detail() gives a human-readable reason for the last failure.
 *   - A plan belongs to the CUDA device that was current when it was created; calls with a
 *     different current device return STENCIL_EINVAL.
 *   - Calls on one plan must not overlap in host threads; separate plans are independent.
 */
#ifndef STENCIL_H
#define STENCIL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STENCIL_ABI_VERSION 1

typedef struct stencil_plan *stencil_t;

typedef enum stencil_status {
    STENCIL_OK = 0,
    STENCIL_EINVAL = 1,       /* an argument is out of range, inconsistent or misaligned */
    STENCIL_ENOMEM = 2,       /* a device or host allocation failed */
    STENCIL_ECUDA = 3,        /* a CUDA call failed (detail string names it) */
    STENCIL_EUNSUPPORTED = 4, /* a valid combination the library does not implement */
    STENCIL_ETIMEOUT = 5      /* a bounded device-side wait expired; the kernel gave up */
} stencil_status;

typedef enum stencil_dtype {
    STENCIL_I32 = 0,  /* int32 storage, arithmetic modulo 2^32 (XCORR only) */
    STENCIL_F64 = 1,
    STENCIL_F32 = 2,
    STENCIL_BF16 = 3  /* bfloat16 storage; arithmetic in FP32 */
} stencil_dtype;

typedef enum stencil_bc {
    STENCIL_BC_PERIODIC = 0,   /* beta(f, i) = f_{i mod n}: library fills the halo */
    STENCIL_BC_CALLER = 1,     /* caller fills the halo; one pass per stencil_step call */
    STENCIL_BC_PERIODIC_XY = 2 /* 3D DIFFUSION / MHD8 z-slab of a grid decomposed along z: x and
                                  y periodic (library), the z halo (r planes below and above the
                                  interior, whole padded planes) supplied by the caller before
                                  every pass -- the neighbouring slabs' edge planes.  One pass
                                  per call: stencil_step(nsteps = 1) for DIFFUSION,
                                  stencil_substep for MHD8.  The z halo of fields_out is
                                  unspecified on return (the caller overwrites it). */
} stencil_bc;

typedef enum stencil_kind {
    STENCIL_XCORR = 0,     /* Eq. 3, ndim = 1, radius 0..1024, caller weights g_{-r..r} */
    STENCIL_DIFFUSION = 1, /* Eqs. 4-7, ndim = 1..3, radius 1..4 (order-2r Laplacian) */
    STENCIL_MHD8 = 2,      /* Eqs. A1-A4 + RK3, ndim = 3, radius 3, 8 fields */
    STENCIL_MAXFILTER = 3  /* Sec. 2.1 nonlinear stencil max_{j=-r..r} f^_{i+j}, ndim = 1, radius 0..1024 */
} stencil_kind;

/* Physical constants.  Unused members are ignored by kinds that do not need them. */
typedef struct stencil_params {
    double dt;     /* time step (DIFFUSION, MHD8) */
    double alpha;  /* diffusion coefficient (DIFFUSION) */
    double dx[3];  /* grid spacing along x, y, z (DIFFUSION, MHD8) */
    double cs0;    /* MHD8: reference sound speed */
    double gamma;  /* MHD8: adiabatic index */
    double cp;     /* MHD8: specific heat at constant pressure */
    double lnrho0; /* MHD8: reference log-density */
    double nu;     /* MHD8: kinematic viscosity */
    double eta;    /* MHD8: magnetic diffusivity */
    double zeta;   /* MHD8: bulk viscosity */
    double mu0;    /* MHD8: vacuum permeability */
    double K;      /* MHD8: radiative heat conductivity of Eq. A3 (constant; 0 switches the
                      conduction term off) */
} stencil_params;

/* Field order of STENCIL_MHD8 (Table A1 symbols). */
enum { STENCIL_MHD_LNRHO = 0, STENCIL_MHD_UX, STENCIL_MHD_UY, STENCIL_MHD_UZ,
       STENCIL_MHD_AX, STENCIL_MHD_AY, STENCIL_MHD_AZ, STENCIL_MHD_SS, STENCIL_MHD_NFIELDS };

/*
 * stencil_create -- validate a problem and build a plan (Sec. 2.4 Eq. 2 for the layout).
 *
 *   ndim     1 (XCORR, MAXFILTER), 1..3 (DIFFUSION) or 3 (MHD8).
 *   dims     interior extents (nx, ny, nz); entries beyond ndim are ignored.  With periodic
 *            boundaries each used extent must be >= 2*radius + 1 (STENCIL_BC_PERIODIC_XY: nx
 *            and ny, and nz >= radius).
 *   radius   stencil radius r: 0..1024 for XCORR (radius > 4: F64 and F32 only; the radius
 *            sweep of Sec. 5.2) and MAXFILTER; 1..4 for DIFFUSION (the central Laplacian of
 *            order 2r; r = 3 is the 6th-order, 19-point step of Eq. 7; the other radii serve the
 *            radius sweep of Sec. 5.3); 3 for MHD8.
 *   coeffs   XCORR only: 2r+1 weights g_{-r..r}, int32_t for STENCIL_I32, double otherwise
 *            (rounded to FP32 for STENCIL_F32).  Copied; may be freed after the call.
 *            NULL for the other kinds.
 *   ncoeffs  2r+1 for XCORR, 0 otherwise.
 *   nfields  1 for XCORR, MAXFILTER and DIFFUSION, 8 for MHD8.
 *   storage  element type of the caller's arrays; compute = arithmetic type:
 *              XCORR:     I32/I32 (radius <= 4), F64/F64, F32/F32
 *              MAXFILTER: I32/I32, F64/F64, F32/F32 (exact: the result equals the definition)
 *              DIFFUSION: F64/F64, F32/F32
 *              MHD8:      F64/F64, F32/F32, BF16/F32 (F32 and BF16 storage use
 *                         Kahan-compensated RK accumulation)
 *   params   physical constants (may be NULL for XCORR and MAXFILTER).
 *   out      receives the plan.
 *
 * The only call that allocates device memory: library-owned scratch (one extra field set for
 * ping-pong, the RK register and Kahan compensation arrays for MHD8, reduction buffers, and
 * for XCORR of radius > 4 a device copy of the weights).
 * Returns EINVAL on invalid arguments, EUNSUPPORTED on valid but unimplemented
 * combinations, ENOMEM/ECUDA if the scratch allocation fails (nothing is leaked).
 */
stencil_status stencil_create(int ndim, const int64_t dims[3], int radius, const void *coeffs,
                              int ncoeffs, int nfields, stencil_bc bc, stencil_kind kind,
                              stencil_dtype storage, stencil_dtype compute,
                              const stencil_params *params, stencil_t *out);

/* Release a plan and its scratch (synchronises the device first).  NULL is a no-op. */
void stencil_destroy(stencil_t plan);

/*
 * stencil_layout -- how the caller must allocate each field (Eq. 2 augmented array).
 *
 * A field is a dense array of padded[0] * padded[1] * padded[2] elements of the storage
 * type, x fastest.  Interior cell (i, j, k) lives at linear element index
 *     (origin[0] + i) + pitch[1] * (origin[1] + j) + pitch[2] * (origin[2] + k),
 * with pitch = {1, padded[0], padded[0] * padded[1]}.  The halo of width r surrounds the
 * interior on every used axis; origin[0] >= r is rounded up so that interior rows start on a
 * 16-byte boundary, and padded[0] is a multiple of 32 bytes.  Any output pointer may be NULL.
 */
stencil_status stencil_layout(stencil_t plan, int64_t padded[3], int64_t pitch[3],
                              int64_t origin[3], int64_t *bytes_per_field);

/*
 * stencil_step -- advance `nsteps` iterations (Sec. 2.4: f'_i = zeta(f^, i) for all i).
 *
 *   XCORR      nsteps sweeps of Eq. 3 (each sweep feeds the next).
 *   MAXFILTER  nsteps max-filter sweeps (each sweep feeds the next).
 *   DIFFUSION  nsteps forward-Euler steps of Eqs. 4-7.
 *   MHD8       nsteps RK3 steps (3 substeps each) of Eqs. A1-A4.
 *
 * fields_in / fields_out: nfields device pointers each, laid out per stencil_layout, in
 * the plan's storage type; in and out must not alias.  The result is in fields_out; the
 * interior of fields_in is not modified.  With STENCIL_BC_PERIODIC the halo of fields_in
 * is (re)filled first and the halo of fields_out is valid on return; with
 * STENCIL_BC_CALLER the halo of fields_in must be filled by the caller, nsteps must be 1
 * and the kind must be XCORR, MAXFILTER or DIFFUSION; with STENCIL_BC_PERIODIC_XY (DIFFUSION
 * only -- MHD8 z-slabs use stencil_substep) nsteps must be 1, the caller supplies the z halo
 * of fields_in and the library its x/y images.  Asynchronous on `stream`: no host sync, no
 * allocation, safe to capture in a CUDA graph.  Bounded device waits that expire are
 * reported by the next stencil_sync / stencil_field_norms on the plan.
 */
stencil_status stencil_step(stencil_t plan, void *const *fields_in, void *const *fields_out,
                            int nsteps, void *stream);

/*
 * stencil_step_host -- stencil_step with the fields in host memory, for callers that keep
 * their state on the host: copies each host_in field (nfields arrays of bytes_per_field bytes
 * in the plan's padded layout, see stencil_layout; only the interior is significant for
 * periodic plans) into dev_in, runs stencil_step(dev_in -> dev_out, nsteps), and copies each
 * dev_out field back into host_out.  dev_in / dev_out are caller-owned device field sets as
 * for stencil_step (dev_in is overwritten).  Host arrays should be page-locked for the copies
 * to run asynchronously.  Synchronises `stream` before returning; errors as stencil_step,
 * ETIMEOUT as stencil_sync.  (Sec. 2.4: f' = zeta(f^) evaluated on the device, the arrays
 * staged through it.)
 */
stencil_status stencil_step_host(stencil_t plan, const void *const *host_in, void *const *host_out,
                                 void *const *dev_in, void *const *dev_out, int nsteps, void *stream);

/* stencil_halo_fill -- fill the halo of each field with the periodic image of its interior
 * (Eq. 2 with periodic beta).  No-op for STENCIL_BC_CALLER; for STENCIL_BC_PERIODIC_XY only the
 * x/y images, on every padded plane (the z-halo planes included, from their own cells).
 * Asynchronous on `stream`. */
stencil_status stencil_halo_fill(stencil_t plan, void *const *fields, void *stream);

/*
 * stencil_substep -- one substep s (0, 1, 2) of the 3-stage Runge-Kutta step of an MHD8 plan
 * (Sec. 3.3; the 2N-storage scheme w <- alpha_s w + dt RHS(f), f <- f + beta_s w of Eqs. A1-A4).
 *
 * Three calls with s = 0, 1, 2, ping-ponging fields_in / fields_out, equal one
 * stencil_step(nsteps = 1).  It exists for decomposed grids (STENCIL_BC_PERIODIC_XY), whose z
 * halo must be exchanged between substeps; it also accepts periodic plans.  The RK register w
 * lives in the plan and carries from substep to substep; for FP32/BF16 storage the Kahan
 * terms are cleared at s = 0.  fields_in / fields_out: 8 device pointers each in the plan's
 * layout, not aliasing.  The halo of fields_in is (re)filled first per the plan's boundary
 * mode.  Asynchronous on `stream`; EINVAL for a non-MHD8 plan or s outside 0..2.
 */
stencil_status stencil_substep(stencil_t plan, void *const *fields_in, void *const *fields_out,
                               int substep, void *stream);

/*
 * stencil_mhd_rhs -- evaluate only the MHD right-hand side phi(gamma(psi(f))) (Sec. 3.3,
 * Eqs. 8-9; Eqs. A1-A4) without time integration.  MHD8 plans only.
 *
 * fields: 8 device pointers in the plan's layout with a valid halo (periodic plans refill
 * it first).  rhs: 8 device pointers to DENSE interior arrays (nx * ny * nz, x fastest) of
 * the plan's compute type (double for F64, float otherwise).  Asynchronous on `stream`.
 */
stencil_status stencil_mhd_rhs(stencil_t plan, void *const *fields, void *const *rhs,
                               void *stream);

/*
 * stencil_field_norms -- per-field reductions over the interior, accumulated in FP64 on
 * the device: out[3*f + 0] = sum f, out[3*f + 1] = sum f^2, out[3*f + 2] = max |f|.  For
 * MHD8 plans out[3*nfields] additionally receives the mass sum exp(lnrho) * dx*dy*dz.
 * `out` is a host array of 3*nfields (+1 for MHD8) doubles.  Synchronises `stream`; returns
 * STENCIL_ETIMEOUT if an earlier kernel on this plan reported an expired wait.
 */
stencil_status stencil_field_norms(stencil_t plan, void *const *fields, double *out,
                                   void *stream);

/*
 * stencil_field_norms_noalloc -- the reductions of stencil_field_norms, for callers that
 * cannot allocate device memory.  The paper has no counterpart: this is an addition of the
 * library.
 *
 * Which callers: a serving loop that has committed its whole HBM budget to resident fields
 * and must not allocate while requests are in flight (an allocation can fail, or
 * synchronise the device), and applications whose device memory is owned by another
 * allocator.  The call needs no plan (creating a plan allocates) and calls no cudaMalloc,
 * cudaFree or allocating library routine.  Its scratch, the pass-1 partials of the two-pass
 * FP64 reduction, is a fixed file-scope device array of 77 824 bytes.  Every GPU that loads
 * the library holds that array until the process exits.
 *
 *   fields        nfields device pointers, each a padded field laid out as stencil_layout
 *                 describes, element type `storage` (I32, F64, F32 or BF16)
 *   nfields       1..8; a larger value returns STENCIL_EINVAL (the array holds 8 fields)
 *   dims          interior extents (nx, ny, nz), 1 on unused axes
 *   padded        padded extents, origin: interior origin -- as stencil_layout reports them
 *   mass_volume   if > 0, out_dev[3*nfields] = sum exp(field 0) * mass_volume (the MHD mass)
 *   out_dev       DEVICE array of 3*nfields doubles (+1 when mass_volume > 0), written in
 *                 stream order as {sum f, sum f^2, max |f|} per field
 *   stream        cudaStream_t as void*; the call returns without synchronising
 *
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current.  Make that first call before any stream capture.  All calls
 * share the one array, and each call overwrites every slot it later reads, so nothing
 * carries over from the previous call.  Calls whose work overlaps on the GPU (different
 * streams, or different host threads) race on the array and give wrong results: serialise
 * them.  Errors: STENCIL_EINVAL for invalid arguments (detail via
 * stencil_last_error_detail(NULL)), STENCIL_ECUDA if a launch fails.
 */
stencil_status stencil_field_norms_noalloc(void *const *fields, int nfields, stencil_dtype storage,
                                           const int64_t dims[3], const int64_t padded[3],
                                           const int64_t origin[3], double mass_volume,
                                           double *out_dev, void *stream);

/*
 * stencil_selftest_wait -- exercise the failure-detection path of the bounded device waits.
 * Launches one CTA that waits on an mbarrier that nothing will ever complete, for at most
 * limit_ns nanoseconds (clamped to 1 us .. 2 s).  The expiry is recorded exactly like a
 * timed-out wait in a stencil kernel: the next stencil_sync (or stencil_field_norms) on
 * the plan returns STENCIL_ETIMEOUT and clears it.  Nothing faults or hangs and the CUDA
 * context stays usable.  The paper has no counterpart; this exists for testing.
 */
stencil_status stencil_selftest_wait(stencil_t plan, int64_t limit_ns, void *stream);

/* stencil_sync -- synchronise `stream` and report (then clear) any expired device wait
 * recorded by this plan's kernels since the last check. */
stencil_status stencil_sync(stencil_t plan, void *stream);

/*
 * Kernel variants and runtime autotuning.  Each kind has a small table of kernel variants
 * (tile shape, pipeline depth, z-chunk length).  2D FP32 DIFFUSION also has temporally
 * blocked variants (1: two, 2: four Euler steps per pass over the field, the remainder one
 * step at a time); they apply with periodic boundaries and nx a multiple of 4 and otherwise
 * run the one-step kernel, with the same results.  As in the paper's automated tuning of the
 * thread-block decomposition (Sec. 5.1), stencil_autotune times every variant on the
 * caller's buffers (one warm-up call, then `reps` timed calls of stencil_step(nsteps) with
 * CUDA events on `stream`), discards variants that fail to launch, and keeps the fastest.
 * For the z-streaming 3D kernels (DIFFUSION in 3D, MHD8) the search also covers the z-chunk
 * length each CTA streams: the kernel's own choice, half of it, or twice it.  It overwrites
 * fields_out and synchronises `stream`.
 *
 * 3D FP32 DIFFUSION has each tile shape in two schedules: one launch per Euler step, and a
 * persistent schedule (variant names ending in "_persist") that runs all nsteps steps of a
 * stencil_step call in one cooperative launch, each tile waiting only for the tiles whose
 * cells it reads to finish the previous step (bounded waits; an expired wait ends the call
 * with STENCIL_ETIMEOUT from the next synchronising call).  Results are bit-identical to the
 * per-step schedule.  Its synchronisation words are allocated by the plan on first use
 * (24 bytes + 8 bytes per tile), so the first call must not be made while `stream` is
 * being captured into a CUDA graph (EINVAL); later calls may be captured.  Two calls of one
 * plan must not run concurrently on different streams.
 *
 * The winner is remembered for the problem class -- GPU name and SM count, kind, storage,
 * radius, boundary, dims and nsteps -- for the rest of the process and, when the environment
 * variable STENCIL_AUTOTUNE_CACHE names a writable file, in that file (one line appended per
 * tuned class; read on first use).  A later stencil_autotune of the same class takes the
 * remembered choice without timing anything.  stencil_autotune_status reports whether the
 * current choice came from that cache (1) or from timing (0), its z-chunk mode (0, 1, 2) and
 * the time of one stencil_step(nsteps) call it measured (ms); outputs may be NULL.
 *
 * stencil_get_variant reports the current variant, the number of variants and the current
 * variant's name (static string); any output pointer may be NULL.  stencil_set_variant selects
 * one (EINVAL if out of range), stencil_set_zmode a z-chunk mode (0 for plans of other kinds;
 * EINVAL if out of range).  Neither changes the results, only how the work is tiled.
 */
stencil_status stencil_get_variant(stencil_t plan, int *variant, int *count, const char **name);
stencil_status stencil_set_variant(stencil_t plan, int variant);
stencil_status stencil_autotune(stencil_t plan, void *const *fields_in, void *const *fields_out,
                                int nsteps, int reps, void *stream);
stencil_status stencil_autotune_status(stencil_t plan, int *from_cache, int *zmode, float *ms);
stencil_status stencil_set_zmode(stencil_t plan, int zmode);

/*
 * Continuous-batching server.  Many independent problems of different kinds and sizes are
 * resident on the device at once and are advanced together: each iteration runs one step
 * of every active problem (a heat Euler step, an MHD RK3 step, or a cross-correlation
 * sweep) through one persistent batched launch per kind.  Problems are admitted in arrival
 * order while an HBM byte budget and an active-slot limit allow, so requests that arrive
 * while others run join the batch as memory and slots free up.  Storage and arithmetic are
 * FP32 (MHD with Kahan-compensated RK); boundaries are periodic, radius 3.  None of this is
 * in the paper: it is the serving layer of this library.
 *
 * A server belongs to the device current at creation and issues all work on `stream`.
 * Calls on one server must come from one host thread at a time.
 */
typedef struct stencil_server *stencil_server_t;

typedef struct stencil_request {
    stencil_kind kind;     /* XCORR (1D, dims[0] cells), DIFFUSION or MHD8 (3D) */
    int64_t dims[3];       /* interior extents: 1D 7 .. 2^31-16; 3D each 7 .. 2^15 */
    int nsteps;            /* sweeps / Euler steps / RK3 steps, >= 1 */
    double coeffs[7];      /* XCORR: weights g_{-3..3}; ignored otherwise */
    stencil_params params; /* DIFFUSION and MHD8 constants (as for stencil_create) */
} stencil_request;

enum { STENCIL_REQ_PENDING = 0, STENCIL_REQ_ACTIVE = 1, STENCIL_REQ_COMPLETING = 2, STENCIL_REQ_DONE = 3,
       STENCIL_REQ_CANCELLED = 4 };

/* Create a server with an HBM budget (bytes of problem data resident at once) and at most
 * max_active problems in flight.  Allocates only small tables; problem memory comes from
 * the device's stream-ordered memory pool at admission. */
stencil_status stencil_server_create(int64_t hbm_budget_bytes, int max_active, void *stream,
                                     stencil_server_t *out);
/* Release the server and every problem's device memory (synchronises its stream). */
void stencil_server_destroy(stencil_server_t server);
/*
 * Queue a problem.  host_in / host_out: nfields (1, or 8 for MHD8) host arrays of
 * dims[0]*dims[1]*dims[2] floats, dense, x fastest.  host_in is read when the problem is
 * admitted and host_out written when it completes; both must stay valid until the ticket
 * reports STENCIL_REQ_DONE, and should be page-locked so that the copies are asynchronous.
 * EINVAL if the request is malformed or needs more memory than the whole budget.
 */
stencil_status stencil_server_submit(stencil_server_t server, const stencil_request *req,
                                     const float *const *host_in, float *const *host_out,
                                     int64_t *ticket);
/* One scheduling iteration: retire finished copy-backs, admit pending problems, launch one
 * step of every active problem, queue copy-back of problems that reached nsteps.  Returns
 * without waiting for the GPU.  Any output pointer may be NULL. */
stencil_status stencil_server_progress(stencil_server_t server, int *n_pending, int *n_active,
                                       int *n_done);
/* Name of the batched kernel's tile shape this server runs for `kind` (static string).  The
 * heat and MHD kernels each come in two tile shapes; at creation the server takes the shape of
 * the per-grid variant that stencil_autotune last chose for an FP32 periodic radius-3 plan of
 * that kind on this GPU (this process, or the STENCIL_AUTOTUNE_CACHE file), else the default. */
const char *stencil_server_variant(stencil_server_t server, stencil_kind kind);
/* State of a ticket (STENCIL_REQ_*). */
stencil_status stencil_server_poll(stencil_server_t server, int64_t ticket, int *state);
/*
 * Cancel a problem that has not started its copy-back.  A pending problem leaves the queue;
 * an active one leaves the batch before the next iteration, and its device memory returns to
 * the pool in stream order (after the iteration already launched).  Its host_out arrays are
 * never written, and host_in / host_out may be released once this returns.  The ticket then
 * reports STENCIL_REQ_CANCELLED.  EINVAL for an unknown ticket or one already COMPLETING, DONE
 * or CANCELLED.
 */
stencil_status stencil_server_cancel(stencil_server_t server, int64_t ticket);
/* Bytes resident now, the peak, and cells x steps of all finished problems. */
stencil_status stencil_server_stats(stencil_server_t server, int64_t *bytes_in_use,
                                    int64_t *peak_bytes, int64_t *cell_updates_done);
/* Synchronise the server's stream; STENCIL_ETIMEOUT if a bounded wait expired in a kernel. */
stencil_status stencil_server_sync(stencil_server_t server);
/* Detail of the last failure on `server` (or of the last failed create when NULL). */
const char *stencil_server_last_error_detail(stencil_server_t server);

/* Human-readable name of a status code (static string). */
const char *stencil_strerror(stencil_status status);

/* Detail of the last failure on `plan` (or, when plan is NULL, of the last failed
 * stencil_create or plan-free call on this host thread).  Valid until the next call. */
const char *stencil_last_error_detail(stencil_t plan);

/* ABI version of the loaded library (STENCIL_ABI_VERSION at build time). */
int stencil_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* STENCIL_H */
