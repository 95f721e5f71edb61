/*
 * lwacm.h — C ABI of the GB300 (sm_103a) Link-wise Artificial Compressibility
 * Method library (Asinari, Ohwada, Chiavazzo, Di Rienzo, "Link-wise Artificial
 * Compressibility Method").
 *
 * The method (Section 2.1, Eq. ACM2.0) advances only the hydrodynamic fields
 * (rho, u) of every lattice node:
 *
 *   f_i(x,t+1) = f_i^(e)(x - c_i, t)
 *              + 2(omega-1)/omega [ f_i^(e,o)(x,t) - f_i^(e,o)(x - c_i,t) ]
 *   rho(x,t+1) = sum_i f_i(x,t+1),   rho u(x,t+1) = sum_i c_i f_i(x,t+1)
 *
 * with the second-order equilibrium of Eq. d2q9_equilibrium_compact (D2Q9; the
 * same form with the weights of Eq. weight_factors_3d for D3Q19), its odd part
 * Eq. feqo, and omega from the viscosity by Eq. viscosity2,
 * nu = (1/omega - 1/2)/3. Populations f_i are never stored.
 *
 * Conventions (all entry points):
 *   - Every call returns an lwacm_status; nothing throws, aborts or exits.
 *   - Fields are structure-of-arrays, one array per field, x fastest:
 *     element (x,y,z) of a field is at [(z*ny + y)*nx + x]. The density field
 *     is stored as d = rho - 1 (not rho), so that no O(1) constant enters the
 *     single-precision sums. D2Q9 has nz = 1 and no uz field.
 *   - Device memory belongs to the caller: the library never allocates or frees
 *     device memory. The caller binds one workspace (lwacm_bind) that holds the
 *     two ping-pong state buffers (Section 2.4: two arrays, toggled each step),
 *     a staging area and reduction scratch.
 *   - Work is enqueued asynchronously on the bound stream. Asynchronous CUDA
 *     errors surface at the next lwacm_sync / lwacm_diagnostics /
 *     lwacm_get_fields call.
 *   - Errors are sticky per context: after LWACM_E_CUDA only lwacm_last_error
 *     and lwacm_destroy are valid.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef LWACM_H
#define LWACM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lwacm_ctx lwacm_ctx; /* opaque; owned by the library */

typedef enum {
    LWACM_OK = 0,
    LWACM_E_ARG = 1,         /* bad argument: null pointer, bad lattice/bc/dtype/size */
    LWACM_E_RANGE = 2,       /* nu outside (0, 1/6], i.e. omega outside [1, 2) */
    LWACM_E_STATE = 3,       /* call order: e.g. step before bind/set_fields */
    LWACM_E_NOMEM = 4,       /* the bound workspace is smaller than required */
    LWACM_E_CUDA = 5,        /* a CUDA runtime error (sticky; see lwacm_last_error) */
    LWACM_E_NONFINITE = 6,   /* diagnostics found a non-finite field value */
    LWACM_E_TIMEOUT = 7,     /* a bounded device-side wait gave up */
    LWACM_E_UNSUPPORTED = 8  /* valid request this build does not implement */
} lwacm_status;

enum { LWACM_D2Q9 = 9, LWACM_D3Q19 = 19 };

/* Boundary types.
 *   PERIODIC: every axis periodic (Section 2.5).
 *   CAVITY:   half-way link-wise walls on every face (Section 2.6, Eq. ACM2.0cccbb2),
 *             the top face of the last axis (y in 2D, z in 3D) moving with the lid
 *             velocity through Eq. ACM2.0ccccbb (lid corners take the lid velocity,
 *             Section 2.6.1).
 *   CHANNEL:  half-way walls at y = -1/2 and y = ny - 1/2, other axes periodic; the
 *             top wall moves with the lid velocity (zero by default: Poiseuille
 *             with a body force, plane Couette with a lid). */
enum { LWACM_BC_PERIODIC = 0, LWACM_BC_CAVITY = 1, LWACM_BC_CHANNEL = 2 };

/* Element types, for storage and for field transfer. */
enum { LWACM_F32 = 0, LWACM_BF16 = 1, LWACM_F16 = 2, LWACM_F64 = 3 };

/* Where a transfer buffer lives. */
enum { LWACM_DEVICE = 0, LWACM_HOST = 1 };

/* Option keys for lwacm_set_option (values are doubles). */
enum {
    LWACM_OPT_LID_X = 0,   /* lid / moving-wall velocity u_w (lattice units) */
    LWACM_OPT_LID_Y = 1,
    LWACM_OPT_LID_Z = 2,
    LWACM_OPT_FORCE_X = 3, /* body acceleration g of Eq. force (lattice units) */
    LWACM_OPT_FORCE_Y = 4,
    LWACM_OPT_FORCE_Z = 5,
    LWACM_OPT_RHO0 = 6,    /* rho_0 of the moving-wall term, Eq. ACM2.0movebb (default 1) */
    LWACM_OPT_STORAGE = 7, /* storage element type: LWACM_F32 (default), BF16, F16;
                              only before lwacm_bind */
    LWACM_OPT_GRAPH_CHUNK = 8, /* steps per captured CUDA graph in lwacm_step (even;
                                  0 disables graphs; default 64) */
    LWACM_OPT_KERNEL = 9,  /* interior kernel: 0 = automatic choice (default),
                              1 = generic gather kernel, 5 = D3Q19 half-row TMA kernel
                              (needs the plain scheme, with or without a constant
                              acceleration but not a force field, nx = 128, 256 or
                              nx >= 72 a multiple of 4 (8 for BF16 / FP16 storage)
                              with nx % 128 == 0 or >= 8, any ny, and runs walled
                              domains with the wall pass
                              after it; FP32, BF16 and FP16 storage: LWACM_E_UNSUPPORTED
                              otherwise); 2 and 3 (earlier row-tiled kernels, superseded
                              by 5) are retired: LWACM_E_ARG; 6 = D2Q9 2D-tile kernel (any boundary, walls
                              and forcing applied in the kernel; omega_p and the
                              bulk-viscosity variant (alone or together) on periodic
                              domains; not the scalar; tile shape from
                              LWACM_OPT_BATCH_TILE, 30x14 when 0). The automatic choice
                              takes 5, else 6, else 1. */
    LWACM_OPT_BATCH_MODE = 10, /* batched contexts: 0 = one launch per step, replayed
                                  from CUDA graphs (default); 1 = one persistent
                                  cooperative launch per lwacm_step call, with a
                                  bounded grid-wide barrier between steps */
    LWACM_OPT_TEST_WITHHOLD = 11, /* batched contexts, tests only: in persistent mode the
                                     first CTA leaves without arriving at the barrier after
                                     this step (-1 = never), so the other CTAs' bounded
                                     waits run out and lwacm_sync reports LWACM_E_TIMEOUT */
    LWACM_OPT_FORCE_FIELD = 12,   /* 1 = reserve room in the workspace for a per-node
                                     acceleration field (lwacm_set_force_field); only
                                     before lwacm_bind; single-domain contexts only */
    LWACM_OPT_BATCH_TILE = 13,    /* how domains are cut into CTA tiles. Batched contexts:
                                     0 (default) = runs of 256 consecutive nodes, one
                                     thread per node, every lattice; 1..6 = 2D tiles of
                                     30x6, 30x14, 62x6, 30x30, 62x14, 126x6 nodes, D2Q9
                                     only (LWACM_E_UNSUPPORTED otherwise), with the link
                                     values computed once per node and exchanged in
                                     shared memory. Single D2Q9 contexts: the shape of
                                     kernel 6. Any time; lwacm_autotune picks one. */
    LWACM_OPT_NU_P = 14,          /* viscosity nu_p of the pressure (density) update,
                                     i.e. omega_p of Section 2.2 item 3 (Eq. FDcompact c
                                     relaxed with omega_p, momentum with omega): in (0,
                                     1/6], or 0 = nu (default). Single periodic domains
                                     only (LWACM_E_UNSUPPORTED otherwise); runs on the
                                     D2Q9 2D-tile kernel, else on the generic kernel;
                                     the adjoint refuses nu_p != nu. */
    LWACM_OPT_SCALAR_ALPHA = 15,  /* > 0: carry a passive scalar T (Eq. ACM2.0t, the
                                     thermal LW-ACM of Appendix "Asymptotic analysis for
                                     energy equation") with diffusivity alpha in (0, 1/6]
                                     (alpha = (1/omega_t - 1/2)/3, Eq. diffusivity2),
                                     advected by the flow velocity at each step's time
                                     level; 0 = none (default). Before lwacm_bind (it
                                     adds one field to the workspace); single periodic
                                     domains only; runs on the generic kernel. */
    LWACM_OPT_BULK_GAMMA = 16,    /* gamma in (-1, 1), 0 = off (default): the bulk-
                                     viscosity variant of Appendix "Computing derivatives
                                     locally", Eq. quasi-equilibrium2. The equilibrium of
                                     Eq. ACM2.0 becomes f^(e) plus the change of the
                                     product-form quasi-equilibrium (Eqs.
                                     d2q9_equilibrium_gen, quasi-equilibrium) when its
                                     trace moves from Tr^(e) = 2/3 + |u|^2 to Tr^(e) +
                                     gamma (Tr^(+) - Tr^(e)), Tr^(+) the trace of
                                     sum_i c_i c_i f_i over rho of the node's last update,
                                     carried as the field Tr^(+) - Tr^(e)
                                     (lwacm_get_trace; lwacm_set_fields sets it to zero).
                                     On a linear longitudinal wave
                                     of wave number k the extra damping per step is
                                     nu gamma k^2 / (1 - gamma) (bulk viscosity raised by
                                     2 rho0 nu gamma / (1 - gamma)); shear waves are
                                     unchanged. Before lwacm_bind (one more field);
                                     periodic D2Q9 domains only, not with the scalar
                                     (LWACM_E_UNSUPPORTED). With LWACM_OPT_NU_P the density
                                     is relaxed with omega_p and the momentum and the
                                     trace with omega. Runs on the D2Q9 2D-tile kernel. */
    LWACM_OPT_SEMI_IMPLICIT = 17, /* 1: semi-implicit pressure update (Section 2.2 item 2,
                                     Eq. FDcompact_si), 0 = explicit (default). The
                                     velocity is that of the explicit step; the density
                                     is then summed again with every link value built
                                     from the old density and the new velocity (one more
                                     pass per step, after the interior kernel). Single
                                     periodic domains, D2Q9 and D3Q19, with or without
                                     forcing and LWACM_OPT_NU_P (the density then uses
                                     nu_p); not with the passive scalar, the
                                     bulk-viscosity variant or the adjoint
                                     (LWACM_E_UNSUPPORTED). */
    LWACM_OPT_STOCHASTIC_ROUNDING = 18 /* 1: BF16 / FP16 stores rounded stochastically,
                                     0 = to nearest (default). A value between two
                                     neighbours of the storage type is stored as the one
                                     further from zero with probability equal to its
                                     distance from the nearer-to-zero one over their
                                     spacing (16 random bits per value from a counter-
                                     based hash of the node, the field and a step counter
                                     kept in the workspace), so that stored values are
                                     unbiased and a per-step change below half a storage
                                     ulp is not lost. Single periodic D3Q19 domains with
                                     BF16 / FP16 storage on the half-row kernel (nx as
                                     for LWACM_OPT_KERNEL 5), plain scheme only (no forcing,
                                     nu_p, scalar, bulk variant or semi-implicit update);
                                     otherwise LWACM_E_UNSUPPORTED, at set_option, bind
                                     or step. Runs are reproducible: the counter starts at
                                     0 at lwacm_bind. */
};

/* Create a single-domain context.
 *   lattice: LWACM_D2Q9 or LWACM_D3Q19; nx, ny, nz >= 1 (nz == 1 for D2Q9;
 *   walled axes need >= 2 nodes); nu: kinematic viscosity in lattice units,
 *   0 < nu <= 1/6 (the stable range 1 <= omega < 2 of Section 2.3) -> otherwise
 *   LWACM_E_RANGE; bc: LWACM_BC_*. On success *out receives a new context. No
 *   device work is done. */
lwacm_status lwacm_create(int lattice, int nx, int ny, int nz, double nu, int bc,
                          lwacm_ctx **out);

/* Create a context holding n independent periodic domains (batched ensemble):
 * domain b has nx[b] x ny[b] x nz[b] nodes (nz may be NULL for D2Q9) and
 * viscosity nu[b] (each checked as in lwacm_create); bc must be
 * LWACM_BC_PERIODIC (else LWACM_E_UNSUPPORTED). The domains are packed one after
 * the other: every field array of the context (lwacm_set_fields, lwacm_get_fields,
 * lwacm_fields) holds domain 0's nodes, then domain 1's, ..., each x fastest;
 * lwacm_diagnostics sums over all of them. One lwacm_step advances every domain. */
lwacm_status lwacm_batch_create(int lattice, int n, const int *nx, const int *ny, const int *nz,
                                const double *nu, int bc, lwacm_ctx **out);

/* offsets[0..n]: first packed node of each domain, then the total node count
 * (n = 1 for a single-domain context). */
lwacm_status lwacm_batch_offsets(const lwacm_ctx *ctx, long long *offsets);

/* Set an option (LWACM_OPT_*). Storage type changes are refused after bind
 * (LWACM_E_STATE). */
lwacm_status lwacm_set_option(lwacm_ctx *ctx, int key, double value);

/* Number of workspace bytes lwacm_bind needs for the current options. */
lwacm_status lwacm_workspace_bytes(const lwacm_ctx *ctx, size_t *bytes);

/* Bind caller-owned device memory (>= lwacm_workspace_bytes, 256-byte aligned)
 * and a CUDA stream (cudaStream_t cast to void*, NULL = legacy default stream).
 * The memory must stay valid until lwacm_destroy or the next bind. Fields are
 * undefined until lwacm_set_fields. */
lwacm_status lwacm_bind(lwacm_ctx *ctx, void *dev_workspace, size_t bytes, void *cuda_stream);

/* Copy an initial state in. d, ux, uy, uz are arrays of nx*ny*nz elements of
 * type dtype (LWACM_F32 or LWACM_F64) on the device or on the host (where =
 * LWACM_DEVICE / LWACM_HOST; host memory should be pinned for asynchronous
 * copies). uz must be NULL for D2Q9. The values are rounded once to the storage
 * type by a device kernel. Resets the step counter. Stream-ordered: host
 * buffers must stay valid until the stream reaches this point. */
lwacm_status lwacm_set_fields(lwacm_ctx *ctx, const void *d, const void *ux, const void *uy,
                              const void *uz, int dtype, int where);

/* Per-node body acceleration g(x) of Eq. force (Section 2.1), for a force that
 * varies in space (and, by calling this between steps, in time: Eq. force uses g
 * at the time level t of the state it updates, so set g(x, t) before the step
 * from t to t+1). gx, gy (and gz for D3Q19; NULL for D2Q9) are arrays of
 * nx*ny*nz elements of type dtype (LWACM_F32 or LWACM_F64) on the device or
 * host (where); they are copied (FP64 rounded once to FP32) into the workspace
 * room reserved by LWACM_OPT_FORCE_FIELD and used by every following step until
 * the next call. The step adds rho(x,t) g(x) to the momentum, on top of any
 * constant LWACM_OPT_FORCE_* vector. All three pointers NULL switches the field
 * off. Stream-ordered on the bound stream (host buffers must stay valid until
 * the stream reaches this point; FP32 host arrays should be pinned). The D3Q19
 * row-tiled kernels have no forcing term, so a D3Q19 context with forcing runs
 * the generic kernel; D2Q9 runs the 2D-tile kernel, which adds it. The adjoint (lwacm_forward_record) refuses a context whose field is on
 * (LWACM_E_UNSUPPORTED).
 * Errors: LWACM_E_STATE (nothing reserved, or not bound), LWACM_E_ARG. */
lwacm_status lwacm_set_force_field(lwacm_ctx *ctx, const void *gx, const void *gy, const void *gz,
                                   int dtype, int where);

/* The passive scalar T of LWACM_OPT_SCALAR_ALPHA: copy nx*ny*nz values of type
 * dtype (LWACM_F32 / LWACM_F64) in from, or out to, the device or the host (where),
 * rounded to the storage type on the way in. lwacm_set_fields sets the scalar to
 * zero, so call lwacm_set_scalar after it. Stream-ordered; lwacm_get_scalar
 * synchronises when where == LWACM_HOST. Errors: LWACM_E_STATE (no scalar, not
 * bound, or fields not set), LWACM_E_ARG. */
lwacm_status lwacm_set_scalar(lwacm_ctx *ctx, const void *T, int dtype, int where);
lwacm_status lwacm_get_scalar(lwacm_ctx *ctx, void *T, int dtype, int where);

/* The trace deviation Tr^(+) - Tr^(e) of LWACM_OPT_BULK_GAMMA (nx*ny values, as
 * lwacm_get_scalar): Tr^(+) the trace of sum_i c_i c_i f_i over rho of each node's
 * last update, Tr^(e) = 2/3 + |u|^2 of the current state. LWACM_E_STATE without
 * the variant. */
lwacm_status lwacm_get_trace(lwacm_ctx *ctx, void *T, int dtype, int where);

/* Advance the state by n >= 0 time steps of Eq. ACM2.0 (plus the wall pass of
 * Eqs. ACM2.0cccbb2 / ACM2.0ccccbb and the forcing of Eq. force when enabled).
 * Asynchronous on the bound stream; long runs are replayed from captured CUDA
 * graphs. */
lwacm_status lwacm_step(lwacm_ctx *ctx, long long n);

/* Capture and instantiate now the CUDA graph that lwacm_step(ctx, n) would replay
 * from the current state's buffer (none when n is below the graph chunk or graphs
 * are off), without advancing the state: lwacm_step builds it on first use, and a
 * caller that times or serves steps can take that one-time cost beforehand. The
 * graph stays valid until an option changes. Needs a bound context with fields set
 * (LWACM_E_STATE); n < 0: LWACM_E_ARG. */
lwacm_status lwacm_prepare(lwacm_ctx *ctx, long long n);

/* Borrowed device pointers to the current state (zero copy). Valid until the
 * next lwacm_step / lwacm_set_fields / lwacm_bind / lwacm_destroy. *dtype gets
 * the storage type, *pitch_elems the row pitch in elements (== nx). uz may be
 * NULL; *uz is NULL for D2Q9. */
lwacm_status lwacm_fields(lwacm_ctx *ctx, void **d, void **ux, void **uy, void **uz,
                          int *dtype, long long *pitch_elems);

/* Copy the current state out, converted by a device kernel to dtype
 * (LWACM_F32 or LWACM_F64), into device or host arrays (where). Synchronises
 * the bound stream when where == LWACM_HOST. */
lwacm_status lwacm_get_fields(lwacm_ctx *ctx, void *d, void *ux, void *uy, void *uz, int dtype,
                              int where);

/* As lwacm_get_fields, but only enqueued: with where == LWACM_HOST the copies
 * are in flight when the call returns, and the host arrays hold the state once
 * the bound stream has reached them (lwacm_sync, or a synchronisation of that
 * stream). Host arrays must be page-locked for the copies to overlap other work,
 * and must stay allocated and untouched until then. Lets a caller stream
 * independent problems through several contexts on several streams, one
 * problem's copy back overlapping the next one's copy in. Same arguments and
 * errors as lwacm_get_fields. */
lwacm_status lwacm_get_fields_async(lwacm_ctx *ctx, void *d, void *ux, void *uy, void *uz, int dtype,
                                    int where);

/* FP64 global quantities of the current state (Eq. global.quantities):
 *   out[0] = sum d (mass minus the node count), out[1..3] = sum rho u_a,
 *   out[4] = 0.5 sum rho |u|^2, out[5] = max |u|, out[6] = 0.5 sum (ux+uy)^2,
 *   out[7] = 0.5 sum (ux-uy)^2 (the M_par / M_perp sums of Eq. 3Dmomenta before
 *   the volume factor, for a lid moving along the x = y diagonal of the top z
 *   plane; zero in 2D).
 * Deterministic two-pass device reduction in FP64; synchronises the stream.
 * Returns LWACM_E_NONFINITE (and still fills out) if any value is NaN/Inf. */
lwacm_status lwacm_diagnostics(lwacm_ctx *ctx, double out[8]);

/* ---- Adjoint (reverse-mode derivative of T steps) -----------------------------
 * The derivative of a scalar loss L of the state after T steps with respect to
 * the initial state (d, u) and to nu, by the chain rule through the moment form
 * of Eq. ACM2.0 (nu enters through a = 1 - 6 nu, Eq. ACM2.0nu, the 18 nu of the
 * pre-combined values and the 36 nu rho0 of the moving-wall term). One domain with
 * FP32 storage, any boundary (the wall rule of Eqs. ACM2.0cccbb2 / ACM2.0ccccbb is
 * differentiated too), optional constant forcing; a force field, omega_p != omega
 * or a passive scalar return LWACM_E_UNSUPPORTED. Memory is the caller's:
 * ceil(T/S) checkpoints of the state plus S+1 segment states and three lambda
 * states, S = stride (0 = ceil(sqrt(T))). */

/* Bytes of adjoint workspace lwacm_forward_record needs for T steps. */
lwacm_status lwacm_adjoint_workspace_bytes(const lwacm_ctx *ctx, long long T, int stride,
                                           size_t *bytes);

/* Advance the current state by T steps (as lwacm_step) while keeping a checkpoint
 * every S steps in the caller's device workspace (256-byte aligned, >=
 * lwacm_adjoint_workspace_bytes). The context then holds the state after T steps
 * and remembers the run for lwacm_backward; the workspace must stay valid until
 * then. */
lwacm_status lwacm_forward_record(lwacm_ctx *ctx, long long T, int stride, void *dev_workspace,
                                  size_t bytes);

/* Given lambda_T = dL/d(d, ux, uy[, uz]) at the end of the recorded run (device
 * arrays of nx*ny*nz elements of dtype LWACM_F32 or LWACM_F64; luz NULL in 2D),
 * write dL/d(d, ux, uy[, uz]) at its start into the device arrays gd, gux, guy,
 * guz (same dtype) and dL/dnu into *g_nu (host). Recomputes each segment from its
 * checkpoint and runs the adjoint step backwards through it; FP32 arithmetic,
 * FP64 accumulation of dL/dnu. Synchronises the bound stream. */
lwacm_status lwacm_backward(lwacm_ctx *ctx, const void *ld, const void *lux, const void *luy,
                            const void *luz, int dtype, void *gd, void *gux, void *guy, void *guz,
                            double *g_nu);

/* Number of completed steps since the last lwacm_set_fields. */
lwacm_status lwacm_step_count(const lwacm_ctx *ctx, long long *steps);

/* Wait for the bound stream and report any asynchronous CUDA error. */
lwacm_status lwacm_sync(lwacm_ctx *ctx);

/* Human-readable description of the last error on this context ("" if none).
 * The string is owned by the context. */
const char *lwacm_last_error(const lwacm_ctx *ctx);

/* Autotuner: measure the kernel configurations that can run this context and
 * keep the fastest (the paper has no counterpart; Section 2.4 discusses tuning the
 * implementation to the machine). The candidates are, for a batched context, every
 * tile layout (LWACM_OPT_BATCH_TILE) the lattice allows times both launch forms
 * (LWACM_OPT_BATCH_MODE); for a single domain, the interior kernels
 * (LWACM_OPT_KERNEL 5 and 1, and for D2Q9 kernel 6 in every tile shape) that
 * support it. Each is timed with CUDA events over
 * trial_steps steps (0 = 256) after a warm-up, from the rest state, on the bound
 * stream; the call synchronises.
 *
 * cache_path (or NULL): a JSON file mapping a problem key (lattice, storage, boundary,
 * shape or the ensemble's sizes and viscosities, forcing, SM count and compute
 * capability) to the chosen configuration. On a hit nothing is timed and the
 * recorded choice is applied; on a miss the measured choice is added (written to a
 * temporary file renamed over the cache). report (or NULL): receives a one-line JSON
 * record (key, "cache" or "measured", the choice, every candidate's time), cut to
 * report_bytes.
 *
 * Call after lwacm_bind and before lwacm_set_fields (LWACM_E_STATE otherwise): the
 * trial steps use the workspace and leave the fields unset. Errors: LWACM_E_ARG,
 * LWACM_E_STATE, LWACM_E_CUDA, LWACM_E_UNSUPPORTED (no candidate ran). */
lwacm_status lwacm_autotune(lwacm_ctx *ctx, const char *cache_path, int trial_steps, char *report,
                            size_t report_bytes);

/* Name of the interior kernel the context runs (for reports). */
const char *lwacm_kernel_name(const lwacm_ctx *ctx);

/* Release the context (host memory and CUDA graphs). Does not touch the bound
 * workspace, which belongs to the caller. NULL is allowed. */
void lwacm_destroy(lwacm_ctx *ctx);

/* Allocation-free diagnostics (the paper has no counterpart; this is a service
 * of the library).
 *
 * For callers that cannot allocate device memory or bind a workspace: code
 * running where cudaMalloc is forbidden or unavailable, or a tool that only sees
 * the field arrays of a running simulation. Computes the same eight FP64 global
 * quantities as lwacm_diagnostics, plus out_dev[8] = the number of nodes with a
 * non-finite value, from caller-owned device arrays d, ux, uy (and uz, or NULL for
 * 2D) of n nodes of type dtype (LWACM_F32, LWACM_BF16 or LWACM_F16), into the
 * caller-owned device array out_dev (9 doubles). Stream-ordered on `stream`
 * (cudaStream_t; NULL = legacy default stream); it does not synchronise.
 *
 * It allocates nothing: the per-block partial sums live in a fixed device array
 * of 72 KiB inside this library (held on every GPU that loads the library until
 * the process exits), which limits n to LWACM_NOALLOC_MAX_N nodes; larger n
 * returns LWACM_E_RANGE without launching anything. The first call on each
 * device looks up that array's device address (with the device current) and
 * keeps it for the life of the process, so make the first call on a device
 * before any stream capture; a cudaDeviceReset() of that device unloads the
 * library's device code and leaves the kept address stale, so do not call this
 * entry point on a device after resetting it. All calls share
 * the array: calls whose kernels overlap on the GPU (different streams, or
 * different host threads) race on it and must be ordered by the caller. Every
 * slot a call reads is written by that same call, so no clearing is needed.
 * Errors: LWACM_E_ARG (null pointer, n < 1, bad dtype), LWACM_E_RANGE,
 * LWACM_E_CUDA (launch failure). */
#define LWACM_NOALLOC_MAX_N 33554432LL
lwacm_status lwacm_diagnostics_noalloc(const void *d, const void *ux, const void *uy,
                                       const void *uz, long long n, int dtype, double *out_dev,
                                       void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LWACM_H */
