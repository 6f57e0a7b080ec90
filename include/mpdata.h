/*
 * mpdata.h -- C ABI of libmpdata_b300.so, a B300 (sm_103a) implementation of
 * one MPDATA advection time step on a structured, halo-padded 3D grid.
 *
 * The step (what the paper's MPDATA dwarf computes; Sec. 5, Listings 4-9):
 *   1. donor-cell pass: F(L,R,C) = max(C,0) L + min(C,0) R on the three face
 *      families (Listings 4/5 horizontally, Listing 7 vertically), then the
 *      flux divergence and solution advance psi1 = psi - (1/G) sum dF
 *      (Listings 8/9, G in the role of the density);
 *   2. iord-1 corrective passes: the antidiffusive pseudo-velocity
 *      Ut = (|U| - U^2/Gf) A - U (Vbar By + Wbar Bz)/Gf (Smolarkiewicz 1984,
 *      G-weighted per Smolarkiewicz & Margolin 1998; the paper defers these
 *      formulas to its companion deliverable, Sec. 5), optionally limited by
 *      the non-oscillatory option (Smolarkiewicz & Grabowski 1990), then the
 *      same flux divergence and advance.
 * Boundaries: periodic in i and j; the bottom face (k = -1/2) and the top
 * face (k = nz-1/2) carry no flux (the boundary factor pivbz = 0 of
 * Listing 7) whatever W holds there.  epsilon = 1e-15 in every ratio.
 *
 * Layout (every field, every call): a C-contiguous array
 * [nz+2h][ny+2h][nx+2h] of the context's dtype, i fastest, interior point
 * (i,j,k) at ((k+h)(ny+2h) + (j+h))(nx+2h) + (i+h).  Staggering follows the
 * C-grid convention of Sec. 3.1.4.1: U[k][j][i] is the face i+1/2, V[k][j][i]
 * the face j+1/2, W[k][j][i] the face k+1/2.  U, V, W are G-weighted Courant
 * numbers (mass fluxes in Courant units: U = G_face u dt/dx).
 *
 * Inputs are read at interior points only: the library applies the periodic
 * and closed boundaries itself, so input halos may hold anything.  Output
 * psi is written at interior points and its halo is filled (periodic in i
 * and j, edge copy in k), so the result is a consistent padded field.
 *
 * Pointers: field pointers are DEVICE pointers (cudaMalloc / torch CUDA
 * tensors) on the context's device, 16-byte aligned, unless a function says
 * HOST.  The caller owns every field buffer; the context owns only its
 * scratch memory, allocated in mpdata_init and freed in mpdata_destroy.
 *
 * Streams and errors: every call is asynchronous on the stream given to
 * mpdata_init (or mpdata_set_stream); none allocates or synchronises, except
 * the HOST-buffer call.  Arguments are checked on the host before any
 * launch; errors are negative return codes (never an abort or a device
 * trap).  A failure reported by the CUDA runtime returns MPDATA_ECUDA and
 * the runtime's message is kept for mpdata_last_error_string().
 */
#ifndef MPDATA_B300_H
#define MPDATA_B300_H

#include <stddef.h>

#if defined(__GNUC__)
#define MPDATA_API __attribute__((visibility("default")))
#else
#define MPDATA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpdata_ctx mpdata_ctx; /* opaque, library-owned */

enum mpdata_status {
  MPDATA_OK = 0,
  MPDATA_EINVAL = -1,  /* bad size, option or null pointer              */
  MPDATA_ENOMEM = -2,  /* scratch allocation failed                     */
  MPDATA_ECUDA = -3,   /* the CUDA runtime reported an error            */
  MPDATA_EALIGN = -4,  /* a field pointer is not 16-byte aligned        */
  MPDATA_EDEVICE = -5, /* no usable device                              */
  MPDATA_ERANGE = -6   /* a size beyond a documented maximum            */
};

enum mpdata_dtype { MPDATA_F64 = 0, MPDATA_F32 = 1 };
enum mpdata_kbc { MPDATA_K_ZEROFLUX = 0, MPDATA_K_PERIODIC = 1 };
enum mpdata_halo_kind {
  MPDATA_HALO_CELL = 0,  /* psi, G, U, V: periodic i-j, edge copy in k   */
  MPDATA_HALO_WFACE = 1  /* W: periodic i-j, closed faces (zero) in k    */
};
enum mpdata_variant {
  MPDATA_FUSED = 0,  /* one kernel per step, intermediates on chip         */
  MPDATA_STAGED = 1, /* one kernel per stage, intermediates in memory      */
  MPDATA_AUTO = 2    /* default: the faster of the two for the dtype on the
                        B300 (FP64: staged, since the fused kernel's halo
                        recompute costs FP64-pipe work, except the plain
                        step of a one-level grid of at most 128 x 128
                        columns, fused on 8 x 4 or 8 x 8 tiles; FP32:
                        fused)                                             */
};

/* Create a context for one grid.
 *   nx, ny, nz  interior sizes, each >= 1 (nz = 1 is a 2D problem);
 *   halo        h >= 1, and h >= 2 when iord >= 2 (the radius a corrective
 *               pass reads, so the output stays usable by h-radius stencils);
 *   iord        number of passes, 1 (donor cell only) to 8;
 *   nonoscillatory  0 or 1 (the limiter of every corrective pass);
 *   dtype       MPDATA_F64 or MPDATA_F32 (storage and arithmetic);
 *   k_bc        MPDATA_K_ZEROFLUX (closed top and bottom, Listing 7) or
 *               MPDATA_K_PERIODIC (k wraps like i and j; every vertical
 *               face carries flux, W at level k is the face k+1/2 and the
 *               one at nz-1 joins the top level to the bottom one);
 *   cuda_stream a cudaStream_t (NULL = the legacy default stream).
 * Allocates the scratch of one step on the current device.
 * Errors: EINVAL (sizes/options/out == NULL), EDEVICE, ENOMEM. */
MPDATA_API int mpdata_init(mpdata_ctx **out, int nx, int ny, int nz, int halo, int iord,
                int nonoscillatory, int dtype, int k_bc, void *cuda_stream);

/* Change the stream later calls are issued on. Errors: EINVAL. */
MPDATA_API int mpdata_set_stream(mpdata_ctx *c, void *cuda_stream);

/* Choose the kernel organisation (mpdata_variant); all give the same step
 * to rounding.  The fused kernel runs only when iord == 2 and nx, ny >= 2h,
 * and with an option set only in FP32; other contexts use the staged
 * kernels whatever is chosen.  Errors: EINVAL. */
MPDATA_API int mpdata_set_variant(mpdata_ctx *c, int variant);

/* Options of the corrective passes (bit flags).  The paper defers the
 * antidiffusive passes to the MPDATA literature (Sec. 5); these are that
 * literature's standard variants:
 *   DFL  the divergent-flow term (Smolarkiewicz 1984): each pseudo-velocity
 *        gains -(1/4) U (D_L + D_R) / G_face, D_c = the sum over the three
 *        directions of the cell's Courant-number differences (second order
 *        in divergent flows);
 *   ABS  signed fields: A and B are formed from |psi|, and the limiter
 *        applies its factors by the direction of each antidiffusive flux
 *        rather than of its velocity (identical results where psi >= 0);
 *   IGA  the infinite gauge (Smolarkiewicz & Clark 1986): the limit of the
 *        scheme applied to psi + c as c grows; the corrective flux of a face
 *        is (|U| - U^2/Gf)(psi_R - psi_L)/2 - U (Vbar N_y + Wbar N_z)/(8 Gf)
 *        with N the numerators of B.  A linear scheme, for signed fields.
 * IGA takes no other option and iord <= 2.  With an option an FP32 step
 * runs on a fused kernel (iord 2: the two-column one with the limiter on
 * and even nx and halo, else the one-column one) and an FP64 step on the
 * staged ones;
 * the adjoint calls (mpdata_adjoint_step, mpdata_step_tape,
 * mpdata_adjoint_step_tape) return EINVAL. */
enum mpdata_option { MPDATA_OPT_DFL = 1, MPDATA_OPT_ABS = 2, MPDATA_OPT_IGA = 4 };

/* Set the option bits of a context (0: the basic scheme, the default).
 * Errors: EINVAL (unknown bits, IGA with another option or iord > 2; the
 * options are left unchanged). */
MPDATA_API int mpdata_set_options(mpdata_ctx *c, int opts);
MPDATA_API int mpdata_get_options(mpdata_ctx *c, int *opts);

/* Advance psi (in/out, device) by nsteps MPDATA steps with Courant fields
 * u, v, w and metric g (device, read-only).  nsteps >= 0.  With the fused
 * kernels the steps alternate between psi and context scratch, and an odd
 * nsteps ends with a device copy back into psi.
 * Errors: EINVAL (null pointer, nsteps < 0), EALIGN, ECUDA. */
MPDATA_API int mpdata_step(mpdata_ctx *c, void *psi, const void *u, const void *v, const void *w,
                const void *g, int nsteps);

/* One step out of place: psi_out = step(psi_in), halo of psi_out filled;
 * psi_in is not modified.  The two buffers must be distinct (a caller that
 * double-buffers its state avoids the copy-back mpdata_step makes when the
 * fused kernels run an odd number of steps).
 * Errors: EINVAL (null pointer, psi_in == psi_out), EALIGN, ECUDA. */
MPDATA_API int mpdata_step_out(mpdata_ctx *c, const void *psi_in, void *psi_out, const void *u,
                               const void *v, const void *w, const void *g);

/* The same from HOST buffers: copies psi, u, v, w, g (padded, HOST) to
 * context-owned device buffers, runs nsteps steps, copies psi back to the
 * HOST buffer and waits for the stream.  The device buffers are allocated on
 * the first call (the only call besides init that allocates).
 * Errors: EINVAL, ENOMEM, ECUDA. */
MPDATA_API int mpdata_step_host(mpdata_ctx *c, void *psi_host, const void *u_host, const void *v_host,
                     const void *w_host, const void *g_host, int nsteps);

/* Pipelined HOST-buffer steps for a stream of problems (a library-interface
 * addition; the paper has none): enqueues, without waiting, the copies of
 * one problem's psi, u, v, w, g (padded, HOST, page-locked for the copies to
 * run asynchronously) to the device, nsteps steps on the context's stream,
 * and the copy of the result to psi_out_host (HOST; may equal psi_in_host).
 * Two problems are in flight: one problem's host-to-device copies run on a
 * copy stream while the previous problem steps and the one before that
 * copies its result back on a third stream, so a stream of problems runs at
 * the rate of the slowest of the three.  The host buffers of a problem must
 * stay untouched until mpdata_host_wait returns.  Device buffers (two sets of
 * five fields), the copy streams and their events are created on the first
 * call.  Errors: EINVAL, ENOMEM, ECUDA. */
MPDATA_API int mpdata_step_host_async(mpdata_ctx *c, const void *psi_in_host, void *psi_out_host,
                                      const void *u_host, const void *v_host,
                                      const void *w_host, const void *g_host, int nsteps);

/* The same for HOST arrays of the interior alone (a library-interface
 * addition): psi_in_host, psi_out_host, u_host, v_host, w_host and g_host
 * each hold the nx*ny*nz interior values, i fastest, then j, then k,
 * page-locked; psi_out_host receives the interior of the result.  Only the
 * interior crosses the host link (one 3D copy a field into the padded
 * device fields): the step reads no input halo and fills its output's.
 * It shares the device buffers, streams and in-flight limit of
 * mpdata_step_host_async.  Errors: EINVAL (also on a slab), ENOMEM, ECUDA. */
MPDATA_API int mpdata_step_host_interior_async(mpdata_ctx *c, const void *psi_in_host,
                                               void *psi_out_host, const void *u_host,
                                               const void *v_host, const void *w_host,
                                               const void *g_host, int nsteps);

/* Wait until every problem enqueued by mpdata_step_host_async or
 * mpdata_step_host_interior_async has been copied back.  Errors: EINVAL,
 * ECUDA. */
MPDATA_API int mpdata_host_wait(mpdata_ctx *c);

/* Adjoint (reverse mode) of one step, iord 1 or 2, with or without the
 * limiter: the derivative of a scalar cost J through the step.
 *   psi_n          the state the step started from (DEVICE, read-only);
 *   u, v, w, g     the step's Courant fields and metric (DEVICE, read-only);
 *   psi_bar        in: dJ/dpsi^(n+1) at interior points; out: dJ/dpsi^n at
 *                  interior points, zero halo;
 *   u_bar, v_bar, w_bar  incremented by dJ/dU, dJ/dV, dJ/dW at interior
 *                  points (the closed top face of W gets nothing).
 * G is held fixed.  The step's intermediates are recomputed from psi_n
 * (mpdata_adjoint_step_tape reuses a recorded tape instead); derivatives
 * follow the branches the forward takes (ties: max(a,b) = a if a >= b,
 * min(a,b) = a if a <= b, sign(0) = 0).  The advance reverses gather
 * without atomics; the limiter and beta reverses, and the FP32
 * pseudo-velocity reverse, add with atomics, so results can differ in the
 * last bits between runs.  Any iord: the corrective passes are reversed in
 * turn.  The first call allocates the adjoint scratch (36 fields plus 11
 * per corrective pass).
 * Errors: EINVAL (null pointer), EALIGN, ENOMEM, ECUDA. */
MPDATA_API int mpdata_adjoint_step(mpdata_ctx *c, const void *psi_n, const void *u,
                                   const void *v, const void *w, const void *g, void *psi_bar,
                                   void *u_bar, void *v_bar, void *w_bar);

/* Taped steps: the adjoint without forward recomputation.
 * mpdata_tape_bytes gives the size of one step's tape: 11 fields for each
 * corrective pass (max(iord-1, 1) blocks): the pass's input state, its
 * unlimited and limited pseudo-velocities, the two betas and the two
 * reciprocals 1/(in+eps), 1/(out+eps) of the limiter's flux sums (which
 * FP32 contexts do not use).
 * mpdata_step_tape runs one forward step psi_in -> psi_out (distinct, halo
 * filled) -- with the fused kernel where mpdata_step would run it, else the
 * staged kernels -- and keeps its intermediates (interior points) in the
 * caller-owned DEVICE buffer tape (16-byte aligned).
 * mpdata_adjoint_step_tape is mpdata_adjoint_step for a step whose tape
 * was recorded from the same psi_n, u, v, w, g.
 * Errors: EINVAL (null pointer, psi_in == psi_out), EALIGN, ENOMEM, ECUDA. */
MPDATA_API int mpdata_tape_bytes(mpdata_ctx *c, size_t *bytes);
MPDATA_API int mpdata_step_tape(mpdata_ctx *c, const void *psi_in, void *psi_out,
                                const void *u, const void *v, const void *w, const void *g,
                                void *tape);
MPDATA_API int mpdata_adjoint_step_tape(mpdata_ctx *c, const void *tape, const void *psi_n,
                                        const void *u, const void *v, const void *w,
                                        const void *g, void *psi_bar, void *u_bar,
                                        void *v_bar, void *w_bar);

/* Reverse of the CELL halo fill for an adjoint field (DEVICE, in place):
 * each halo entry's adjoint is added to the interior value it copies, then
 * the halo is cleared.  Errors: EINVAL, EALIGN, ECUDA. */
MPDATA_API int mpdata_fold_halo_adjoint(mpdata_ctx *c, void *field);

/* Fill the halo of a padded field in place (kind: mpdata_halo_kind).
 * Periodic in i and j, corners included; in k an edge copy (CELL) or zero
 * (WFACE, which also zeroes the top face k = nz-1).
 * This is the boundary-condition component of Sec. 3.1.1, item 2.
 * Errors: EINVAL, EALIGN, ECUDA. */
MPDATA_API int mpdata_fill_halo(mpdata_ctx *c, void *field, int kind);

/* Mass: the sum over the interior of psi*G, accumulated in FP64 for either
 * dtype with a deterministic two-level reduction (fixed partition and fixed
 * tree order, so repeated calls give identical bits); the result is written
 * to *out_dev, a DEVICE double.  Errors: EINVAL, EALIGN, ECUDA. */
MPDATA_API int mpdata_mass(mpdata_ctx *c, const void *psi, const void *g, double *out_dev);

/* ------------------------------------------------------------------------
 * Batches: many independent problems in one persistent launch.
 *
 * Each domain has its own grid and Courant fields and ntracers tracers that
 * share them.  One batch step advances every tracer of every domain by one
 * MPDATA step (iord 2, zero-flux vertical boundary) from one tracer buffer
 * into the other (ping-pong).
 * Domains need nx, ny >= 2*halo and halo >= 2.  The work is split into items
 * (domain, column tile, level chunk, tracer) that the CTAs of one persistent
 * kernel take from an atomic counter; the tracers of one tile are
 * consecutive items, so their shared U, V, W, G columns come from L2.
 * ---------------------------------------------------------------------- */
typedef struct mpdata_domain_desc {
  int nx, ny, nz, halo;  /* grid of this domain                              */
  int ntracers;          /* tracers sharing its Courant fields                */
  void *psi_a, *psi_b;   /* DEVICE: ntracers padded fields each, consecutive  */
                         /* (tracer stride = one padded field); distinct      */
  const void *u, *v, *w, *g; /* DEVICE padded fields of the domain           */
} mpdata_domain_desc;

typedef struct mpdata_batch mpdata_batch; /* opaque */

/* Create a batch from a HOST array of ndomains descriptors (copied; the
 * buffers they point to stay owned by the caller).  Allocates the device
 * descriptor table.  Errors: EINVAL, EALIGN, ERANGE, ENOMEM, EDEVICE, ECUDA. */
MPDATA_API int mpdata_batch_init(mpdata_batch **out, const mpdata_domain_desc *domains,
                                 int ndomains, int nonoscillatory, int dtype, void *cuda_stream);

/* One step of every tracer: direction 0 reads psi_a and writes psi_b,
 * direction 1 the reverse.  With use_graph = 1 the launch (counter reset +
 * persistent kernel) is captured once per direction into a CUDA graph and
 * replayed (needs a non-default stream).  Errors: EINVAL, ECUDA. */
MPDATA_API int mpdata_batch_step(mpdata_batch *b, int direction, int use_graph);

/* Tile shape (index into the compiled shapes: FP32 32x16, 64x8, 32x8,
 * 16x16, and 32x8, 32x12 with two tracers per item (4, 5: each thread
 * advances one column of two tracers of the domain; a field of fewer than
 * 2^31 elements, else ERANGE); FP64 32x8, 16x16, 16x8; one thread per
 * column of the tile and a 2-cell ring) and level-chunk length (0 = whole
 * columns).  Setting waits for the stream and drops captured graphs.
 * Errors: EINVAL, ERANGE (the shape cannot take this batch; the previous
 * configuration stays), ECUDA. */
MPDATA_API int mpdata_batch_set_config(mpdata_batch *b, int shape, int kchunk_levels);
MPDATA_API int mpdata_batch_get_config(mpdata_batch *b, int *shape, int *kchunk_levels,
                                       int *tile_x, int *tile_y, int *threads,
                                       long long *items);

/* Time every shape x chunk length (0, 32, 16, 8) over reps steps (the
 * shapes that can take the batch) and keep the fastest; *best_ms gets its
 * time per step.  It runs steps on the
 * batch's buffers, so their contents change.  Errors: EINVAL, ECUDA. */
MPDATA_API int mpdata_batch_autotune(mpdata_batch *b, int reps, double *best_ms);

MPDATA_API long long mpdata_batch_launch_count(mpdata_batch *b);
MPDATA_API const char *mpdata_batch_last_error_string(mpdata_batch *b);
MPDATA_API void mpdata_batch_destroy(mpdata_batch *b);

/* Instrumentation.  Stage ids of the kernels the library launches. */
enum mpdata_stage {
  MPDATA_STAGE_HALO = 0,     /* halo fill of psi (a1)                        */
  MPDATA_STAGE_DONOR = 1,    /* donor-cell fluxes (a2)                       */
  MPDATA_STAGE_ADVANCE = 2,  /* flux divergence + advance (a2, a6)           */
  MPDATA_STAGE_PSEUDO = 3,   /* antidiffusive pseudo-velocities (a3)         */
  MPDATA_STAGE_BETA = 4,     /* limiter bounds and beta (a4, a5)             */
  MPDATA_STAGE_LIMIT = 5,    /* limited velocities and fluxes (a6)           */
  MPDATA_STAGE_MASS = 6,     /* mass reduction (a7)                          */
  MPDATA_STAGE_FUSED = 7,    /* fused corrective pass (a3-a6)                */
  MPDATA_STAGE_FUSED_DONOR = 8, /* fused donor pass (a2)                     */
  MPDATA_STAGE_EXCHANGE = 9, /* halo strip pack/unpack of a slab            */
  MPDATA_NSTAGES = 10
};

/* Number of kernels this context has launched since it was created. */
MPDATA_API long long mpdata_launch_count(mpdata_ctx *c);

/* Per-stage timing with CUDA events recorded on the context's stream around
 * every launch while enabled (enable = 1; 0 stops).  Enabling clears the
 * totals.  At most 65536 launches are timed; later ones are counted but not
 * timed.  Errors: EINVAL, ENOMEM, ECUDA. */
MPDATA_API int mpdata_profile(mpdata_ctx *c, int enable);

/* Waits for the stream, then returns the summed event time (ms) and number
 * of timed launches of one stage.  Errors: EINVAL, ECUDA. */
MPDATA_API int mpdata_profile_read(mpdata_ctx *c, int stage, double *ms, int *launches);

/* Mass without a context and without allocating: the same deterministic
 * sum over the interior of psi*G as mpdata_mass, for callers that cannot call
 * cudaMalloc -- applications whose device memory is all handed out by their
 * own pool or arena, and hosts that forbid allocation after start-up (real-
 * time or certified codes).  (mpdata_init allocates, so those callers cannot
 * get a context.)
 * The paper has no counterpart: this is a library-interface addition.
 *   psi, g   padded DEVICE fields [nz+2h][ny+2h][nx+2h] of dtype, 16-byte
 *            aligned, read at interior points only;
 *   out_dev  DEVICE double that receives the sum (8-byte aligned);
 *   cuda_stream  the stream the two kernels run on (NULL = legacy default).
 * Scratch: a file-scope device array of MPDATA_MASS_NOALLOC_PARTIALS doubles
 * (9472 bytes) that every GPU loading the library keeps until exit.  All
 * calls on one device share it: two calls whose kernels overlap on that GPU
 * (for example on two streams) race on it, so the caller must order them.
 * Each call overwrites every partial before reading it, so nothing carries
 * over from the previous call.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current
 * and keeps it for the life of the process; make that first call before any
 * stream capture.  A cudaDeviceReset of that device makes the kept address
 * stale: do not call this entry point on a device after resetting it.
 * Limits: ny*nz <= MPDATA_MASS_MAX_ROWS and (nx+2h)(ny+2h) < 2^31, else
 * MPDATA_ERANGE, checked before anything is launched.
 * Errors: EINVAL, EALIGN, ERANGE, EDEVICE, ECUDA. */
#define MPDATA_MASS_NOALLOC_PARTIALS 1184
/* The mass reduction walks the ny*nz interior rows with a 32-bit counter that
 * runs up to 16 x 1184 rows past the last one, so the row count stays below
 * 2^31 by that margin (mpdata_init enforces the same bound). */
#define MPDATA_MASS_MAX_ROWS (2147483647LL - 16LL * 1184LL)
#define MPDATA_MASS_NOALLOC_MAX_ROWS MPDATA_MASS_MAX_ROWS
MPDATA_API int mpdata_mass_noalloc(const void *psi, const void *g, int nx, int ny, int nz,
                                   int halo, int dtype, double *out_dev, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Slabs of an i-j decomposed domain (Sec. 3.1.1, item 2: halo exchange and
 * boundary conditions as a library component; Fig. 8: the grid split into
 * partitions).  A domain of NX x NY x nz is cut into px x py slabs, one
 * context each (sizes nx_r x ny_r x nz, halo h >= 3).  A slab's i-j halo
 * belongs to its neighbours: its step reads the halo instead of wrapping,
 * so one exchange of psi's halo before each step (depth 3, corners
 * included) makes the step of every slab equal, point for point, to the
 * step of the undivided domain under the same kernel.  U, V, W, G are
 * exchanged once, before the first step.
 * ------------------------------------------------------------------------ */
enum mpdata_ij_boundary {
  MPDATA_IJ_PERIODIC = 0, /* the context is the whole domain (default)       */
  MPDATA_IJ_HALO = 1      /* the context is one slab: i-j halo from neighbours */
};

/* Make a context a slab (MPDATA_IJ_HALO) or the whole periodic domain
 * again.  A slab runs the one-kernel step of iord 2 in both dtypes,
 * whatever the variant; its output's i-j halo is left to the exchange (the
 * k halo is still filled).  Requires iord == 2, halo >= 3, no options,
 * nx, ny >= halo.  The adjoint calls, mpdata_fill_halo and
 * mpdata_set_options(nonzero) return EINVAL on a slab.
 * Errors: EINVAL, ECUDA (the kernel cannot run on this device). */
MPDATA_API int mpdata_set_ij_boundary(mpdata_ctx *c, int mode);

/* Halo strips.  Face f: 0 = -x, 1 = +x, 2 = -y, 3 = +y.
 * mpdata_halo_pack copies the h-deep interior strip of field next to face f
 * into buf; the neighbour across face f passes that buffer to
 * mpdata_halo_unpack with face f ^ 1, which writes it into the halo strip
 * beyond that face.  x faces carry the interior rows (j in [0, ny)); y
 * faces carry whole padded rows (i in [-h, nx+h)), so exchanging x first
 * and y second fills the halo's corners.  Levels k in [0, nz).
 * buf: DEVICE, 16-byte aligned, mpdata_halo_strip_elems(face) elements of
 * the context's dtype, laid out [nz][rows][cols] with (rows, cols) =
 * (ny, h) for x faces and (h, nx + 2h) for y faces.  Both calls run one
 * kernel on the context's stream and work in either boundary mode.
 * Errors: EINVAL (null context, face out of range, buf == field), EALIGN,
 * ECUDA. */
MPDATA_API int mpdata_halo_strip_elems(mpdata_ctx *c, int face, long long *n);
MPDATA_API int mpdata_halo_pack(mpdata_ctx *c, const void *field, int face, void *buf);
MPDATA_API int mpdata_halo_unpack(mpdata_ctx *c, const void *buf, int face, void *field);

/* Destroy a context and free its scratch (NULL is ignored). */
MPDATA_API void mpdata_destroy(mpdata_ctx *c);

/* Static description of a status code. */
MPDATA_API const char *mpdata_strerror(int code);

/* The CUDA runtime's message for the last MPDATA_ECUDA on this context. */
MPDATA_API const char *mpdata_last_error_string(mpdata_ctx *c);

/* Library version (major*10000 + minor*100 + patch). */
MPDATA_API int mpdata_version(void);

/* Measurement helper, not part of the method: the device's FP64 FMA rate,
 * which bounds every FP64 kernel of the step on the B300.  Launches one
 * kernel of `blocks` CTAs x 256 threads on cuda_stream; each thread runs 8
 * independent chains of `iters` fused multiply-adds.  *flops (HOST) receives
 * the launch's flop count (2 per FMA); the caller times the launch (CUDA
 * events on the same stream) and divides.  out_dev is a DEVICE double that
 * is never written in practice (it keeps the work from being optimised
 * away).  Errors: EINVAL (null pointer, blocks or iters < 1), ECUDA. */
MPDATA_API int mpdata_probe_fp64_fma(double *out_dev, int blocks, int iters, void *cuda_stream,
                                     double *flops);

/* ------------------------------------------------------------------------
 * Edge-based flux stages on a structured triangular patch.
 *
 * The subset of the MPDATA dwarf the paper shows on its octahedral grid
 * (Sec. 5): the upwind flux on every edge (Listings 4/5), the vertical
 * upwind flux on every node (Listings 6/7), their divergence over each
 * node's dual cell and the advance (the calls of Listing 8, composed into
 * one kernel as Listing 9 composes its stages):
 *   flux_e   = max(0, vn_e) pD(first node) + min(0, vn_e) pD(second node);
 *   fluz_k   = max(0, W_k) pD_{k-1} + min(0, W_k) pD_k    (faces 1..nz-1),
 *   fluz_0   = pivbz fluz_1,  fluz_nz = pivbz fluz_{nz-1};
 *   divVD    = (sum over the node's own edges of flux - sum over the
 *               edges ending at it of flux + fluz_{k+1} - fluz_k) / vol;
 *   pD_out   = pD - divVD / rho.
 * The paper names the last two calls without their bodies; these are the
 * plain finite-volume divergence and density-weighted update.
 *
 * The patch: nr x nc nodes, periodic in both directions (one parallelogram
 * of the octahedral grid without its corner irregularities).  Structured
 * numbering, direct access (Figs. 9 and 11): node (r, c) owns the edges of
 * colours 0: (r,c)->(r,c+1), 1: (r,c)->(r+1,c), 2: (r,c)->(r+1,c+1); a
 * positive vn moves mass from the first node to the second.  With nr or
 * nc equal to 1 a colour's edges join a node to itself and carry no net
 * flux.  DEVICE fields of the context's dtype, level-major, C-contiguous,
 * 16-byte aligned, no halo:
 *   pD, rho    [nz][nr][nc]       nodes (rho > 0)
 *   vn         [nz][nr][3][nc]    edges, (row, colour, column) per level
 *   wn         [nz+1][nr][nc]     vertical faces, face k between levels k-1
 *                                 and k; faces 0 and nz are never read
 *   vol        [nr][nc]           dual volume of each node (> 0)
 * ---------------------------------------------------------------------- */
typedef struct mpdata_edge mpdata_edge; /* opaque, library-owned */

/* Create a context for one patch: nr, nc >= 1, nz >= 2 (the boundary
 * faces take their flux from an interior face), dtype MPDATA_F64 or
 * MPDATA_F32, pivbz the boundary factor (0: closed top and bottom).
 * Allocates the staged organisation's scratch (5 nz + 1 node planes).
 * Errors: EINVAL, ERANGE (nz > 65534 or nr > 524280), EDEVICE, ENOMEM. */
MPDATA_API int mpdata_edge_init(mpdata_edge **out, int nr, int nc, int nz, int dtype,
                                double pivbz, void *cuda_stream);
MPDATA_API int mpdata_edge_set_stream(mpdata_edge *e, void *cuda_stream);

/* MPDATA_FUSED (one kernel; also MPDATA_AUTO, the default) or
 * MPDATA_STAGED (four kernels, one per call of Listing 8). Errors: EINVAL. */
MPDATA_API int mpdata_edge_set_variant(mpdata_edge *e, int variant);

/* One application of the four stages: pD_out = step(pD_in); the two
 * buffers must be distinct.  Asynchronous on the context's stream.
 * Errors: EINVAL (null pointer, pD_in == pD_out), EALIGN, ECUDA. */
MPDATA_API int mpdata_edge_step(mpdata_edge *e, const void *pD_in, void *pD_out,
                                const void *vn, const void *wn, const void *rho,
                                const void *vol);

/* Nodes per thread of the fused kernel: 1, or 4 (consecutive columns read
 * as 16-byte vectors; FP32 with nc a multiple of 4, the default there); 0
 * restores the default.  Errors: EINVAL (other values, or 4 where it does
 * not apply). */
MPDATA_API int mpdata_edge_set_width(mpdata_edge *e, int width);
MPDATA_API int mpdata_edge_get_width(mpdata_edge *e, int *width);

/* Kernel launches issued so far (-1 for NULL). */
MPDATA_API long long mpdata_edge_launch_count(mpdata_edge *e);
MPDATA_API const char *mpdata_edge_last_error_string(mpdata_edge *e);
MPDATA_API void mpdata_edge_destroy(mpdata_edge *e);

/* ------------------------------------------------------------------------
 * Cell-neighbour reduction (Table 1).
 *
 * The on_cells operation of Fig. 5 that Table 1 times under different
 * numberings and access methods: for every cell s and level k
 *   B[k][s] = fac * (A[k][n0] + A[k][n1] + A[k][n2]),
 * n0, n1, n2 the three cells across s's edges, summed in that order; the
 * two-stage operator of Table 1 is two calls (A -> B with fac1, B -> C with
 * fac2).  Fields are DEVICE arrays [nz][ncells] of the context's dtype in
 * the numbering's storage order, 16-byte aligned.
 *
 * Access methods (Sec. 3.2):
 *   direct    structured numbering of the triangles of a periodic nr x nc
 *             patch: cell (row r, colour, column c) -> (2 r + colour) nc + c,
 *             colour 0 the upward triangle (r,c), (r,c+1), (r+1,c+1) and 1
 *             the downward (r,c), (r+1,c+1), (r+1,c); the neighbours, found
 *             by index arithmetic, are D(r-1,c), D(r,c+1), D(r,c) for U(r,c)
 *             and U(r,c), U(r+1,c), U(r,c-1) for D(r,c);
 *   indirect  a neighbour table [3][ncells] of int32 in any numbering (the
 *             structured one, a mesh library's, a space-filling curve's).
 * ---------------------------------------------------------------------- */
typedef struct mpdata_cells mpdata_cells; /* opaque, library-owned */

/* table == NULL: direct access, structured numbering, ncells = 2 nr nc.
 * table != NULL: indirect access; HOST array [3][ncells], every entry in
 * [0, ncells) (checked), copied to the device (nr, nc ignored).
 * Errors: EINVAL (sizes, dtype, a table entry out of range), ERANGE
 * (ncells >= 2^31), EDEVICE, ENOMEM. */
MPDATA_API int mpdata_cells_init(mpdata_cells **out, long long ncells, int nz, int dtype,
                                 const int *table, int nr, int nc, void *cuda_stream);
MPDATA_API int mpdata_cells_set_stream(mpdata_cells *c, void *cuda_stream);

/* B = fac * neighbour sum of A (A and B distinct).  Asynchronous on the
 * context's stream.  Errors: EINVAL (null, A == B), EALIGN, ECUDA. */
MPDATA_API int mpdata_cells_sum(mpdata_cells *c, const void *A, void *B, double fac);
MPDATA_API long long mpdata_cells_launch_count(mpdata_cells *c);
MPDATA_API const char *mpdata_cells_last_error_string(mpdata_cells *c);
MPDATA_API void mpdata_cells_destroy(mpdata_cells *c);

#ifdef __cplusplus
}
#endif

#endif /* MPDATA_B300_H */
