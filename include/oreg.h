/*
 * oreg.h -- C ABI of the GB300 (sm_103a) Onsager-Regularized lattice
 * Boltzmann library liboreg.so (D2Q9, arXiv 2501.16000).
 *
 * The library advances a periodic nx x ny D2Q9 lattice with the fused
 * stream-and-collide update of the paper:
 *
 *   f_i(x + c_i, t + 1) = f_i^eq(x, t) + (1 - 1/tau) f_i^OReg(x, t)   (Eq. 7)
 *
 * where f^eq is the guided equilibrium (Eq. 11) or the second-order
 * polynomial equilibrium (Eq. 15) and f^OReg is the local OReg projection of
 * the non-equilibrium part f - f^eq (Eq. 6).  Lattice BGK (Eq. 1) is the
 * switchable special case.  theta is a fixed per-lattice temperature
 * (isothermal flow, Sec. II).
 *
 * Conventions shared by every call:
 *   - Velocity order i = 0..8: (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1)
 *     (-1,-1) (1,-1).
 *   - Host population arrays are double[9][ny][nx] (index (i*ny + y)*nx + x);
 *     host field arrays are double[ny][nx] (index y*nx + x).
 *   - The state of a lattice is always the canonical pre-collision
 *     populations S_t at integer time t; storage precision, layout (A-B or
 *     in-place AA) and parity are hidden behind the calls.
 *   - Every call returns an olb_status and never aborts the process; on an
 *     error the calling thread's message is available from olb_last_error().
 *   - Calls that only enqueue device work are asynchronous on the lattice's
 *     stream; calls that return data in host memory synchronise that stream.
 *   - A lattice handle must not be used from two host threads at once.
 */
#ifndef OREG_H
#define OREG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct olb_lattice olb_lattice; /* opaque; owned by the library */

typedef enum {
    OLB_OK = 0,
    OLB_ERR_INVALID = 1,   /* bad argument or parameter combination */
    OLB_ERR_NOMEM = 2,     /* device or host allocation failed */
    OLB_ERR_CUDA = 3,      /* a CUDA runtime call or launch failed */
    OLB_ERR_NONFINITE = 4, /* the state holds NaN or Inf (outputs still written) */
    OLB_ERR_TIMEOUT = 5,   /* a bounded wait ended before the work it waits
                              for (olb_batch_wait_for); that work goes on */
    OLB_ERR_STATE = 6      /* call not valid in the lattice's current state */
} olb_status;

typedef enum { OLB_EQ_GUIDED = 0, OLB_EQ_POLY2 = 1 } olb_equilibrium;
typedef enum { OLB_COLL_OREG = 0, OLB_COLL_BGK = 1 } olb_collision;

/* Population storage.  Every format stores shifted values g_i = f_i - s_i,
 * with s_i the rest equilibrium w_i(theta) rho0 rounded to the compute type
 * (w = (1-theta)^2, theta(1-theta)/2, theta^2/4 for rest, axis and diagonal
 * directions).  F64 computes in double; F32, F16 and BF16 compute in float
 * (F32 in double with OLB_OPT_F64_COLLISION).
 * F16 stores g * 2^8 (exact scaling) to keep small deviations out of the f16
 * subnormal range; |f_i - s_i| must stay below 255. */
typedef enum {
    OLB_F64 = 0,
    OLB_F32 = 1,
    OLB_F16_SHIFTED = 2,
    OLB_BF16_SHIFTED = 3
} olb_storage;

/* A-B: two population buffers, pull streaming, buffers swap each step.
 * AA: one buffer updated in place; even steps read and write a node's own
 * slots (writing direction i into the opposite slot), odd steps read from
 * and write to the neighbours.  Same results, half the memory. */
typedef enum { OLB_LAYOUT_AB = 0, OLB_LAYOUT_AA = 1 } olb_layout;

/* PERIODIC: periodic in x and y.  WALLS_X: columns x = 0 and x = nx - 1 are
 * solid wall nodes with full-way bounce-back (the shock tube of Sec. IV):
 * a wall node does not collide, it returns every population along the link
 * it arrived on, post_i = f_opp(i), so the no-slip wall lies halfway between
 * the wall column and the first fluid column; y stays periodic.  Wall nodes
 * keep populations in the state (moments there are not fluid fields); the
 * total mass over all nodes stays exactly conserved.  Needs nx >= 3. */
typedef enum { OLB_BOUNDARY_PERIODIC = 0, OLB_BOUNDARY_WALLS_X = 1 } olb_boundary;

/* FIXED: theta is the lattice's fixed temperature in the guided equilibrium
 * (Eq. 11) and in Eq. 6 (isothermal flow, Sec. II; the paper's runs).
 * LOCAL: every node uses its own temperature
 * theta = (<f,c^2> - rho u^2) / (2 rho) (Eq. 2a: E = (D p + rho u^2)/2,
 * p = rho theta); the guided equilibrium then carries the node's energy, so
 * BGK conserves <f,c^2> and sound travels at sqrt(2 theta) (gamma = 2 in two
 * dimensions); p->theta is the reference temperature of the storage shift
 * and of the initialisers.  Guided equilibrium only. */
typedef enum { OLB_THETA_FIXED = 0, OLB_THETA_LOCAL = 1 } olb_theta_mode;

typedef struct {
    int32_t nx, ny;        /* lattice size, >= 1 each */
    double tau;            /* relaxation time, > 0.5 */
    double theta;          /* guided: lattice temperature in (0, 1);
                              poly2: must be 1/3 (theta0 of Eq. 15) */
    double rho0;           /* reference density of the storage shift, > 0 (1 if unsure) */
    int32_t eq;            /* olb_equilibrium */
    int32_t coll;          /* olb_collision */
    int32_t storage;       /* olb_storage */
    int32_t layout;        /* olb_layout */
    void *device_buffer;   /* optional caller-owned device memory for the
                              populations (>= olb_required_bytes, 256-byte
                              aligned); NULL: the library allocates.  Caller
                              memory must outlive the lattice. */
    size_t buffer_bytes;   /* size of device_buffer in bytes (ignored if NULL) */
    void *cuda_stream;     /* cudaStream_t for all work of this lattice;
                              NULL: the library creates and owns one */
    int32_t boundary;      /* olb_boundary (0: periodic) */
    int32_t theta_mode;    /* olb_theta_mode (0: fixed) */
} olb_params;

/* Tuning and precision options of a lattice (olb_set_option). */
typedef enum {
    /* OLB_F32 storage.  1 (default): the conserved moments (mass and
       momentum) of the FP32 collision are exact sums of the stored
       populations, rounded once (an error-free split of each population
       against a power-of-two constant; about 50 more FP32 additions per
       node, two nodes per packed instruction).  Plain FP32 sums round each
       partial sum, and the rounding repeats identically at every node of a
       uniform region and every step: on the 2048 x 4 shock tube (tau =
       0.51, 2000 steps) they end ~3e-5 from the FP64 scheme, the exact
       sums ~5e-6.  0: plain sums (the rest of the FP32 collision is the
       same; olb_batch_add rejects an FP32 lattice with 0).  Ignored by the
       other formats. */
    OLB_OPT_COMPENSATED = 1,
    /* warps per thread block of the stream-collide kernels: 1, 2, 4 or 8
       (default 4).  A warp pass updates 32 consecutive 16-byte vectors of
       V nodes each (V = 16 bytes / element size) of the row-major planes,
       whose rows are nx rounded up to V elements, back to back; a pass may
       span rows. */
    OLB_OPT_WARPS_PER_BLOCK = 2,
    /* 1 (default for OLB_F16_SHIFTED and OLB_BF16_SHIFTED): round the
       post-collision values to the half format stochastically, with random
       bits drawn from a counter-based hash of (x, y, t, direction), so that
       rounding adds no bias to slow, small-amplitude dynamics (round-to-
       nearest there changes a shear wave's decay rate by up to ~1e-1 at
       tau = 0.52); results stay deterministic and independent of batching
       and layout.  0: round to nearest even.  Ignored by F32 and F64. */
    OLB_OPT_STOCHASTIC_ROUNDING = 3,
    /* OLB_F32 storage only.  1: olb_step computes the collision in FP64
       (decode, Eqs. 6-7, encode) while the populations stay stored in
       FP32, so the store is the only FP32 rounding of a step (2048 x 4
       shock tube, tau = 0.51, 2000 steps: ~5e-6 from the FP64 result,
       like the default FP32 collision with exact conserved sums); a
       reference mode for accuracy studies, at the GPU's FP64 rate (a few
       GLUPS).  The stored state is that of the FP32 collision
       (same elements and shifts), so the option may change between steps.
       0 (default): FP32 collision.  OLB_ERR_INVALID for value 1 on another
       storage format; olb_batch_add rejects a lattice with it set. */
    OLB_OPT_F64_COLLISION = 4
} olb_option;

/* Version of this ABI (bumped on incompatible change); 5 since
 * olb_batch_params.item_passes (work items of warp passes). */
int32_t olb_abi_version(void);

/* Bytes of device memory the populations of a lattice with these
 * parameters occupy (for admission control and caller allocation);
 * 0 if the parameters are invalid.  Library scratch is extra and always
 * library-owned: ~60 KB of reduction partials per lattice from
 * olb_create_lattice, and, from the first olb_init_fields / olb_moments /
 * olb_get_populations / olb_get_region / olb_set_populations call on, an
 * FP64 staging buffer of at most 128 MiB (for a small lattice 2 x ny x nx
 * x 3 doubles for fields, ny x nx x 9 for populations), held until
 * olb_destroy. */
size_t olb_required_bytes(const olb_params *p);

/* Validates p, allocates the lattice and (unless p->device_buffer is
 * given) its population memory.  The state is undefined until one of the
 * olb_init_* or olb_set_populations calls.  *out receives the handle.
 * OLB_ERR_INVALID for a lattice of more than 2^36 nodes or more than
 * 2^31 - 64 16-byte vectors per population plane (ceil(nx / V) x ny,
 * V = 16 / element size); OLB_ERR_NOMEM when its memory cannot be
 * allocated. */
olb_status olb_create_lattice(const olb_params *p, olb_lattice **out);

/* Rebinds a lattice to another stream: the work of every later call on it
 * is enqueued there (a serving loop reads a finished lattice back on its own
 * stream while the batch's next round runs).  Work already enqueued on the
 * previous stream is not waited for: the caller orders it, e.g. with an
 * event.  cuda_stream NULL: back to the stream the library created for the
 * lattice (OLB_ERR_INVALID if it was created on a caller stream).
 * OLB_ERR_STATE while the lattice is a batch member. */
olb_status olb_set_stream(olb_lattice *lat, void *cuda_stream);

/* S_0 = f^eq(rho, u) of a rotated decaying shear wave (Sec. IV, Eq. 18 with
 * any integer wave vector): k = 2 pi (m/nx, n/ny), u = u0 sin(k.x) e_perp,
 * e_perp = (-k_y, k_x)/|k|, rho = rho0.  (m, n) != (0, 0).  Sets t = 0. */
olb_status olb_init_shear_wave(olb_lattice *lat, double rho0, double u0, int32_t m,
                               int32_t n);

/* The same shear wave carried by a uniform mean flow U = (ux_mean, uy_mean):
 * u = U + u0 sin(k.x) e_perp (the Mach sweep of Sec. IV, Fig. 2, uses
 * U = (0, Ma sqrt(theta))).  first_order = 0 starts from S_0 = f^eq;
 * first_order = 1 starts from S_0 = f^eq + f^(1), the first-order
 * populations of Eq. 5 evaluated with the analytic velocity gradient
 * grad_b u_a = u0 cos(k.x) e_perp,a k_b, the lattice's tau and the theta of
 * Eq. 6 (the lattice theta for the guided equilibrium, 1/3 for the
 * polynomial one); this removes the start-up transient of an equilibrium
 * start.  OLB_ERR_INVALID for (m, n) = (0, 0), rho0 <= 0, non-finite
 * u0 / U, or first_order not 0 or 1.  Sets t = 0. */
olb_status olb_init_shear_flow(olb_lattice *lat, double rho0, double u0, int32_t m, int32_t n,
                               double ux_mean, double uy_mean, int32_t first_order);

/* S_0 = f^eq of the isothermal shock tube (Sec. IV): rho = rho_left for
 * x < x_split, rho_right otherwise, u = 0.  Sets t = 0. */
olb_status olb_init_shock_tube(olb_lattice *lat, double rho_left, double rho_right,
                               int32_t x_split);

/* S_0 = f^eq(rho(x), u(x)) from host fields rho, ux, uy (double[ny][nx]).
 * Copies host -> device inside the call; the arrays may be reused on return.
 * Sets t = 0. */
olb_status olb_init_fields(olb_lattice *lat, const double *rho, const double *ux,
                           const double *uy);

/* Advances nsteps >= 0 time steps (Eq. 7, or Eq. 1 for BGK) asynchronously
 * on the lattice's stream. */
olb_status olb_step(olb_lattice *lat, int64_t nsteps);

/* Sets an olb_option; takes effect from the next olb_step. */
olb_status olb_set_option(olb_lattice *lat, int32_t option, int64_t value);

/* Current integer time t of the canonical state (-1 before any init). */
int64_t olb_time(const olb_lattice *lat);

/* Macroscopic fields of S_t into host arrays double[ny][nx]:
 * rho = <f,1>, u = <f,c>/rho (Eq. 2a) and, if theta_loc != NULL, the local
 * temperature (<f,c^2> - rho u^2)/(2 rho) (from E = (D p + rho u^2)/2,
 * p = rho theta).  Synchronises the stream. */
olb_status olb_moments(olb_lattice *lat, double *rho, double *ux, double *uy,
                       double *theta_loc);

/* Same fields written to caller device arrays (double[ny][nx], any may be
 * NULL except rho), asynchronously on the lattice's stream. */
olb_status olb_moments_device(olb_lattice *lat, double *d_rho, double *d_ux,
                              double *d_uy, double *d_theta_loc);

/* Canonical S_t into host double[9][ny][nx].  Synchronises the stream. */
olb_status olb_get_populations(olb_lattice *lat, double *f9);

/* Canonical S_t of the window [x0, x0 + wx) x [y0, y0 + wy) into host
 * double[9][wy][wx] (sampled checks of lattices too large to copy whole).
 * Synchronises the stream. */
olb_status olb_get_region(olb_lattice *lat, int32_t x0, int32_t y0, int32_t wx, int32_t wy,
                          double *f9);

/* Replaces the state by host double[9][ny][nx] (canonical populations) at
 * time t (>= 0); the arrays may be reused on return. */
olb_status olb_set_populations(olb_lattice *lat, const double *f9, int64_t t);

/* FP64 reductions of S_t: total mass sum rho, momentum sum rho u, and the
 * number of nodes whose populations are not all finite.  Returns
 * OLB_ERR_NONFINITE (after writing the outputs) if that number is > 0.
 * Synchronises the stream. */
olb_status olb_diagnostics(olb_lattice *lat, double *mass, double *mom_x, double *mom_y,
                           int64_t *nonfinite);

/* Largest difference between the canonical populations of two lattices of
 * the same size, in any storage formats: *max_abs_diff = max over nodes and
 * directions of |f_a - f_b| and, if max_abs_ref is not NULL, *max_abs_ref =
 * max |f_b| (b is the reference, e.g. an FP64 run of the same problem),
 * both in FP64, reduced on the GPU over the whole lattice; a difference
 * that is not finite reads as infinity.  Waits for b's stream, runs on a's
 * and synchronises it.  Allocates 16 bytes of scratch with a on first use.
 * OLB_ERR_INVALID for different sizes, OLB_ERR_STATE if one is not
 * initialised. */
olb_status olb_compare(olb_lattice *a, olb_lattice *b, double *max_abs_diff,
                       double *max_abs_ref);

/* FP64 projection of the velocity of S_t on a shear-wave mode:
 * A = (2 / (nx ny)) sum_x u(x) . e_perp sin(k . x), k = 2 pi (m/nx, n/ny);
 * the decay statistic of Sec. IV.  Synchronises the stream. */
olb_status olb_wave_amplitude(olb_lattice *lat, int32_t m, int32_t n, double *amp);

/* Both quadratures of that projection,
 * a_sin = (2 / (nx ny)) sum_x u(x) . e_perp sin(k . x) (= olb_wave_amplitude) and
 * a_cos = (2 / (nx ny)) sum_x u(x) . e_perp cos(k . x),
 * so that a wave advected by a mean flow has amplitude hypot(a_sin, a_cos)
 * and phase atan2(a_cos, a_sin).  Either pointer may be NULL, not both.
 * Returns OLB_ERR_NONFINITE if the state holds non-finite populations.
 * Synchronises the stream. */
olb_status olb_wave_mode(olb_lattice *lat, int32_t m, int32_t n, double *a_sin,
                         double *a_cos);

/* ------------------------------------------------------------------------
 * Batched path: many independent lattices advanced together.
 *
 * One kernel per time step and slot, whose warps stride over a flattened
 * table of warp work items (up to item_passes consecutive warp passes over
 * one member lattice each); steps_per_launch steps of such launches are
 * captured in a CUDA graph and replayed per round.  Each
 * member keeps its own size, relaxation time, temperature, equilibrium and
 * collision; all members share the batch's storage format and layout and
 * must have been created on the batch's stream.  Members are grouped into
 * slots of one kernel (walls, equilibrium kind, collision) and one class of
 * collision constants (the same theta, rho0 and equilibrium; tau is per
 * member), and every step launches one kernel per slot, whose class constants
 * are a launch parameter; within the graph the kernels of different slots
 * run side by side (each slot's steps in order).  Joining and leaving rewrite the device tables
 * only; the graph is captured again when a member brings a new slot (at most
 * 64 slots are in use at a time: olb_batch_add returns OLB_ERR_NOMEM beyond).
 * A member is advanced exactly the number of steps it was added with, then
 * idles until removed.
 * Results are bitwise those of olb_step on the same lattice: each node's
 * update depends only on that lattice's state.
 * ---------------------------------------------------------------------- */
typedef struct olb_batch olb_batch; /* opaque; owned by the library */

typedef struct {
    int32_t storage;           /* olb_storage of every member */
    int32_t layout;            /* olb_layout of every member */
    int32_t max_lattices;      /* descriptor capacity */
    int64_t max_items;         /* work-item capacity: sum over members of
                                  ceil(P / R), P = ceil(ceil(nx / V) * ny / 32)
                                  the member's warp passes (32 vectors of
                                  V = 16 / element size nodes each, rows
                                  rounded up to V), R = item_passes */
    int32_t steps_per_launch;  /* K: time steps per graph replay (1..10000) */
    int32_t warps_per_block;   /* 1, 2 or 4 */
    int32_t blocks_per_sm;     /* grid = blocks_per_sm x SMs (0..256);
                                  0 = the kernel's occupancy limit (every
                                  block resident); above it, blocks start as
                                  earlier ones finish, which evens out uneven
                                  work items */
    void *cuda_stream;         /* stream of the batch and of every member;
                                  NULL: the library creates and owns one */
    int32_t item_passes;       /* R: warp passes per work item (1..64); a
                                  warp reads the member's descriptor once
                                  per item; 0 = 4 */
} olb_batch_params;

olb_status olb_batch_create(const olb_batch_params *p, olb_batch **out);

/* Adds an initialised lattice that will advance nsteps more steps over the
 * following rounds.  Does not wait for the batch: the change of the device
 * tables is enqueued on the batch's stream and takes effect from the next
 * round enqueued after this call (rounds enqueued before it run without the
 * lattice).  While a member, the lattice is advanced only by olb_batch_run
 * (olb_step and the init calls return OLB_ERR_STATE); its readback calls may
 * be used between rounds (they run on the batch's stream). */
olb_status olb_batch_add(olb_batch *b, olb_lattice *lat, int64_t nsteps);

/* Removes a member, without waiting: rounds enqueued before the call still
 * advance it (up to its step count), rounds enqueued after it do not.  Its
 * state is final once those rounds have run (stream order on the batch's
 * stream, e.g. an event recorded there before olb_set_stream moves the
 * lattice to another stream).  olb_destroy of a member removes it first and
 * synchronises the stream before freeing anything. */
olb_status olb_batch_remove(olb_batch *b, olb_lattice *lat);

/* Enqueues nrounds graph replays of steps_per_launch steps each
 * (asynchronous on the batch's stream); member times advance accordingly. */
olb_status olb_batch_run(olb_batch *b, int64_t nrounds);

/* Waits until the batch's enqueued rounds have finished. */
olb_status olb_batch_wait(olb_batch *b);

/* Waits at most `seconds` (0 .. 1e6) for the rounds enqueued so far: OLB_OK once
 * they have finished, OLB_ERR_TIMEOUT if they are still running when the time
 * is up (nothing is cancelled; a later wait can succeed), OLB_ERR_CUDA if the
 * stream reported an error.  Polls an event recorded on the batch's stream,
 * sleeping ~50 us between polls; seconds = 0 polls once. */
olb_status olb_batch_wait_for(olb_batch *b, double seconds);

/* Steps a member still has to take. */
olb_status olb_batch_remaining(const olb_batch *b, const olb_lattice *lat, int64_t *steps);

/* Number of members / of work items in the batch's tables. */
int32_t olb_batch_size(const olb_batch *b);
int64_t olb_batch_work_items(const olb_batch *b);

/* Releases the batch (waits first); members stay valid lattices. */
olb_status olb_batch_destroy(olb_batch *b);

/* Largest ny olb_diagnostics_noalloc accepts. */
#define OLB_NOALLOC_MAX_ROWS 16384

/* olb_diagnostics for callers that cannot allocate device memory.  The
 * paper has no counterpart: this is plumbing for embedding the library.
 *
 * Some callers own the GPU memory budget themselves and must not let a
 * library call cudaMalloc: a serving loop that admits work against an HBM
 * budget it accounts for byte by byte, or a host loop on a latency budget in
 * which cudaMalloc/cudaFree would add device-wide synchronisation.  Such a
 * caller keeps the populations in its own device buffer and still needs the
 * mass, momentum and non-finite count.  This call allocates nothing: no
 * cudaMalloc, no cudaFree, no allocating library routine.  Its reduction
 * scratch is a fixed static device array of OLB_NOALLOC_MAX_ROWS x 4 doubles
 * (512 KiB) that every GPU which loads liboreg.so holds until the process
 * exits.
 *
 * d_populations: device memory laid out exactly as a lattice created with
 *   the same olb_params keeps it (the device_buffer of olb_create_lattice,
 *   olb_required_bytes(p) bytes, 16-byte aligned).
 * p: nx, ny, tau, theta, rho0, eq, storage, layout and cuda_stream describe
 *   that state; device_buffer and buffer_bytes are ignored.  ny must not
 *   exceed OLB_NOALLOC_MAX_ROWS (larger lattices are rejected with
 *   OLB_ERR_INVALID).
 * t: the time of the state (selects the A-B buffer and the AA parity).
 * d_out: device double[4] receiving total mass, momentum x, momentum y and
 *   the number of nodes holding a non-finite population.
 *
 * Asynchronous on p->cuda_stream (NULL: the legacy default stream); the
 * caller synchronises before reading d_out.  Results equal olb_diagnostics
 * up to the order of the FP64 additions.  The first call on a device looks
 * up the device address of the static array (with that device current);
 * make that first call before any stream capture.  All calls share the
 * array: calls whose work overlaps on the GPU race and must be ordered by
 * the caller.  Every partial the call reads is written by the same call, so
 * the array needs no clearing between calls.  On failure the message is
 * available from olb_last_error(). */
olb_status olb_diagnostics_noalloc(const void *d_populations, const olb_params *p, int64_t t,
                                   double *d_out);

/* Releases the lattice and everything it allocated (NULL is a no-op).
 * Waits for the lattice's pending work first. */
olb_status olb_destroy(olb_lattice *lat);

/* Message of the last failed call on this host thread ("" if none). */
const char *olb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* OREG_H */
