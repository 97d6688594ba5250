/*
 * maclab.h -- C ABI of the GB300 MacLAB library (libmaclab.so).
 *
 * The library advances the macroscopic lattice Boltzmann method of Zhou,
 * "Macroscopic Lattice Boltzmann Method (MacLAB)": with relaxation time
 * tau = 1 no distribution function is stored, and each node's new density and
 * momentum are the zeroth and first moments of the equilibria, Eq. (2), of its
 * upstream neighbours x - e_a dt (Eqs. (4) and (5)); the particle speed is
 * e = 6 nu / dx (Eq. (6)) and the time step dt = dx / e.  Walls keep the
 * physical values they are given (procedure step (iv); Tests 2, 3 and 5);
 * periodic axes wrap (Tests 1 and 4).
 *
 * Conventions for every call:
 *  - Return a maclab_status: 0 = OK, > 0 warning, < 0 error.  Nothing throws,
 *    nothing aborts.  maclab_status_string() names a status.
 *  - Arrays are structure-of-arrays with x fastest: node index
 *    (z * ny + y) * nx + x; a velocity field is d consecutive arrays of N
 *    values (all x-components, then y, then z).  N = nx * ny * nz counts wall
 *    nodes too.  D2Q9 uses nz = 1.
 *  - "where" = MACLAB_HOST (pageable or pinned host memory) or MACLAB_DEVICE
 *    (memory of the handle's GPU).  Caller buffers stay owned by the caller
 *    and are not retained after the call returns.
 *  - Work is queued on the handle's CUDA stream (the one given in the config,
 *    or the default stream).  Calls that return data to the host synchronise
 *    that stream; the others are asynchronous, and a device-side failure
 *    surfaces as MACLAB_ERR_CUDA at the next synchronising call.
 *  - A handle may be used from one host thread at a time.
 */
#ifndef MACLAB_H
#define MACLAB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t maclab_status;
#define MACLAB_OK 0
#define MACLAB_WARN_RLE 1          /* lattice Reynolds number U dx / nu > 1 (stated
                                      stability bound, sentence after Eq. (6)) */
#define MACLAB_ERR_INVALID (-1)    /* bad argument, size, pointer or mask */
#define MACLAB_ERR_CUDA (-2)       /* CUDA runtime error (launch, copy, device fault) */
#define MACLAB_ERR_NONFINITE (-3)  /* NaN or Inf found in the state */
#define MACLAB_ERR_TIMEOUT (-4)    /* a bounded device-side wait ran out */
#define MACLAB_ERR_OOM (-5)        /* device or host allocation failed */
#define MACLAB_ERR_UNSUPPORTED (-6)/* valid request that this library does not serve */

typedef enum { MACLAB_D2Q9 = 0, MACLAB_D3Q19 = 1 } maclab_lattice;

/* How the state is stored on the device.  Arithmetic is FP64 for MACLAB_F64
 * and FP32 for the others.  The density is stored as drho = rho / rho0 - 1 and
 * the velocity in lattice units u / e. */
typedef enum {
  MACLAB_F64 = 0,
  MACLAB_F32 = 1,
  MACLAB_BF16_STORE = 2,
  MACLAB_F16_STORE = 3
} maclab_precision;

typedef enum { MACLAB_HOST = 0, MACLAB_DEVICE = 1 } maclab_where;
typedef enum { MACLAB_DTYPE_F64 = 0, MACLAB_DTYPE_F32 = 1 } maclab_dtype;

typedef struct maclab_ctx *maclab_handle;

/*
 * Problem statement, following the paper's procedure step (i): choose dx,
 * give nu; the library derives e = 6 nu / dx and dt = dx / e (Eq. (6)).
 */
typedef struct {
  int32_t lattice;          /* maclab_lattice */
  int32_t precision;        /* maclab_precision */
  int64_t dims[3];          /* nx, ny, nz (nz = 1 for D2Q9); each >= 1 */
  double dx;                /* lattice spacing, > 0 */
  double nu;                /* kinematic viscosity, > 0 */
  double rho0;              /* reference density (<= 0 means 1, as in the tests) */
  uint32_t periodic;        /* bit0 x, bit1 y, bit2 z */
  const uint8_t *node_type; /* HOST array of N bytes, or NULL (all fluid):
                               0 = fluid, k >= 1 = wall node with wall id k.  On a
                               non-periodic axis the first and last layers must
                               be wall nodes. */
  int32_t n_wall_ids;       /* number of wall ids (ids 1..n_wall_ids) */
  const double *wall_rho;   /* HOST, n_wall_ids physical densities (NULL = rho0) */
  const double *wall_u;     /* HOST, n_wall_ids * 3 physical velocities (x,y,z) */
  double body_force[3];     /* physical body acceleration, e.g. -(1/rho0) dp/dx of
                               Test 2; 0 = none.  Added after the division of
                               Eq. (5) as force * dt / e in lattice units. */
  void *stream;             /* cudaStream_t to run on, or NULL (default stream) */
} maclab_config;

/* Create a solver for one domain.  Copies the config and its tables, allocates
 * the device state (two buffers of (d + 1) * N values) and sets the state to
 * rest (rho = rho0, u = 0) with wall values in place.  Returns
 * MACLAB_WARN_RLE (with a valid handle) if a wall speed exceeds the stated
 * stability bound.  Errors: MACLAB_ERR_INVALID (dims, dx, nu, lattice,
 * precision, wall ids, or an open boundary on a non-periodic axis),
 * MACLAB_ERR_OOM, MACLAB_ERR_CUDA.  On error *out is NULL. */
maclab_status maclab_create(const maclab_config *cfg, maclab_handle *out);

/* Free the handle and its device memory (synchronises its stream). NULL is OK.
 * No paper counterpart: the end of the procedure after Eq. (6) (step (v):
 * repeat until a solution is reached) leaves the owner to release the state. */
maclab_status maclab_destroy(maclab_handle h);

/* out[0] = e (Eq. (6)), out[1] = dt = dx / e, out[2] = lattice Reynolds number
 * of the fastest wall, max|U_w| dx / nu, out[3..5] = body force per step in
 * lattice units, out[6] = fluid node count, out[7] = steps taken so far. */
maclab_status maclab_params(maclab_handle h, double out[8]);

/* Set the state from physical fields: rho (N values) and u (d * N values) of
 * the given dtype, in host or device memory -- step (i) of the procedure after
 * Eq. (6), the initial rho and u, stored in lattice units (u / e with e from
 * Eq. (6), rho / rho0).  Wall nodes are overwritten with their wall id's
 * values (the physical variables retained on walls, Tests 1-3 and 5).  Resets
 * the step counter.  Host buffers that are
 * page-locked and mapped for the handle's device (cudaHostAlloc,
 * cudaHostRegister) are read by the conversion kernel directly; other host
 * memory goes through a device staging buffer.  Either way the call returns
 * only after the host buffers have been read. */
maclab_status maclab_set_state(maclab_handle h, const void *rho, const void *u,
                               int32_t where, int32_t dtype);

/* Per-node wall values: every wall node takes the physical (rho, u) given at
 * its position in rho (N values) and u (d * N values, logical order, same
 * layout, dtype and host/device rules as maclab_set_state); entries at fluid
 * nodes are not read.  Wall nodes keep these values through every step: the
 * paper retains the physical variables on walls with no calculation there
 * (the boundary treatment of Tests 1-3 and 5), and this extends the per-id
 * table of maclab_config to any field over the walls (a moving or curved
 * body, an inflow profile).  Written into both state buffers; may be called
 * between steps (the step counter is kept).  maclab_set_state afterwards puts
 * the id table's values back.  A handle without wall nodes ignores the call.
 * Errors: MACLAB_ERR_INVALID, MACLAB_ERR_OOM (host staging), MACLAB_ERR_CUDA. */
maclab_status maclab_set_wall_state(maclab_handle h, const void *rho, const void *u,
                                    int32_t where, int32_t dtype);

/* Read the current physical state into rho (N) and u (d * N): the macroscopic
 * variables of Eqs. (4)-(5) mapped back to physical units (u = e ut,
 * rho = rho0 (1 + drho)).  Synchronises.
 * Page-locked host buffers mapped for the device are written by the
 * conversion kernel directly, other host memory through a staging buffer. */
maclab_status maclab_get_state(maclab_handle h, void *rho, void *u, int32_t where,
                               int32_t dtype);

/* Raw stored state, (d + 1) * N values in the storage type of the precision
 * (double, float, bfloat16 or half): drho, then the d lattice velocity
 * components.  This is the checkpoint format: setting a state read earlier
 * resumes bit-identically. maclab_state_bytes gives the size in bytes. */
maclab_status maclab_state_bytes(maclab_handle h, size_t *bytes);
maclab_status maclab_get_lattice_state(maclab_handle h, void *state, int32_t where);
maclab_status maclab_set_lattice_state(maclab_handle h, const void *state, int32_t where);

/* Advance n >= 0 MacLAB steps (Eqs. (4)-(5), walls kept, periodic wrap),
 * asynchronously on the handle's stream. */
maclab_status maclab_step(maclab_handle h, int64_t n);

/* Step kernels.  MACLAB_KERNEL_AUTO lets the library choose (the default);
 * MACLAB_KERNEL_REFERENCE is the simple one-thread-per-node gather, kept as the
 * GPU-side yardstick; MACLAB_KERNEL_TILED is the staged, vectorised kernel;
 * MACLAB_KERNEL_FOLDED is its D3Q19 FP32 form without halo-row threads (the
 * tile's edge rows fold their halo rows in; needs ny divisible by the tile's
 * rows); MACLAB_KERNEL_SEGMENT is the batched D2Q9 kernel run on one domain
 * (a warp per 30-quad row segment, x exchange by warp shuffles; with two
 * steps per launch the rows are staged four ahead in the warp's own shared
 * memory; nx % 4 == 0; the tile's tz is its rows per work item, default 2
 * up to 65,536 quads, 4 above and 32 with two steps above 524,288 quads, and
 * ty the time steps per launch, 1 or 2, default 2 below 200,000 quads and,
 * with FP32 storage, above 524,288 quads, where two steps are supported, see
 * maclab_batch_set_depth), the default for D2Q9 grids with nx % 4 == 0 that the
 * block kernel does not take (below).  All compute Eqs.
 * (4)-(5) with the same terms per node (the folded kernel sums them in
 * another order; the segment and tiled kernels give identical bits).
 * MACLAB_KERNEL_ROWS2 is the D3Q19 kernel with two rows per thread (FP32,
 * BF16 or FP16 storage; nx % 4 == 0 with nx <= 128; ny divisible by the
 * tile's rows, 8 by default; the tile's ty is its rows, 4 or 8, and 8 for
 * 16-bit storage; the default for FP32 storage where it applies): the
 * equilibria moving between a thread's rows stay in registers and the rest of
 * the y exchange is read 16 bytes per direction; its terms are formed and
 * summed in yet another order, so it agrees with the others to rounding.
 * MACLAB_KERNEL_BLOCK is the block-resident D2Q9 kernel (FP32 or FP64
 * storage, nx % 4 == 0): a launch takes ty steps (1, 2, 4 or, with FP32, 8;
 * default 8 up to 65,536 node pairs and 4 above; FP64 4 up to 16,384 pairs
 * and 2 above) on tiles of 32 x 32 node pairs (pair j of a row holds x = j
 * and x = j + nx / 2; FP32: 2 x 2 pairs per thread, FP64: 32 x 16 pairs, one
 * per thread) held in registers, exchanging equilibria through warp shuffles
 * and shared memory, each tile with a halo of ty pairs and rows, so the state
 * passes through global memory once per ty steps; a run of n steps ends with
 * a one-step launch (the previous state is step n - 1).  Its sums run in the
 * tiled kernel's order: identical bits.  The default for FP32 and FP64 D2Q9
 * grids of up to 131,072 node pairs (512^2). */
#define MACLAB_KERNEL_AUTO 0
#define MACLAB_KERNEL_REFERENCE 1
#define MACLAB_KERNEL_TILED 2
#define MACLAB_KERNEL_FOLDED 3
#define MACLAB_KERNEL_SEGMENT 4
#define MACLAB_KERNEL_ROWS2 5
#define MACLAB_KERNEL_BLOCK 6

/* Choose the step kernel.  MACLAB_ERR_UNSUPPORTED if the tiled kernel cannot
 * serve this domain (then the handle keeps its previous choice). */
maclab_status maclab_set_kernel(maclab_handle h, int32_t kernel);

/* Programmatic dependent launch of the tiled, folded and segment step kernels
 * (on = 1, the default): a launch may be scheduled onto the GPU while the
 * previous step's kernel is still running; on the device it waits for that
 * kernel to complete, and for its writes to be visible, before reading or
 * writing any state, so the results are bit-identical with on = 0 (plain
 * stream-ordered launches).  It shortens the gap between consecutive steps.
 * The reference kernel is always launched plainly; maclab_tune may change the
 * setting.  No paper counterpart (a launch detail of Eqs. (4)-(5)'s time
 * loop).  Drops the handle's captured graphs.  Errors: MACLAB_ERR_INVALID (NULL
 * handle, on not 0 or 1). */
maclab_status maclab_set_launch_overlap(maclab_handle h, int32_t on);

/* *on receives the handle's launch-overlap setting (1 or 0).  Errors:
 * MACLAB_ERR_INVALID (NULL argument). */
maclab_status maclab_get_launch_overlap(maclab_handle h, int32_t *on);

/* Tile shape of the kernel in use.  Tiled and folded kernels: ty rows of y per
 * block (3D only) and tz planes of the slowest axis per block.  Segment kernel:
 * ty time steps per launch (1 or 2; 2 needs FP32 or FP64 storage and nx >= 8,
 * and a run of n steps then ends with a one-step launch so that the previous
 * state is step n - 1) and tz rows per work item; ty = 3 runs the two-step
 * launches of one maclab_step call as the sweeps of a single persistent
 * cooperative launch, each block waiting between sweeps (bounded, see
 * maclab_set_wait_limit) only for the blocks that own rows within two of its
 * own; the results are bit-identical with ty = 2.  0 keeps the library's
 * default (for the segment kernel it depends on the grid's size).  MACLAB_ERR_UNSUPPORTED if no built instance has that shape for this
 * domain (the previous shape is kept). */
maclab_status maclab_set_tile(maclab_handle h, int32_t ty, int32_t tz);

/* Describe the kernel in use: out[0] = kernel id (REFERENCE, TILED, FOLDED or SEGMENT),
 * out[1] = time steps advanced per launch, out[2] = kernel launches per
 * launch group, out[3] = threads per block (out[3] = 0 and out[1..2] = 1 for
 * the reference kernel's grid-stride launch of 256-thread blocks).  *name (may be NULL) receives a
 * static string naming the kernel instance. */
maclab_status maclab_kernel_info(maclab_handle h, int32_t out[4], const char **name);

/* FP64 diagnostics over the fluid nodes (walls excluded), physical units:
 * out[0] mass, sum of rho; out[1] kinetic energy, sum of rho |u|^2 / 2;
 * out[2..4] momentum, sum of rho u_i (out[4] = 0 in 2D); out[5] steady
 * residual ||u^n - u^(n-1)||_2 / ||u^n||_2 (lattice units; -1 when the
 * previous step's state is not held, e.g. right after a set_state);
 * out[6] largest |u| / e (lattice Mach number); out[7] number of non-finite
 * stored values.  Mass and momentum are invariants of the periodic update
 * (Eq. (15)).  Synchronises the stream.  Returns MACLAB_ERR_NONFINITE (with
 * out filled) if out[7] > 0. */
maclab_status maclab_diagnostics(maclab_handle h, double out[8]);

/* The same reduction as raw FP64 sums over the fluid nodes, in lattice units,
 * so that the diagnostics of several sub-domains (maclab_get_planes) can be
 * added up exactly: out[0] sum drho, out[1] sum rho |u|^2, out[2..4] sum
 * rho u_i, out[5] sum |u - u_prev|^2 and out[6] sum |u|^2 (both -1 when the
 * previous state is not held), out[7] max |u|, out[8] non-finite count (the
 * layout of maclab_diagnostics_noalloc).  Mass and momentum are the
 * invariants of Eq. (15).  Synchronises the stream. */
maclab_status maclab_diagnostics_sums(maclab_handle h, double out[9]);

/* The same raw sums written to device memory (out: 9 doubles on the handle's
 * device; out[5] and out[6] are the residual sums over the state one step
 * back, meaningful only when that state is held), asynchronously on the
 * handle's stream: no host round trip, so it can sit between steps of a
 * running loop.  Errors: MACLAB_ERR_INVALID, MACLAB_ERR_CUDA. */
maclab_status maclab_diagnostics_device(maclab_handle h, double *out);

/* Raw planes of the march axis (z in 3D, y in 2D) of the current lattice
 * state, for decomposing a domain into slabs along that axis.  A slab is a
 * domain closed along the axis whose first and last planes are wall nodes
 * (never computed into, Tests 1-3 and 5: values retained) that hold copies of
 * the neighbouring slabs' edge planes: the one-layer ghost exchange of a
 * radius-1 stencil (every c_a has |c_a,z| <= 1 in Eqs. (4)-(5)).
 * maclab_get_planes copies planes [p0, p0 + count) of every field into dst
 * laid out [field][plane][stored values of a plane] (storage order, storage
 * type); maclab_set_planes writes src (same layout) into them.  where:
 * MACLAB_HOST or MACLAB_DEVICE (a device buffer may be on another device with
 * peer access).  One copy per field on the handle's stream; with host buffers
 * the call synchronises.  set_planes changes the current state only: the
 * residual of maclab_diagnostics compares it with the previous step's state as
 * that is held (ghost planes are walls and take no part).  Errors: MACLAB_ERR_INVALID (range, where),
 * MACLAB_ERR_CUDA. */
maclab_status maclab_get_planes(maclab_handle h, int64_t p0, int64_t count, void *dst, int32_t where);
maclab_status maclab_set_planes(maclab_handle h, int64_t p0, int64_t count, const void *src, int32_t where);

/* Capture maclab_step's launches in CUDA graphs of `steps` time steps each
 * (rounded up to an even count; 0 turns graphs off, the default is 32).
 * Graphs are built on first use and rebuilt after any change of kernel or
 * tile shape. */
maclab_status maclab_set_graph(maclab_handle h, int32_t steps);

/* ---------------------------------------------------------------- batches
 * Many independent domains advanced together: every maclab_batch_step is one
 * kernel launch over the work items of all domains (D2Q9 domains whose nx is a
 * multiple of 4), or one launch per domain otherwise, and runs of steps are
 * captured in CUDA graphs.  Domains may differ in size, dx, nu, walls and
 * force; they must share lattice, precision, device and stream. */
typedef struct maclab_batch_ctx *maclab_batch;

/* Create a batch from `count` configurations (see maclab_create).  Returns
 * MACLAB_WARN_RLE if any member warned. */
maclab_status maclab_batch_create(const maclab_config *cfgs, int32_t count, maclab_batch *out);
maclab_status maclab_batch_destroy(maclab_batch b);

/* Handle of member i, for maclab_set_state / get_state / diagnostics and the
 * other per-domain calls.  The batch owns it (do not destroy it).  Stepping a
 * member with maclab_step puts it out of step with the batch, which
 * maclab_batch_step then reports as MACLAB_ERR_INVALID. */
maclab_status maclab_batch_member(maclab_batch b, int32_t i, maclab_handle *out);

/* Advance every member by n steps.  With two steps per launch
 * (maclab_batch_set_depth) the last of the n steps is a one-step launch, so
 * every member's other buffer holds step n - 1 as after single steps. */
maclab_status maclab_batch_step(maclab_batch b, int64_t n);

/* Rows of a domain per work item (the tuning knob of the single launch);
 * 0 = library default.  Rebuilds the work list. */
maclab_status maclab_batch_set_rows(maclab_batch b, int32_t rows);

/* Time steps per launch of the single launch (temporal blocking): 1 (0 =
 * the default, 1) or 2.  With 2, each warp carries its row segment through two
 * updates of Eqs. (4)-(5) in registers, a two-quad and two-row halo wide, and
 * the intermediate state never goes to memory; results are bit-identical to
 * single steps.  3 is the persistent form of 2: every step pair of one
 * maclab_batch_step call runs in a single cooperative launch (the procedure
 * after Eq. (6), step (ii) repeated, on all domains at once), where between
 * two sweeps a block waits only for the blocks owning rows of its domains
 * within two rows of its own (per-block finished-sweep counters, acquire and
 * release ordering).  Every block is resident, so every wait ends; each is
 * bounded all the same (maclab_batch_set_wait_limit), and one that runs out
 * ends that block's sweeps and sets the status word that maclab_sync (on any
 * member) returns as MACLAB_ERR_TIMEOUT.  Bit-identical to depth 2.
 * MACLAB_ERR_UNSUPPORTED unless the batch uses one launch per step, stores
 * FP32 or FP64 and every nx >= 8 (depth 3 also when the cooperative launch
 * does not fit on the device; the batch then keeps two steps per launch).
 * Rebuilds the work list. */
maclab_status maclab_batch_set_depth(maclab_batch b, int32_t depth);

/* Polls a wait between blocks of the persistent batch launch may take before
 * it gives up (as maclab_set_wait_limit; < 0 restores the default).  No paper
 * counterpart.  Errors: MACLAB_ERR_INVALID (NULL batch, above 2^32 - 1). */
maclab_status maclab_batch_set_wait_limit(maclab_batch b, int64_t polls);

/* maclab_set_launch_overlap for the batch's launches and its members
 * (maclab_batch_tune may change it).  Errors: MACLAB_ERR_INVALID (NULL batch,
 * on not 0 or 1). */
maclab_status maclab_batch_set_launch_overlap(maclab_batch b, int32_t on);

/* out[0] members, out[1] total nodes, out[2] fluid nodes, out[3] work items
 * per launch (0 when one launch per member is used), out[4] rows per item,
 * out[5] kernel launches per step, out[6] time steps per launch (3: the
 * persistent form of two, maclab_batch_set_depth). */
maclab_status maclab_batch_info(maclab_batch b, int64_t out[7]);

/* ---------------------------------------------------------------- tuning
 * Time the candidate shapes of the tiled, folded and segment kernels (rows
 * per tile, planes per block; rows per work item and steps per launch) on
 * this handle's domain and keep the fastest kernel and shape, then time that
 * shape with and without launch overlap (maclab_set_launch_overlap) and turn
 * the overlap off only if plain launches are faster by more than 0.5 %; the
 * state is saved before and restored after (temporary device buffers are
 * allocated).
 * Results are cached per (lattice, precision, dims, periodicity, wall mode,
 * device model) for the process.  If the environment variable
 * MACLAB_TUNE_CACHE names a file, a shape not yet tuned in this process is
 * looked up there first (lines "<key> <kernel> <ty> <tz> [<overlap>]", the
 * last line for a key wins) and each newly tuned one is appended to it; an
 * unreadable file or malformed lines are ignored.  out (may be NULL) receives
 * the chosen ty, tz. */
maclab_status maclab_tune(maclab_handle h, int32_t out[2]);

/* The same for a batch: chooses the rows per work item and the time steps per
 * launch (1, 2 or the persistent form 3, compared per step), then the launch
 * overlap as above; *rows receives the rows. */
maclab_status maclab_batch_tune(maclab_batch b, int32_t *rows);

/* ---------------------------------------------------------------- adjoint
 * Reverse mode of maclab_step, for gradients of a loss on the final state
 * with respect to the initial fields, the wall values, the body force and nu.
 * Not in the paper; it is the chain rule applied to Eqs. (2), (4), (5) (see
 * adjoint.cu).  Adjoint arrays hold (d + 1) * N values of the arithmetic type
 * (double for MACLAB_F64, float otherwise) -- the adjoint of drho, then of
 * the d lattice velocity components -- in the same node order as the raw
 * state of maclab_get_lattice_state.  All array arguments of these calls are
 * DEVICE pointers; the calls run on the handle's stream. */

/* Size in bytes of one adjoint array. */
maclab_status maclab_adjoint_bytes(maclab_handle h, size_t *bytes);

/* One reverse step.  state_n: raw state at step n; state_np1: the raw state
 * one maclab_step later; lam_np1: adjoint of state_np1; lam_n (output, must
 * not alias lam_np1): adjoint of state_n.  grad_force (d doubles, or NULL)
 * accumulates the gradient with respect to the lattice-unit body-force
 * increment.  The first call allocates a scratch array of the adjoint size
 * owned by the handle. */
maclab_status maclab_adjoint_step(maclab_handle h, const void *state_n, const void *state_np1,
                                  const void *lam_np1, void *lam_n, double *grad_force);

/* The viscosity term of one reverse step: *acc (device, one double,
 * accumulated) += sum over fluid nodes x of lam_np1(x) . D_n(x), where state_n
 * is the raw state a maclab_step consumed and lam_np1 the adjoint of the state
 * it produced.  nu enters a rollout only through the particle speed e = 6 nu
 * / dx of Eq. (6) (initial and wall velocities u / e, force increment g dt / e,
 * output u = e ut; the update of Eqs. (4)-(5) itself does not depend on e), and
 * D_n is the defect of one step under that scaling: with ut'_nf = m' / rho'
 * the output without the force F and J (0, ut) the step's derivative along the
 * velocities, D_n = (ut'_nf - J (0, ut) - F, -J (0, ut) on drho).  Summed over
 * the steps of a rollout, e dL/de = sum_n sum_x lam_(n+1) . D_n, so
 * dL/dnu = (6 / dx) (1 / e) sum; each term is formed directly, without the
 * near-cancellation of the end-point products that maclab_adjoint_finish
 * subtracts (which loses accuracy in FP32 when the flow is nearly linear in u).
 * state_np1 (optional, may be NULL): the raw state that step produced.  With
 * it, on FP32 storage where the two-rows-per-thread D3Q19 step is built, the
 * term is one tiled pass: it gathers the moments of
 * g_a = w_a (drho + rho (3/2 u.u - 9/2 (c.u)^2)) and takes rho' and m' / rho'
 * from state_np1 (J (0, ut) on drho = R - sum g, with R = 36 drho').  Without
 * it (or elsewhere) a per-node kernel gathers the 19 neighbours of every node.
 * Asynchronous on the handle's stream.  Errors: MACLAB_ERR_INVALID,
 * MACLAB_ERR_CUDA. */
maclab_status maclab_adjoint_nu_term(maclab_handle h, const void *state_n, const void *state_np1,
                                     const void *lam_np1, double *acc);

/* Seed the reverse pass: the gradients of the loss with respect to the
 * physical output fields rho (N values) and u (d * N values, logical order;
 * either may be NULL = zero) of dtype, for the raw final state state_T, give
 * the adjoint array lam_T.  *dot_T receives sum over nodes of lam_u . u
 * (lattice units), which maclab_adjoint_finish needs for dL/dnu.
 * Synchronises the stream. */
maclab_status maclab_adjoint_seed(maclab_handle h, const void *grad_rho, const void *grad_u,
                                  int32_t dtype, const void *state_T, void *lam_T, double *dot_T);

/* Finish the reverse pass from lam_0, the adjoint of the raw initial state
 * state_0 (the state maclab_set_state produced).  Outputs (any may be NULL):
 * grad_rho0 / grad_u0 (device, dtype, logical order): gradients with respect
 * to the physical rho and u given to maclab_set_state (zero on wall nodes,
 * whose values come from the wall tables); grad_wall (HOST, n_wall_ids * 4
 * doubles): gradient with respect to each wall id's physical (rho, u_x, u_y,
 * u_z); grad_scalars (HOST, 5 doubles): [0] dL/dnu, [1] dL/de, [2..4]
 * gradient with respect to the physical body acceleration.  dot_T comes from
 * maclab_adjoint_seed; grad_force_lat (HOST, d doubles) is the sum of all
 * maclab_adjoint_step grad_force outputs.  The loss is taken at a fixed
 * number of steps: changing nu changes e = 6 nu / dx and so the lattice
 * velocities of the initial field, the walls and the output, and the force
 * increment force * dx / e^2.  Synchronises the stream. */
maclab_status maclab_adjoint_finish(maclab_handle h, const void *lam_0, const void *state_0,
                                    void *grad_rho0, void *grad_u0, int32_t dtype, double dot_T,
                                    const double *grad_force_lat, double *grad_wall,
                                    double *grad_scalars);

/* Diagnostics sums without any device allocation.  (Not part of the method:
 * the paper has no counterpart.)  For callers that cannot allocate device
 * memory while they run -- for example a host loop that reserved all device
 * memory for its own pool up front, or code that may not block on an
 * allocation.  The per-block partial sums live in a fixed array of 288 KiB
 * that every GPU loading the library holds until the process exits; one call
 * reduces at most 33,554,432 nodes (larger n_nodes: MACLAB_ERR_INVALID).
 *
 * state: device, (d + 1) * n_nodes stored values of the precision's storage
 *   type, drho then the d lattice velocity components, in any node order
 *   (e.g. a buffer filled by maclab_get_lattice_state).
 * prev_state: device, the same layout one step earlier, or NULL (then the
 *   residual sums are 0).
 * exclude: device, n_nodes bytes in the same node order, nonzero = leave the
 *   node out (walls), or NULL.
 * out_sums: device, 9 doubles written with the raw lattice-unit sums over the
 *   included nodes: [0] sum drho, [1] sum rho |u|^2, [2..4] sum rho u_i,
 *   [5] sum |u - u_prev|^2, [6] sum |u|^2, [7] max |u|, [8] non-finite count.
 * stream: cudaStream_t (NULL = default stream); the call is asynchronous.
 *
 * All four pointers must be device (or managed) memory usable by the current
 * device; anything else (a host buffer, another GPU's memory) is rejected with
 * MACLAB_ERR_INVALID before any launch.
 *
 * The first call on a device (and again after the device's context is
 * replaced, e.g. by cudaDeviceReset) sets up, with that device current: it
 * loads the reduction kernels, whose code lazy module loading would otherwise
 * load -- possibly taking device memory -- at their first launch, and looks up
 * the array's address.  Make that first call before reserving the device's
 * memory for other uses and before any stream capture.
 * Every call on a device reuses the same array: calls that overlap on the GPU
 * race.  Nothing in it needs clearing between calls (each call writes the
 * entries it reads).  No cudaMalloc, cudaFree or other allocating routine is
 * called.  Errors: MACLAB_ERR_INVALID (arguments, size, pointers),
 * MACLAB_ERR_CUDA. */
maclab_status maclab_diagnostics_noalloc(int32_t lattice, int32_t precision, int64_t n_nodes,
                                         const void *state, const void *prev_state,
                                         const uint8_t *exclude, double *out_sums,
                                         void *stream);

/* Self-check of the reciprocal the FP32 kernels use for u' = m' / rho'
 * (Eq. (5)): evaluates it on the device at n points spaced geometrically over
 * [lo, hi] (0 < lo < hi, 1 <= n <= 2^24) and stores the largest relative error
 * against 1/x in FP64 in *max_rel_err.  No paper counterpart: it checks an
 * implementation choice (a hardware approximation refined by one
 * Newton-Raphson step).  Runs on the current device, synchronously.
 * Errors: MACLAB_ERR_INVALID (arguments), MACLAB_ERR_OOM, MACLAB_ERR_CUDA. */
maclab_status maclab_check_reciprocal(float lo, float hi, int32_t n, double *max_rel_err);

/* Measure the current device's paired-FP32 FMA rate (the arithmetic the FP32
 * kernels use: one instruction, two fused multiply-adds on a float2) in
 * TFLOP/s, counting two operations per FMA: independent chains at full
 * occupancy, the best of three timed launches after a warm-up.  The D3Q19
 * step is checked against it beside the memory roofline.  No paper
 * counterpart (a measurement of the device).  Runs on the current device and
 * the default stream, synchronously; allocates 2 KB of device memory for the
 * call.  Errors: MACLAB_ERR_INVALID (NULL tflops), MACLAB_ERR_OOM,
 * MACLAB_ERR_CUDA. */
maclab_status maclab_measure_fp32_peak(double *tflops);

/* Debug builds only (compiled with -DMACLAB_BOUNDS_CHECK, libmaclab_bounds.so):
 * the number of out-of-bounds indices the checked kernels met on the current
 * device since the last call (out[0]) and the first such index (out[1]); the
 * log is cleared.  The checked kernels (the D3Q19 two-rows-per-thread step)
 * compare every global and shared-memory index with the size of its buffer
 * and skip a bad access instead of making it; nothing traps.  No paper
 * counterpart (a verification aid).  Synchronises the device.  Errors:
 * MACLAB_ERR_UNSUPPORTED in normal builds, MACLAB_ERR_INVALID, MACLAB_ERR_CUDA. */
maclab_status maclab_debug_bounds(int64_t out[2]);

/* Run the handle's stream to completion and report any CUDA error.  Also
 * reads and clears the device's status word: MACLAB_ERR_TIMEOUT if, since the
 * last check, a step kernel's bounded wait (for a tile copy, or for another
 * block of a persistent launch) ran out (the kernel then finished with
 * undefined values in the state it wrote). */
maclab_status maclab_sync(maclab_handle h);

/* Budget of the bounded waits between blocks of the persistent segment launch
 * (maclab_set_tile ty = 3): polls of a neighbouring block's counter before the
 * wait gives up.  polls < 0 restores the default (2^22); 0 makes every such
 * wait give up at once, so that the next maclab_sync returns
 * MACLAB_ERR_TIMEOUT and the state is undefined until the next set_state.  A
 * verification aid: with every block resident the waits always end.  No paper
 * counterpart.  Errors: MACLAB_ERR_INVALID (NULL handle, polls > 2^32 - 1). */
maclab_status maclab_set_wait_limit(maclab_handle h, int64_t polls);

/* The persistent segment launch's work items and wait lists for a D2Q9 domain
 * of nx x ny nodes (nx % 4 == 0, nx >= 8; periodic_y != 0 if y wraps), rows
 * rows per item and `blocks` blocks of four warps (warp w takes items w,
 * w + 4 blocks, ...).  items receives 4 ints per item (0, x segment, first
 * row, end row); waits receives blocks + 1 offsets into waits itself, then
 * each block's list of the other blocks it waits for between sweeps.  lens[0]
 * and lens[1] receive the number of ints each needs; with a capacity that is
 * too small nothing is copied and MACLAB_ERR_INVALID is returned (call with
 * 0 capacities to size the arrays).  Host only, no device work.  A
 * verification aid with no paper counterpart. */
maclab_status maclab_debug_segment_waits(int32_t nx, int32_t ny, int32_t periodic_y, int32_t rows,
                                         int32_t blocks, int32_t *items, int64_t items_cap, int32_t *waits,
                                         int64_t waits_cap, int64_t lens[2]);

/* The same for the persistent batch launch (maclab_batch_set_depth 3): the
 * work items and wait lists of `count` D2Q9 domains of nx[i] x ny[i] nodes
 * (nx[i] % 4 == 0, nx[i] >= 8; periodic_y[i] != 0 if domain i wraps in y),
 * rows rows per item.  items: 4 ints per item (domain, x segment, first row,
 * end row), the domains' items in order; waits, lens and the capacity rule as
 * above.  A block waits only for blocks owning rows of the same domain within
 * two rows of its own.  Host only, no device work.  A verification aid with
 * no paper counterpart. */
maclab_status maclab_debug_batch_waits(int32_t count, const int32_t *nx, const int32_t *ny,
                                       const int32_t *periodic_y, int32_t rows, int32_t blocks,
                                       int32_t *items, int64_t items_cap, int32_t *waits,
                                       int64_t waits_cap, int64_t lens[2]);

/* Name of a status code (static string). */
const char *maclab_status_string(maclab_status s);

/* Library build tag, e.g. "maclab sm_103a". */
const char *maclab_version(void);

/* Message of the last failing call on this host thread (empty if none). */
const char *maclab_last_error(void);

/* ---------------------------------------------------------------- comparator
 * The scheme MacLAB replaces: the single-relaxation-time lattice Boltzmann
 * method of Eq. (1) (BGK collision, relaxation time tau), which stores the
 * distributions f and streams and collides them every step.  Fully periodic
 * D2Q9 grids in lattice units (lattice viscosity (tau - 1/2) / 3); no walls,
 * force or adjoint.  It holds 2 x 9 values per node and moves 9 + 9 per update
 * (72 B in FP32, against MacLAB's 2 x 3 held and 24 B moved), which is the
 * memory and traffic claim of the paper's introduction and discussion; at
 * tau = 1 it gives MacLAB's (rho, u) (Methods, Eqs. (9)-(13)).  One kernel per
 * step: every node gathers the streamed post-collision distributions of its
 * upstream neighbours, forms (rho, u) (Eq. (3)) and the equilibria (Eq. (2)),
 * relaxes and stores the nine post-collision values.  Velocity order and
 * weights as the paper lists them with Eq. (1). */
typedef struct maclab_lbm_ctx *maclab_lbm;

/* nx, ny >= 1 nodes; tau > 1/2; precision MACLAB_F32 or MACLAB_F64 (values
 * stored and computed in that type); stream: a cudaStream_t or NULL for the
 * default stream.  Allocates the two distribution buffers and a staging
 * buffer on the current device.  Errors: MACLAB_ERR_INVALID, MACLAB_ERR_OOM,
 * MACLAB_ERR_CUDA. */
maclab_status maclab_lbm_create(int32_t nx, int32_t ny, double tau, int32_t precision, void *stream,
                                maclab_lbm *out);
maclab_status maclab_lbm_destroy(maclab_lbm h);

/* Start from f = f^eq(rho, u) (Eq. (2)).  Host arrays, x fastest: rho[ny][nx],
 * u[2][ny][nx] (lattice units, u / e).  Synchronises the stream. */
maclab_status maclab_lbm_set_state(maclab_lbm h, const double *rho, const double *u);

/* n steps, queued on the stream. */
maclab_status maclab_lbm_step(maclab_lbm h, int64_t n);

/* The moments (rho, u) of the current distributions (Eq. (3)) into host
 * arrays shaped as in maclab_lbm_set_state.  Synchronises the stream. */
maclab_status maclab_lbm_get_state(maclab_lbm h, double *rho, double *u);

/* out[0] nodes, out[1] bytes of device state (both distribution buffers),
 * out[2] bytes read and written per node update, out[3] steps taken. */
maclab_status maclab_lbm_info(maclab_lbm h, int64_t out[4]);

#ifdef __cplusplus
}
#endif

#endif /* MACLAB_H */
