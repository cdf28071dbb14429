/*
 * lbm.h -- C ABI of the GB300 D3Q19 lattice Boltzmann library.
 *
 * The library advances a 3D D3Q19 BGK lattice (Guo body force, periodic or
 * half-way bounce-back faces, one moving lid) on one GPU, in place, with a
 * single copy of the populations.  It implements the hot path of Fu & Song,
 * "Designing a 3D Parallel Memory-Aware Lattice Boltzmann Algorithm on
 * Manycore Systems" (arXiv 2208.05429): the fused collide-and-stream update
 * (Sec. 3, Alg. 1) and its merge of two collision-streaming cycles into one
 * sweep over memory (Sec. 4.1, Alg. 2; Sec. 4.2, Alg. 3), re-designed for the
 * GPU as an AA-pattern even/odd pair and a tiled kernel that performs both
 * steps per HBM round trip.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Return value: an lbm_status (0 = success, negative = error).  Nothing
 *    throws across the ABI; lbm_strerror() gives a static message.
 *  - Pointers documented as "device" are CUDA device pointers owned by the
 *    caller (for example torch tensors); the library never frees them and
 *    only reads/writes them on the handle's stream.  Arguments documented as
 *    "host" are plain host memory.
 *  - Canonical field layout (inputs and outputs): x fastest, then y, then z:
 *      scalar field  a[z][y][x]              (N = nx*ny*nz elements)
 *      vector field  a[3][z][y][x]           (component-major)
 *      populations   f[q][z][y][x]           (direction-major, q = 19, or
 *                                             15 / 27 for those lattices,
 *                                             directions in the order
 *                                             lbm_lattice_q() reports)
 *  - Every launch is asynchronous on the stream given at creation.  Only
 *    lbm_reduce() and lbm_adjoint_* with host outputs synchronise it.
 *  - A handle is not thread-safe; use one handle per host thread.
 *  - The populations held by a handle always represent the post-stream state
 *    f^n after n time steps; the AA parity used internally is hidden.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_handle lbm_handle;

/* Status codes. */
enum lbm_status {
    LBM_OK = 0,
    LBM_EINVAL = -1,        /* invalid argument or configuration            */
    LBM_ENOMEM = -2,        /* device allocation failed / buffer too small  */
    LBM_ECUDA = -3,         /* a CUDA runtime call failed                   */
    LBM_ESTATE = -4,        /* call not valid in the handle's current state */
    LBM_ENONFINITE = -5,    /* a reduction met a NaN or Inf                 */
    LBM_ETIMEOUT = -6,      /* a bounded device wait gave up                */
    LBM_EUNSUPPORTED = -7   /* combination not built in this library        */
};

/* Face boundary types; faces are ordered x-, x+, y-, y+, z-, z+.  The two
 * faces of one axis are either both PERIODIC or both non-periodic. */
enum { LBM_BC_PERIODIC = 0, LBM_BC_WALL = 1, LBM_BC_LID = 2 };

/* Population storage.  F64 and F32 store f_i; the "S" forms store the
 * shifted value f_i - w_i (w_i the lattice weight), which keeps the small
 * deviations from rest at full relative precision.  All forms except F64
 * compute in FP32 registers; F64 computes in FP64. */
enum { LBM_STORAGE_F64 = 0, LBM_STORAGE_F32 = 1, LBM_STORAGE_F32S = 2,
       LBM_STORAGE_F16S = 3, LBM_STORAGE_BF16S = 4 };

/* Update schedule.  All of them give bit-identical populations for the same
 * storage (Sec. 5.1 of the paper verifies its two-step solvers against the
 * single-step ones the same way).
 *   TWO_LATTICE  fused collide-and-push into a second lattice (reference
 *                form of Alg. 1; needs twice the population memory)
 *   AA           single copy: even step collides in place into the opposite
 *                slots (the "revert" of Sec. 3), odd step gathers, collides
 *                and scatters (the "swap_stream" half of Sec. 3)
 *   MERGED       single copy of the lattice, two time steps per sweep
 *                (Sec. 4): one CTA per 32 x 14 column tile (32 x 4 in F64)
 *                marches z; each interval it does the odd step of plane k and
 *                the even step of plane k+2, handing post-collision values
 *                between the two through shared-memory rings.  Two kernels
 *                make the tiles safe where they meet (the role of the
 *                intersection layers of Alg. 3):
 *                - neighbour-synchronised sweep (every face a wall or lid,
 *                  4- and 2-byte storage, at least half as many tiles as
 *                  SMs, all tiles resident at once): one cooperative launch;
 *                  a tile pushes into a plane only after its eight neighbour
 *                  tiles have copied that plane, which they announce in
 *                  per-tile progress words in global memory (bounded waits,
 *                  status bit 8);
 *                - shadow-shell sweep (otherwise): the tile-boundary cells
 *                  also live in a double-buffered shadow that the sweep
 *                  reads from the current copy and writes to the next, so
 *                  tiles need no synchronisation (with fewer tiles than
 *                  SMs, z is split into chunks of at least 4 planes; the
 *                  environment variable LBM_MERGED_ZCHUNKS sets the chunk
 *                  count at handle creation).
 *                LBM_MERGED_SWEEP=shadow at handle creation selects the
 *                shadow-shell sweep, =neighbour the neighbour-synchronised
 *                one for any tile count it can hold resident.  Where
 *                neither sweep can run (a periodic z with nz = 1, or a
 *                shadow beyond 2^31 elements) MERGED runs the AA pair.
 *   KSTEP        K = sweep_steps (3 or 4) time steps per sweep on two
 *                lattices, the merge of more than two steps the paper
 *                leaves as future work (Sec. 6): each 16 x 8 (K = 3) or
 *                16 x 4 (K = 4) column tile marches z with K levels of
 *                post-collision planes in shared memory, the level-s values
 *                on the tile widened by K - s cells (halos recomputed by
 *                every tile that reads them, no tile waits on another).
 *                4- and 2-byte storage, D3Q19, BGK (LBM_EUNSUPPORTED
 *                otherwise); step counts not divisible by K end with
 *                two-lattice steps. */
enum { LBM_VARIANT_TWO_LATTICE = 0, LBM_VARIANT_AA = 1, LBM_VARIANT_MERGED = 2, LBM_VARIANT_KSTEP = 3 };

/* Body force (Guo forcing): none, one vector for every cell, or a per-cell
 * FP32 field [3][z][y][x] set with lbm_set_force(). */
enum { LBM_FORCE_NONE = 0, LBM_FORCE_UNIFORM = 1, LBM_FORCE_FIELD = 2 };

/* Collision operator.  BGK: one relaxation rate 1/tau.  TRT: the parts of
 * the populations that are symmetric / antisymmetric under c -> -c relax
 * with 1/tau and with omega-, where (tau - 1/2)(1/omega- - 1/2) = trt_lambda.
 * REG (regularised BGK): before relaxing with 1/tau, f - feq is replaced by
 * its projection on the Hermite polynomials up to second order,
 * w_i (3 c_i.J + 4.5 (c_i c_i - I/3) : Pi) with J, Pi its first and second
 * moments, which removes the higher ("ghost") moments.  MRT: f - feq is split
 * into its parts of Hermite order up to two, three and four (orthogonal in
 * sum_i w_i a_i b_i on D3Q19), relaxed with 1/tau, mrt_s3 and mrt_s4
 * (mrt_s3 = mrt_s4 = 1/tau is BGK, = 1 is REG).  (The paper's solver
 * builds on "collision models" without naming one, Sec. 1; the schedules of
 * Sec. 3-4 are independent of the model.)  Every schedule runs all three;
 * MERGED runs TRT and REG with the neighbour-synchronised sweep where that
 * can run and as the AA pair elsewhere (the shadow-shell sweep is BGK only).
 * The adjoint calls return LBM_EUNSUPPORTED for a handle without BGK. */
enum { LBM_COLLISION_BGK = 0, LBM_COLLISION_TRT = 1, LBM_COLLISION_REG = 2, LBM_COLLISION_MRT = 3 };

/* Velocity set (lbm_config.lattice): D3Q19, the paper's lattice, or the two
 * other cubic sets for which its dependency guard holds (Sec. 4.1): D3Q15
 * (rest, 6 faces, 8 corners; w = 2/9, 1/9, 1/72) and D3Q27 (every vector of
 * {-1, 0, 1}^3; w = 8/27, 2/27, 1/54, 1/216).  c_s^2 = 1/3 on all three.
 * D3Q15 and D3Q27 run the single-step schedules (TWO_LATTICE, AA; MERGED
 * runs the AA pair) with every storage format and the BGK, TRT and REG
 * collisions; MRT and the adjoint calls return LBM_EUNSUPPORTED for them.
 * 0 means D3Q19. */
enum { LBM_LATTICE_D3Q15 = 15, LBM_LATTICE_D3Q19 = 19, LBM_LATTICE_D3Q27 = 27 };

/* Element type of caller-provided field buffers. */
enum { LBM_DTYPE_F32 = 0, LBM_DTYPE_F64 = 1 };

typedef struct lbm_config {
    int64_t nx, ny, nz;       /* cells per axis, each >= 1                     */
    double tau;               /* BGK relaxation time, > 0.5                    */
    int32_t face_bc[6];       /* x-, x+, y-, y+, z-, z+ (LBM_BC_*)             */
    double u_lid[3];          /* velocity of every LID face, |u_lid| < 0.3     */
    double rho_wall;          /* density in the moving-wall term (default 1)   */
    int32_t storage;          /* LBM_STORAGE_*                                 */
    int32_t variant;          /* LBM_VARIANT_*                                 */
    int32_t force_mode;       /* LBM_FORCE_*                                   */
    double force_uniform[3];  /* the force of LBM_FORCE_UNIFORM                */
    int32_t collision;        /* LBM_COLLISION_* (default BGK)                  */
    double trt_lambda;        /* TRT magic product, > 0 (default 3/16)          */
    double mrt_s3, mrt_s4;    /* MRT rates of the third- and fourth-order
                                 moments, in (0, 2) (default 1)                 */
    int32_t lattice;          /* LBM_LATTICE_* (default D3Q19; 0 = D3Q19)       */
    int32_t sweep_steps;      /* time steps per KSTEP sweep: 3 or 4 (0 = 3)     */
} lbm_config;

/* Fill cfg with a 32^3 fully periodic FP32 AA D3Q19 lattice, tau = 0.6, BGK
 * (trt_lambda = 3/16 and mrt_s3 = mrt_s4 = 1 for a later switch to TRT or
 * MRT). */
void lbm_config_default(lbm_config *cfg);

/* Check a configuration without allocating.  LBM_EINVAL on: a dimension < 1,
 * cell count beyond 2^31, tau <= 0.5, a face type out of range, an axis with
 * one periodic and one non-periodic face, |u_lid| >= 0.3, rho_wall <= 0,
 * unknown storage/variant/force mode, collision or lattice, a trt_lambda that
 * is not positive and finite, or an MRT rate outside (0, 2).
 * LBM_EUNSUPPORTED for MRT on D3Q15 or D3Q27, and for KSTEP with FP64
 * storage, another lattice or another collision; LBM_EINVAL for a
 * sweep_steps other than 0, 3 or 4. */
int lbm_validate(const lbm_config *cfg);

/* Device bytes a handle of this configuration uses (populations, second
 * lattice for TWO_LATTICE and KSTEP, tile-shell shadow or progress words for MERGED,
 * reduction scratch), each region aligned to
 * 256 bytes.
 * *bytes is a host output.  For MERGED the figure depends on the current
 * device (its SM count and the resident CTAs choose the sweep and the z
 * chunks) and on LBM_MERGED_SWEEP and LBM_MERGED_ZCHUNKS, all read at each
 * call: query with the device and environment the handle will be created
 * with. */
int lbm_required_bytes(const lbm_config *cfg, size_t *bytes);

/* Create a handle that allocates its own device memory (stream-ordered,
 * cudaMallocAsync on `stream`, current device; released with cudaFreeAsync
 * on the same stream by lbm_destroy) and launches on `stream` (a
 * cudaStream_t; NULL = legacy default stream).  Populations start at zero: call lbm_init_equilibrium()
 * or lbm_init_populations() before stepping.  *out receives the handle. */
int lbm_create(const lbm_config *cfg, void *stream, lbm_handle **out);

/* Same as lbm_create() but uses `device_buffer` (device, at least
 * lbm_required_bytes() bytes, 256-byte aligned, owned by the caller and
 * kept alive until lbm_destroy()).  LBM_ENOMEM if `bytes` is too small. */
int lbm_create_with_buffer(const lbm_config *cfg, void *stream, void *device_buffer,
                           size_t bytes, lbm_handle **out);

/* Release the handle (and the memory lbm_create() allocated).  NULL is a
 * no-op.  Synchronises the handle's stream first. */
void lbm_destroy(lbm_handle *h);

/* Static message for a status code. */
const char *lbm_strerror(int status);

/* The library's D3Q19 table: c[19][3] integer velocities and w[19] weights
 * (host outputs, either may be NULL).  Directions 1..9 are those whose first
 * non-zero component is -1 (the half of the neighbours the swap algorithm of
 * Sec. 3 streams to), direction i+9 is the opposite of i, 0 is rest. */
int lbm_lattice(int32_t *c, double *w);

/* The table of lattice q (LBM_LATTICE_*, 0 = D3Q19): c[q][3] and w[q] (host
 * outputs, either may be NULL), ordered by the same rule: 0 is rest,
 * directions 1 .. (q-1)/2 have -1 as first non-zero component (in
 * lexicographic (cx, cy, cz) order for D3Q15 and D3Q27), direction
 * i + (q-1)/2 is the opposite of i.  LBM_EINVAL for another q. */
int lbm_lattice_q(int32_t q, int32_t *c, double *w);

/* Populations of every cell := equilibrium feq(rho, u) (second-order BGK
 * equilibrium) and the time counter := 0.  rho: device [z][y][x] or NULL
 * (rho = 1); u: device [3][z][y][x] or NULL (u = 0); both of element type
 * `dtype`.  This is the initial state of the cavity of Sec. 5.1. */
int lbm_init_equilibrium(lbm_handle *h, const void *rho, const void *u, int32_t dtype);

/* Set the per-cell body force used when force_mode == LBM_FORCE_FIELD.
 * F: device FP32 [3][z][y][x], borrowed: it must stay valid and unchanged
 * while steps are in flight.  LBM_ESTATE for other force modes. */
int lbm_set_force(lbm_handle *h, const float *F);

/* Advance n >= 0 time steps (one step = collide then stream, Sec. 3).  With
 * MERGED, pairs of steps run as one two-step sweep (Sec. 4) and
 * an odd remainder as one AA step; with KSTEP, groups of sweep_steps steps
 * run as one K-step sweep and a remainder as two-lattice steps.  Asynchronous on the handle's stream.
 * Calls with n >= 32 (outside profiling) capture the launches of 32 steps
 * once into a CUDA graph and replay it, on an internal stream ordered after
 * and before the handle's stream; a new force field drops the graph. */
int lbm_step(lbm_handle *h, int64_t n);

/* Time steps taken since the last init (host output). */
int lbm_time(const lbm_handle *h, int64_t *t);

/* Density and velocity of the current state (the per-cell velocity norm the
 * paper's verification logs is |u|, Sec. 5.1): rho = sum_i f_i,
 * u = (sum_i f_i c_i + F/2) / rho.  rho: device [z][y][x] or NULL; u: device
 * [3][z][y][x] or NULL; element type `dtype`. */
int lbm_moments(lbm_handle *h, void *rho, void *u, int32_t dtype);

/* Copy out the post-stream populations f^n in canonical layout
 * f[q][z][y][x] (device, element type `dtype`, directions as lbm_lattice_q()
 * of the handle's lattice). */
int lbm_populations(lbm_handle *h, void *f_out, int32_t dtype);

/* Replace the state with caller populations f_in (device, canonical layout,
 * element type `dtype`, rounded to the storage format) and reset time to 0. */
int lbm_init_populations(lbm_handle *h, const void *f_in, int32_t dtype);

/* Global FP64 sums of the current state, written to out[5] (host):
 *   out[0] = sum rho              (mass)
 *   out[1..3] = sum_cells sum_i f_i c_i   (momentum, without the half force)
 *   out[4] = sum 1/2 rho |u|^2    (kinetic energy, u as in lbm_moments)
 * Deterministic (fixed summation tree).  Synchronises the stream.
 * LBM_ENONFINITE if any cell has a non-finite density or velocity; out is
 * still written.  LBM_ETIMEOUT if, since the previous call, a MERGED sweep
 * gave up waiting for one of its asynchronous plane copies or for a
 * neighbouring tile's progress word (every wait in the kernels is
 * bounded); the lattice is then
 * invalid and the flag is cleared. */
int lbm_reduce(lbm_handle *h, double *out);

/* The sums of lbm_reduce() for a population field the caller holds, computed
 * without allocating any device memory and without a handle.  The paper has
 * no counterpart: this is for callers that cannot call cudaMalloc -- a
 * process whose free device memory is all held by a caching allocator (such
 * as PyTorch's, where cudaMalloc fails although the pool has room), a
 * serving or stepping loop that must not take the device-wide
 * synchronisation of cudaMalloc / cudaFree, or code running inside an
 * allocator callback.
 *   cfg    lattice sizes and body force (force_mode, force_uniform); the
 *          whole config must pass lbm_validate(), so lattices beyond
 *          2^31 - 1 cells are rejected with LBM_EINVAL; storage, variant
 *          and collision are ignored; the lattice must be D3Q19
 *          (LBM_EUNSUPPORTED otherwise)
 *   f      device, canonical natural-parity populations f[19][z][y][x] of
 *          element type `dtype` (LBM_DTYPE_F32 or _F64), directions as
 *          lbm_lattice() -- what lbm_populations() writes
 *   F      device FP32 [3][z][y][x] when force_mode == LBM_FORCE_FIELD
 *          (else ignored, may be NULL)
 *   out    host double[5], as lbm_reduce(): mass, momentum xyz, kinetic energy
 *   stream cudaStream_t to run on (NULL = legacy default stream); the call
 *          synchronises it
 * Scratch: one file-scope device array of 41,088 bytes (1024 x 5 FP64
 * partial sums, the five results and a flag), present on every GPU that
 * loads the library until the process exits; enough for every lattice
 * lbm_validate() accepts.  The first call on a device looks up that array's
 * device address (once per device, with the device current): make that
 * first call before any stream capture on the device.  All calls in the
 * process share the array and it keeps the last call's contents (the flag
 * is cleared at the start of each call), so calls that overlap on the GPU
 * -- on two streams, or from two host threads -- race and must be
 * serialised by the caller.  Returns LBM_ENONFINITE (out still written) as
 * lbm_reduce() does, LBM_EINVAL for bad arguments, LBM_ECUDA on a CUDA
 * error, LBM_EUNSUPPORTED for a device ordinal of 64 or more. */
int lbm_reduce_populations(const lbm_config *cfg, const void *f, int32_t dtype, const float *F, double *out,
                           void *stream);

/* ---------------- per-kernel timing ----------------
 * Kernel classes launched by lbm_step(). */
enum { LBM_KERNEL_TWO_LATTICE = 0, LBM_KERNEL_AA_EVEN = 1, LBM_KERNEL_AA_ODD = 2,
       LBM_KERNEL_SNAPSHOT = 3, LBM_KERNEL_MERGED = 4, LBM_KERNEL_KSTEP = 5, LBM_KERNEL_COUNT = 6 };
/* LBM_KERNEL_SNAPSHOT: the shadow-shell sweep's copies made before a sweep
 * (the tile shells after a single step, the planes at z-chunk boundaries);
 * LBM_KERNEL_MERGED: either two-step sweep; LBM_KERNEL_KSTEP: the K-step
 * sweep. */

/* enable = 1: from now on every kernel lbm_step() launches is bracketed by
 * two CUDA events recorded on the handle's stream (earlier records are
 * dropped); enable = 0 stops recording and keeps the records.  The events
 * are created on first use and owned by the handle. */
int lbm_profile(lbm_handle *h, int32_t enable);

/* Launch count and summed device time (milliseconds, from the events) of
 * one kernel class (LBM_KERNEL_*) since profiling was last enabled; host
 * outputs.  Synchronises on the recorded events. */
int lbm_profile_read(lbm_handle *h, int32_t kernel, int64_t *launches, double *total_ms);

/* Self-test of the failure detection of a MERGED handle that runs the
 * neighbour-synchronised sweep: runs one sweep in which the tile in the
 * middle of the grid never announces its progress, so that its neighbours'
 * bounded waits for it run out (a second or two), they give up, and so does
 * every tile that waits for them.  No kernel faults, traps or spins without
 * a limit.  The populations are left undefined (partly stepped): re-create
 * the state with lbm_init_equilibrium() or lbm_init_populations() before
 * stepping again; the step count is unchanged.  Returns LBM_ETIMEOUT when
 * the give-up was recorded in the status word (which is cleared again),
 * LBM_OK if nothing was recorded, LBM_ESTATE for a handle without that
 * sweep, at odd parity (after an odd number of steps) or with a force
 * field not yet set.  Synchronises the stream. */
int lbm_selftest_wait_timeout(lbm_handle *h);

/* ---------------- adjoint (reverse-mode) ----------------
 * The reverse of one step f^t -> f^{t+1} of this handle's configuration,
 * derived by hand from the collide and stream rules above (the paper has no
 * counterpart).  The wall-density rho_wall is a constant, so the lid term
 * carries no derivative.  Computation in the handle's compute precision,
 * gradient accumulation in FP64. */

/* lambda_out = (d f^{t+1} / d f^t)^T lambda_in, and dLdF += (d f^{t+1}/dF)^T
 * lambda_in per cell.  f_t: device canonical populations of the state the
 * forward step started from; lambda_in / lambda_out: device canonical
 * populations (distinct buffers); all three of element type `dtype`.
 * dLdF: device FP64 [3][z][y][x], accumulated (may be NULL). */
int lbm_adjoint_step(lbm_handle *h, const void *f_t, const void *lambda_in, void *lambda_out,
                     int32_t dtype, double *dLdF);

/* Seed of the reverse sweep for a loss L(rho, u) of the moments of the
 * current state: lambda = dL/df (device canonical, `dtype`), and
 * dLdF += dL/du / (2 rho) (the half-force path of u; FP64, may be NULL).
 * dLdrho: device [z][y][x] or NULL; dLdu: device [3][z][y][x]; both `dtype`. */
int lbm_adjoint_seed(lbm_handle *h, const void *dLdrho, const void *dLdu, void *lambda,
                     int32_t dtype, double *dLdF);

/* Workspace bytes for lbm_adjoint_forward/backward with T steps and a
 * checkpoint every K steps: ceil(T/K)+1 checkpoints, two segment buffers
 * (one segment is recomputed while the adjoint runs through the other), each
 * two states and the moments rho, u of K states (all of f^t the adjoint step
 * reads), and two adjoint buffers.  Host output. */
int lbm_adjoint_workspace_bytes(const lbm_handle *h, int64_t T, int64_t K, size_t *bytes);

/* Run T >= 1 steps forward from the current state (which becomes f^0),
 * keeping a checkpoint every K >= 1 steps in `work` (device, at least the
 * bytes above, owned by the caller and left untouched until
 * lbm_adjoint_backward returns).  Leaves the handle at f^T, bit-identical to
 * lbm_step(T). */
int lbm_adjoint_forward(lbm_handle *h, int64_t T, int64_t K, void *work, size_t work_bytes);

/* Reverse sweep of the last lbm_adjoint_forward: seeds with dL/drho, dL/du of
 * f^T (device, `dtype`, dLdrho may be NULL), recomputes each K-step segment
 * from its checkpoint and applies lbm_adjoint_step backwards.  Writes
 * dLdf0 = dL/df^0 (device canonical populations, `dtype`, may be NULL) and
 * accumulates dLdF += dL/dF (device FP64 [3][z][y][x], may be NULL).
 * Asynchronous on the handle's stream: the segment recomputes run on an
 * internal stream of the handle, ordered after the work already on the
 * handle's stream and before the adjoint steps that read them (events), so
 * that the recompute of one segment overlaps the adjoint of the next. */
int lbm_adjoint_backward(lbm_handle *h, const void *dLdrho, const void *dLdu, int32_t dtype,
                         void *dLdf0, double *dLdF, void *work, size_t work_bytes);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
