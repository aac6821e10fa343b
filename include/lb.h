/*
 * lb.h -- C ABI of the GB300 (sm_103a) forced D3Q19 lattice Boltzmann
 * library with off-lattice singular point forces, after Nash, Adhikari &
 * Cates, "Singular forces and point-like colloids in lattice Boltzmann
 * hydrodynamics".
 *
 * Model (lattice units, dt = dx = 1, rest density rho0 = 1):
 *   - D3Q19 populations, advanced as the auxiliary distribution
 *     fbar = f - (dt/2) R of Sec. II, Eq. (transformf), stored as the
 *     deviation df_i = fbar_i - w_i from the rest state;
 *   - multiple-relaxation-time collision with the second-order forcing
 *     term, Sec. II, Eq. (fiexp): ghost modes projected out, traceless
 *     stress relaxed at 1/(tau_shear + 1/2), its trace at
 *     1/(tau_bulk + 1/2); shear viscosity eta = tau_shear / 3;
 *   - pull streaming, fused with the collision in one kernel;
 *   - singular forces spread to the lattice with Peskin's 4-point
 *     regularised delta function, Sec. III, Eq. (deltadef);
 *   - lattice velocity interpolated back with the same kernel and point
 *     colloids moved by the Faxen relation with the a_L subtraction,
 *     Sec. IV, Eq. (a_Ldefn).
 *
 * Conventions for every call:
 *   - Every function returns an lb_status and never aborts; on failure
 *     lb_last_error() describes it.  Arguments are validated on the host
 *     before anything is launched.
 *   - The context owns its device memory (allocated in lb_create, freed in
 *     lb_destroy).  Pointer arguments stay owned by the caller.  A pointer
 *     argument may point to host memory or to device memory of the
 *     context's GPU; the library tells them apart with
 *     cudaPointerGetAttributes.
 *   - Work is issued on the stream given to lb_create.  Calls whose
 *     outputs are all in device memory return without waiting; a call
 *     that writes host memory waits for its own copies.
 *   - Positions are in lattice units with nodes at integer coordinates
 *     0 .. n-1 in each axis, periodic.  Forces are force densities per
 *     lattice site (a point force F spreads to F delta^P).
 *   - Population layout (lb_get_populations / lb_set_populations):
 *     df[i][z][y][x] as double, i in the order
 *       0:(0,0,0) 1:(1,0,0) 2:(-1,0,0) 3:(0,1,0) 4:(0,-1,0) 5:(0,0,1)
 *       6:(0,0,-1) 7:(1,1,0) 8:(-1,-1,0) 9:(1,-1,0) 10:(-1,1,0)
 *       11:(1,0,1) 12:(-1,0,-1) 13:(1,0,-1) 14:(-1,0,1) 15:(0,1,1)
 *       16:(0,-1,-1) 17:(0,1,-1) 18:(0,-1,1)
 *     with weights 1/3 (rest), 1/18 (axes), 1/36 (diagonals).  The state
 *     held between steps is the post-collision df* of the last step.
 */
#ifndef GB300_LB_H
#define GB300_LB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_ctx lb_ctx;

typedef enum {
    LB_OK = 0,
    LB_ERR_ARG = 1,        /* invalid argument; nothing was launched */
    LB_ERR_CUDA = 2,       /* a CUDA call failed; see lb_last_error */
    LB_ERR_OOM = 3,        /* device allocation failed */
    LB_ERR_NONFINITE = 4,  /* a non-finite value was found in an input */
    LB_ERR_STATE = 5,      /* call not valid in the context's state */
    LB_ERR_TIMEOUT = 6     /* a bounded device-side wait ran out; see lb_mlp_last_error */
} lb_status;

/* Storage precision of the populations.  F64: double storage and
 * arithmetic.  F32: float storage and arithmetic.  F16S / BF16S: df
 * stored as half / bfloat16 multiplied by a power-of-two scale (the
 * deviation from the rest state is small, so half precision needs the
 * scale to stay out of subnormals); arithmetic in float. */
typedef enum { LB_F64 = 0, LB_F32 = 1, LB_F16S = 2, LB_BF16S = 3 } lb_precision;

/* Kinds of singular force (Sec. III and IV). */
typedef enum {
    LB_STOKESLET = 0, /* one fixed force monopole F at pos */
    LB_STRESSLET = 1, /* collinear pair: +F at pos + (sep/2) F^, -F at pos - (sep/2) F^ */
    LB_ROTLET = 2,    /* four tangential forces of magnitude |T|/(2 arm) at
                         pos +- (arm/2) e1, pos +- (arm/2) e2 (Fig. rotlet);
                         (e1, e2, T^) right-handed, e1 = the coordinate axis
                         least aligned with T^ (lowest index on ties),
                         orthogonalised to T^; +F e2 at +e1, -F e2 at -e1,
                         -F e1 at +e2, +F e1 at -e2; torque T, net force 0 */
    LB_COLLOID = 3    /* a mobile point colloid of radius a pushed by the
                         external force F (Sec. IV) */
} lb_kind;

/* Create a lattice of grid[0] x grid[1] x grid[2] sites (x fastest), each
 * >= 1 and their product < 2^32, at rest (df = 0).  tau_shear, tau_bulk
 * > 0 are the relaxation times of Sec. II in the convention
 * eta = rho cs^2 tau_shear (rate 1/(tau + 1/2)); precision is an
 * lb_precision; stream is a cudaStream_t (NULL: the legacy default
 * stream).  Allocates two population buffers, a force field and the
 * point arrays on the current device.  Sec. II, Eqs. (mrtlbe), (fiexp). */
lb_status lb_create(lb_ctx **out, const int grid[3], double tau_shear, double tau_bulk,
                    int precision, void *stream);

/* Free everything the context owns.  Waits for its stream.  NULL is a no-op. */
void lb_destroy(lb_ctx *ctx);

/* Description of the last failure on this context (or of a failed
 * lb_create when ctx is NULL); never NULL. */
const char *lb_last_error(const lb_ctx *ctx);

/* Uniform body-force density g (3 doubles, host memory) on every fluid
 * site, the smooth "gravity" forcing of Sec. I. */
lb_status lb_set_body_force(lb_ctx *ctx, const double g[3]);

/* Make the z-planes z_lo and z_hi solid (halfway bounce-back; walls at
 * z_lo + 1/2 and z_hi - 1/2).  -1 disables a plane.  Walls are not part
 * of the paper; they serve the body-force channel flow. */
lb_status lb_set_walls_z(lb_ctx *ctx, int z_lo, int z_hi);

/* Enable (default) or disable the uniform counter-force -sum F / V_fluid
 * on fluid sites that cancels the net point force in a periodic box
 * (the k = 0 removal of Appendix A). */
lb_status lb_set_counterforce(lb_ctx *ctx, int enabled);

/* Lattice offset parameter a_L of Eq. (a_Ldefn) used by the colloid update
 * (a_L > 0; +inf turns the subtraction off).  Default +inf. */
lb_status lb_set_colloid_aL(lb_ctx *ctx, double a_L);

/* Append n singular forces of one kind.  pos, F: 3n doubles (xyz per
 * point; host or device), F is the force (STOKESLET, COLLOID), the pair
 * force (STRESSLET) or the torque (ROTLET).  param: n doubles (host or
 * device) -- separation (STRESSLET), arm (ROTLET), radius a (COLLOID);
 * may be NULL for STOKESLET.  Positions are wrapped into the box.  The
 * points are expanded into monopoles on the device; the total count
 * after expansion must stay below 2^31 / 64.  Sec. III, IV. */
lb_status lb_add_point_forces(lb_ctx *ctx, int n, const double *pos, const double *F, int kind,
                              const double *param);

/* Remove every point force. */
lb_status lb_clear_point_forces(lb_ctx *ctx);

/* Number of monopoles after expansion. */
lb_status lb_num_points(const lb_ctx *ctx, int *n_out);

/* Replace the positions of all monopoles (3 * lb_num_points doubles, host
 * or device, in the order they were created), each wrapped into the box;
 * forces are kept.  A NaN or an infinity anywhere rejects the whole update
 * with LB_ERR_NONFINITE and leaves every position as it was.  Device
 * positions are checked on the device, so that case waits for the stream. */
lb_status lb_set_positions(lb_ctx *ctx, const double *pos);

/* Host memory without waiting (default off).  With on != 0, a call that
 * copies results into host memory (lb_velocity_at, lb_colloid_velocity,
 * lb_moments, lb_particles, lb_get_populations) enqueues the copy on the
 * context's stream and returns without waiting for it; host inputs are
 * read by copies enqueued likewise.  The caller leaves every host buffer
 * it passed untouched until lb_synchronize returns.  Host buffers should be
 * page-locked (cudaHostAlloc, cudaHostRegister) for the copies to run
 * asynchronously.  Calls that read a device status on the host
 * (lb_add_point_forces, lb_set_positions with device positions, lb_save,
 * ...) still wait. */
lb_status lb_set_host_async(lb_ctx *ctx, int on);

/* Advance nsteps >= 0 time steps.  Each step: spread the point forces at
 * their current positions (unless the previous step already did), collide
 * and stream every site, then interpolate the velocity at each colloid,
 * move it (forward Euler, dt = 1) and spread the forces at the new
 * positions for the next step.  Sec. II-IV. */
lb_status lb_step(lb_ctx *ctx, int nsteps);

/* Velocity v = (sum fbar c + F/2) / rho (Eq. macrovariables2) interpolated
 * with delta^P at n query points pos (3n doubles) into v_out (3n
 * doubles); host or device pointers. */
lb_status lb_velocity_at(lb_ctx *ctx, int n, const double *pos, double *v_out);

/* Fields at the current time: rho (V doubles) and u (3V doubles, u[a][z][y][x])
 * -- either may be NULL -- and totals[4] = {sum rho, sum rho u} over fluid
 * sites accumulated in FP64 (NULL allowed).  Solid sites report rho = 1,
 * u = 0.  Host or device pointers. */
lb_status lb_moments(lb_ctx *ctx, double *rho, double *u, double *totals);

/* Current monopole positions and forces (3 * lb_num_points doubles each;
 * either may be NULL; host or device). */
lb_status lb_particles(lb_ctx *ctx, double *pos_out, double *f_out);

/* Copy the population state out / in, as df[i][z][y][x] doubles (19V;
 * host or device).  Reduced-precision storage is converted. */
lb_status lb_get_populations(lb_ctx *ctx, double *df);
lb_status lb_set_populations(lb_ctx *ctx, const double *df);

/* Number of kernels this context has launched since lb_create (a running
 * count kept on the host; copies and memsets are not counted). */
lb_status lb_kernel_launches(const lb_ctx *ctx, long long *count);

/* Phase timing of lb_step, for measurement (not part of the paper).  With
 * on != 0 every lb_step records a pair of CUDA events on the context's
 * stream around each phase of each step; lb_phase_times waits for the
 * stream and returns, per phase, the summed elapsed time in milliseconds
 * (ms, 5 doubles, host) and the number of timed occurrences (counts, 5
 * long longs, host, may be NULL) since the last call, then recycles the
 * events.  Phases: 0 spreading at the current positions (the first step,
 * or after the points changed), 1 collide + stream, 2 point phase
 * (interpolation, colloid update, spreading at the new positions), 3 the
 * periodic cell-order sort, 4 learned correction (features and forward).  The
 * events are host-side objects: no device memory is allocated.  Turning
 * timing off waits for the stream and discards unread pairs.  LB_ERR_STATE
 * if a step failed between the two events of a pair. */
lb_status lb_set_phase_timing(lb_ctx *ctx, int on);
lb_status lb_phase_times(lb_ctx *ctx, double ms[5], long long counts[5]);

/* Checkpoint of the whole state of a context: lattice parameters, the
 * expanded point list (positions, forces, radii, mobility), the populations
 * of the current step in the storage format (raw bytes: the restored state
 * is the saved one bit for bit), and the stochastic-rounding seed, followed
 * by a 64-bit FNV-1a hash of the file.  The continued run equals the
 * uninterrupted one bit for bit wherever no two stencils overlap (where
 * they do, the order of the spreading atomics may change the last bits).  lb_save waits for the context's stream
 * and writes `path` (LB_ERR_ARG if it cannot be written).  lb_load reads a
 * checkpoint into a context of the same grid and precision and replaces
 * its state; LB_ERR_ARG for a missing, foreign, truncated or corrupt file
 * or a grid or precision mismatch (the context is then unchanged).  Host
 * memory of one population buffer is used while loading.  Not part of the
 * paper: restart support for long runs. */
lb_status lb_save(lb_ctx *ctx, const char *path);
lb_status lb_load(lb_ctx *ctx, const char *path);

/* Wait for all work issued on the context's stream. */
lb_status lb_synchronize(lb_ctx *ctx);

/* a_L of Appendix A for a lattice grid[3] and a point R (3 doubles, host):
 * 1/a_L = (6 pi / V) sum_{k != 0} |delta^P(k;R)|^2 / k^2 d.(1 - k^k^).d
 * along the unit vector d = dir (host, 3 doubles), or one third of the
 * trace when dir is NULL; k = 2 pi m / n, continuum |k|^2.  Evaluated on
 * the current device (allocates temporary device memory). */
lb_status lb_compute_aL(const int grid[3], const double R[3], const double dir[3], double *a_L);

/* Colloid velocity of Sec. IV at n query points: the interpolated fluid
 * velocity plus the Faxen term with the a_L subtraction,
 *   U = v(R) + F (1/a - 1/a_L) / (6 pi eta),
 * for forces F (3n doubles) and radii a (n doubles); host or device
 * pointers.  lb_step moves colloids with exactly this velocity. */
lb_status lb_colloid_velocity(lb_ctx *ctx, int n, const double *pos, const double *F, const double *radius,
                              double *U_out);

/* ------------------------------------------------------------------------
 * Learned correction of the colloid velocity: a 27 -> 64 -> 64 -> 3
 * perceptron with SiLU activations in bfloat16 (FP32 accumulation and
 * master weights), trained on pairs of runs of the method at two lattice
 * resolutions.  Input of a colloid: its fractional lattice offset and the
 * minimum-image vectors to its 8 nearest others within 8 lattice units
 * (nearest first, equal distances by lower index, in units of 4 lattice
 * spacings, zero where absent).  The vectors and the distances that select
 * and order them are float32, each operation rounded once: positions
 * rounded to float, d = x_j - x_i, then d -+ box beyond +-box/2, squared
 * distance (dx^2 + dy^2) + dz^2, kept up to 64.
 * Parameters: one float vector, W1[64][27] b1[64] W2[64][64] b2[64]
 * W3[3][64] b3[3] (lb_mlp_num_params() floats).  n-sized arrays are device
 * pointers; parameter vectors host or device.  Work runs on the stream
 * given at creation.  Not part of the paper: the method itself stays the
 * reference the correction is judged against.
 * --------------------------------------------------------------------- */
typedef struct lb_mlp lb_mlp;
int lb_mlp_num_params(void);
lb_status lb_mlp_create(lb_mlp **out, const float *init_params, void *stream);
void lb_mlp_destroy(lb_mlp *net);
const char *lb_mlp_last_error(const lb_mlp *net);
lb_status lb_mlp_get_params(lb_mlp *net, float *out);
lb_status lb_mlp_set_params(lb_mlp *net, const float *in);  /* also resets Adam */
/* feat[n][27] (float) from positions pos[n][3] (double) in a periodic box */
lb_status lb_mlp_features(lb_mlp *net, long long n, const double *pos, const int box[3], float *feat);
/* out[n][3] = network(feat); the two hidden layers run on the tensor cores
 * (tcgen05, bfloat16 operands, FP32 accumulation).  Waits for completion;
 * LB_ERR_TIMEOUT if the tensor-core pipeline did not complete within its
 * bounded wait (out is then incomplete). */
lb_status lb_mlp_forward(lb_mlp *net, long long n, const float *feat, float *out);
/* Bound of every wait of the tensor-core kernels on their own pipeline, in
 * polls of an mbarrier (default 2^26, far beyond any completion).  0 makes
 * the waits time out at once, which drives the timeout path: the forward
 * stops, waits with the default bound for the work it issued, frees its
 * tensor memory and returns LB_ERR_TIMEOUT; the network stays usable.
 * LB_ERR_ARG for polls < 0. */
lb_status lb_mlp_set_wait_limit(lb_mlp *net, long long polls);
/* gradient of (1/3n) sum (y - target)^2 (grad: num_params floats, host or
 * device, may be NULL) and the sum of squared errors (*sse, may be NULL);
 * waits for completion */
lb_status lb_mlp_grad(lb_mlp *net, long long n, const float *feat, const float *target, float *grad,
                      float *sse);
/* one Adam step (beta 0.9 / 0.999, eps 1e-8) on that gradient; *sse (may
 * be NULL) receives the sum of squared errors before the step */
lb_status lb_mlp_train_step(lb_mlp *net, long long n, const float *feat, const float *target, float lr,
                            float *sse);
/* `steps` Adam steps on minibatches drawn on the device: minibatch s takes
 * `batch` samples of (feat[n][27], target[n][3]) (device pointers), sample
 * b the row j = h(seed, s, b) mod n, h the SplitMix64 finaliser of
 * seed + (s * batch + b + 1) * 0x9E3779B97F4A7C15 shifted right by 11 (with
 * replacement); targets are divided by target_scale (> 0) as they are
 * gathered.  The learning rate of step s is max(lr (1 + cos(pi s / steps)) / 2,
 * 1e-6).  loss (host, may be NULL) receives the minibatch's mean squared
 * error before steps 0, e, 2e, ... (e = loss_every >= 1) and before the last
 * step: floor((steps - 1) / e) + 2 floats at most (the last step listed
 * once).  The draws and steps run on the network's stream without waiting;
 * the call waits once at the end.  Allocates its minibatch buffers on first
 * use (grown on demand).  LB_ERR_ARG for n < 1, batch < 1, steps < 1,
 * lr <= 0, target_scale <= 0 or non-finite, loss_every < 1. */
lb_status lb_mlp_train(lb_mlp *net, long long n, const float *feat, const float *target, float target_scale,
                       int batch, int steps, float lr, unsigned long long seed, int loss_every, float *loss);

/* Attach (net != NULL) or detach the learned correction to the colloid
 * update of lb_step: each mobile colloid then moves by
 *   U + y |F| / (6 pi eta a),  y = net(features of all points),
 * U the colloid velocity of lb_colloid_velocity.  The network is used, not
 * owned (keep it alive while attached; do not use it concurrently on
 * another stream).  Without a network the plain method of Sec. IV runs. */
lb_status lb_set_colloid_correction(lb_ctx *ctx, lb_mlp *net);

/* ------------------------------------------------------------------------
 * Batches: independent lattices (replicas of uneven sizes, e.g. many small
 * sedimentation boxes) advanced together, one persistent cooperative kernel
 * launch per time step over all members.  Inside the launch, every 64
 * steps the cell order of all colloids (a counting sort) and, on the first
 * step of a call whose force fields are not spread, the spread, each
 * followed by a grid-wide barrier; then a work queue that the blocks drain:
 * the collide + stream of every site of every member in chunks, member
 * after member (32-site windows of each member's flat site index when
 * every nx is a multiple of 8 and every member has fewer than 2^24 sites,
 * else 4 x 32-site tiles), then the point items -- interpolation, colloid
 * update and the spread of the forces at the new positions for the next
 * step -- each started once the collide of its own member is complete.
 * Every wait (barrier or queue) is bounded.  Two steps are replayed from a
 * CUDA graph.  The method per member is exactly that of lb_step.
 * --------------------------------------------------------------------- */
typedef struct lb_batch lb_batch;

/* Group n contexts (same device and precision) into a batch.  The batch
 * snapshots each member's configuration (points, forces, walls, body
 * force, relaxation times, a_L); the members keep their memory and every
 * per-context call (lb_moments, lb_particles, lb_velocity_at, ...) still
 * works between batch steps.  Reconfiguring or stepping a member on its own
 * makes the next lb_batch_step fail with LB_ERR_STATE: recreate the batch.
 * The batch orders its work after `stream` and every member's stream and
 * makes them wait for it.  Allocates a private stream and small tables. */
lb_status lb_batch_create(lb_batch **out, int n, lb_ctx *const *ctxs, void *stream);
void lb_batch_destroy(lb_batch *batch);
const char *lb_batch_last_error(const lb_batch *batch);

/* Autotune the grid of the persistent kernel: time whole batch steps for
 * grids of 2, 4, 6 and 8 blocks of 128 threads per SM (as many as can be
 * resident together), keep the fastest, report its block count in *blocks
 * (may be NULL).  Leaves every member's state unchanged: the trial steps
 * write only the spare population buffers, and the positions and counters
 * they move are put back; the force fields they spread are cleared (the
 * next step spreads again).  Waits for the batch's stream; LB_ERR_TIMEOUT
 * if a wait ran out during the trials. */
lb_status lb_batch_tune(lb_batch *batch, int *blocks);

/* Advance every member nsteps >= 0 time steps (Sec. II-IV, as lb_step).
 * Returns without waiting.  Afterwards each member's force field holds
 * the forces at its new positions (queries on a member use it as is). */
lb_status lb_batch_step(lb_batch *batch, int nsteps);

/* Wait for the batch's stream; LB_ERR_TIMEOUT if a wait (grid barrier or
 * work queue) of the steps issued since the last call ran out (those steps
 * are then incomplete and the members' state is undefined; the barrier and
 * the queue are reset so that the batch can be used again). */
lb_status lb_batch_synchronize(lb_batch *batch);

/* Bound of every wait of the batch kernel (grid barrier, or a point item
 * waiting for its member's collide), in polls of the word waited on with a
 * short sleep between polls (default 2^22, about a second).  0 makes every
 * wait that is not already satisfied give up at once, which drives the
 * timeout path.  Waits for the batch's stream; LB_ERR_ARG for polls < 0. */
lb_status lb_batch_set_wait_limit(lb_batch *batch, long long polls);

/* Sites and points over all members, the persistent grid size and the
 * number of kernels launched by the batch so far (any pointer may be NULL). */
lb_status lb_batch_info(const lb_batch *batch, long long *sites, long long *points, int *blocks,
                        long long *launches);

/* Totals {sum rho, sum rho u} over the fluid sites of a population array
 * that the caller owns, computed without allocating any device memory.
 * The paper has no counterpart to this call: it exists for callers that
 * cannot use cudaMalloc -- code whose device memory belongs to its own pool
 * allocator or fixed arena, and code that cannot tolerate cudaFree's
 * device-wide wait or an out-of-memory failure in the middle of a run --
 * and therefore cannot create an lb_ctx.
 *   df        device pointer, 19 * V elements laid out as df[i][z][y][x]
 *             (the order of lb_get_populations) in the storage format of
 *             `precision`: double (LB_F64), float (LB_F32), half holding
 *             df * 2^20 (LB_F16S) or bfloat16 (LB_BF16S).  It is read as
 *             the post-collision state; the totals are those of the pulled
 *             (streamed) state, as lb_moments reports them.
 *   grid      nx, ny, nz >= 1 with nx * ny * nz < 2^32 (host).
 *   z_lo, z_hi  solid z-planes with bounce-back, -1 for none.
 *   F         uniform force density on fluid sites (3 doubles, host; NULL
 *             for zero); it enters rho u = sum df c + F / 2.
 *   totals    device pointer to 4 doubles, written.
 *   stream    cudaStream_t the two kernels are launched on; the call does
 *             not wait for them.
 * Scratch: a library-wide static device array of 1024 x 4 doubles
 * (32 KiB) that every GPU using the library keeps until the process
 * exits.  Its device address is looked up (with the device current) by
 * every call whose stream is not capturing, so a device reset or a new
 * context never leaves a stale address; a call on a capturing stream
 * reuses the address found by the last such lookup on that device, so the
 * first call on a device should come before any stream capture (else
 * LB_ERR_STATE).  All calls share the array; calls whose kernels overlap
 * on the GPU race on it.
 * Errors: LB_ERR_ARG (NULL pointer, bad precision, grid or plane, or a
 * lattice beyond the limit above), LB_ERR_NONFINITE (F), LB_ERR_STATE,
 * LB_ERR_CUDA.  The pointers are trusted: df must hold 19 V elements of
 * the storage type and totals 4 doubles, both in device memory.
 * Does not call cudaMalloc, cudaFree or any allocating routine, and does
 * not touch lb_last_error. */
lb_status lb_totals_noalloc(const void *df, int precision, const int grid[3], int z_lo, int z_hi,
                            const double F[3], double *totals, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GB300_LB_H */
