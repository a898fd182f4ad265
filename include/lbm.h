/*
 * lbm.h - C ABI of the GB300 (sm_103a) variable-speed-of-sound D2Q9 lattice
 * Boltzmann library (liblbm.so).
 *
 * The method (Buick & Cosgrove, "Investigation of a Lattice Boltzmann Model
 * with a Variable Speed of Sound"):
 *
 *   Section 3, Eq. 5 (nbm):
 *     f_i(x + e_i, t + 1) - f_i(x, t) = -(f_i - fbar_i)/tau + 3 w_i alpha grad(rho).e_i
 *   Section 2, Eq. 2: fbar_i = w_i rho [1 + 3 e_i.u + 9/2 (e_i.u)^2 - 3/2 u^2]
 *   Section 2, Eq. 3: rho = sum_i f_i,  rho u = sum_i f_i e_i
 *   Section 3, Eq. 8 (cef): effective sound speed c_e^2 = c_1^2 - alpha, with
 *     c_1^2 = 1/3 on this lattice; the library takes c2 = c_e^2 and uses
 *     alpha = 1/3 - c2, so the sound speed is set independently of tau.
 *   Section 3, Eq. 7: viscosity nu = (2 tau - 1)/6, independent of alpha.
 *   Section 4: grad(rho) by central differences, (rho(x+1) - rho(x-1))/2 along
 *     x and y (the stable choice; lbm_set_gradient selects the forward
 *     difference the paper found unstable, for reproducing that result).
 *
 * Grids are periodic in x and y.  Fields passed in or out are row-major
 * [ny][nx] arrays of double (x fastest): element (x, y) is at index y*nx + x.
 *
 * Ownership: a handle owns its device memory (two distribution buffers and a
 * small reduction scratch area), freed by lbm_destroy.  Caller pointers are
 * only read or written during the call that receives them.  No call keeps a
 * caller pointer.  Per device, the library also keeps, for the life of the
 * process, a pool of staging memory for host fields and a copy stream.
 *
 * Errors: every call returns a status (LBM_OK = 0, negative on error, positive
 * for a warning); no C++ exception crosses this interface.  lbm_strerror maps
 * a status to text; lbm_last_error gives the detail of the calling thread's
 * most recent failure (for example the CUDA error string).
 *
 * Streams: work is queued on the handle's CUDA stream (the one passed to
 * lbm_create or lbm_set_stream, or the legacy default stream if NULL).
 * lbm_step only queues work; lbm_moments, lbm_sums, lbm_mode, lbm_get_state
 * and lbm_sync wait for the stream.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define LBM_OK 0
#define LBM_EINVAL (-1)      /* an argument is out of range or NULL */
#define LBM_ENOMEM (-2)      /* device or host allocation failed */
#define LBM_ECUDA (-3)       /* a CUDA runtime call failed (see lbm_last_error) */
#define LBM_ENONFINITE (-4)  /* a reduction met NaN or Inf */
#define LBM_ETIMEOUT (-5)    /* a bounded in-kernel wait ran out */
#define LBM_WUNSTABLE 1      /* warning: c2 > 1.2656 (c_e > 1.125), beyond the
                                largest sound speed the paper found stable
                                (Section 4); the handle is still created */

/* Storage of the distributions in device memory.  Arithmetic is FP32 in all
 * cases.  Every storage keeps h_i = (f_i - w_i rho0) / w_i, the deviation from
 * the rest equilibrium scaled by the weight, so that small waves keep their
 * precision; the 16-bit kinds round h_i on every store, to nearest-even or
 * stochastically (lbm_set_rounding). */
#define LBM_F32 0
#define LBM_F16D 1
#define LBM_BF16D 2

/* Rounding of the 16-bit stores (lbm_set_rounding). */
#define LBM_ROUND_NEAREST 0     /* round to nearest even (default) */
#define LBM_ROUND_STOCHASTIC 1  /* unbiased stochastic rounding */

/* Fields for lbm_mode. */
#define LBM_FIELD_RHO 0   /* rho - rho0 */
#define LBM_FIELD_UX 1
#define LBM_FIELD_UY 2

typedef struct lbm_grid *lbm_t;
typedef struct lbm_batch *lbm_batch_t;

/* Creates a periodic nx x ny grid (Section 2-3).
 *   nx, ny      >= 1, nx * ny <= 2^31 - 1
 *   tau         relaxation time, > 0.5 (Section 4: the model turns unstable as
 *               tau -> 0.5).  With a large sound speed the force lowers the
 *               margin for modes that vary in both x and y: at c_e = 0.9 to
 *               1.0 the linearised update has growing 2-D modes below
 *               tau = 0.52 to 0.53, while plane waves stay stable down to
 *               0.501 (no warning is returned for this)
 *   c2          squared sound speed c_e^2 > 0 (Eq. 8); alpha = 1/3 - c2
 *   storage     LBM_F32, LBM_F16D or LBM_BF16D
 *   cuda_stream a cudaStream_t (NULL: legacy default stream)
 *   out         receives the handle
 * The reference density rho0 of the stored deviations is 1 (the paper's
 * ambient density).  The state is undefined until lbm_init or lbm_set_state.
 * Returns LBM_OK, LBM_WUNSTABLE (created, see above), LBM_EINVAL, LBM_ENOMEM
 * or LBM_ECUDA. */
int lbm_create(int nx, int ny, double tau, double c2, int storage,
               void *cuda_stream, lbm_t *out);

/* As lbm_create with an explicit reference density rho0 > 0. */
int lbm_create_ex(int nx, int ny, double tau, double c2, double rho0,
                  int storage, void *cuda_stream, lbm_t *out);

/* Frees the handle and its device memory (waits for its stream first).
 * NULL is accepted. */
int lbm_destroy(lbm_t h);

/* Sets the state at t = 0 to the local equilibrium f_i = fbar_i(rho, u)
 * (Eq. 2) of the given fields (the paper gives rho and u only).
 *   rho, ux, uy  [ny][nx] doubles, rho > 0; host pointers if on_device == 0,
 *                device pointers otherwise
 * Resets the step counter to 0.  Returns after the fields have been read:
 * host fields once they are copied to the device, device fields once the
 * initialisation kernel has run.  Host fields are copied on a stream of the
 * library's, so the call does not wait for work already queued on the
 * handle's stream; the kernel is queued there behind that work. */
int lbm_init(lbm_t h, const double *rho, const double *ux, const double *uy,
             int on_device);

/* Queues n >= 0 time steps of Eq. 5 (stream, moments, central grad(rho),
 * collide with force) on the handle's stream.  Calls either launch the step
 * kernel once per step with the handle's tile configuration (replayed from
 * CUDA graphs from 8 steps on), or run all n steps as one persistent launch:
 * the batched kernel (see lbm_batch_create) with this grid alone, warps
 * taking tiles dynamically, a bounded grid barrier between steps.  Which one
 * is set by lbm_set_persistent; by default (LBM_PERSISTENT_AUTO) every call
 * launches the step kernel, measured the faster for single grids of 64^2 to
 * 8192^2 in every storage.  A slab always steps persistent; a driven grid or
 * the forward-difference gradient never.  All forms give bitwise the same result.
 * Asynchronous: errors of the kernels surface at the next synchronising call
 * (LBM_ETIMEOUT if a bounded wait ran out). */
int lbm_step(lbm_t h, long long n);

/* Persistent mode of lbm_step:
 *   LBM_PERSISTENT_OFF   every call uses the step kernel
 *   LBM_PERSISTENT_ON    calls of 64 steps or more, or of 8 or more on grids
 *                        of at least 2^20 sites, run one persistent launch
 *   LBM_PERSISTENT_AUTO  the default: as described at lbm_step (the step
 *                        kernel, except for slabs)
 * LBM_EINVAL for other values. */
#define LBM_PERSISTENT_OFF 0
#define LBM_PERSISTENT_ON 1
#define LBM_PERSISTENT_AUTO 2
int lbm_set_persistent(lbm_t h, int on);

/* Writes rho, ux, uy (Eq. 3) of the current state, computed in FP64 from the
 * stored distributions.
 *   rho, ux, uy  [ny][nx] doubles (host if on_device == 0, else device);
 *                any of them may be NULL to skip it
 * Waits for the stream. */
int lbm_moments(lbm_t h, double *rho, double *ux, double *uy, int on_device);

/* Grid totals of mass sum rho and momentum sum rho u (Eq. 3 summed over all
 * sites), reduced in FP64 on the device in a fixed order (bitwise
 * reproducible).  out3 (host) receives {mass, momentum_x, momentum_y}.
 * Returns LBM_ENONFINITE if any total is NaN or Inf.  Waits for the stream. */
int lbm_sums(lbm_t h, double *out3);

/* FP64 Fourier coefficient of a field over the grid, used to measure the
 * sound speed and the viscosity (Section 4, the plane-wave runs and the decay
 * formula of Eq. 10):
 *   out2[0] = (2/N) sum_x v(x) cos(2 pi (kx x/nx + ky y/ny))
 *   out2[1] = (2/N) sum_x v(x) sin(2 pi (kx x/nx + ky y/ny))
 * with v = rho - rho0, ux or uy (field = LBM_FIELD_*), N = nx * ny.  A field
 * v = A sin(2 pi kx x / nx) gives out2 = {0, A}.  Waits for the stream. */
int lbm_mode(lbm_t h, int field, int kx, int ky, double *out2);

/* Driven channel in x, the setup of the sound-speed runs of Section 4
 * (Fig. 1): a plane wave launched from x = 0, where the density varies
 * sinusoidally at zero velocity, into fluid held at rho = 1, u = 0 at the far
 * end.  The paper gives the boundary values but no scheme; this library
 * uses equilibrium columns.  After every step, the post-collision values
 * of column 0 become fbar_i(rho_b(t), u = 0) = w_i rho_b(t) with
 *   rho_b(t) = 1 + amplitude sin(2 pi t / period),
 * t the step number (the step from t to t+1, mod 2^32), and those of columns
 * nx-2 and nx-1 become w_i * 1.  The far end spans two columns, so the
 * periodic wrap in x, which links column nx-1 to column 0, carries nothing
 * into the interior.  y stays periodic.
 *   on         1 to drive, 0 to return to a fully periodic grid
 *   amplitude  |amplitude| < 1 (the paper's runs are small-amplitude)
 *   period     steps per cycle, finite and > 0 (500 in the paper)
 * Needs nx >= 4.  Each step then runs one extra small kernel (27 ny
 * stores), and long step calls use CUDA graphs instead of the persistent
 * launch.  A driven grid cannot join a batch: lbm_batch_create and
 * lbm_batch_step return LBM_EINVAL.  Waits for the grid's stream; returns
 * LBM_EINVAL for a bad argument. */
int lbm_set_drive(lbm_t h, int on, double amplitude, double period);

/* Spatially varying sound speed (the paper's Section 5 outlook: alpha set per
 * site, for example for a temperature gradient or an acoustic lens).  c2 is a
 * [ny][nx] array of c_e^2 > 0 (host if on_device == 0, else device; host
 * values are checked); the force at site x uses alpha(x) = 1/3 - c2(x) in
 * Eq. 5.  NULL returns to the grid's uniform c2.  The field costs one more
 * 4-byte read per site and step.  While a field is set the single-grid step
 * kernel uses at most 4 sites per lane, no bulk-copy pipeline and nearest
 * rounding (an FP32 grid configured for 4 sites per lane steps with 2 sites
 * per lane and one row of loads prefetched, its tile height raised to fill
 * one wave of resident warps where that helps).  The grid can join a batch,
 * where 16-bit grids with nx a multiple of 8 take the 8-site walk, and with
 * LBM_PERSISTENT_ON long lbm_step calls run that batch kernel. */
int lbm_set_c2_field(lbm_t h, const double *c2, int on_device);

/* Steps taken since lbm_init / lbm_set_state. */
long long lbm_time(lbm_t h);

/* Waits for all work queued on the handle's stream. */
int lbm_sync(lbm_t h);

/* Moves the handle to another stream (NULL: the legacy default stream).
 * Work queued on it afterwards runs on `cuda_stream`, after the work already
 * queued on the old stream (an event wait; the host does not block).  If a
 * long lbm_step call has run as a persistent launch, that launch is waited
 * for and its status returned first (LBM_ETIMEOUT leaves the stream
 * unchanged).  Typical use: move a grid created and initialised on one
 * stream onto the stream of the batch it joins. */
int lbm_set_stream(lbm_t h, void *cuda_stream);

/* Bytes of device state (both distribution buffers) a grid of this size and
 * storage needs; 0 for invalid arguments. */
size_t lbm_bytes_required(int nx, int ny, int storage);

/* Free and total device memory (cudaMemGetInfo) of the current device.
 * Host fields passed to lbm_init and lbm_moments are staged in device memory
 * from a pool owned by the library (one per device) that keeps up to 1 GiB
 * reserved between calls; that reservation counts as used here.  lbm_create
 * releases it and retries when a grid's buffers do not fit otherwise. */
int lbm_mem_info(size_t *free_bytes, size_t *total_bytes);

/* Checkpoint: the raw stored distributions (9 planes of nx*ny elements of the
 * storage type, plane-major, each plane [ny][nx]) of the current state.  The
 * steps pull, so a buffer holds values at the site they stream from: plane i
 * at site x is the value the next step reads as f_i(x + e_i), stored as
 * h_i = (f_i - w_i rho0)/w_i.
 * lbm_state_bytes gives the size; lbm_get_state copies it to host memory and
 * the step counter to *t (may be NULL); lbm_set_state restores both.  A run
 * resumed from a checkpoint is bitwise identical to an uninterrupted one. */
size_t lbm_state_bytes(lbm_t h);
int lbm_get_state(lbm_t h, void *dst_host, long long *t);
int lbm_set_state(lbm_t h, const void *src_host, long long t);

/* Tile configuration of the step kernel: each warp walks a strip of 32*vec
 * columns down `rows` rows; blocks hold `warps` warps.  vec is the number of
 * adjacent sites per lane (vectorised loads of vec elements): 1, 2 or 4 for
 * any storage, 8 for the 16-bit storages; nx must be a multiple of vec.
 * rows in [1, 4096], warps in {1, 2, 4, 8}.  At vec 8 with 4 warps and no
 * pipeline (lbm_set_pipeline 0) rows move through shared memory (cp.async),
 * as in the batch kernels; the default for 16-bit grids with nx a multiple of
 * 8 and enough tiles.  The result of a step does not depend on the
 * configuration (bitwise).  Until this is called (or
 * lbm_tune), a grid has the default configuration (rows 16), whose register
 * walks adapt the tile height at launch to the resident warps: fewer rows
 * (down to 2) when the grid has too few tiles to occupy them, more (up to
 * 32) when its tiles need between one and two waves; lbm_get_config reports
 * the configured 16. */
int lbm_set_config(lbm_t h, int vec, int rows, int warps);
int lbm_get_config(lbm_t h, int *vec, int *rows, int *warps);

/* Row pipeline of the step kernel.  stages = 2..4: each warp streams the rows
 * it needs into that many shared-memory stages with asynchronous bulk copies
 * (cp.async.bulk with mbarrier completion), which keeps stages - 1 rows of
 * loads in flight per warp; used when vec is 4 (FP32) or 8 (16-bit), i.e. 16
 * bytes of elements per lane.  stages = 0: the lanes load directly into
 * registers.  Results are bitwise the same either way.  *active tells whether
 * the pipeline is in use with the current vec. */
int lbm_set_pipeline(lbm_t h, int stages);
int lbm_get_pipeline(lbm_t h, int *stages, int *active);

/* Rounding of the 16-bit stores.  With LBM_ROUND_NEAREST a stored value whose
 * per-step change is below half a unit in the last place never changes, so
 * slow processes freeze: the viscous decay of a shear wave of amplitude 1e-3
 * and wavelength 256 (tau = 0.9) stops completely in FP16 storage.
 * LBM_ROUND_STOCHASTIC rounds up with probability equal to the discarded
 * fraction (as many random bits as dropped bits: 13 for FP16, 16 for BF16),
 * so each stored value is the FP32 result in expectation; the random bits are
 * a hash of (pair of sites, direction, step), so runs stay deterministic and
 * independent of the tile configuration and of batching.  Stochastic rounding
 * uses the register walks (vec 1, 2 or 4) and the shared-memory walk at vec 8
 * with 4 warps; it moves other vec-8 configurations to 4 and turns the
 * bulk-copy pipeline off.  FP32 storage
 * accepts only LBM_ROUND_NEAREST.  Because the dither differs from site to
 * site, it breaks symmetries a deterministic rounding keeps exactly: above c2
 * of about 1.16 (c_e > 1.08) a grid started uniform in y has transverse modes
 * that grow (linear analysis), and the dither seeds them, so keep nearest
 * rounding there. */
int lbm_set_rounding(lbm_t h, int mode);
int lbm_get_rounding(lbm_t h, int *mode);

/* Discretisation of grad(rho) in the force (Section 4).
 *   LBM_GRAD_CENTRAL  the default and the paper's scheme:
 *                     (rho(x+1) - rho(x-1))/2 along x and y
 *   LBM_GRAD_FORWARD  rho(x+1) - rho(x) along x and y, the scheme the paper
 *                     found unstable as c_e approaches 1; for reproducing that
 *                     instability.  FP32 storage without a c2 field only; the
 *                     grid then steps with the one-site-per-lane step kernel
 *                     (no persistent launch) and cannot join a batch.
 * Waits for the handle's stream.  LBM_EINVAL for other modes, 16-bit storage,
 * a grid with a c2 field or a slab. */
#define LBM_GRAD_CENTRAL 0
#define LBM_GRAD_FORWARD 1
int lbm_set_gradient(lbm_t h, int mode);
int lbm_get_gradient(lbm_t h, int *mode);

/* Autotuner: times the valid tile configurations on this grid (without
 * changing its state) and keeps the fastest.  If cache_path is not NULL the
 * choice is read from / stored in that JSON file, keyed by device, storage
 * and grid size.  Waits for the stream. */
int lbm_tune(lbm_t h, const char *cache_path);

/* Mean device time in milliseconds of the step kernel over the last
 * lbm_step call made with timing enabled (lbm_set_timing(h, 1)); the events
 * are recorded on the handle's stream around each launch. */
int lbm_set_timing(lbm_t h, int on);
int lbm_kernel_ms(lbm_t h, double *ms, long long *launches);

/* ---- Batches: many uneven grids advanced in one persistent launch ------- */

/* Groups n >= 1 existing handles (any sizes, tau, c2, storage and rounding;
 * all on the same device) into a batch stepped by persistent cooperative
 * kernels over a tile work-list, with a grid-wide barrier between time steps
 * (one launch per kind group, see lbm_batch_get_groups).  Every grid reaches
 * bitwise the state it reaches when stepped alone.  The batch refers to the
 * handles; they must outlive it and must not be stepped individually while
 * it is being stepped.  The batch's work runs on the stream grids[0] had
 * when the batch was created.  Each step call first makes it wait for the
 * work queued on every member's current stream, and then makes those streams
 * wait for the batch's work, so calls on a member's own stream stay ordered
 * with the batch.
 * Grids with a c2 field may join; driven grids are refused (LBM_EINVAL). */
int lbm_batch_create(const lbm_t *grids, int n, lbm_batch_t *out);
int lbm_batch_destroy(lbm_batch_t b);

/* Advances grid g of the batch by min(n, limits[g]) steps (limits may be NULL:
 * n steps each), one persistent launch per kind group, replayed from a CUDA
 * graph (see lbm_batch_set_launch).  Asynchronous.  A barrier wait that exceeds its time limit makes the
 * kernel stop and the next synchronising batch call return LBM_ETIMEOUT.
 * If a grid's c2 field or rounding mode changed since the batch was built,
 * the work-list is rebuilt first (the call then waits for the stream).
 * LBM_EINVAL if a grid has gained a drive or the forward-difference gradient. */
int lbm_batch_step(lbm_batch_t b, long long n, const long long *limits);

/* Waits for the batch's stream and returns the kernel's status
 * (LBM_OK or LBM_ETIMEOUT). */
int lbm_batch_sync(lbm_batch_t b);

/* Tile height (rows per warp) and persistent-grid occupancy (0: as many
 * blocks per SM as fit) of the batch kernels; lbm_batch_tune picks the tile
 * height and the 16-bit walk from timed dry steps (the grids' states and step
 * counts are unchanged; on an error the previous configuration is restored
 * and the error returned).  Until one of them is called, a lockstep batch
 * whose tiles at 16 rows would fill less than 3/4 of the resident warps
 * (16 per SM) takes shorter tiles, down to 2 rows, as many as those warps
 * hold. */
int lbm_batch_set_config(lbm_batch_t b, int rows, int blocks_per_sm);
int lbm_batch_tune(lbm_batch_t b);
/* Current tile height (of the lockstep work-list as built), resident blocks
 * per SM of the first kind group, and whether every kind group runs a
 * specialised kernel rather than the general one. */
int lbm_batch_get_config(lbm_batch_t b, int *rows, int *blocks_per_sm, int *specialised);
/* The work-list as last built (at creation, by a configuration, schedule or
 * walk change, or by a step call that found a grid's field or rounding
 * changed): *tiles = warp walks per time step, *paired = how many of them
 * walk two segments of a narrow grid, a half-warp each (lockstep kind groups
 * of one 8-site 16-bit kind under LBM_WALK16_AUTO pair the tiles of grids at
 * most 128 columns wide when those are at least a fifth of the group's tiles;
 * results are bitwise those of single walks).  Either pointer may be NULL. */
int lbm_batch_get_tiles(lbm_batch_t b, int *tiles, int *paired);

/* Number of persistent launches one lbm_batch_step makes (kind groups).  The
 * grids of one walk (storage kind, sites per lane, rounding; nx a multiple of
 * 4) that together move at least 64 MiB per step run in a launch of their
 * own specialised kernel; the other grids share one launch of the general
 * kernel.  A batch of one walk is one group.  The groups hold disjoint grids
 * and run one after the other on the batch's stream, each advancing its
 * grids by all the steps of the call. */
int lbm_batch_get_groups(lbm_batch_t b, int *groups);

/* The walk of 16-bit grids in a batch (results are bitwise the same for all):
 *   LBM_WALK16_AUTO    the default: LBM_WALK16_V8, the faster on GB300 for
 *                      both roundings
 *   LBM_WALK16_V8      8 sites per lane, 128-bit loads, when nx is a multiple
 *                      of 8 (else as LBM_WALK16_V4)
 *   LBM_WALK16_V4      4 sites per lane, 64-bit loads, one row of loads in
 *                      flight ahead of the row being pulled
 *   LBM_WALK16_V4_PF2  as LBM_WALK16_V4 with two rows in flight (more
 *                      registers, 12 warps per SM instead of 16)
 * lbm_batch_tune tries them all.  Waits for the batch's stream; LBM_EINVAL
 * for other values. */
#define LBM_WALK16_AUTO 0
#define LBM_WALK16_V8 1
#define LBM_WALK16_V4 2
#define LBM_WALK16_V4_PF2 3
int lbm_batch_set_walk16(lbm_batch_t b, int walk);
int lbm_batch_get_walk16(lbm_batch_t b, int *walk);

/* Schedule of lbm_batch_step:
 *   LBM_SCHEDULE_LOCKSTEP  the default: one persistent launch per kind group
 *                          runs every time step of all its grids, with a
 *                          grid-wide barrier between steps
 *   LBM_SCHEDULE_FLOW      one launch over all grids with no barrier: each
 *                          grid advances on its own, a tile's step starting
 *                          as soon as the tiles it reads from have finished
 *                          the previous step (per-tile progress counters,
 *                          bounded waits).  Warps share the GPU round-robin
 *                          between grids, so a small grid takes many steps
 *                          while a large one takes few: each grid's
 *                          time-to-result follows its own size instead of the
 *                          whole batch's.  Every call still runs until each
 *                          grid has taken min(n, limits[g]) steps; n at most
 *                          2^31 - 1.
 * Every grid reaches bitwise the same state in both schedules.  Waits for the
 * batch's stream; LBM_EINVAL for other values. */
#define LBM_SCHEDULE_LOCKSTEP 0
#define LBM_SCHEDULE_FLOW 1
int lbm_batch_set_schedule(lbm_batch_t b, int schedule);
int lbm_batch_get_schedule(lbm_batch_t b, int *schedule);

/* How lbm_batch_step issues its persistent launches:
 *   LBM_LAUNCH_AUTO    the default: the launches of a call (one per kind group,
 *                      with their parameter copies) are captured once per step
 *                      count into a CUDA graph and replayed; if the capture
 *                      fails, the batch switches to direct launches for good
 *                      and reports it below
 *   LBM_LAUNCH_GRAPH   always replay the graph; a failed capture is an error
 *                      (LBM_ECUDA from lbm_batch_step)
 *   LBM_LAUNCH_DIRECT  cooperative launches issued one by one, no graph
 * Results are bitwise the same in every mode.  lbm_batch_set_launch waits for
 * the batch's stream.  lbm_batch_get_launch gives the mode, how the last step
 * call ran (*last: LBM_LAUNCH_GRAPH or LBM_LAUNCH_DIRECT; 0 before the first
 * call) and whether an AUTO capture failed (*capture_failed: 1).  Any output
 * pointer may be NULL. */
#define LBM_LAUNCH_AUTO 0
#define LBM_LAUNCH_GRAPH 1
#define LBM_LAUNCH_DIRECT 2
int lbm_batch_set_launch(lbm_batch_t b, int mode);
int lbm_batch_get_launch(lbm_batch_t b, int *mode, int *last, int *capture_failed);

/* Barrier wait limit of the batch kernel in microseconds (default 1e6). */
int lbm_batch_set_timeout_us(lbm_batch_t b, long long us);

/* ---- Slab decomposition in y (one grid over several GPUs) ---------------- */

/* A slab of a grid split along y between ranks (one GPU each): rank r of N
 * owns the global rows [r*ny_local, (r+1)*ny_local); the grid stays
 * periodic in x and in y (rank 0's lower neighbour is rank N-1).  A step of
 * Eq. 5 at a row reads the stored values up to two rows away (the pull, and
 * the central gradient of the pulled density, Section 4), so the handle's
 * buffers hold ny_local + 4 rows: ghost rows 0 and 1 (copies of the lower
 * neighbour's two highest rows), the own rows 2 .. ny_local+1, and ghost rows
 * ny_local+2 and ny_local+3 (copies of the upper neighbour's two lowest).
 *   nx, tau, c2, storage, cuda_stream, out  as lbm_create
 *   ny_local  own rows, >= 2
 * The handle is an ordinary one otherwise: lbm_init, lbm_moments,
 * lbm_get_state, lbm_set_c2_field and so on see the whole local buffer,
 * [ny_local + 4][nx], ghost rows included.  lbm_step takes n = 1 only (the
 * ghost rows must be refreshed between steps; LBM_EINVAL otherwise) and
 * computes the own rows, with the batch kernel over their tiles; a slab can
 * also join a batch.  Driven slabs are refused.  Returns as lbm_create. */
int lbm_slab_create(int nx, int ny_local, double tau, double c2, int storage,
                    void *cuda_stream, lbm_t *out);

/* Bytes of one side's halo: 9 planes x 2 rows x nx elements of the storage
 * type (0 for a handle that is not a slab). */
size_t lbm_slab_halo_bytes(lbm_t h);

/* Halo exchange, queued on the handle's stream (asynchronous):
 *   lbm_slab_pack(h, dst, 0)    own rows 2, 3 (to send to the lower
 *                               neighbour)          -> dst
 *   lbm_slab_pack(h, dst, 1)    own rows ny_local, ny_local+1 (to send to
 *                               the upper neighbour) -> dst
 *   lbm_slab_unpack(h, src, 0)  src -> ghost rows 0, 1 (from the lower
 *                               neighbour's side-1 pack)
 *   lbm_slab_unpack(h, src, 1)  src -> ghost rows ny_local+2, +3 (from the
 *                               upper neighbour's side-0 pack)
 * dst/src are device buffers of lbm_slab_halo_bytes bytes, packed as
 * [9][2][nx] of the current state (after the last lbm_step).  The transfer
 * between ranks is the caller's; order it with the handle's stream.  A
 * single slab exchanging with itself (side 0 into side 1 and back) is the
 * periodic grid.  LBM_EINVAL for a bad side, NULL or a handle that is not a
 * slab. */
int lbm_slab_pack(lbm_t h, void *dst, int side);
int lbm_slab_unpack(lbm_t h, const void *src, int side);

/* ---- Grid totals without allocation ------------------------------------- */

/* The paper has no counterpart to this call; it is a service for callers that
 * cannot allocate device memory at the point where they need the totals: code
 * that runs inside its own memory pool or under an allocator that forbids
 * outside cudaMalloc, code whose device memory is budgeted up front, or code
 * that must not make an allocating CUDA call there.  It computes what
 * lbm_sums computes, for a state buffer the caller already holds, and calls
 * no cudaMalloc, cudaFree or other allocating routine.
 *   f             device pointer to 9 planes of the stored distributions, plane
 *                 i starting at element i * plane_stride (the checkpoint
 *                 layout of lbm_get_state has plane_stride = nx * ny); element
 *                 type per `storage`, h_i = (f_i - w_i rho0)/w_i
 *   nx, ny        grid size, nx * ny <= 2^31 - 1 (larger grids: LBM_EINVAL)
 *   plane_stride  elements between planes, >= nx * ny
 *   storage       LBM_F32, LBM_F16D or LBM_BF16D; rho0 > 0 as at creation
 *   cuda_stream   stream to run on (NULL: legacy default stream)
 *   out3          host array receiving {mass, momentum_x, momentum_y}
 * Scratch: a fixed 24.1 KiB array in the library's device memory (one partial
 * triple for each of at most 1024 reduction blocks, plus the result), held on
 * every GPU that loads the library until the process exits.  The first call on
 * a device also does a one-time set-up: it looks up that array's device
 * address (cudaGetSymbolAddress, with that device current) and keeps it for
 * later calls; make that first call on each device before any stream capture
 * begins.  All calls share the array and leave their values in it; each call
 * writes every slot it reads, so nothing needs clearing, but calls that
 * overlap on the GPU race and can return wrong totals.  Every call is
 * synchronous: it queues the reduction on cuda_stream, copies the three totals
 * to out3 and waits for that stream before it returns.  Returns LBM_OK,
 * LBM_EINVAL, LBM_ECUDA or LBM_ENONFINITE. */
int lbm_sums_noalloc(const void *f, int nx, int ny, size_t plane_stride,
                     int storage, double rho0, void *cuda_stream, double *out3);

/* ---- Errors --------------------------------------------------------------- */
const char *lbm_strerror(int status);
const char *lbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
